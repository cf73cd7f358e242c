// cluster.cuh -- the whole p-BiCGStab iteration loop (Algorithm 2) of a small
// system in one launch over one thread-block cluster, held in shared memory.
//
// A system of a few thousand rows leaves the multi-pass launch graph bound by
// latency: every iteration pays two kernel launches, two grid-wide merges
// through global memory and an atomic ticket, and the ramp of a grid that has
// only a handful of tiles.  Here one cluster of up to 16 CTAs (one SM each)
// runs the iterations inside one kernel:
//   - each CTA keeps its rows of the 11 solver vectors and of the SELL-32
//     matrix in its own shared memory for the whole launch;
//   - the SpMV gathers w (pass X) and z (pass Y) from the owning CTA's shared
//     memory through distributed shared memory;
//   - each reduction point is a cluster merge: every CTA adds its exact
//     accumulator digits (or writes its plain partial) into CTA 0's shared
//     memory, the cluster syncs (a hardware barrier), CTA 0 rounds (exact) or
//     sums in CTA order (plain) and takes the pass's scalar step on its shared
//     copy of the control block, and the cluster syncs again before the
//     other CTAs read the scalars from it.
// The row arithmetic, the SpMV's fma order, the exact rounding and the
// scalar steps are the functions the passes use, so exact mode is
// bit-identical to the multi-pass path and to the oracle.  The vectors and
// the control block go back to global memory when the status leaves RUNNING.
//
// There is no spin-wait: every CTA executes the same sequence of cluster
// barriers (the exit test reads a status that CTA 0 wrote before the last
// barrier), and the final barrier keeps every CTA's shared memory alive
// until no other CTA reads it.
#pragma once
#include <cooperative_groups.h>
#include "kernels.cuh"

namespace pbcg {

constexpr int CLUSTER_MAX_CTAS = 16;     // non-portable cluster size (opt-in)
constexpr int CLUSTER_MAX_RPT = 4;       // rows per thread (1, 2 or 4: rows per CTA a power of two)
constexpr int CL_NV = 11;                // vectors held in shared memory
enum { CV_X, CV_R, CV_W, CV_T, CV_P, CV_S, CV_Z, CV_V, CV_Q, CV_Y, CV_R0 };

// CTA 0's merge target and control block (declared in every CTA, used in CTA 0)
struct ClusterHub {
    unsigned long long dig[4][NDIG];     // carry-save digits of the cluster's exact dots
    int kmin[4], kmax[4], nf[4], pad;
    double part[4][CLUSTER_MAX_CTAS];    // plain partials, one per CTA
    Ctl ctl;                             // the solve's control block during the launch
};

// Dynamic shared memory of a CTA holding `rows` rows and `emax` SELL entries.
__host__ __device__ constexpr size_t cluster_smem_bytes(int rows, int emax)
{
    return (size_t)CL_NV * rows * sizeof(double) + (size_t)emax * (sizeof(double) + sizeof(uint32_t)) +
           (size_t)rows * sizeof(int) + (size_t)(rows / 32 + 1) * sizeof(int);
}

// Row of the CTA (local row lr, local slice lr / 32): acc = +0;
// acc = fma(val_j, x[col_j], acc) for j < len in the CSR order, x gathered
// from the CTA owning col_j (code = owner << 16 | local row).
__device__ __forceinline__ double spmv_cluster(const double *mva, const uint32_t *mcode, int soff, int width, int len,
                                               int lane, const double *const *gx)
{
    double acc = 0.0;
    for (int j0 = 0; j0 < width; j0 += UNR) {        // warp-uniform bound
        double v[UNR], xv[UNR];
        uint32_t cd[UNR];
#pragma unroll
        for (int j = 0; j < UNR; j++) {
            if (j0 + j < len) {
                const int e = soff + (j0 + j) * 32 + lane;
                cd[j] = mcode[e];
                v[j] = mva[e];
            }
        }
#pragma unroll
        for (int j = 0; j < UNR; j++)
            if (j0 + j < len)
                xv[j] = gx[cd[j] >> 16][cd[j] & 0xffffu];
#pragma unroll
        for (int j = 0; j < UNR; j++)
            if (j0 + j < len)
                acc = __fma_rn(v[j], xv[j], acc);
    }
    return acc;
}

// Merge the cluster's ND dots into dv (valid in CTA 0).  Every thread of every CTA calls.
template <int ND, int MODE>
__device__ __forceinline__ void cluster_merge(DotSet<ND, MODE> &D, Shm<ND> &sh, ClusterHub &hub, ClusterHub *hub0,
                                              cooperative_groups::cluster_group &cl)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (MODE == 1) {
#pragma unroll
        for (int d = 0; d < ND; d++) {
            win_flush<ND>(D.win[d], sh.acc, d);
            if (D.nf[d])
                atomicOr(&sh.acc.nf[d], 1);
        }
    } else {
        double tot[ND];
        warp_sum_plain<ND>(D.s, tot);
        if (lane == 0) {
#pragma unroll
            for (int d = 0; d < ND; d++)
                sh.wpart[d][warp] = tot[d];
        }
    }
    __syncthreads();
    if (MODE == 1) {
        for (int d = 0; d < ND; d++) {
            const int k0 = sh.acc.kmin[d], k1 = sh.acc.kmax[d];
            for (int k = k0 + (int)threadIdx.x; k <= k1; k += THREADS) {
                const unsigned long long v = sh.acc.dig[d][k];
                if (v != 0ull)
                    atomicAdd(&hub0->dig[d][k], v);
            }
            if (threadIdx.x == 0) {
                if (k1 >= k0) {
                    atomicMin(&hub0->kmin[d], k0);
                    atomicMax(&hub0->kmax[d], k1);
                }
                if (sh.acc.nf[d])
                    atomicOr(&hub0->nf[d], 1);
            }
        }
    } else if (threadIdx.x < ND) {
        double v = sh.wpart[threadIdx.x][0];
        for (int w = 1; w < WARPS; w++)
            v = __dadd_rn(v, sh.wpart[threadIdx.x][w]);
        hub0->part[threadIdx.x][blockIdx.x] = v;
    }
    cl.sync();
    if (blockIdx.x != 0)
        return;
    if (MODE == 1) {
        // round, then clear the touched digits for the next merge
        if (threadIdx.x < ND) {
            const int d = threadIdx.x;
            sh.dv[d] = round_digits(hub.dig[d], hub.kmin[d], hub.kmax[d], hub.nf[d], sh.scratch[d]);
        }
        __syncthreads();
        for (int d = 0; d < ND; d++)
            for (int k = hub.kmin[d] + (int)threadIdx.x; k <= hub.kmax[d]; k += THREADS)
                hub.dig[d][k] = 0ull;
        __syncthreads();
        if (threadIdx.x < ND) {
            hub.kmin[threadIdx.x] = NDIG;
            hub.kmax[threadIdx.x] = -1;
            hub.nf[threadIdx.x] = 0;
        }
    } else if (warp < ND) {
        // the order of finalize(): lane c takes CTA c, then a butterfly
        double v = 0.0;
        for (int c = lane; c < (int)gridDim.x; c += 32)
            v = __dadd_rn(v, hub.part[warp][c]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            v = __dadd_rn(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (lane == 0)
            sh.dv[warp] = v;
    }
    __syncthreads();
}

// Iterations of Algorithm 2 from the state the setup passes (or an earlier
// launch) left, until the status leaves RUNNING.  The grid is one cluster;
// CTA b holds rows [b * rows, (b + 1) * rows), rows = rpt * THREADS = 2^lg,
// and at most emax SELL entries.  Residual replacement is not taken here
// (the multi-pass path runs it).
template <int MODE>
__global__ void __launch_bounds__(THREADS, 1)
    k_pipe_cluster(Mat A, Vecs V, Ctl *c, int rpt, int lg, int emax)
{
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ __align__(128) uint8_t dsm[];
    __shared__ Shm<4> sx;
    __shared__ Shm<3> sy;
    __shared__ ClusterHub hub;
    __shared__ const double *gw[CLUSTER_MAX_CTAS], *gz[CLUSTER_MAX_CTAS];
    const int rows = rpt * THREADS, nsl = rows / 32, me = (int)blockIdx.x, row0 = me * rows;
    double *vec = reinterpret_cast<double *>(dsm);               // [CL_NV][rows]
    double *mva = vec + (size_t)CL_NV * rows;                    // [emax]
    uint32_t *mcode = reinterpret_cast<uint32_t *>(mva + emax);  // [emax]
    int *mlen = reinterpret_cast<int *>(mcode + emax);           // [rows]
    int *msoff = mlen + rows;                                    // [nsl + 1]
    double *const Vx = vec + CV_X * rows, *const Vr = vec + CV_R * rows, *const Vw = vec + CV_W * rows;
    double *const Vt = vec + CV_T * rows, *const Vp = vec + CV_P * rows, *const Vs = vec + CV_S * rows;
    double *const Vz = vec + CV_Z * rows, *const Vv = vec + CV_V * rows, *const Vq = vec + CV_Q * rows;
    double *const Vy = vec + CV_Y * rows, *const Vr0 = vec + CV_R0 * rows;

    // ---- load this CTA's rows: matrix slices, row lengths, vectors
    const int gs0 = min(me * nsl, A.nslices), gs1 = min(gs0 + nsl, A.nslices);
    const int e0 = A.sl_off[gs0], ne = A.sl_off[gs1] - e0;
    for (int t = threadIdx.x; t <= nsl; t += THREADS)
        msoff[t] = A.sl_off[min(gs0 + t, gs1)] - e0;
    for (int e = threadIdx.x; e < ne; e += THREADS) {
        const int col = A.ci[e0 + e];
        mva[e] = A.va[e0 + e];
        mcode[e] = ((uint32_t)(col >> lg) << 16) | (uint32_t)(col & (rows - 1));
    }
    double *const gsrc[CL_NV] = {V.x, V.r, V.w, V.t, V.p, V.s, V.z, V.v, V.q, V.y, V.r0};
    for (int r = threadIdx.x; r < rows; r += THREADS) {
        const int i = row0 + r;
        mlen[r] = (i < A.nslices * 32) ? A.rlen[i] : 0;
#pragma unroll
        for (int v = 0; v < CL_NV; v++)
            vec[v * rows + r] = (i < A.n) ? gsrc[v][i] : 0.0;
    }
    if (me == 0 && threadIdx.x == 0) {
        hub.ctl = *c;
        for (int d = 0; d < 4; d++) {
            hub.kmin[d] = NDIG;
            hub.kmax[d] = -1;
            hub.nf[d] = 0;
        }
    }
    if (me == 0)
        for (int k = threadIdx.x; k < 4 * NDIG; k += THREADS)
            (&hub.dig[0][0])[k] = 0ull;
    if (threadIdx.x < gridDim.x) {
        gw[threadIdx.x] = cl.map_shared_rank(Vw, threadIdx.x);
        gz[threadIdx.x] = cl.map_shared_rank(Vz, threadIdx.x);
    }
    ClusterHub *const hub0 = cl.map_shared_rank(&hub, 0);
    const volatile Ctl *const c0 = &hub0->ctl;     // read after each cluster barrier
    cl.sync();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (;;) {
        if (c0->status != ST_RUNNING)
            break;
        const bool first = c0->it == 0;
        {
            // pass X: t = A w (i >= 1), p, s, z, q, y; dots (q,y), (y,y), (r0,s), (r0,z)
            const double beta = c0->beta, nalpha = -c0->alpha, nomega = -c0->omega;
            shm_init<4, MODE>(sx);
            __syncthreads();
            DotSet<4, MODE> D;
            D.init();
            for (int k = 0; k < rpt; k++) {
                const int r = k * THREADS + (int)threadIdx.x, ls = k * WARPS + warp;
                const bool act = row0 + r < A.n;
                double q = 0.0, y = 0.0, r0i = 0.0, si = 0.0, zi = 0.0;
                if (act) {
                    const double ri = Vr[r], wi = Vw[r];
                    r0i = Vr0[r];
                    double ti, pold = 0.0, sold = 0.0, zold = 0.0, vold = 0.0;
                    if (first) {
                        ti = Vt[r];
                    } else {
                        ti = spmv_cluster(mva, mcode, msoff[ls], (msoff[ls + 1] - msoff[ls]) >> 5, mlen[r], lane, gw);
                        pold = Vp[r];
                        sold = Vs[r];
                        zold = Vz[r];
                        vold = Vv[r];
                    }
                    const XRow X = pipe_x_row(first, false, nalpha, beta, nomega, ri, wi, ti, pold, sold, zold, vold);
                    Vt[r] = ti;
                    Vp[r] = X.p;
                    Vs[r] = X.s;
                    Vz[r] = X.z;
                    Vq[r] = X.q;
                    Vy[r] = X.y;
                    q = X.q;
                    y = X.y;
                    si = X.s;
                    zi = X.z;
                }
                const Dec dq = decode(q), dy = decode(y), dr = decode(r0i), ds = decode(si), dz = decode(zi);
                D.template add2<false>(sx, 0, q, y, dq, dy, act);
                D.template add2<true>(sx, 1, y, y, dy, dy, act);
                D.template add2<false>(sx, 2, r0i, si, dr, ds, act);
                D.template add2<false>(sx, 3, r0i, zi, dr, dz, act);
            }
            cluster_merge<4, MODE>(D, sx, hub, hub0, cl);
            if (me == 0 && threadIdx.x == 0)
                pipe_x_tail(&hub.ctl, sx.dv);
            cl.sync();
        }
        if (c0->status != ST_RUNNING)
            break;
        {
            // pass Y: v = A z, x, r, w; dots (r0,r), (r0,w), (r,r)
            const double alpha = c0->alpha, omega = c0->omega;
            const double nalpha = -alpha, nomega = -omega;
            shm_init<3, MODE>(sy);
            __syncthreads();
            DotSet<3, MODE> D;
            D.init();
            for (int k = 0; k < rpt; k++) {
                const int r = k * THREADS + (int)threadIdx.x, ls = k * WARPS + warp;
                const bool act = row0 + r < A.n;
                double rn = 0.0, wn = 0.0, r0i = 0.0;
                if (act) {
                    const double vi = spmv_cluster(mva, mcode, msoff[ls], (msoff[ls + 1] - msoff[ls]) >> 5, mlen[r],
                                                   lane, gz);
                    const YRow Yr = pipe_y_row(alpha, omega, nalpha, nomega, Vq[r], Vy[r], Vp[r], Vx[r], Vt[r], vi);
                    Vx[r] = Yr.x;
                    Vv[r] = vi;
                    Vr[r] = Yr.r;
                    Vw[r] = Yr.w;
                    rn = Yr.r;
                    wn = Yr.w;
                    r0i = Vr0[r];
                }
                const Dec dr0 = decode(r0i), dr = decode(rn), dw = decode(wn);
                D.template add_row<3, false, false, true>(sy, act, r0i, rn, dr0, dr, r0i, wn, dr0, dw, rn, rn, &dr,
                                                          &dr);
            }
            cluster_merge<3, MODE>(D, sy, hub, hub0, cl);
            if (me == 0 && threadIdx.x == 0)
                pipe_y_tail(&hub.ctl, sy.dv);
            cl.sync();
        }
    }

    // ---- write back: the vectors of this CTA's rows and the control block
    for (int r = threadIdx.x; r < rows; r += THREADS) {
        const int i = row0 + r;
        if (i < A.n) {
#pragma unroll
            for (int v = 0; v < CL_NV - 1; v++)          // r0 is never written
                gsrc[v][i] = vec[v * rows + r];
        }
    }
    if (me == 0 && threadIdx.x == 0)
        *c = hub.ctl;
    cl.sync();       // no CTA leaves while another may still read its shared memory
}

}  // namespace pbcg
