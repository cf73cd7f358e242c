// cluster.cuh -- the whole iteration loop of a small system (Algorithm 2, and
// Algorithm 1 beside it) in one launch over one thread-block cluster, held in
// shared memory.
//
// A system of a few thousand rows leaves the multi-pass launch graph bound by
// latency: every iteration pays two kernel launches, two grid-wide merges
// through global memory and an atomic ticket, and the ramp of a grid that has
// only a handful of tiles.  Here one cluster of up to 16 CTAs (one SM each)
// runs the iterations inside one kernel:
//   - each CTA keeps its rows of the 11 solver vectors and of the SELL-32
//     matrix in its own shared memory for the whole launch;
//   - the SpMV gathers its operand (w and z in Algorithm 2, p and s, r in
//     Algorithm 1) from the owning CTA's shared memory through distributed
//     shared memory;
//   - each reduction point is a cluster merge: every CTA adds its exact
//     accumulator digits (or writes its plain partial) into CTA 0's shared
//     memory, the cluster syncs (a hardware barrier), CTA 0 rounds (exact) or
//     sums in CTA order (plain) and takes the pass's scalar step on its shared
//     copy of the control block, pushes the scalars the next step reads into
//     every CTA's shared memory, and the cluster syncs again.
// The row arithmetic, the SpMV's fma order, the exact rounding and the
// scalar steps are the functions the passes use, so exact mode is
// bit-identical to the multi-pass path and to the oracle.  The vectors and
// the control block go back to global memory when the status leaves RUNNING.
//
// There is no spin-wait: every CTA executes the same sequence of cluster
// barriers (the exit test reads a status that CTA 0 pushed before the last
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

// same, with the gathered operand formed as fma(na, s[col], r[col]) (pass B of Algorithm 1)
__device__ __forceinline__ double spmv_cluster_axpy(const double *mva, const uint32_t *mcode, int soff, int width,
                                                    int len, int lane, double na, const double *const *gs,
                                                    const double *const *gr)
{
    double acc = 0.0;
    for (int j0 = 0; j0 < width; j0 += UNR) {
        double v[UNR], xs[UNR], xr[UNR];
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
        for (int j = 0; j < UNR; j++) {
            if (j0 + j < len) {
                xs[j] = gs[cd[j] >> 16][cd[j] & 0xffffu];
                xr[j] = gr[cd[j] >> 16][cd[j] & 0xffffu];
            }
        }
#pragma unroll
        for (int j = 0; j < UNR; j++)
            if (j0 + j < len)
                acc = __fma_rn(v[j], __fma_rn(na, xs[j], xr[j]), acc);
    }
    return acc;
}

// This CTA's rows in shared memory (dynamic): CL_NV vectors of `rows`
// entries, the SELL entries of its slices (value and owner/local code), the
// row lengths and the slices' local entry offsets.  gv[k][b] is vector k of
// CTA b through distributed shared memory.
struct ClusterRows {
    double *vec, *mva;
    uint32_t *mcode;
    int *mlen, *msoff;
    int rows, nsl, row0;
    __device__ __forceinline__ double *v(int k) const { return vec + (size_t)k * rows; }
    __device__ __forceinline__ int soff(int ls) const { return msoff[ls]; }
    __device__ __forceinline__ int width(int ls) const { return (msoff[ls + 1] - msoff[ls]) >> 5; }
};

// The scalars every CTA reads after a merge.  CTA 0 pushes them into each
// CTA's own copy (one distributed-shared-memory store per CTA) before the
// barrier that ends the merge, so that after it every thread reads local
// shared memory instead of loading them from CTA 0.
struct ClusterScal {
    double alpha, beta, omega;
    int status, it;
};

struct ClusterGather {
    const double *gv[CL_NV][CLUSTER_MAX_CTAS];
    ClusterScal *scp[CLUSTER_MAX_CTAS];      // every CTA's sc
    ClusterScal sc;                          // this CTA's copy of the scalars
};

// CTA 0, every thread: after its scalar step (thread 0), push the scalars to
// every CTA of the cluster (the caller's cluster barrier publishes them)
__device__ __forceinline__ void push_scal(const ClusterHub &hub, const ClusterGather &G)
{
    __syncthreads();
    if (threadIdx.x < gridDim.x) {
        ClusterScal s;
        s.alpha = hub.ctl.alpha;
        s.beta = hub.ctl.beta;
        s.omega = hub.ctl.omega;
        s.status = hub.ctl.status;
        s.it = hub.ctl.it;
        *G.scp[threadIdx.x] = s;
    }
}

// Fill this CTA's rows from global memory, CTA 0's hub from the control
// block, the gather tables; ends with a cluster barrier.
__device__ __forceinline__ ClusterRows cluster_load(const Mat &A, const Vecs &V, const Ctl *c, int rpt, int lg,
                                                    int emax, uint8_t *dsm, ClusterHub &hub, ClusterGather &G,
                                                    cooperative_groups::cluster_group &cl)
{
    ClusterRows R;
    R.rows = rpt * THREADS;
    R.nsl = R.rows / 32;
    R.row0 = (int)blockIdx.x * R.rows;
    R.vec = reinterpret_cast<double *>(dsm);
    R.mva = R.vec + (size_t)CL_NV * R.rows;
    R.mcode = reinterpret_cast<uint32_t *>(R.mva + emax);
    R.mlen = reinterpret_cast<int *>(R.mcode + emax);
    R.msoff = R.mlen + R.rows;
    const int gs0 = min((int)blockIdx.x * R.nsl, A.nslices), gs1 = min(gs0 + R.nsl, A.nslices);
    const int e0 = A.sl_off[gs0];
    const int ne = PBCG_IN(A.sl_off[gs1] - e0, emax + 1, CHK_CLUSTER) ? A.sl_off[gs1] - e0 : 0;
    for (int t = threadIdx.x; t <= R.nsl; t += THREADS)
        R.msoff[t] = A.sl_off[min(gs0 + t, gs1)] - e0;
    for (int e = threadIdx.x; e < ne; e += THREADS) {
        int col = A.ci[e0 + e];
        if (!PBCG_IN(col, A.n, CHK_COL))
            col = 0;
        R.mva[e] = A.va[e0 + e];
        R.mcode[e] = ((uint32_t)(col >> lg) << 16) | (uint32_t)(col & (R.rows - 1));
    }
    const double *const gsrc[CL_NV] = {V.x, V.r, V.w, V.t, V.p, V.s, V.z, V.v, V.q, V.y, V.r0};
    for (int r = threadIdx.x; r < R.rows; r += THREADS) {
        const int i = R.row0 + r;
        R.mlen[r] = (i < A.nslices * 32) ? A.rlen[i] : 0;
#pragma unroll
        for (int k = 0; k < CL_NV; k++)
            R.vec[(size_t)k * R.rows + r] = (i < A.n) ? gsrc[k][i] : 0.0;
    }
    if (blockIdx.x == 0) {
        if (threadIdx.x == 0) {
            hub.ctl = *c;
            for (int d = 0; d < 4; d++) {
                hub.kmin[d] = NDIG;
                hub.kmax[d] = -1;
                hub.nf[d] = 0;
            }
        }
        for (int k = threadIdx.x; k < 4 * NDIG; k += THREADS)
            (&hub.dig[0][0])[k] = 0ull;
    }
    for (int t = threadIdx.x; t < CL_NV * (int)gridDim.x; t += THREADS)
        G.gv[t / gridDim.x][t % gridDim.x] = cl.map_shared_rank(R.v(t / gridDim.x), t % gridDim.x);
    for (int t = threadIdx.x; t < (int)gridDim.x; t += THREADS)
        G.scp[t] = cl.map_shared_rank(&G.sc, t);
    cl.sync();
    // (every CTA is running from here on) the scalars of the first step
    if (blockIdx.x == 0)
        push_scal(hub, G);
    cl.sync();
    return R;
}

// Write this CTA's rows of the vectors (all but r0) and CTA 0's control block
// back to global memory; the final barrier keeps every CTA's shared memory
// alive until no other CTA reads it.
__device__ __forceinline__ void cluster_store(const Mat &A, const Vecs &V, Ctl *c, const ClusterRows &R,
                                              const ClusterHub &hub, cooperative_groups::cluster_group &cl)
{
    double *const gdst[CL_NV - 1] = {V.x, V.r, V.w, V.t, V.p, V.s, V.z, V.v, V.q, V.y};
    for (int r = threadIdx.x; r < R.rows; r += THREADS) {
        const int i = R.row0 + r;
        if (i < A.n) {
#pragma unroll
            for (int k = 0; k < CL_NV - 1; k++)
                gdst[k][i] = R.vec[(size_t)k * R.rows + r];
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0)
        *c = hub.ctl;
    cl.sync();
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
        if (warp < ND) {                                // warp d rounds dot d
            const double v = round_digits_warp(hub.dig[warp], hub.kmin[warp], hub.kmax[warp], hub.nf[warp],
                                               sh.scratch[warp]);
            if ((threadIdx.x & 31) == 0)
                sh.dv[warp] = v;
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
    __shared__ ClusterGather G;
    const ClusterRows R = cluster_load(A, V, c, rpt, lg, emax, dsm, hub, G, cl);
    ClusterHub *const hub0 = cl.map_shared_rank(&hub, 0);
    const volatile ClusterScal *const c0 = &G.sc;  // pushed by CTA 0 before each cluster barrier
    const int me = (int)blockIdx.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double *const Vx = R.v(CV_X), *const Vr = R.v(CV_R), *const Vw = R.v(CV_W), *const Vt = R.v(CV_T);
    double *const Vp = R.v(CV_P), *const Vs = R.v(CV_S), *const Vz = R.v(CV_Z), *const Vv = R.v(CV_V);
    double *const Vq = R.v(CV_Q), *const Vy = R.v(CV_Y), *const Vr0 = R.v(CV_R0);
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
                const bool act = R.row0 + r < A.n;
                double q = 0.0, y = 0.0, r0i = 0.0, si = 0.0, zi = 0.0;
                if (act) {
                    const double ri = Vr[r], wi = Vw[r];
                    r0i = Vr0[r];
                    double ti, pold = 0.0, sold = 0.0, zold = 0.0, vold = 0.0;
                    if (first) {
                        ti = Vt[r];
                    } else {
                        ti = spmv_cluster(R.mva, R.mcode, R.soff(ls), R.width(ls), R.mlen[r], lane, G.gv[CV_W]);
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
            if (me == 0) {
                if (threadIdx.x == 0)
                    pipe_x_tail(&hub.ctl, sx.dv);
                push_scal(hub, G);
            }
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
                const bool act = R.row0 + r < A.n;
                double rn = 0.0, wn = 0.0, r0i = 0.0;
                if (act) {
                    const double vi = spmv_cluster(R.mva, R.mcode, R.soff(ls), R.width(ls), R.mlen[r], lane, G.gv[CV_Z]);
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
            if (me == 0) {
                if (threadIdx.x == 0)
                    pipe_y_tail(&hub.ctl, sy.dv);
                push_scal(hub, G);
            }
            cl.sync();
        }
    }
    cluster_store(A, V, c, R, hub, cl);
}

// Iterations of Algorithm 1 (BiCGStab) in the same form: the passes P, A, B
// and C of the launch graph become phases separated by cluster barriers
// (after P) and cluster merges (after A, B and C).
template <int MODE>
__global__ void __launch_bounds__(THREADS, 1)
    k_bicg_cluster(Mat A, Vecs V, Ctl *c, int rpt, int lg, int emax)
{
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ __align__(128) uint8_t dsm[];
    __shared__ Shm<1> sa;
    __shared__ Shm<2> sb;
    __shared__ ClusterHub hub;
    __shared__ ClusterGather G;
    const ClusterRows R = cluster_load(A, V, c, rpt, lg, emax, dsm, hub, G, cl);
    ClusterHub *const hub0 = cl.map_shared_rank(&hub, 0);
    const volatile ClusterScal *const c0 = &G.sc;  // pushed by CTA 0 before each cluster barrier
    const int me = (int)blockIdx.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double *const Vx = R.v(CV_X), *const Vr = R.v(CV_R), *const Vp = R.v(CV_P), *const Vs = R.v(CV_S);
    double *const Vy = R.v(CV_Y), *const Vr0 = R.v(CV_R0);
    for (;;) {
        if (c0->status != ST_RUNNING)
            break;
        if (c0->it > 0) {
            // P: p = fma(beta, fma(-omega, s, p), r)
            const double beta = c0->beta, nomega = -c0->omega;
            for (int k = 0; k < rpt; k++) {
                const int r = k * THREADS + (int)threadIdx.x;
                if (R.row0 + r < A.n)
                    Vp[r] = __fma_rn(beta, __fma_rn(nomega, Vs[r], Vp[r]), Vr[r]);
            }
            cl.sync();
        }
        {
            // A: s = A p; dot (r0, s); alpha
            shm_init<1, MODE>(sa);
            __syncthreads();
            DotSet<1, MODE> D;
            D.init();
            for (int k = 0; k < rpt; k++) {
                const int r = k * THREADS + (int)threadIdx.x, ls = k * WARPS + warp;
                const bool act = R.row0 + r < A.n;
                double si = 0.0, r0i = 0.0;
                if (act) {
                    si = spmv_cluster(R.mva, R.mcode, R.soff(ls), R.width(ls), R.mlen[r], lane, G.gv[CV_P]);
                    Vs[r] = si;
                    r0i = Vr0[r];
                }
                const Dec dr = decode(r0i), ds = decode(si);
                D.template add2<false>(sa, 0, r0i, si, dr, ds, act);
            }
            cluster_merge<1, MODE>(D, sa, hub, hub0, cl);
            if (me == 0) {
                if (threadIdx.x == 0)
                    bicg_a_scalar(&hub.ctl, sa.dv[0]);
                push_scal(hub, G);
            }
            cl.sync();
        }
        if (c0->status != ST_RUNNING)
            break;
        {
            // B: y = A q with q_j = fma(-alpha, s_j, r_j); dots (q,y), (y,y); omega
            const double nalpha = -c0->alpha;
            shm_init<2, MODE>(sb);
            __syncthreads();
            DotSet<2, MODE> D;
            D.init();
            for (int k = 0; k < rpt; k++) {
                const int r = k * THREADS + (int)threadIdx.x, ls = k * WARPS + warp;
                const bool act = R.row0 + r < A.n;
                double qi = 0.0, yi = 0.0;
                if (act) {
                    yi = spmv_cluster_axpy(R.mva, R.mcode, R.soff(ls), R.width(ls), R.mlen[r], lane, nalpha,
                                           G.gv[CV_S], G.gv[CV_R]);
                    qi = __fma_rn(nalpha, Vs[r], Vr[r]);
                    Vy[r] = yi;
                }
                const Dec dq = decode(qi), dy = decode(yi);
                D.template add_row<2, false, true>(sb, act, qi, yi, dq, dy, yi, yi, dy, dy);
            }
            cluster_merge<2, MODE>(D, sb, hub, hub0, cl);
            if (me == 0) {
                if (threadIdx.x == 0)
                    bicg_b_scalar(&hub.ctl, sb.dv[0], sb.dv[1]);
                push_scal(hub, G);
            }
            cl.sync();
        }
        if (c0->status != ST_RUNNING)
            break;
        {
            // C: x, r updates; dots (r0,r), (r,r); beta, stop test
            const double alpha = c0->alpha, omega = c0->omega;
            const double nalpha = -alpha, nomega = -omega;
            shm_init<2, MODE>(sb);
            __syncthreads();
            DotSet<2, MODE> D;
            D.init();
            for (int k = 0; k < rpt; k++) {
                const int r = k * THREADS + (int)threadIdx.x;
                const bool act = R.row0 + r < A.n;
                double rn = 0.0, r0i = 0.0;
                if (act) {
                    const double q = __fma_rn(nalpha, Vs[r], Vr[r]);
                    Vx[r] = __fma_rn(omega, q, __fma_rn(alpha, Vp[r], Vx[r]));
                    rn = __fma_rn(nomega, Vy[r], q);
                    Vr[r] = rn;
                    r0i = Vr0[r];
                }
                const Dec dr0 = decode(r0i), dr = decode(rn);
                D.template add_row<2, false, true>(sb, act, r0i, rn, dr0, dr, rn, rn, dr, dr);
            }
            cluster_merge<2, MODE>(D, sb, hub, hub0, cl);
            if (me == 0) {
                if (threadIdx.x == 0)
                    bicg_c_scalar(&hub.ctl, sb.dv[0], sb.dv[1]);
                push_scal(hub, G);
            }
            cl.sync();
        }
    }
    cluster_store(A, V, c, R, hub, cl);
}

}  // namespace pbcg
