// batched.cuh -- many independent systems in one sweep per pass.
//
// The systems of a block-diagonal matrix are laid out one after another, each
// padded to whole 256-row tiles, so every tile belongs to exactly one system.
// A batched pass walks its CTA's tiles (tile blockIdx.x, + gridDim.x, ...),
// skips tiles of systems that are not in the state the pass serves, and
// computes the same row formulas as the single-system passes.  Dot terms are
// accumulated while consecutive tiles of the CTA belong to the same system and
// are flushed into that system's accumulators when the system changes.  The
// CTA whose flush completes a system's tile count (an atomic counter per
// system) rounds that system's dots and runs its scalar step, so every system
// advances with its own alpha, beta, omega, residual, history, tolerance and
// status -- bit for bit the arithmetic of a single solve of its block in
// exact mode.
#pragma once
#include "kernels.cuh"

namespace pbcg {

struct Batch {
    int nsys, ntiles;
    const int *__restrict__ tile_sys;    // [ntiles] system of each tile
    const int *__restrict__ sys_t0;      // [nsys] first tile of each system
    const int *__restrict__ sys_t1;      // [nsys] end tile of each system
    Ctl *ctl;                            // [nsys]
    GAcc *acc;                           // [nsys * MAXD]
    double *part;                        // [ntiles * MAXD] plain partial of the flush group starting at a tile
    unsigned *done;                      // [nsys] tiles merged in the current pass
    int *flag;                           // [1] loop condition scratch
    // pools only (NULL otherwise): the tiles of the live systems, listed system by
    // system: lv_n = {live systems, live tiles}; live system j owns list entries
    // [lv_pre[j], lv_pre[j+1]), which are tiles lv_t0[j], lv_t0[j] + 1, ...
    const int *lv_n, *lv_pre, *lv_t0;
};

// ---------------------------------------------------------------------------
// generic batched pass
// ---------------------------------------------------------------------------
template <int ND, int MODE, class Step>
__device__ __forceinline__ void b_flush(DotSet<ND, MODE> &D, Shm<ND> &sh, const Batch &B, int sys, int t_first,
                                        int cnt, const Vecs &V)
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
        cta_to_global<ND>(sh.acc, B.acc + (size_t)sys * MAXD);
    } else if (threadIdx.x < ND) {
        double v = sh.wpart[threadIdx.x][0];
        for (int w = 1; w < WARPS; w++)
            v = __dadd_rn(v, sh.wpart[threadIdx.x][w]);
        B.part[(size_t)t_first * MAXD + threadIdx.x] = v;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned need = (unsigned)(B.sys_t1[sys] - B.sys_t0[sys]);
        const unsigned old = atomicAdd(&B.done[sys], (unsigned)cnt);
        sh.last = (old + (unsigned)cnt == need);
    }
    __syncthreads();
    if (sh.last) {
        __threadfence();
        GAcc *g = B.acc + (size_t)sys * MAXD;
        if (MODE == 1) {
            gacc_round_reset_cta<ND>(g, sh.acc, sh.scratch, sh.dv);
        } else if (warp < ND) {
            // partials of the system's flush groups, in tile order (non-first tiles hold +0)
            const int t0 = B.sys_t0[sys], t1 = B.sys_t1[sys];
            double v = 0.0;
            for (int ta = t0 + lane; ta < t1; ta += 32 * 8) {     // eight loads per round trip, same order
                double u[8];
#pragma unroll
                for (int j = 0; j < 8; j++)
                    u[j] = ta + 32 * j < t1 ? __ldcg(B.part + (size_t)(ta + 32 * j) * MAXD + warp) : 0.0;
#pragma unroll
                for (int j = 0; j < 8; j++)
                    if (ta + 32 * j < t1)
                        v = __dadd_rn(v, u[j]);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
                v = __dadd_rn(v, __shfl_xor_sync(0xffffffffu, v, o));
            if (lane == 0)
                sh.dv[warp] = v;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            B.done[sys] = 0u;
            Step::fin(B.ctl + sys, sh.dv, V);
        }
    }
    __syncthreads();
    // fresh CTA accumulator for the next group
    if (MODE == 1)
        cta_acc_init<ND>(sh.acc);
    if (threadIdx.x == 0)
        sh.last = 0;
    __syncthreads();
}

template <int MODE, class Step>
__global__ void __launch_bounds__(THREADS) k_batched(Mat A, Vecs V, Batch B)
{
    constexpr int ND = Step::ND;
    __shared__ Shm<ND> sh;
    shm_init<ND, MODE>(sh);
    __syncthreads();
    DotSet<ND, MODE> D;
    D.init();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int cur = -1, t_first = -1, cnt = 0;
    bool run = false;
    typename Step::Scal S;
    // each CTA serves one contiguous chunk of the tile list (the live list of a
    // pool, else all tiles), so a system's tiles form few flush groups
    const bool listed = B.lv_n != nullptr;
    const int nq = listed ? B.lv_n[1] : B.ntiles;
    const int q0 = (int)(((long long)nq * blockIdx.x) / gridDim.x);
    const int q1 = (int)(((long long)nq * (blockIdx.x + 1)) / gridDim.x);
    int j = 0;
    if (listed && q0 < q1) {
        int lo = 0, hi = B.lv_n[0] - 1;           // last live system with lv_pre[j] <= q0
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (B.lv_pre[mid] <= q0)
                lo = mid;
            else
                hi = mid - 1;
        }
        j = lo;
    }
    for (int q = q0; q < q1;) {
        int t = q;
        if (listed) {
            while (B.lv_pre[j + 1] <= q)
                j++;
            t = B.lv_t0[j] + (q - B.lv_pre[j]);
        }
        const int sys = PBCG_IN(t, B.ntiles, CHK_TILE) ? B.tile_sys[t] : -1;
        if (sys < 0 || !PBCG_IN(sys, B.nsys, CHK_SYS)) {
            q++;
            continue;                    // unallocated tile of a pool
        }
        if (sys != cur) {
            if (cur >= 0 && cnt > 0) {
                b_flush<ND, MODE, Step>(D, sh, B, cur, t_first, cnt, V);
                D.init();
            }
            cur = sys;
            t_first = t;
            cnt = 0;
            const Ctl *c = B.ctl + sys;
            run = Step::wants(c);
            if (run)
                S = Step::load(c);
        }
        if (!run) {                      // skip the rest of this system
            const int qend = listed ? B.lv_pre[j + 1] : B.sys_t1[sys];
            q = max(q + 1, min(q1, qend));
            continue;
        }
        q++;
        if (MODE == 0 && threadIdx.x < ND)
            B.part[(size_t)t * MAXD + threadIdx.x] = 0.0;
        const int sl = t * TILE_SLICES + warp;
        const int i = sl * 32 + lane;
        const bool act = sl < A.nslices && i < A.n;
        double a[ND], b[ND];
        Step::row(A, V, S, sl, lane, i, act, a, b);
#pragma unroll
        for (int d = 0; d < ND; d++)
            D.add(sh, d, a[d], b[d], act);
        cnt++;
    }
    if (cur >= 0 && cnt > 0)
        b_flush<ND, MODE, Step>(D, sh, B, cur, t_first, cnt, V);
}

// ---------------------------------------------------------------------------
// steps.  Row formulas are those of the single-system passes.
// ---------------------------------------------------------------------------
struct NoScal {
};

// S1: r0 = b - A x0, r = r0 (p = r0 for BiCGStab); dots (b,b), (r0,r0)
struct StepSetup1 {
    static constexpr int ND = 2;
    struct Scal {
        bool bicg;
    };
    static __device__ bool wants(const Ctl *c) { const int st = c->status; return st == ST_RUNNING; }
    static __device__ Scal load(const Ctl *c) { return Scal{c->alg == ALG_BICGSTAB}; }
    static __device__ void row(const Mat &A, const Vecs &V, const Scal &S, int sl, int lane, int i, bool act,
                               double (&a)[ND], double (&b)[ND])
    {
        double bi = 0.0, r0i = 0.0;
        if (sl < A.nslices) {
            RowRef R = row_ref(A, sl, lane);
            double ax = spmv_row(A, R, V.x);
            if (act) {
                bi = V.b[i];
                r0i = __dsub_rn(bi, ax);
                V.r0[i] = r0i;
                V.r[i] = r0i;
                if (S.bicg)
                    V.p[i] = r0i;
            }
        }
        a[0] = bi, b[0] = bi, a[1] = r0i, b[1] = r0i;
    }
    static __device__ void fin(Ctl *c, const double *dv, const Vecs &)
    {
        c->bb = dv[0];
        c->rho = dv[1];
        if (c->alg == ALG_BICGSTAB)
            setup_scalar(c, dv[0], dv[1], 0.0);
    }
};

// S2 (p-BiCGStab): w0 = A r0; dot (r0, w0); setup scalars
struct StepSetup2 {
    static constexpr int ND = 1;
    using Scal = NoScal;
    static __device__ bool wants(const Ctl *c) { const int st = c->status; return st == ST_RUNNING; }
    static __device__ Scal load(const Ctl *) { return Scal{}; }
    static __device__ void row(const Mat &A, const Vecs &V, const Scal &, int sl, int lane, int i, bool act,
                               double (&a)[ND], double (&b)[ND])
    {
        double r0i = 0.0, wi = 0.0;
        if (sl < A.nslices) {
            RowRef R = row_ref(A, sl, lane);
            wi = spmv_row(A, R, V.r0);
            if (act) {
                r0i = V.r0[i];
                V.w[i] = wi;
            } else {
                wi = 0.0;
            }
        }
        a[0] = r0i, b[0] = wi;
    }
    static __device__ void fin(Ctl *c, const double *dv, const Vecs &) { setup_scalar(c, c->bb, c->rho, dv[0]); }
};

// S3 (p-BiCGStab): t0 = A w0 (no dots)
struct StepSetup3 {
    static constexpr int ND = 1;
    using Scal = NoScal;
    static __device__ bool wants(const Ctl *c) { const int st = c->status; return st == ST_RUNNING || st == ST_CANDIDATE; }
    static __device__ Scal load(const Ctl *) { return Scal{}; }
    static __device__ void row(const Mat &A, const Vecs &V, const Scal &, int sl, int lane, int i, bool act,
                               double (&a)[ND], double (&b)[ND])
    {
        if (sl < A.nslices) {
            RowRef R = row_ref(A, sl, lane);
            double ti = spmv_row(A, R, V.w);
            if (act)
                V.t[i] = ti;
        }
        a[0] = 0.0, b[0] = 0.0;
    }
    static __device__ void fin(Ctl *, const double *, const Vecs &) {}
};

// X(i) (p-BiCGStab)
struct StepPipeX {
    static constexpr int ND = 4;
    struct Scal {
        double alpha, beta, omega;
        bool first, rr;
    };
    static __device__ bool wants(const Ctl *c) { const int st = c->status; return st == ST_RUNNING; }
    static __device__ Scal load(const Ctl *c) { return Scal{c->alpha, c->beta, c->omega, c->it == 0, rr_now(c)}; }
    static __device__ void fin(Ctl *c, const double *dv, const Vecs &)
    {
        double qy = dv[0], yy = dv[1];
        c->qy = qy;
        c->yy = yy;
        c->rs = dv[2];
        c->rz = dv[3];
        if (!pbcg::fin(qy) || !pbcg::fin(yy))
            c->status = 3;
        else
            c->omega = (yy == 0.0) ? 0.0 : __ddiv_rn(qy, yy);
    }
};

// Y(i) (p-BiCGStab)
struct StepPipeY {
    static constexpr int ND = 3;
    struct Scal {
        double alpha, omega;
    };
    static __device__ bool wants(const Ctl *c) { const int st = c->status; return st == ST_RUNNING; }
    static __device__ Scal load(const Ctl *c) { return Scal{c->alpha, c->omega}; }
    static __device__ void fin(Ctl *c, const double *dv, const Vecs &)
    {
        double rho_new = dv[0], rw = dv[1], rr = dv[2];
        c->rho_new = rho_new;
        c->rw = rw;
        c->rr = rr;
        c->phase = PH_ITER;
        if (!pbcg::fin(rho_new) || !pbcg::fin(rw) || !pbcg::fin(c->rs) || !pbcg::fin(c->rz) || !pbcg::fin(rr)) {
            c->status = 3;
        } else {
            c->it += 1;
            residual_step(c, rr);
        }
    }
};

// ---------------------------------------------------------------------------
// staged batched passes (p-BiCGStab X and Y)
//
// The tiles a CTA serves travel through two shared-memory stages by bulk
// copies, as in the single-system passes.  Thread 0 walks the CTA's tile
// positions ahead of the warps, skips whole systems the pass does not serve,
// and records each staged tile's system; the loop stays CTA-synchronous so a
// flush group can close at any tile.  Row arithmetic and dots are those of
// the generic steps (pipe_x_row / pipe_y_row), so results are bit-identical.
// ---------------------------------------------------------------------------
constexpr int BLIST = 512;     // tile positions of a CTA's chunk scheduled per round

// one scheduled tile of a staged batched pass
struct BEntry {
    int tile, sys, first;        // first: pass X at the system's first iteration
    int e0, e1;                  // the tile's SELL entry range
};

struct BPipeX : StepPipeX {
    static constexpr int NV = 7;     // r, w, r0, p (t when first), s, z, v
    static __device__ int flags(const Ctl *c) { return c->it == 0; }
    static __device__ void srcs(const Vecs &V, int first, const double *(&src)[NV], const double *&gx)
    {
        src[0] = V.r;
        src[1] = V.w;
        src[2] = V.r0;
        src[3] = first ? V.t : V.p;
        src[4] = V.s;
        src[5] = V.z;
        src[6] = V.v;
        gx = first ? nullptr : V.w;
    }
    template <int MODE>
    static __device__ __forceinline__ void row(const TilePipe<NV, true, false> &P, int k, const Mat &A, const Vecs &V,
                                               const Scal &S, int tile, int warp, int lane, DotSet<ND, MODE> &D,
                                               Shm<ND> &sh)
    {
        const int sl = tile * TILE_SLICES + warp;
        const int i = sl * 32 + lane;
        const bool act = sl < A.nslices && i < A.n;
        const int o = warp * 32 + lane;
        const double ri = P.vec(k, 0)[o], wi = P.vec(k, 1)[o], r0i = P.vec(k, 2)[o];
        const double ti = S.first ? P.vec(k, 3)[o] : P.spmv(k, A, warp, lane, V.w);
        const XRow X = S.first ? pipe_x_row(true, false, -S.alpha, S.beta, -S.omega, ri, wi, ti, 0.0, 0.0, 0.0, 0.0)
                               : pipe_x_row(false, S.rr, -S.alpha, S.beta, -S.omega, ri, wi, ti, P.vec(k, 3)[o],
                                            P.vec(k, 4)[o], P.vec(k, 5)[o], P.vec(k, 6)[o]);
        if (act) {
            if (!S.first)
                V.t[i] = ti;
            V.p[i] = X.p;
            V.s[i] = X.s;
            V.z[i] = X.z;
            V.q[i] = X.q;
            V.y[i] = X.y;
        }
        const double q = act ? X.q : 0.0, y = act ? X.y : 0.0, r0 = act ? r0i : 0.0;
        const double s = act ? X.s : 0.0, z = act ? X.z : 0.0;
        const Dec dq = decode(q), dy = decode(y), dr = decode(r0), ds = decode(s), dz = decode(z);
        D.template add2<false>(sh, 0, q, y, dq, dy, act);
        D.template add2<true>(sh, 1, y, y, dy, dy, act);
        D.template add2<false>(sh, 2, r0, s, dr, ds, act);
        D.template add2<false>(sh, 3, r0, z, dr, dz, act);
    }
};

struct BPipeY : StepPipeY {
    static constexpr int NV = 6;     // q, y, p, x, t, r0
    static __device__ int flags(const Ctl *) { return 0; }
    static __device__ void srcs(const Vecs &V, int, const double *(&src)[NV], const double *&gx)
    {
        src[0] = V.q;
        src[1] = V.y;
        src[2] = V.p;
        src[3] = V.x;
        src[4] = V.t;
        src[5] = V.r0;
        gx = V.z;
    }
    template <int MODE>
    static __device__ __forceinline__ void row(const TilePipe<NV, true, false> &P, int k, const Mat &A, const Vecs &V,
                                               const Scal &S, int tile, int warp, int lane, DotSet<ND, MODE> &D,
                                               Shm<ND> &sh)
    {
        const int sl = tile * TILE_SLICES + warp;
        const int i = sl * 32 + lane;
        const bool act = sl < A.nslices && i < A.n;
        const int o = warp * 32 + lane;
        const double vi = P.spmv(k, A, warp, lane, V.z);
        const YRow Yr = pipe_y_row(S.alpha, S.omega, -S.alpha, -S.omega, P.vec(k, 0)[o], P.vec(k, 1)[o],
                                   P.vec(k, 2)[o], P.vec(k, 3)[o], P.vec(k, 4)[o], vi);
        if (act) {
            V.x[i] = Yr.x;
            V.v[i] = vi;
            V.r[i] = Yr.r;
            V.w[i] = Yr.w;
        }
        const double r0 = act ? P.vec(k, 5)[o] : 0.0, rn = act ? Yr.r : 0.0, wn = act ? Yr.w : 0.0;
        const Dec dr0 = decode(r0), dr = decode(rn), dw = decode(wn);
        D.template add_row<3, false, false, true>(sh, act, r0, rn, dr0, dr, r0, wn, dr0, dw, rn, rn, &dr, &dr);
    }
};

// ---------------------------------------------------------------------------
// Staged batched passes (p-BiCGStab X and Y).
//
// Each CTA serves one contiguous chunk of the tile list.  A round first
// schedules up to BLIST positions of the chunk in parallel: the tiles of the
// systems this pass serves, in order, with their entry ranges, into a list
// in shared memory.  The list is then run like the single-system tile loop:
// bulk copies into two stages, each warp waiting on the stage's mbarrier for
// its own data, the last warp out of a stage refilling it from the list.
// Warps only meet at system boundaries, where the CTA closes the system's
// flush group.  Row arithmetic and dots are those of the generic steps.
// ---------------------------------------------------------------------------
template <int MODE, class Step>
__global__ void __launch_bounds__(THREADS, 2) k_bstaged(Mat A, Vecs V, Batch B)
{
    constexpr int ND = Step::ND, NV = Step::NV;
    extern __shared__ __align__(128) uint8_t dsm[];
    __shared__ Shm<ND> sh;
    __shared__ uint64_t bar[NSTAGE];
    __shared__ StageInfo info[NSTAGE];
    __shared__ BEntry list[BLIST];
    __shared__ int cnts[THREADS];
    __shared__ int done_cnt[NSTAGE], uses[NSTAGE], nlist, tmo;
    shm_init<ND, MODE>(sh);
    TilePipe<NV, true, false> P{dsm, bar, info};
    DotSet<ND, MODE> D;
    D.init();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, tid = threadIdx.x;
    const bool listed = B.lv_n != nullptr;
    const int nq = listed ? B.lv_n[1] : B.ntiles;
    const int q0 = (int)(((long long)nq * blockIdx.x) / gridDim.x);
    const int q1 = (int)(((long long)nq * (blockIdx.x + 1)) / gridDim.x);
    auto issue = [&](int k, const BEntry &e) {        // one lane
        const double *src[NV];
        const double *gx;
        Step::srcs(V, e.first, src, gx);
        int rec[TMETA];
        rec[0] = e.e0;
        rec[1] = e.e1;
#pragma unroll
        for (int g = 2; g < TMETA; g++)
            rec[g] = -1;
        uses[k] += 1;
        P.issue(k, e.tile, rec, A, src, NV, gx, -1);
    };
    if (tid == 0) {
        for (int k = 0; k < NSTAGE; k++) {
            mbar_init(&bar[k], 1);
            uses[k] = 0;
        }
        tmo = 0;
        fence_mbar_init();
        fence_async_shared();
    }
    __syncthreads();
    int cur = -1, t_first = -1, cnt = 0;
    typename Step::Scal S;
    for (int qa = q0; qa < q1 && !*(volatile int *)&tmo; qa += BLIST) {
        const int qb = min(q1, qa + BLIST);
        // schedule positions [qa, qb): thread tid takes a contiguous piece, then an ordered compaction
        const int per = (qb - qa + THREADS - 1) / THREADS;
        const int pa = min(qb, qa + tid * per), pb = min(qb, pa + per);
        BEntry mine[2];
        int nm = 0;
        for (int q = pa; q < pb; q++) {
            int t = q;
            if (listed) {
                int lo = 0, hi = B.lv_n[0] - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (B.lv_pre[mid] <= q)
                        lo = mid;
                    else
                        hi = mid - 1;
                }
                t = B.lv_t0[lo] + (q - B.lv_pre[lo]);
            }
            const int sys = PBCG_IN(t, B.ntiles, CHK_TILE) ? B.tile_sys[t] : -1;
            if (sys < 0 || !PBCG_IN(sys, B.nsys, CHK_SYS) || !Step::wants(B.ctl + sys))
                continue;
            BEntry &e = mine[nm++];
            e.tile = t;
            e.sys = sys;
            e.first = Step::flags(B.ctl + sys);
            const int s0 = t * TILE_SLICES;
            e.e0 = A.sl_off[s0];
            e.e1 = A.sl_w ? A.sl_off[s0 + TILE_SLICES - 1] + 32 * A.sl_w[s0 + TILE_SLICES - 1]
                          : A.sl_off[s0 + TILE_SLICES];
        }
        cnts[tid] = nm;
        __syncthreads();
        if (tid == 0) {
            int run = 0;
            for (int u = 0; u < THREADS; u++) {
                const int cu = cnts[u];
                cnts[u] = run;
                run += cu;
            }
            nlist = run;
            for (int k = 0; k < NSTAGE; k++)
                done_cnt[k] = 0;
        }
        __syncthreads();
        for (int m = 0; m < nm; m++)
            list[cnts[tid] + m] = mine[m];
        __syncthreads();
        const int n = nlist;
        int base[NSTAGE];
#pragma unroll
        for (int k = 0; k < NSTAGE; k++)
            base[k] = uses[k];                             // stage uses before this round
        __syncthreads();
        if (tid == 0)
            for (int k = 0; k < NSTAGE && k < n; k++)
                issue(k, list[k]);
        __syncthreads();
        for (int j = 0; j < n; j++) {
            const int k = j % NSTAGE;
            const BEntry e = list[j];
            if (e.sys != cur) {                            // every warp reaches this entry: CTA-uniform
                if (cur >= 0 && cnt > 0) {
                    b_flush<ND, MODE, Step>(D, sh, B, cur, t_first, cnt, V);
                    D.init();
                }
                cur = e.sys;
                t_first = e.tile;
                cnt = 0;
                S = Step::load(B.ctl + cur);
            }
            // after an expired wait every warp keeps walking the list (so the
            // CTA-wide flush points stay matched) but skips waits, rows and refills
            if (!*(volatile int *)&tmo) {
                const bool ok = __all_sync(0xffffffffu,
                                           mbar_wait_bounded(&bar[k], (uint32_t)(base[k] + j / NSTAGE) & 1u));
                if (!ok && lane == 0)
                    tmo = 1;
            }
            if (__any_sync(0xffffffffu, *(volatile int *)&tmo))
                continue;
            if (MODE == 0 && warp == 0 && lane < ND)
                B.part[(size_t)e.tile * MAXD + lane] = 0.0;
            Step::template row<MODE>(P, k, A, V, S, e.tile, warp, lane, D, sh);
            cnt++;
            __syncwarp();
            if (lane == 0) {
                __threadfence_block();
                if (atomicAdd(&done_cnt[k], 1) == WARPS - 1) {   // last warp out refills the stage
                    __threadfence_block();
                    done_cnt[k] = 0;
                    if (j + NSTAGE < n)
                        issue(k, list[j + NSTAGE]);
                }
            }
        }
        __syncthreads();
    }
    if (tmo) {
        // give up: wait (bounded) for copies still in flight, flag the systems
        if (tid == 0) {
            for (int k = 0; k < NSTAGE; k++)
                if (uses[k] > 0)
                    mbar_wait_bounded(&bar[k], (uint32_t)(uses[k] - 1) & 1u);
            if (cur >= 0)
                atomicOr(&B.ctl[cur].err, 1);
        }
        __syncthreads();
        return;
    }
    if (cur >= 0 && cnt > 0)
        b_flush<ND, MODE, Step>(D, sh, B, cur, t_first, cnt, V);
}

// P(i), i >= 1 (BiCGStab): p = fma(beta, fma(-omega, s, p), r)
struct StepBicgP {
    static constexpr int ND = 1;
    struct Scal {
        double beta, omega;
        bool first;
    };
    static __device__ bool wants(const Ctl *c) { const int st = c->status; return st == ST_RUNNING; }
    static __device__ Scal load(const Ctl *c) { return Scal{c->beta, c->omega, c->it == 0}; }
    static __device__ void row(const Mat &, const Vecs &V, const Scal &S, int, int, int i, bool act,
                               double (&a)[ND], double (&b)[ND])
    {
        if (act && !S.first)
            V.p[i] = __fma_rn(S.beta, __fma_rn(-S.omega, V.s[i], V.p[i]), V.r[i]);
        a[0] = 0.0, b[0] = 0.0;
    }
    static __device__ void fin(Ctl *, const double *, const Vecs &) {}
};

// A(i) (BiCGStab): s = A p; (r0, s); alpha
struct StepBicgA {
    static constexpr int ND = 1;
    using Scal = NoScal;
    static __device__ bool wants(const Ctl *c) { const int st = c->status; return st == ST_RUNNING; }
    static __device__ Scal load(const Ctl *) { return Scal{}; }
    static __device__ void row(const Mat &A, const Vecs &V, const Scal &, int sl, int lane, int i, bool act,
                               double (&a)[ND], double (&b)[ND])
    {
        double si = 0.0, r0i = 0.0;
        if (sl < A.nslices) {
            RowRef R = row_ref(A, sl, lane);
            si = spmv_row(A, R, V.p);
            if (act) {
                V.s[i] = si;
                r0i = V.r0[i];
            } else {
                si = 0.0;
            }
        }
        a[0] = r0i, b[0] = si;
    }
    static __device__ void fin(Ctl *c, const double *dv, const Vecs &)
    {
        double rs = dv[0];
        c->rs = rs;
        if (!pbcg::fin(rs)) {
            c->status = 3;
        } else {
            double al = __ddiv_rn(c->rho, rs);
            if (!pbcg::fin(al))
                c->status = 2;
            else
                c->alpha = al;
        }
    }
};

// B(i) (BiCGStab): y = A q, q_j = fma(-alpha, s_j, r_j) in the gather; (q,y), (y,y); omega
struct StepBicgB {
    static constexpr int ND = 2;
    struct Scal {
        double alpha;
    };
    static __device__ bool wants(const Ctl *c) { const int st = c->status; return st == ST_RUNNING; }
    static __device__ Scal load(const Ctl *c) { return Scal{c->alpha}; }
    static __device__ void row(const Mat &A, const Vecs &V, const Scal &S, int sl, int lane, int i, bool act,
                               double (&a)[ND], double (&b)[ND])
    {
        double qi = 0.0, yi = 0.0;
        if (sl < A.nslices) {
            RowRef R = row_ref(A, sl, lane);
            yi = spmv_row_axpy(A, R, -S.alpha, V.s, V.r);
            if (act) {
                qi = __fma_rn(-S.alpha, V.s[i], V.r[i]);
                V.y[i] = yi;
            } else {
                yi = 0.0;
            }
        }
        a[0] = qi, b[0] = yi, a[1] = yi, b[1] = yi;
    }
    static __device__ void fin(Ctl *c, const double *dv, const Vecs &)
    {
        double qy = dv[0], yy = dv[1];
        c->qy = qy;
        c->yy = yy;
        if (!pbcg::fin(qy) || !pbcg::fin(yy))
            c->status = 3;
        else
            c->omega = (yy == 0.0) ? 0.0 : __ddiv_rn(qy, yy);
    }
};

// C(i) (BiCGStab): x, r; (r0,r), (r,r); beta, stop test
struct StepBicgC {
    static constexpr int ND = 2;
    struct Scal {
        double alpha, omega;
    };
    static __device__ bool wants(const Ctl *c) { const int st = c->status; return st == ST_RUNNING; }
    static __device__ Scal load(const Ctl *c) { return Scal{c->alpha, c->omega}; }
    static __device__ void row(const Mat &, const Vecs &V, const Scal &S, int, int, int i, bool act,
                               double (&a)[ND], double (&b)[ND])
    {
        double rn = 0.0, r0i = 0.0;
        if (act) {
            const double q = __fma_rn(-S.alpha, V.s[i], V.r[i]);
            V.x[i] = __fma_rn(S.omega, q, __fma_rn(S.alpha, V.p[i], V.x[i]));
            rn = __fma_rn(-S.omega, V.y[i], q);
            V.r[i] = rn;
            r0i = V.r0[i];
        }
        a[0] = r0i, b[0] = rn, a[1] = rn, b[1] = rn;
    }
    static __device__ void fin(Ctl *c, const double *dv, const Vecs &)
    {
        double rho_new = dv[0], rr = dv[1];
        c->rho_new = rho_new;
        c->rr = rr;
        c->phase = PH_ITER;
        if (!pbcg::fin(rho_new) || !pbcg::fin(rr)) {
            c->status = 3;
        } else {
            c->it += 1;
            residual_step(c, rr);
        }
    }
};

// residual replacement steps (p-BiCGStabRR), on systems replacing at this iteration
template <int WHICH>
struct StepRR {
    static constexpr int ND = 1;
    struct Scal {
        double beta, omega;
    };
    static __device__ bool wants(const Ctl *c) { return c->status == ST_RUNNING && rr_now(c); }
    static __device__ Scal load(const Ctl *c) { return Scal{c->beta, c->omega}; }
    static __device__ void row(const Mat &A, const Vecs &V, const Scal &S, int sl, int lane, int i, bool act,
                               double (&a)[ND], double (&b)[ND])
    {
        if (sl < A.nslices) {
            RowRef R = row_ref(A, sl, lane);
            const double *src = WHICH == 1 ? V.x : WHICH == 2 ? V.r : WHICH == 3 ? V.p : V.s;
            double y = spmv_row(A, R, src);
            if (act) {
                if (WHICH == 1) {
                    V.r[i] = __dsub_rn(V.b[i], y);
                } else if (WHICH == 2) {
                    V.w[i] = y;
                    V.p[i] = __fma_rn(S.beta, __fma_rn(-S.omega, V.s[i], V.p[i]), V.r[i]);
                } else if (WHICH == 3) {
                    V.s[i] = y;
                } else {
                    V.z[i] = y;
                }
            }
        }
        a[0] = 0.0, b[0] = 0.0;
    }
    static __device__ void fin(Ctl *, const double *, const Vecs &) {}
};

// true residual of candidate systems (resolve) or of every system (report)
template <bool REPORT>
struct StepTrueRes {
    static constexpr int ND = 2;
    using Scal = NoScal;
    static __device__ bool wants(const Ctl *c) { const int st = c->status; return REPORT || st == ST_CANDIDATE; }
    static __device__ Scal load(const Ctl *) { return Scal{}; }
    static __device__ void row(const Mat &A, const Vecs &V, const Scal &, int sl, int lane, int i, bool act,
                               double (&a)[ND], double (&b)[ND])
    {
        double ri = 0.0, bi = 0.0;
        if (sl < A.nslices) {
            RowRef R = row_ref(A, sl, lane);
            double ax = spmv_row(A, R, V.x);
            if (act) {
                bi = V.b[i];
                ri = __dsub_rn(bi, ax);
            }
        }
        a[0] = ri, b[0] = ri, a[1] = bi, b[1] = bi;
    }
    static __device__ void fin(Ctl *c, const double *dv, const Vecs &)
    {
        double nb = __dsqrt_rn(dv[1]);
        if (nb == 0.0)
            nb = 1.0;
        double tr = __ddiv_rn(__dsqrt_rn(dv[0]), nb);
        c->trueres = tr;
        c->bbx = dv[1];
        if (c->status == ST_CANDIDATE) {
            if (tr <= c->tol) {
                c->status = 0;
            } else {
                c->target = __dmul_rn(c->tol, __ddiv_rn(c->tol, tr));
                c->status = ST_RUNNING;
                post_stop(c);
            }
        }
    }
};

// ---------------------------------------------------------------------------
// pool (continuous batching): slots are admitted in state ST_SETUP1 between
// steps and go through the setup passes inside the step loop
// ---------------------------------------------------------------------------
struct PoolSetup1 : StepSetup1 {
    static __device__ bool wants(const Ctl *c) { return c->status == ST_SETUP1; }
    static __device__ void fin(Ctl *c, const double *dv, const Vecs &)
    {
        c->bb = dv[0];
        c->rho = dv[1];
        if (c->alg == ALG_BICGSTAB)
            setup_scalar(c, dv[0], dv[1], 0.0);
        else
            c->status = ST_SETUP2;
    }
};

struct PoolSetup2 : StepSetup2 {
    static __device__ bool wants(const Ctl *c) { return c->status == ST_SETUP2; }
    static __device__ void fin(Ctl *c, const double *dv, const Vecs &)
    {
        setup_scalar(c, c->bb, c->rho, dv[0]);
        c->need_t = 1;
    }
};

struct PoolSetup3 : StepSetup3 {
    static __device__ bool wants(const Ctl *c) { return c->need_t == 1; }
    static __device__ void fin(Ctl *c, const double *, const Vecs &) { c->need_t = 0; }
};

// step control of a pool (one CTA of 1024 threads): lists the tiles of the
// slots that are still live for the next iteration (in slot order, so that a
// CTA meets each system in one run of consecutive list entries) and, unless
// `first`, counts down `left` and sets the loop condition
__device__ __forceinline__ bool pool_live(const Ctl &c)
{
    const int st = c.status;
    return c.err == 0 && (st == ST_RUNNING || st == ST_CANDIDATE || st == ST_SETUP1 || st == ST_SETUP2 || c.need_t == 1);
}

__global__ void __launch_bounds__(1024) k_pool_ctl(Batch B, int *lv_n, int *lv_pre, int *lv_t0, int *left,
                                                   unsigned long long handle, int first)
{
    __shared__ unsigned long long wsum[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int C = (B.nsys + (int)blockDim.x - 1) / (int)blockDim.x;
    const int s0 = min(tid * C, B.nsys), s1 = min(s0 + C, B.nsys);
    // (systems, tiles) of this thread's slots, packed as systems << 32 | tiles
    unsigned long long v = 0;
    for (int s = s0; s < s1; s++)
        if (pool_live(B.ctl[s]))
            v += (1ull << 32) | (unsigned long long)(B.sys_t1[s] - B.sys_t0[s]);
    unsigned long long inc = v;
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long u = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o)
            inc += u;
    }
    if (lane == 31)
        wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const int nw = (int)blockDim.x >> 5;
        unsigned long long w = lane < nw ? wsum[lane] : 0ull;
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long u = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o)
                w += u;
        }
        if (lane < nw)
            wsum[lane] = w;                       // inclusive over warps
    }
    __syncthreads();
    unsigned long long ex = inc - v + (warp > 0 ? wsum[warp - 1] : 0ull);
    int js = (int)(ex >> 32), ts = (int)(ex & 0xffffffffull);
    for (int s = s0; s < s1; s++) {
        if (pool_live(B.ctl[s])) {
            lv_t0[js] = B.sys_t0[s];
            lv_pre[js] = ts;
            ts += B.sys_t1[s] - B.sys_t0[s];
            js++;
        }
    }
    if (tid == (int)blockDim.x - 1) {
        const unsigned long long tot = wsum[((int)blockDim.x >> 5) - 1];
        const int nl = (int)(tot >> 32), nt = (int)(tot & 0xffffffffull);
        lv_pre[nl] = nt;
        lv_n[0] = nl;
        lv_n[1] = nt;
        if (!first) {
            const int l = *left - 1;
            *left = l;
            cudaGraphSetConditional((cudaGraphConditionalHandle)handle, (nl > 0 && l > 0) ? 1u : 0u);
        }
    }
}

// admission of a request into a pool slot: its CSR rows (staged in device
// memory, rows in caller order) into the slot's SELL-32 entries.  nrows = the
// slot's whole tiles; slices sl_off / sl_w are the slot's own.  A column
// outside [0, n) raises *bad and is stored as column 0 with value 0.
__global__ void k_pool_scatter(int n, int nrows, int row0, const int *__restrict__ rp, const int *__restrict__ ci,
                               const double *__restrict__ va, const int *__restrict__ sl_off,
                               const int *__restrict__ sl_w, int *rlen, int *ci_out, double *va_out, int *bad)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nrows; i += gridDim.x * blockDim.x) {
        const int sl = i >> 5;
        const long long base = (long long)sl_off[sl] + (i & 31);
        const int w = sl_w[sl];
        int k0 = 0, len = 0;
        if (i < n) {
            k0 = rp[i];
            len = rp[i + 1] - k0;
        }
        rlen[row0 + i] = len;
        for (int j = 0; j < w; j++) {
            int c = 0;
            double v = 0.0;
            if (j < len) {
                c = ci[k0 + j];
                v = va[k0 + j];
                if (c < 0 || c >= n) {
                    *bad = 1;
                    c = 0;
                    v = 0.0;
                }
            }
            ci_out[base + 32ll * j] = row0 + c;
            va_out[base + 32ll * j] = v;
        }
    }
}

// Jacobi for a pool request (right preconditioning, M = diag(A)), from the
// request's staged CSR: d_i = the sum, in stored order, of row i's entries
// in column i; an absent, zero or non-finite diagonal marks the request bad.
// Padding rows of the slot get d = 1.
__global__ void k_pool_diag(int n, int nrows, int row0, const int *__restrict__ rp, const int *__restrict__ ci,
                            const double *__restrict__ va, double *diag, int *bad)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nrows; i += gridDim.x * blockDim.x) {
        double d = 1.0;
        if (i < n) {
            bool found = false;
            double s = 0.0;
            for (int k = rp[i]; k < rp[i + 1]; k++)
                if (ci[k] == i) {
                    s = found ? __dadd_rn(s, va[k]) : va[k];
                    found = true;
                }
            if (!found || s == 0.0 || !isfinite(s))
                *bad = 1;
            d = s;
        }
        diag[row0 + i] = d;
    }
}

// the slot's stored entries become those of A M^-1: v / d_col (one IEEE division)
__global__ void k_pool_jscale(int nrows, int row0, const int *__restrict__ sl_off, const int *__restrict__ rlen,
                              const int *__restrict__ ci, double *va, const double *__restrict__ diag)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nrows; i += gridDim.x * blockDim.x) {
        const int sl = i >> 5;
        const long long base = (long long)sl_off[sl] + (i & 31);
        const int len = rlen[row0 + i];
        for (int j = 0; j < len; j++) {
            const long long e = base + 32ll * j;
            va[e] = __ddiv_rn(va[e], diag[ci[e]]);
        }
    }
}

// a slot joins the sweep: its tiles, its tile range and its control block
__global__ void k_pool_activate(int *tile_sys, int *sys_t0, int *sys_t1, Ctl *ctl, int sid, int t0, int ntl,
                                Ctl init, const int *bad, unsigned *done, GAcc *acc)
{
    for (int t = threadIdx.x; t < ntl; t += blockDim.x)
        tile_sys[t0 + t] = sid;
    // a previous occupant stopped by an expired wait may have left partial sums
    GAcc *g = acc + (size_t)sid * MAXD;
    for (int k = threadIdx.x; k < MAXD * NDIG; k += blockDim.x)
        g[k / NDIG].dig[k % NDIG] = 0ull;
    if (threadIdx.x < MAXD) {
        g[threadIdx.x].kmin = NDIG;
        g[threadIdx.x].kmax = -1;
        g[threadIdx.x].nf = 0;
    }
    if (threadIdx.x == 0)
        done[sid] = 0u;
    if (threadIdx.x == 0) {
        sys_t0[sid] = t0;
        sys_t1[sid] = t0 + ntl;
        if (bad[sid])
            init.status = ST_INVALID;
        ctl[sid] = init;
    }
}

// a retired slot's tiles leave the sweep
__global__ void k_pool_clear(int *tile_sys, int t0, int ntl)
{
    for (int t = threadIdx.x; t < ntl; t += blockDim.x)
        tile_sys[t0 + t] = -1;
}

__global__ void k_pool_arm(int *left, int iters)
{
    *left = iters;
}

// loop condition of a batched solve: some system still running or awaiting its true-residual check
__global__ void k_batch_ctl(Batch B, unsigned long long handle, int use_cond)
{
    __shared__ int any;
    if (threadIdx.x == 0)
        any = 0;
    __syncthreads();
    for (int s = threadIdx.x; s < B.nsys; s += blockDim.x) {
        int st = B.ctl[s].status;
        if ((st == ST_RUNNING || st == ST_CANDIDATE) && B.ctl[s].err) {
            B.ctl[s].status = ST_TIMEOUT;             // a bounded wait expired: the system stops
            st = ST_TIMEOUT;
        }
        if (st == ST_RUNNING || st == ST_CANDIDATE)
            any = 1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        B.flag[0] = any;
        if (use_cond)
            cudaGraphSetConditional((cudaGraphConditionalHandle)handle, any ? 1u : 0u);
    }
}

// batched vectors <-> caller order: dst[p] = src[map[p]] (0 for padding rows, map < 0)
__global__ void k_bgather(int np, const int *__restrict__ map, const double *__restrict__ src, double *dst)
{
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < np; p += gridDim.x * blockDim.x) {
        int c = map[p];
        dst[p] = c >= 0 ? src[c] : 0.0;
    }
}

__global__ void k_bscatter(int np, const int *__restrict__ map, const double *__restrict__ src, double *dst)
{
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < np; p += gridDim.x * blockDim.x) {
        int c = map[p];
        if (c >= 0)
            dst[c] = src[p];
    }
}

}  // namespace pbcg
