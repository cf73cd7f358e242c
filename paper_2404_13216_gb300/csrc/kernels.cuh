// kernels.cuh -- fused solver passes for BiCGStab (Algorithm 1) and
// p-BiCGStab (Algorithm 2) of arXiv 2404.13216 on sm_103a, FP64.
//
// Each pass streams the rows once: it forms the SpMV row (fma chain in stored
// column order), the vector recurrences of its step, and the dot products of
// that step, all in one launch.  Dots are merged grid-wide (exact: integer
// superaccumulator; plain: fixed-order FP64 partials) and the last CTA to
// finish computes the scalars of the step (alpha, omega, beta, the residual,
// the stop and breakdown tests) and, inside a CUDA graph, sets the loop's
// conditional handle.  Pass boundaries are the global reduction points of
// Section 2; p-BiCGStab has two per iteration, BiCGStab three.
//
// Matrix layout: SELL-32.  Rows are grouped in slices of 32; inside a slice
// entry j of every row is stored contiguously (column-major), so the 32 lanes
// of a warp read one 256-byte line per entry.  Each row keeps its entries in
// stored CSR order and padding is never read, so every SpMV row is exactly
// the CSR fma chain.  Rows may be permuted (sorted by length) at upload; all
// solver vectors then live in that order, which changes no result in exact
// mode.
//
// Grid: persistent, one contiguous run of slices per warp.
#pragma once
#include "exdot.cuh"
#include "tma.cuh"

namespace pbcg {

#ifndef PBCG_UNR
#define PBCG_UNR 8                      // SpMV entries loaded per batch
#endif
#ifndef PBCG_MINB_PLAIN
#define PBCG_MINB_PLAIN 2               // resident CTAs per SM the plain passes are compiled for
#endif
#ifndef PBCG_MINB_EXACT
#define PBCG_MINB_EXACT 2               // same, exact passes
#endif
#ifndef PBCG_MINB_WIDE
#define PBCG_MINB_WIDE 2                // same, passes over matrices whose tiles are too wide to stage
#endif
#define PBCG_MINB(MODE, MATS) ((MATS) ? ((MODE) ? PBCG_MINB_EXACT : PBCG_MINB_PLAIN) : PBCG_MINB_WIDE)
#ifndef PBCG_INTERLEAVE
#define PBCG_INTERLEAVE 1               // 1: warp w takes slices w, w + W, ...; 0: one contiguous run per warp
#endif

// ---------------------------------------------------------------------------
// device-side bounds checks (a build with PBCG_CHECKS=1 only)
//
// Every index a kernel takes from the matrix layout, a tile record or a tile
// list is checked before it is used; a failed check records what failed
// (the first failure: kind << 56 | the offending value) in g_check_word,
// which the host reads with pbcg_check_word, and the access is skipped (a
// clamped index stands in).  No trap, no assert: the context stays usable.
// In the ordinary build the checks compile to nothing.
// ---------------------------------------------------------------------------
#ifndef PBCG_CHECKS
#define PBCG_CHECKS 0
#endif
enum : int {
    CHK_COL = 1,        // a column index outside the gathered vector
    CHK_LOCAL = 2,      // a staged local column outside the tile's staged blocks
    CHK_RLEN = 3,       // a row longer than its slice
    CHK_SPAN = 4,       // a slice's entries outside its tile's staged span
    CHK_BLOCK = 5,      // a gather block outside the vector
    CHK_TILE = 6,       // a tile index outside the matrix
    CHK_SYS = 7,        // a tile's system outside the batch
    CHK_CLUSTER = 8     // a cluster row's entries or owner outside the cluster
};
#if PBCG_CHECKS
static __device__ unsigned long long g_check_word;
static __device__ __noinline__ void check_fail(int kind, long long v)
{
    atomicCAS(&g_check_word, 0ull, ((unsigned long long)kind << 56) | ((unsigned long long)v & ((1ull << 56) - 1)));
}
__device__ __forceinline__ bool check_in(long long v, long long hi, int kind)
{
    const bool ok = v >= 0 && v < hi;
    if (!ok)
        check_fail(kind, v);
    return ok;
}
#define PBCG_IN(v, hi, kind) check_in((long long)(v), (long long)(hi), (kind))
#else
#define PBCG_IN(v, hi, kind) true
#endif

constexpr int THREADS = 256;
constexpr int WARPS = THREADS / 32;
constexpr int MAXD = 4;                 // most dots merged in one pass
constexpr int UNR = PBCG_UNR;

// streamed matrix entries: read once, so they go first when L2 needs room
// (the gathered vector, reused across rows, stays)
__device__ __forceinline__ unsigned long long l2_evict_first_policy()
{
    unsigned long long p;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ int ld_stream(const int *a, unsigned long long pol)
{
    int v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(a), "l"(pol));
    return v;
}
__device__ __forceinline__ double ld_stream(const double *a, unsigned long long pol)
{
    double v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(a), "l"(pol));
    return v;
}

enum : int { ST_RUNNING = 100, ST_CANDIDATE = 101, ST_SETUP1 = 110, ST_SETUP2 = 111, ST_FREE = 120, ST_INVALID = 130, ST_TIMEOUT = 200 };
enum : int { PH_SETUP = 0, PH_ITER = 1 };
enum : int { ALG_BICGSTAB = 0, ALG_PIPELINED = 1 };

// device control block of one solve (one per system in batched solves)
struct Ctl {
    double alpha, beta, omega, rho;
    double rho_new, rw, rs, rz;
    double qy, yy, rr, bb;
    double normb, res, target, tol;
    double trueres, bbx, pad_d0, pad_d1;
    int it, maxit, status, phase;
    int alg, use_cond, err, rr_period;  // err: a bounded device wait expired; rr_period: 0 = no replacement
    unsigned long long cond;            // cudaGraphConditionalHandle of the loop
    double *hist;
    int hist_cap, need_t;               // need_t: t0 = A w0 still to be formed (pool slots)
    int gen;                            // admission number of a pool slot's occupant
    int order;                          // tile order of the staged passes: 0 default, 1 round-robin, 2 claimed
};

// grid-wide merge workspace
struct Work {
    GAcc g[MAXD];
    unsigned int ticket;
    unsigned int tile_next;              // next tile to claim in a pass that schedules tiles dynamically
    int maxgrid;
    int dist;                            // 1: this grid is one rank of a row-partitioned solve
    double *part;                        // plain partials [MAXD][maxgrid]
    double loc[MAXD];                    // dist, plain: this rank's dots, its CTAs' partials summed in CTA order
};

// SELL-32 matrix in the solver's (possibly permuted) row order
struct Mat {
    int n;                               // rows
    int ncols;                           // entries of the gathered vector (n, or n plus a partition's halo)
    int nslices;                         // ceil(n / 32)
    const int *__restrict__ sl_off;      // [nslices + 1] first entry of each slice; width = diff / 32
    const int *__restrict__ rlen;        // [nslices * 32] row lengths (0 past n)
    const int *__restrict__ ci;          // padded column indices (solver order)
    const double *__restrict__ va;       // padded values
    const int *__restrict__ sl_w;        // [nslices] slice widths, or NULL: width = (sl_off[s+1] - sl_off[s]) / 32
    const uint16_t *__restrict__ lci;    // padded local indices (< GMAX * 256) into a tile's staged blocks (or NULL)
    const int *__restrict__ tmeta;       // [ntiles * TMETA] per tile: first and end SELL entry, then the GMAX
                                         // 256-row blocks it gathers from (-1 pad; all -1: gathers from global)
};

struct Vecs {
    double *x, *b, *r0, *r, *w, *t, *p, *s, *z, *v, *y, *q;
};

// Whether a staged pass hands its tiles out from a grid-wide counter (claimed
// in index order) rather than round-robin: by default only when its tiles are
// not staged (wide rows); Ctl::order overrides (a tuned launch variant).
// Either order gives bit-identical exact dots.
template <bool MATS>
__device__ __forceinline__ bool claimed_tiles(const Ctl *c)
{
    return c->order >= 2 || (c->order == 0 && !MATS);
}

// Ctl::order 3: round-robin, with the last TAIL_CLAIMED tiles of each CTA's
// share claimed (tile_loop's rounds); other orders claim every tile or none
constexpr int TAIL_CLAIMED = 2;
__device__ __forceinline__ int rr_rounds(const Ctl *c, int nslices)
{
    const int ntiles = (nslices + TILE_SLICES - 1) / TILE_SLICES;
    return c->order == 3 ? max(0, ntiles / (int)gridDim.x - TAIL_CLAIMED) : 0;
}

// Programmatic dependent launch.  A pass launched behind a programmatic graph
// edge (pass Y after pass X; BiCGStab's A after P, B after A, C after B) may
// become resident once every CTA of the pass before it has left its tile
// loop (grid_dep_launch), while that pass's last CTA still merges; it runs
// grid_dep_wait -- which returns once the earlier grid has completed and its
// stores are visible -- before its first global read.  Launched otherwise,
// both are no-ops.
__device__ __forceinline__ void grid_dep_wait()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
}
__device__ __forceinline__ void grid_dep_launch()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// residual replacement at the start of iteration it (every rr_period iterations, never at 0)
__device__ __forceinline__ bool rr_now(const Ctl *c)
{
    return c->rr_period > 0 && c->it > 0 && c->it % c->rr_period == 0;
}

__device__ __forceinline__ bool fin(double v)
{
    return ((unsigned long long)__double_as_longlong(v) & 0x7ff0000000000000ull) != 0x7ff0000000000000ull;
}

// the slices of this warp: s0, s0 + step, ... below s1
struct WarpRange {
    int s0, s1, step, lane;
};

__device__ __forceinline__ WarpRange warp_range(int nslices)
{
    WarpRange R;
    const int nw = (gridDim.x * THREADS) >> 5;
    const int gw = (blockIdx.x * THREADS + threadIdx.x) >> 5;
#if PBCG_INTERLEAVE
    R.s0 = gw;
    R.s1 = nslices;
    R.step = nw;
#else
    const int per = (nslices + nw - 1) / nw;
    R.s0 = min(gw * per, nslices);
    R.s1 = min(R.s0 + per, nslices);
    R.step = 1;
#endif
    R.lane = threadIdx.x & 31;
    return R;
}

// SpMV row of slice s, lane `lane`: acc = +0; acc = fma(val_j, x[col_j], acc) for j < len
struct RowRef {
    int base, width, len;
};

__device__ __forceinline__ RowRef row_ref(const Mat &A, int s, int lane)
{
    RowRef R;
    R.base = __ldg(A.sl_off + s);
    R.width = A.sl_w ? __ldg(A.sl_w + s) : (__ldg(A.sl_off + s + 1) - R.base) >> 5;
    R.len = __ldg(A.rlen + s * 32 + lane);
    R.base += lane;
    return R;
}

__device__ __forceinline__ double spmv_row(const Mat &A, const RowRef &R, const double *__restrict__ x)
{
    double acc = 0.0;
    const int len = PBCG_IN(R.len, R.width + 1, CHK_RLEN) ? R.len : R.width;
    for (int j0 = 0; j0 < R.width; j0 += UNR) {      // warp-uniform bound
        int c[UNR];
        double v[UNR], xv[UNR];
#pragma unroll
        for (int j = 0; j < UNR; j++) {
            if (j0 + j < len) {
                c[j] = __ldg(A.ci + R.base + (j0 + j) * 32);
                v[j] = __ldg(A.va + R.base + (j0 + j) * 32);
                if (!PBCG_IN(c[j], A.ncols, CHK_COL))
                    c[j] = 0;
            }
        }
#pragma unroll
        for (int j = 0; j < UNR; j++)
            if (j0 + j < len)
                xv[j] = __ldg(x + c[j]);
#pragma unroll
        for (int j = 0; j < UNR; j++)
            if (j0 + j < len)
                acc = __fma_rn(v[j], xv[j], acc);
    }
    return acc;
}

// same, with the gathered operand formed on the fly as fma(na, s[col], r[col])
__device__ __forceinline__ double spmv_row_axpy(const Mat &A, const RowRef &R, double na,
                                                const double *__restrict__ s, const double *__restrict__ r)
{
    double acc = 0.0;
    const int len = PBCG_IN(R.len, R.width + 1, CHK_RLEN) ? R.len : R.width;
    for (int j0 = 0; j0 < R.width; j0 += UNR) {
        int c[UNR];
        double v[UNR], xs[UNR], xr[UNR];
#pragma unroll
        for (int j = 0; j < UNR; j++) {
            if (j0 + j < len) {
                c[j] = __ldg(A.ci + R.base + (j0 + j) * 32);
                v[j] = __ldg(A.va + R.base + (j0 + j) * 32);
                if (!PBCG_IN(c[j], A.ncols, CHK_COL))
                    c[j] = 0;
            }
        }
#pragma unroll
        for (int j = 0; j < UNR; j++) {
            if (j0 + j < len) {
                xs[j] = __ldg(s + c[j]);
                xr[j] = __ldg(r + c[j]);
            }
        }
#pragma unroll
        for (int j = 0; j < UNR; j++)
            if (j0 + j < len)
                acc = __fma_rn(v[j], __fma_rn(na, xs[j], xr[j]), acc);
    }
    return acc;
}

// ---------------------------------------------------------------------------
// dot accumulation shared by all passes
// ---------------------------------------------------------------------------
template <int ND>
struct Shm {
    CtaAcc<ND> acc;
    double wpart[ND][WARPS];
    uint32_t scratch[ND][NDIG];
    double dv[ND];
    int last;
};

template <int ND, int MODE>
struct DotSet {
    Win win[MODE == 1 ? ND : 1];
    double s[ND];
    bool nf[ND];

    __device__ __forceinline__ void init()
    {
#pragma unroll
        for (int d = 0; d < ND; d++) {
            if (MODE == 1)
                win_init(win[d]);
            s[d] = 0.0;
            nf[d] = false;
        }
    }
    // all lanes of the warp call add() together for the same d
    __device__ __forceinline__ void add(Shm<ND> &sh, int d, double a, double b, bool act)
    {
        if (MODE == 1) {
            win_deposit<ND>(win[d], sh.acc, d, a, b, act, nf[d]);
        } else if (act) {
            s[d] = __fma_rn(a, b, s[d]);
        }
    }
    // same, with operands already decoded (exact mode); SQUARE when a == b
    template <bool SQUARE>
    __device__ __forceinline__ void add2(Shm<ND> &sh, int d, double a, double b, const Dec &da, const Dec &db,
                                         bool act)
    {
        if (MODE == 1) {
            win_add<ND, SQUARE>(win[d], sh.acc, d, da, db, act, nf[d]);
        } else if (act) {
            s[d] = __fma_rn(a, b, s[d]);
        }
    }
    // Dots 0 and 1 (and 2 when K == 3) of one row, each a (value, decoded)
    // operand pair; SQk when dot k is a square.  Exact mode takes one vote for
    // the common case in which every term lands in its window.
    template <int K, bool SQ0, bool SQ1, bool SQ2 = false>
    __device__ __forceinline__ void add_row(Shm<ND> &sh, bool act, double a0, double b0, const Dec &da0,
                                            const Dec &db0, double a1, double b1, const Dec &da1, const Dec &db1,
                                            double a2 = 0.0, double b2 = 0.0, const Dec *da2 = nullptr,
                                            const Dec *db2 = nullptr)
    {
        static_assert(K == 2 || K == 3, "two or three terms");
        if constexpr (MODE == 1) {
            const WinTerm t0 = win_term<SQ0>(win[0], da0, db0, act, nf[0]);
            const WinTerm t1 = win_term<SQ1>(win[1], da1, db1, act, nf[1]);
            WinTerm t2;
            if constexpr (K == 3)
                t2 = win_term<SQ2>(win[2], *da2, *db2, act, nf[2]);
            bool odd = t0.odd || t1.odd;
            if constexpr (K == 3)
                odd = odd || t2.odd;
            if (__any_sync(0xffffffffu, odd)) {
                win_settle<ND, SQ0>(win[0], sh.acc, 0, t0);
                win_settle<ND, SQ1>(win[1], sh.acc, 1, t1);
                if constexpr (K == 3)
                    win_settle<ND, SQ2>(win[2], sh.acc, 2, t2);
            } else {
                win_put<SQ0>(win[0], t0);
                win_put<SQ1>(win[1], t1);
                if constexpr (K == 3)
                    win_put<SQ2>(win[2], t2);
            }
        } else if (act) {
            s[0] = __fma_rn(a0, b0, s[0]);
            s[1] = __fma_rn(a1, b1, s[1]);
            if constexpr (K == 3)
                s[2] = __fma_rn(a2, b2, s[2]);
        }
    }
};

template <int ND, int MODE>
__device__ __forceinline__ void shm_init(Shm<ND> &sh)
{
    if (MODE == 1)
        cta_acc_init<ND>(sh.acc);
    if (threadIdx.x == 0)
        sh.last = 0;
}

// Warp sum of ND plain partials with a reduce-scatter: the dots are split
// between lane halves (and quarters) before the butterfly, so a lane performs
// 5 additions for ND = 1 or 2 and 6 for ND = 3 or 4 instead of 5 per dot.
// Every lane receives every total; the order of additions is fixed.
template <int ND>
__device__ __forceinline__ void warp_sum_plain(const double (&s)[ND], double (&out)[ND])
{
    const int lane = threadIdx.x & 31;
    const bool h16 = lane & 16, h8 = lane & 8;
    double v;
    if (ND == 1) {
        v = s[0];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            v = __dadd_rn(v, __shfl_xor_sync(0xffffffffu, v, o));
        out[0] = v;
        return;
    } else if (ND == 2) {
        // lanes < 16 keep dot 0, lanes >= 16 dot 1
        double k = h16 ? s[ND - 1] : s[0], g = h16 ? s[0] : s[ND - 1];
        v = __dadd_rn(k, __shfl_xor_sync(0xffffffffu, g, 16));
#pragma unroll
        for (int o = 8; o > 0; o >>= 1)
            v = __dadd_rn(v, __shfl_xor_sync(0xffffffffu, v, o));
#pragma unroll
        for (int d = 0; d < ND; d++)
            out[d] = __shfl_sync(0xffffffffu, v, 16 * d);
        return;
    } else {
        // quarters: dot d = 2*h16 + h8 ends in lane 8*d
        double a0 = s[0], a1 = s[1], a2 = s[2], a3 = ND > 3 ? s[ND > 3 ? 3 : 0] : 0.0;
        double k0 = h16 ? a2 : a0, k1 = h16 ? a3 : a1;
        double g0 = h16 ? a0 : a2, g1 = h16 ? a1 : a3;
        k0 = __dadd_rn(k0, __shfl_xor_sync(0xffffffffu, g0, 16));
        k1 = __dadd_rn(k1, __shfl_xor_sync(0xffffffffu, g1, 16));
        double kk = h8 ? k1 : k0, gg = h8 ? k0 : k1;
        v = __dadd_rn(kk, __shfl_xor_sync(0xffffffffu, gg, 8));
#pragma unroll
        for (int o = 4; o > 0; o >>= 1)
            v = __dadd_rn(v, __shfl_xor_sync(0xffffffffu, v, o));
#pragma unroll
        for (int d = 0; d < ND; d++)
            out[d] = __shfl_sync(0xffffffffu, v, 8 * d);
    }
}

// First half of a merge: the CTA's windows (exact) or plain partials are
// summed within the CTA and published in global memory (wk->g digits or
// wk->part[d][blockIdx.x]).  Called by every thread.
template <int ND, int MODE>
__device__ __forceinline__ void merge_publish(DotSet<ND, MODE> &D, Shm<ND> &sh, Work *wk)
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
        cta_to_global<ND>(sh.acc, wk->g);
    } else if (threadIdx.x < ND) {
        double v = sh.wpart[threadIdx.x][0];
        for (int w = 1; w < WARPS; w++)
            v = __dadd_rn(v, sh.wpart[threadIdx.x][w]);
        wk->part[threadIdx.x * wk->maxgrid + blockIdx.x] = v;
    }
    __threadfence();
}

// Second half, in one CTA once every CTA has published: round the exact
// accumulators (and reset them) or sum the plain partials in CTA order, into
// sh.dv.  Called by every thread of that CTA.
template <int ND, int MODE>
__device__ __forceinline__ void merge_finish(Shm<ND> &sh, Work *wk, const void *pre = nullptr)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __threadfence();
    if (pre && threadIdx.x == THREADS - 1) {
        // the control block the scalar step reads next, into L1 while the merge runs
        asm volatile("prefetch.global.L1 [%0];" ::"l"(pre));
        asm volatile("prefetch.global.L1 [%0];" ::"l"((const char *)pre + 128));
    }
    if (MODE == 1) {
        gacc_round_reset_cta<ND>(wk->g, sh.acc, sh.scratch, sh.dv);
    } else if (warp < ND) {
        const double *pp = wk->part + warp * wk->maxgrid;
        double v = 0.0;
        // lane l adds partials l, l + 32, ... in that order; they are loaded
        // eight at a time, so the sum waits on one round trip per eight
        const int grid = (int)gridDim.x;
        for (int c0 = lane; c0 < grid; c0 += 32 * 8) {
            double t[8];
#pragma unroll
            for (int j = 0; j < 8; j++)
                t[j] = c0 + 32 * j < grid ? __ldcg(pp + c0 + 32 * j) : 0.0;
#pragma unroll
            for (int j = 0; j < 8; j++)
                if (c0 + 32 * j < grid)
                    v = __dadd_rn(v, t[j]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            v = __dadd_rn(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (lane == 0)
            sh.dv[warp] = v;
    }
}

// Merge the CTA's dots grid-wide.  Returns true in the last CTA, whose
// sh.dv[] then holds the finished dot values.  Called by every thread.  pre:
// the control block the last CTA's scalar step reads (prefetched), or NULL.
template <int ND, int MODE>
__device__ bool finalize(DotSet<ND, MODE> &D, Shm<ND> &sh, Work *wk, const void *pre = nullptr)
{
    const int dist = wk->dist;       // loaded here, used by the last CTA: off the path after the ticket
    merge_publish<ND, MODE>(D, sh, wk);
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int t = atomicAdd(&wk->ticket, 1u);
        sh.last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!sh.last)
        return false;
    if (dist) {
        // one rank of a row-partitioned solve: the exact digits stay in wk->g
        // and the plain partials are summed into wk->loc; the host adds them
        // over the ranks and k_dist_finish rounds and takes the scalar step
        if (MODE == 0) {
            merge_finish<ND, MODE>(sh, wk);
            __syncthreads();
            if (threadIdx.x < ND)
                wk->loc[threadIdx.x] = sh.dv[threadIdx.x];
        }
        if (threadIdx.x == 0) {
            wk->ticket = 0u;
            wk->tile_next = 0u;
        }
        __syncthreads();
        return false;
    }
    merge_finish<ND, MODE>(sh, wk, pre);
    if (threadIdx.x == 0) {
        wk->ticket = 0u;
        wk->tile_next = 0u;          // every CTA has left its tile loop
    }
    __syncthreads();
    return true;
}

// ---------------------------------------------------------------------------
// scalar steps (one thread of the last CTA)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void set_cond(Ctl *c)
{
    if (c->use_cond)
        cudaGraphSetConditional((cudaGraphConditionalHandle)c->cond, c->status == ST_RUNNING ? 1u : 0u);
}

// the part of a step after the stop test: breakdown checks, beta, alpha, maxit
static __device__ void post_stop(Ctl *c)
{
    if (c->phase == PH_SETUP) {
        if (c->alg == ALG_PIPELINED) {
            double a0 = __ddiv_rn(c->rho, c->rw);
            if (!fin(a0))
                c->status = 2;
            else
                c->alpha = a0;
        }
    } else {
        double om = c->omega;
        if (om == 0.0) {
            c->status = 2;
        } else {
            double beta = __dmul_rn(__ddiv_rn(c->alpha, om), __ddiv_rn(c->rho_new, c->rho));
            if (c->alg == ALG_PIPELINED) {
                double den = __dsub_rn(__dadd_rn(c->rw, __dmul_rn(beta, c->rs)),
                                       __dmul_rn(__dmul_rn(beta, om), c->rz));
                double an = __ddiv_rn(c->rho_new, den);
                if (!fin(beta) || !fin(an) || c->rho_new == 0.0) {
                    c->status = 2;
                } else {
                    c->beta = beta;
                    c->alpha = an;
                    c->rho = c->rho_new;
                }
            } else {
                if (!fin(beta) || c->rho_new == 0.0) {
                    c->status = 2;
                } else {
                    c->beta = beta;
                    c->rho = c->rho_new;
                }
            }
        }
    }
    if (c->status == ST_RUNNING && c->it >= c->maxit)
        c->status = 1;
}

// residual of step k, stop test, then post_stop
static __device__ void residual_step(Ctl *c, double rr)
{
    double res = __ddiv_rn(__dsqrt_rn(rr), c->normb);
    c->res = res;
    if (c->it < c->hist_cap)
        c->hist[c->it] = res;
    if (res <= c->target)
        c->status = ST_CANDIDATE;
    else
        post_stop(c);
}

// after the setup dots (b,b), (r0,r0) [, (r0,w0)]
static __device__ void setup_scalar(Ctl *c, double bb, double rho, double rw)
{
    c->bb = bb;
    c->rho = rho;
    c->rw = rw;
    c->it = 0;
    c->phase = PH_SETUP;
    c->target = c->tol;
    double nb = __dsqrt_rn(bb);
    c->normb = (nb == 0.0) ? 1.0 : nb;
    double res = __ddiv_rn(__dsqrt_rn(rho), c->normb);
    c->res = res;
    if (c->hist_cap > 0)
        c->hist[0] = res;
    if (!fin(bb) || !fin(rho) || !fin(rw)) {
        c->status = 3;
        return;
    }
    c->status = ST_RUNNING;
    if (res <= c->target)
        c->status = ST_CANDIDATE;
    else
        post_stop(c);
}

#define PBCG_SLICE_LOOP(A)                                 \
    const WarpRange wr_ = warp_range((A).nslices);         \
    for (int sl_ = wr_.s0; sl_ < wr_.s1; sl_ += wr_.step)

#define PBCG_ROW (sl_ * 32 + wr_.lane)

// ---------------------------------------------------------------------------
// setup passes
// ---------------------------------------------------------------------------
// S1: r0 = b - A x0, r = r0 (and p = r0 for BiCGStab); dots (b,b), (r0,r0)
template <int MODE>
__global__ void __launch_bounds__(THREADS) k_setup1(Mat A, Vecs V, Ctl *c, Work *wk)
{
    __shared__ Shm<2> sh;
    shm_init<2, MODE>(sh);
    __syncthreads();
    const bool bicg = c->alg == ALG_BICGSTAB;
    DotSet<2, MODE> D;
    D.init();
    PBCG_SLICE_LOOP(A)
    {
        int i = PBCG_ROW;
        bool act = i < A.n;
        RowRef R = row_ref(A, sl_, wr_.lane);
        double ax = spmv_row(A, R, V.x);
        double bi = 0.0, r0i = 0.0;
        if (act) {
            bi = V.b[i];
            r0i = __dsub_rn(bi, ax);
            V.r0[i] = r0i;
            V.r[i] = r0i;
            if (bicg)
                V.p[i] = r0i;
        }
        D.add(sh, 0, bi, bi, act);
        D.add(sh, 1, r0i, r0i, act);
    }
    if (!finalize<2, MODE>(D, sh, wk))
        return;
    if (threadIdx.x == 0) {
        c->bb = sh.dv[0];
        c->rho = sh.dv[1];
        if (bicg) {
            setup_scalar(c, sh.dv[0], sh.dv[1], 0.0);
            set_cond(c);
        }
    }
}

// S2 (p-BiCGStab): w0 = A r0; dot (r0, w0); setup scalars
template <int MODE>
__global__ void __launch_bounds__(THREADS) k_setup2(Mat A, Vecs V, Ctl *c, Work *wk)
{
    __shared__ Shm<1> sh;
    shm_init<1, MODE>(sh);
    __syncthreads();
    DotSet<1, MODE> D;
    D.init();
    PBCG_SLICE_LOOP(A)
    {
        int i = PBCG_ROW;
        bool act = i < A.n;
        RowRef R = row_ref(A, sl_, wr_.lane);
        double wi = spmv_row(A, R, V.r0);
        double r0i = 0.0;
        if (act) {
            r0i = V.r0[i];
            V.w[i] = wi;
        }
        D.add(sh, 0, r0i, wi, act);
    }
    if (!finalize<1, MODE>(D, sh, wk))
        return;
    if (threadIdx.x == 0) {
        setup_scalar(c, c->bb, c->rho, sh.dv[0]);
        set_cond(c);
    }
}

// S3 (p-BiCGStab): t0 = A w0
static __global__ void __launch_bounds__(THREADS) k_setup3(Mat A, Vecs V, const Ctl *c)
{
    if (c->status != ST_RUNNING && c->status != ST_CANDIDATE)
        return;
    PBCG_SLICE_LOOP(A)
    {
        int i = PBCG_ROW;
        RowRef R = row_ref(A, sl_, wr_.lane);
        double ti = spmv_row(A, R, V.w);
        if (i < A.n)
            V.t[i] = ti;
    }
}

// ---------------------------------------------------------------------------
// true residual ||b - A x|| / ||b|| with exact dots; resolves a candidate stop
// ---------------------------------------------------------------------------
// the scalar step after the dots (r,r) and (b,b) of the true residual (one thread)
static __device__ void true_res_tail(Ctl *c, const double *dv)
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

static __global__ void __launch_bounds__(THREADS) k_true_res(Mat A, Vecs V, Ctl *c, Work *wk)
{
    __shared__ Shm<2> sh;
    shm_init<2, 1>(sh);
    __syncthreads();
    DotSet<2, 1> D;
    D.init();
    PBCG_SLICE_LOOP(A)
    {
        int i = PBCG_ROW;
        bool act = i < A.n;
        RowRef R = row_ref(A, sl_, wr_.lane);
        double ax = spmv_row(A, R, V.x);
        double ri = 0.0, bi = 0.0;
        if (act) {
            bi = V.b[i];
            ri = __dsub_rn(bi, ax);
        }
        D.add(sh, 0, ri, ri, act);
        D.add(sh, 1, bi, bi, act);
    }
    if (!finalize<2, 1>(D, sh, wk))
        return;
    if (threadIdx.x == 0)
        true_res_tail(c, sh.dv);
}

// ---------------------------------------------------------------------------
// right Jacobi preconditioning: A M^-1 with M = diag(A) as scaled entries,
// y0 = d x0 before the solve and x = y / d after it (one rounding each)
// ---------------------------------------------------------------------------
static __global__ void k_jacobi_scale(long long ne, const int *__restrict__ ci, const double *__restrict__ va,
                                      const double *__restrict__ d, double *vs)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < ne; e += (long long)gridDim.x * blockDim.x)
        vs[e] = __ddiv_rn(va[e], d[ci[e]]);
}

static __global__ void k_vmul(int n, const double *__restrict__ d, double *x)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        x[i] = __dmul_rn(x[i], d[i]);
}

static __global__ void k_vdiv(int n, const double *__restrict__ d, double *x)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        x[i] = __ddiv_rn(x[i], d[i]);
}

// ---------------------------------------------------------------------------
// standalone kernels: dot, SpMV, permutation gather/scatter
// ---------------------------------------------------------------------------
template <int MODE>
__global__ void __launch_bounds__(THREADS) k_dot(long long n, const double *a, const double *b, double *out,
                                                 Work *wk)
{
    __shared__ Shm<1> sh;
    shm_init<1, MODE>(sh);
    __syncthreads();
    DotSet<1, MODE> D;
    D.init();
    const int lane = threadIdx.x & 31;
    const long long nw = ((long long)gridDim.x * THREADS) >> 5;
    const long long gw = ((long long)blockIdx.x * THREADS + threadIdx.x) >> 5;
    const long long nt = (n + 31) >> 5;
    const long long per = (nt + nw - 1) / nw;
    const long long t0 = gw * per < nt ? gw * per : nt;
    const long long t1 = t0 + per < nt ? t0 + per : nt;
    for (long long t = t0; t < t1; t++) {
        long long i = t * 32 + lane;
        bool act = i < n;
        double ai = act ? a[i] : 0.0, bi = act ? b[i] : 0.0;
        D.add(sh, 0, ai, bi, act);
    }
    if (!finalize<1, MODE>(D, sh, wk))
        return;
    if (threadIdx.x == 0)
        *out = sh.dv[0];
}

static __global__ void __launch_bounds__(THREADS) k_spmv(Mat A, const double *x, double *y)
{
    PBCG_SLICE_LOOP(A)
    {
        int i = PBCG_ROW;
        RowRef R = row_ref(A, sl_, wr_.lane);
        double yi = spmv_row(A, R, x);
        if (i < A.n)
            y[i] = yi;
    }
}

// Device-side validation of an uploaded SELL-32 layout (every build): slice
// offsets non-decreasing in whole 32-entry columns, every row no longer than
// its slice (rows past n empty), every stored column inside the gathered
// vector, every tile record matching the slice offsets with gather blocks
// inside the vector, and every staged local index pointing at the entry's
// column.  *word receives the first failure found (CHK_* << 56 | position),
// or stays 0.  Reads only inside the arrays' sizes.
static __global__ void k_mat_check(Mat A, long long padded, unsigned long long *word)
{
    auto bad = [&](int kind, long long pos) {
        atomicCAS(word, 0ull, ((unsigned long long)kind << 56) | ((unsigned long long)pos & ((1ull << 56) - 1)));
    };
    const int ntiles = (A.nslices + TILE_SLICES - 1) / TILE_SLICES;
    const long long nrows = (long long)A.nslices * 32;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < nrows; p += stride) {
        const int s = (int)(p >> 5), lane = (int)(p & 31);
        const int o0 = A.sl_off[s], o1 = A.sl_off[s + 1];
        if (o1 < o0 || ((o1 - o0) & 31) || o1 > padded) {
            bad(CHK_SPAN, s);
            continue;
        }
        const int width = (o1 - o0) >> 5, len = A.rlen[p];
        if (len < 0 || len > width || (p >= A.n && len != 0)) {
            bad(CHK_RLEN, p);
            continue;
        }
        for (int j = 0; j < len; j++) {
            const long long e = o0 + lane + 32ll * j;
            const int c = A.ci[e];
            if (c < 0 || c >= A.ncols)
                bad(CHK_COL, e);
        }
    }
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; A.tmeta && t < ntiles; t += stride) {
        const int *r = A.tmeta + t * TMETA;
        const int sa = (int)t * TILE_SLICES, sb = min(A.nslices, sa + TILE_SLICES);
        if (r[0] != A.sl_off[sa] || r[1] != A.sl_off[sb]) {
            bad(CHK_TILE, t);
            continue;
        }
        int nblk = 0;
        for (int g = 0; g < GMAX; g++) {
            if (r[2 + g] < 0)
                continue;
            nblk++;
            if (r[2 + g] >= (A.ncols + TILE_ROWS - 1) / TILE_ROWS)
                bad(CHK_BLOCK, t);
        }
        if (nblk == 0 || !A.lci || r[1] - r[0] > MCAP)
            continue;
        for (int e = r[0]; e < r[1]; e++) {
            const int l = A.lci[e], g = l / TILE_ROWS;
            if (g >= nblk || r[2 + g] * TILE_ROWS + l % TILE_ROWS != A.ci[e])
                bad(CHK_LOCAL, e);
        }
    }
}

// dst[p] = src[perm[p]] (into solver order)
static __global__ void k_gather(int n, const int *__restrict__ perm, const double *__restrict__ src, double *dst)
{
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x)
        dst[p] = src[perm[p]];
}

// dst[perm[p]] = src[p] (back to caller order)
static __global__ void k_scatter(int n, const int *__restrict__ perm, const double *__restrict__ src, double *dst)
{
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x)
        dst[perm[p]] = src[p];
}


// ---------------------------------------------------------------------------
// residual replacement (p-BiCGStabRR): at the start of iteration i, i > 0,
// i mod k == 0: r = b - A x, w = A r (and p from its recurrence with the new
// r), s = A p, z = A s.  Each step needs the whole previous vector, so each is
// its own launch; on other iterations they return at once.
// ---------------------------------------------------------------------------
static __global__ void __launch_bounds__(THREADS) k_rr1(Mat A, Vecs V, const Ctl *c)
{
    if (c->status != ST_RUNNING || !rr_now(c))
        return;
    PBCG_SLICE_LOOP(A)
    {
        int i = PBCG_ROW;
        RowRef R = row_ref(A, sl_, wr_.lane);
        double ax = spmv_row(A, R, V.x);
        if (i < A.n)
            V.r[i] = __dsub_rn(V.b[i], ax);
    }
}

static __global__ void __launch_bounds__(THREADS) k_rr2(Mat A, Vecs V, const Ctl *c)
{
    if (c->status != ST_RUNNING || !rr_now(c))
        return;
    const double beta = c->beta, nomega = -c->omega;
    PBCG_SLICE_LOOP(A)
    {
        int i = PBCG_ROW;
        RowRef R = row_ref(A, sl_, wr_.lane);
        double wi = spmv_row(A, R, V.r);
        if (i < A.n) {
            V.w[i] = wi;
            V.p[i] = __fma_rn(beta, __fma_rn(nomega, V.s[i], V.p[i]), V.r[i]);
        }
    }
}

static __global__ void __launch_bounds__(THREADS) k_rr3(Mat A, Vecs V, const Ctl *c)
{
    if (c->status != ST_RUNNING || !rr_now(c))
        return;
    PBCG_SLICE_LOOP(A)
    {
        int i = PBCG_ROW;
        RowRef R = row_ref(A, sl_, wr_.lane);
        double si = spmv_row(A, R, V.p);
        if (i < A.n)
            V.s[i] = si;
    }
}

static __global__ void __launch_bounds__(THREADS) k_rr4(Mat A, Vecs V, const Ctl *c)
{
    if (c->status != ST_RUNNING || !rr_now(c))
        return;
    PBCG_SLICE_LOOP(A)
    {
        int i = PBCG_ROW;
        RowRef R = row_ref(A, sl_, wr_.lane);
        double zi = spmv_row(A, R, V.s);
        if (i < A.n)
            V.z[i] = zi;
    }
}

// ---------------------------------------------------------------------------
// staged passes: tiles of 256 rows double-buffered in shared memory by TMA
// ---------------------------------------------------------------------------
template <int NV, bool MATS, bool WIN = MATS>
struct TilePipe {
    using L = StageLayout<NV, MATS, WIN>;
    uint8_t *smem;
    uint64_t *bar;
    StageInfo *info;

    __device__ __forceinline__ uint8_t *stage(int k) const { return smem + (size_t)k * L::STAGE; }
    __device__ __forceinline__ const double *vec(int k, int v) const
    {
        return reinterpret_cast<const double *>(stage(k)) + v * TILE_ROWS;
    }
    __device__ __forceinline__ const double *gwin(int k) const
    {
        return reinterpret_cast<const double *>(stage(k) + L::VEC);
    }
    __device__ __forceinline__ const double *va(int k) const
    {
        return reinterpret_cast<const double *>(stage(k) + L::VEC + L::GWIN);
    }
    __device__ __forceinline__ const int *ci(int k) const
    {
        return reinterpret_cast<const int *>(stage(k) + L::VEC + L::GWIN + L::VA);
    }
    __device__ __forceinline__ const int *rlen(int k) const
    {
        return reinterpret_cast<const int *>(stage(k) + L::VEC + L::GWIN + L::VA + L::CI);
    }
    __device__ __forceinline__ const int *sloff(int k) const
    {
        return reinterpret_cast<const int *>(stage(k) + L::VEC + L::GWIN + L::VA + L::CI + L::RLEN);
    }
    __device__ __forceinline__ const int *meta(int k) const
    {
        return reinterpret_cast<const int *>(stage(k) + L::VEC + L::GWIN + L::VA + L::CI + L::RLEN + L::SLOFF);
    }

    // thread 0 or the refilling lane: copy tile `tile` (nv of the NV vectors),
    // described by its record rec, into stage k, together with the record of
    // tile tn, the next one for this stage (-1: none); gx is the vector the
    // tile's SpMV gathers from (NULL: no SpMV in this pass)
    __device__ __forceinline__ void issue(int k, int tile, const int (&rec)[TMETA], const Mat &A,
                                          const double *const (&src)[NV], int nv, const double *gx, int tn)
    {
        const int s0 = tile * TILE_SLICES;
        const int e0 = rec[0], span = rec[1] - rec[0];
        const bool staged = MATS && span > 0 && span <= MCAP;
        const bool windowed = WIN && staged && gx != nullptr && A.lci != nullptr && rec[2] >= 0;
        int nblk = 0;
        if (windowed) {
#pragma unroll
            for (int g = 0; g < GMAX; g++)
                nblk += rec[2 + g] >= 0;
        }
        info[k].e0 = e0;
        info[k].staged = staged;
        info[k].windowed = windowed;
        info[k].tile = tile;
        info[k].span = span;
        info[k].nblk = nblk;
        uint32_t bytes = (uint32_t)nv * TILE_ROWS * 8 + L::RLEN + L::SLOFF + (staged ? (uint32_t)span * (windowed ? 10u : 12u) : 0u) +
                         (uint32_t)nblk * TILE_ROWS * 8 + (tn >= 0 ? TMETA * 4u : 0u);
        fence_async_shared();
        mbar_arrive_expect_tx(&bar[k], bytes);
        const size_t row0 = (size_t)tile * TILE_ROWS;
        for (int v = 0; v < nv; v++)
            bulk_g2s(stage(k) + (size_t)v * TILE_ROWS * 8, src[v] + row0, TILE_ROWS * 8, &bar[k]);
        uint8_t *tail = stage(k) + L::VEC + L::GWIN + L::VA + L::CI;
        bulk_g2s(tail, A.rlen + row0, L::RLEN, &bar[k]);
        bulk_g2s(tail + L::RLEN, A.sl_off + s0, L::SLOFF, &bar[k]);
        if (tn >= 0)
            bulk_g2s(tail + L::RLEN + L::SLOFF, A.tmeta + (size_t)tn * TMETA, TMETA * 4, &bar[k]);
        if (staged) {
            if (windowed)
                bulk_g2s(stage(k) + L::VEC + L::GWIN + L::VA, A.lci + e0, (uint32_t)span * 2u, &bar[k]);
            else
                bulk_g2s(stage(k) + L::VEC + L::GWIN + L::VA, A.ci + e0, (uint32_t)span * 4u, &bar[k]);
            bulk_g2s(stage(k) + L::VEC + L::GWIN, A.va + e0, (uint32_t)span * 8u, &bar[k]);
        }
        if (windowed) {
#pragma unroll
            for (int g = 0; g < GMAX; g++)
                if (rec[2 + g] >= 0) {
                    // (a checked build copies block 0 in place of a block outside the vector)
                    const int blk = PBCG_IN(rec[2 + g], (A.ncols + TILE_ROWS - 1) / TILE_ROWS, CHK_BLOCK) ? rec[2 + g] : 0;
                    bulk_g2s(stage(k) + L::VEC + (size_t)g * TILE_ROWS * 8, gx + (size_t)blk * TILE_ROWS,
                             TILE_ROWS * 8, &bar[k]);
                }
        }
    }

    // SpMV row of this lane from stage k (matrix from shared memory when staged)
    __device__ __forceinline__ double spmv(int k, const Mat &A, int warp, int lane, const double *__restrict__ x) const
    {
        const int *so = sloff(k);
        const int off = so[warp];
        // the slice's width: explicit for pools (a tile's last slice need not be
        // followed by the same slot's entries), else the distance to the next slice
        int width = A.sl_w ? __ldg(A.sl_w + (size_t)(info[k].tile * TILE_SLICES + warp)) : (so[warp + 1] - off) >> 5;
        int len = rlen(k)[warp * 32 + lane];
        const bool st = info[k].staged;
#if PBCG_CHECKS
        if (!PBCG_IN(len, width + 1, CHK_RLEN))
            len = width;
        if (st && !(PBCG_IN(off - info[k].e0, info[k].span + 1, CHK_SPAN) &&
                    PBCG_IN(off - info[k].e0 + 32 * width, info[k].span + 1, CHK_SPAN)))
            width = len = 0;
#endif
        const int *cp = st ? ci(k) + (off - info[k].e0) + lane : A.ci + off + lane;
        const double *vp = st ? va(k) + (off - info[k].e0) + lane : A.va + off + lane;
        double acc = 0.0;
        if (WIN && info[k].windowed) {                  // gather from the staged blocks (16-bit local indices)
            const double *xw = gwin(k);
            const uint16_t *lp = reinterpret_cast<const uint16_t *>(ci(k)) + (off - info[k].e0) + lane;
            for (int j0 = 0; j0 < width; j0 += UNR) {
#pragma unroll
                for (int j = 0; j < UNR; j++)
                    if (j0 + j < len) {
                        int l = lp[(j0 + j) * 32];
                        if (!PBCG_IN(l, info[k].nblk * TILE_ROWS, CHK_LOCAL))
                            l = 0;
                        acc = __fma_rn(vp[(j0 + j) * 32], xw[l], acc);
                    }
            }
            return acc;
        }
        const unsigned long long pol = l2_evict_first_policy();
        for (int j0 = 0; j0 < width; j0 += UNR) {
            int c[UNR];
            double v[UNR], xv[UNR];
            if (st) {                                  // warp-uniform: entries in shared memory
#pragma unroll
                for (int j = 0; j < UNR; j++) {
                    if (j0 + j < len) {
                        c[j] = cp[(j0 + j) * 32];
                        v[j] = vp[(j0 + j) * 32];
                    }
                }
            } else {                                   // entries in global memory, streamed
#pragma unroll
                for (int j = 0; j < UNR; j++) {
                    if (j0 + j < len) {
                        c[j] = ld_stream(cp + (j0 + j) * 32, pol);
                        v[j] = ld_stream(vp + (j0 + j) * 32, pol);
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < UNR; j++)
                if (j0 + j < len && !PBCG_IN(c[j], A.ncols, CHK_COL))
                    c[j] = 0;
#pragma unroll
            for (int j = 0; j < UNR; j++)
                if (j0 + j < len)
                    xv[j] = __ldg(x + c[j]);
#pragma unroll
            for (int j = 0; j < UNR; j++)
                if (j0 + j < len)
                    acc = __fma_rn(v[j], xv[j], acc);
        }
        return acc;
    }
};

// Common tile loop.  No CTA-wide barrier per tile: each warp waits on the
// stage's mbarrier for its own data, and the last warp to finish with a stage
// (a shared counter) issues the copies of the tile that reuses it, reading
// that tile's record from the stage itself (no global load on the refill
// path).  Warps thus drift apart by up to NSTAGE - 1 tiles, so one
// warp's integer (exact-dot) work overlaps another's FP64 and memory work.
// Every wait is bounded; a warp that gives up raises a flag that stops the
// others, and before the CTA returns one thread waits (bounded) for copies
// still in flight.
//
// Tiles go to CTAs round-robin (CTA b takes b, b + grid, ...), or, with dyn
// (a grid-wide counter that the pass's last CTA resets), in claim order: the
// thread that refills a stage claims the next tile.  With dyn and rounds > 0
// the first `rounds` tiles of every CTA are dealt round-robin and only the
// rest are claimed (tiles rounds * grid, ... in claim order), so that the
// SMs that run ahead take over the tail without paying a claim per tile.  A matrix with wide rows
// keeps its rows sorted by length, so claiming hands out the heaviest tiles
// first and lets the light ones fill in around them (round-robin leaves the
// CTA holding the heaviest tile of every round with the most work).  When the
// counter is exhausted the refilling thread completes the stage's phase with
// no data and a tile of -1, which ends every warp's loop at that stage.
template <int NV, bool MATS, class Body>
__device__ __forceinline__ void tile_loop(const Mat &A, const double *const (&src)[NV], int nv, const double *gx,
                                          Ctl *c, uint8_t *dsm, Body body, unsigned int *dyn = nullptr,
                                          int rounds = 0)
{
    __shared__ uint64_t bar[NSTAGE];
    __shared__ StageInfo info[NSTAGE];
    __shared__ int done_cnt[NSTAGE];         // warps finished with the stage's current tile
    __shared__ int nissued[NSTAGE];          // tiles issued into each stage
    __shared__ int tmo;
    TilePipe<NV, MATS> P{dsm, bar, info};
    const int ntiles = (A.nslices + TILE_SLICES - 1) / TILE_SLICES;
    // round-robin tiles of this CTA (all of its tiles without dyn)
    const int my = dyn ? min(rounds, ntiles / (int)gridDim.x)
                       : (ntiles > (int)blockIdx.x ? (ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x : 0);
    const unsigned int claim0 = dyn ? (unsigned int)my * gridDim.x : 0u;     // first claimed tile
    auto tile_of = [&](int jj) { return jj < my ? (int)blockIdx.x + jj * (int)gridDim.x : -1; };
    const bool recs = A.tmeta != nullptr;     // tile records travel with the stages
    auto record = [&](int t, int (&rec)[TMETA]) {   // from global memory
        if (recs) {
#pragma unroll
            for (int q = 0; q < TMETA; q++)
                rec[q] = A.tmeta[(size_t)t * TMETA + q];
        } else {
            rec[0] = A.sl_off[t * TILE_SLICES];
            rec[1] = A.sl_off[min((t + 1) * TILE_SLICES, A.nslices)];
#pragma unroll
            for (int q = 2; q < TMETA; q++)
                rec[q] = -1;
        }
    };
    // dynamic: claim a tile into stage k (or end the stage's sequence)
    auto claim_issue = [&](int k) {
        const unsigned int t = claim0 + atomicAdd(dyn, 1u);
        if (t < (unsigned int)ntiles) {
            int rec[TMETA];
            record((int)t, rec);
            nissued[k] += 1;
            P.issue(k, (int)t, rec, A, src, nv, gx, -1);
        } else {
            info[k].tile = -1;
            mbar_arrive(&bar[k]);
        }
    };
    if (threadIdx.x == 0) {
        for (int k = 0; k < NSTAGE; k++) {
            mbar_init(&bar[k], 1);
            done_cnt[k] = 0;
            nissued[k] = 0;
        }
        tmo = 0;
        fence_mbar_init();
        fence_async_shared();
        for (int k = 0; k < NSTAGE; k++) {
            if (k < my) {
                int rec[TMETA];
                record(tile_of(k), rec);
                nissued[k] += 1;
                P.issue(k, tile_of(k), rec, A, src, nv, gx, recs ? tile_of(k + NSTAGE) : -1);
            } else if (dyn) {
                claim_issue(k);
            }
        }
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int j = 0; dyn != nullptr || j < my; j++) {
        const int k = j % NSTAGE;
        const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&bar[k], (uint32_t)(j / NSTAGE) & 1u));
        if (!ok || *(volatile int *)&tmo) {
            if (lane == 0)
                tmo = 1;
            break;
        }
        const int tile = dyn ? *(volatile int *)&info[k].tile : tile_of(j);
        if (tile < 0)
            break;                                // dynamic: no tiles left (the same for every warp)
        body(P, k, tile, warp, lane);
        __syncwarp();
        if (lane == 0) {
            __threadfence_block();
            if (atomicAdd(&done_cnt[k], 1) == WARPS - 1) {
                // last warp out of this stage: every warp has read it
                __threadfence_block();
                done_cnt[k] = 0;
                const int jn = j + NSTAGE;
                if (jn < my) {
                    int rec[TMETA];
                    if (recs) {
                        const int *m = P.meta(k);
#pragma unroll
                        for (int q = 0; q < TMETA; q++)
                            rec[q] = m[q];
                    } else {
                        record(tile_of(jn), rec);
                    }
                    nissued[k] += 1;
                    P.issue(k, tile_of(jn), rec, A, src, nv, gx, recs ? tile_of(jn + NSTAGE) : -1);
                } else if (dyn) {
                    claim_issue(k);
                }
            }
        }
    }
    __syncthreads();
    if (tmo) {
        if (threadIdx.x == 0) {
            for (int k = 0; k < NSTAGE; k++)
                if (nissued[k] > 0)
                    mbar_wait_bounded(&bar[k], (uint32_t)(nissued[k] - 1) & 1u);
            atomicOr(&c->err, 1);
        }
        __syncthreads();
    }
}

// Scalar tails of the p-BiCGStab passes (one thread, after the merge):
// pass X stores (q,y), (y,y), (r0,s), (r0,z) and forms omega_i; pass Y stores
// (r0,r), (r0,w), (r,r), counts the iteration and takes the stop test, beta
// and alpha.
static __device__ void pipe_x_tail(Ctl *c, const double *dv)
{
    double qy = dv[0], yy = dv[1];
    c->qy = qy;
    c->yy = yy;
    c->rs = dv[2];
    c->rz = dv[3];
    if (c->err) {
        c->status = ST_TIMEOUT;
        set_cond(c);
    } else if (!fin(qy) || !fin(yy)) {
        c->status = 3;
        set_cond(c);
    } else {
        c->omega = (yy == 0.0) ? 0.0 : __ddiv_rn(qy, yy);
    }
}

static __device__ void pipe_y_tail(Ctl *c, const double *dv)
{
    double rho_new = dv[0], rw = dv[1], rr = dv[2];
    c->rho_new = rho_new;
    c->rw = rw;
    c->rr = rr;
    c->phase = PH_ITER;
    if (c->err) {
        c->status = ST_TIMEOUT;
    } else if (!fin(rho_new) || !fin(rw) || !fin(c->rs) || !fin(c->rz) || !fin(rr)) {
        c->status = 3;
    } else {
        c->it += 1;
        residual_step(c, rr);
    }
    set_cond(c);
}

// The bounded barrier wait of the tile loop on a phase that nothing
// completes (failure-detection check): out[0] = 1 when it gave up, out[1..2]
// the clock64 cycles it took (low, high words).  One CTA of one warp.
static __global__ void __launch_bounds__(32) k_check_wait(unsigned probes, unsigned *out)
{
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncwarp();
    const long long t0 = clock64();
    const bool done = mbar_wait_bounded(&bar, 0u, probes);
    const long long t1 = clock64();
    if (threadIdx.x == 0) {
        out[0] = done ? 0u : 1u;
        out[1] = (unsigned)(unsigned long long)(t1 - t0);
        out[2] = (unsigned)((unsigned long long)(t1 - t0) >> 32);
    }
}

// Row arithmetic of the p-BiCGStab passes (Algorithm 2), shared by the
// single-system and batched passes so that both round identically.
// Pass X: p, s, z (bit copies of r, w, t at i = 0; kept as they are right
// after a residual replacement), then q and y.
struct XRow {
    double p, s, z, q, y;
};

__device__ __forceinline__ XRow pipe_x_row(bool first, bool rr, double nalpha, double beta, double nomega, double ri,
                                           double wi, double ti, double pold, double sold, double zold, double vold)
{
    XRow o;
    if (first) {
        o.p = ri;
        o.s = wi;
        o.z = ti;
    } else if (rr) {
        o.p = pold;
        o.s = sold;
        o.z = zold;
    } else {
        o.p = __fma_rn(beta, __fma_rn(nomega, sold, pold), ri);
        o.s = __fma_rn(beta, __fma_rn(nomega, zold, sold), wi);
        o.z = __fma_rn(beta, __fma_rn(nomega, vold, zold), ti);
    }
    o.q = __fma_rn(nalpha, o.s, ri);
    o.y = __fma_rn(nalpha, o.z, wi);
    return o;
}

// Pass Y: x_{i+1}, r_{i+1}, w_{i+1} from q, y, p, x, t and v = A z.
struct YRow {
    double x, r, w;
};

__device__ __forceinline__ YRow pipe_y_row(double alpha, double omega, double nalpha, double nomega, double q, double y,
                                           double p, double x, double t, double v)
{
    YRow o;
    o.x = __fma_rn(omega, q, __fma_rn(alpha, p, x));
    o.r = __fma_rn(nomega, y, q);
    o.w = __fma_rn(nomega, __fma_rn(nalpha, v, t), y);
    return o;
}

// X(i) staged: t_i = A w_i (i >= 1), p, s, z, q, y; dots (q,y), (y,y), (r0,s), (r0,z); omega_i
template <int MODE, bool MATS>
__global__ void __launch_bounds__(THREADS, PBCG_MINB(MODE, MATS))
    k_pipe_x_tma(Mat A, Vecs V, Ctl *c, Work *wk)
{
    extern __shared__ __align__(128) uint8_t dsm[];
    __shared__ Shm<4> sh;
    shm_init<4, MODE>(sh);
    grid_dep_wait();
    if (c->status != ST_RUNNING)
        return;
    const bool first = (c->it == 0);
    const bool rr = rr_now(c);       // p, s, z were just recomputed: no recurrence this iteration
    const double alpha = c->alpha, beta = c->beta, omega = c->omega;
    const double nalpha = -alpha, nomega = -omega;
    DotSet<4, MODE> D;
    D.init();
    // stage slots: 0 r, 1 w, 2 r0, 3 p (t when first), 4 s, 5 z, 6 v
    const double *const src[7] = {V.r, V.w, V.r0, first ? V.t : V.p, V.s, V.z, V.v};
    tile_loop<7, MATS>(A, src, first ? 4 : 7, first ? nullptr : V.w, c, dsm,
                       [&](const TilePipe<7, MATS> &P, int k, int tile, int warp, int lane) {
        const int sl = tile * TILE_SLICES + warp;
        const int i = sl * 32 + lane;
        const bool act = sl < A.nslices && i < A.n;
        const int o = warp * 32 + lane;
        double q = 0.0, y = 0.0, r0i = 0.0, si = 0.0, zi = 0.0;
        if (sl < A.nslices) {
            const double ri = P.vec(k, 0)[o], wi = P.vec(k, 1)[o];
            r0i = P.vec(k, 2)[o];
            double ti, pold = 0.0, sold = 0.0, zold = 0.0, vold = 0.0;
            if (first) {
                ti = P.vec(k, 3)[o];
            } else {
                ti = P.spmv(k, A, warp, lane, V.w);
                pold = P.vec(k, 3)[o];
                sold = P.vec(k, 4)[o];
                zold = P.vec(k, 5)[o];
                vold = P.vec(k, 6)[o];
            }
            const XRow X = pipe_x_row(first, rr, nalpha, beta, nomega, ri, wi, ti, pold, sold, zold, vold);
            si = X.s;
            zi = X.z;
            q = X.q;
            y = X.y;
            if (act) {
                if (!first)
                    V.t[i] = ti;
                V.p[i] = X.p;
                V.s[i] = X.s;
                V.z[i] = X.z;
                V.q[i] = q;
                V.y[i] = y;
            }
        }
        // (one vote for all four terms, as add_row does, needs more registers than pass X has: spills)
        const Dec dq = decode(q), dy = decode(y), dr = decode(r0i), ds = decode(si), dz = decode(zi);
        D.template add2<false>(sh, 0, q, y, dq, dy, act);
        D.template add2<true>(sh, 1, y, y, dy, dy, act);
        D.template add2<false>(sh, 2, r0i, si, dr, ds, act);
        D.template add2<false>(sh, 3, r0i, zi, dr, dz, act);
    }, claimed_tiles<MATS>(c) ? &wk->tile_next : nullptr, rr_rounds(c, A.nslices));
    grid_dep_launch();               // pass Y may take the SMs this CTA leaves
    if (!finalize<4, MODE>(D, sh, wk, c))
        return;
    if (threadIdx.x == 0)
        pipe_x_tail(c, sh.dv);
}

// Y(i) staged: v_i = A z_i, x_{i+1}, r_{i+1}, w_{i+1}; dots (r0,r), (r0,w), (r,r); beta, alpha, stop test
template <int MODE, bool MATS>
__global__ void __launch_bounds__(THREADS, PBCG_MINB(MODE, MATS))
    k_pipe_y_tma(Mat A, Vecs V, Ctl *c, Work *wk)
{
    extern __shared__ __align__(128) uint8_t dsm[];
    __shared__ Shm<3> sh;
    shm_init<3, MODE>(sh);
    grid_dep_wait();                 // pass X's merge and omega_i complete
    if (c->status != ST_RUNNING)
        return;
    const double alpha = c->alpha, omega = c->omega;
    const double nalpha = -alpha, nomega = -omega;
    DotSet<3, MODE> D;
    D.init();
    // stage slots: 0 q, 1 y, 2 p, 3 x, 4 t, 5 r0
    const double *const src[6] = {V.q, V.y, V.p, V.x, V.t, V.r0};
    tile_loop<6, MATS>(A, src, 6, V.z, c, dsm, [&](const TilePipe<6, MATS> &P, int k, int tile, int warp, int lane) {
        const int sl = tile * TILE_SLICES + warp;
        const int i = sl * 32 + lane;
        const bool act = sl < A.nslices && i < A.n;
        const int o = warp * 32 + lane;
        double rn = 0.0, wn = 0.0, r0i = 0.0;
        if (sl < A.nslices) {
            const double vi = P.spmv(k, A, warp, lane, V.z);
            const YRow Yr = pipe_y_row(alpha, omega, nalpha, nomega, P.vec(k, 0)[o], P.vec(k, 1)[o], P.vec(k, 2)[o],
                                       P.vec(k, 3)[o], P.vec(k, 4)[o], vi);
            rn = Yr.r;
            wn = Yr.w;
            r0i = P.vec(k, 5)[o];
            if (act) {
                V.x[i] = Yr.x;
                V.v[i] = vi;
                V.r[i] = rn;
                V.w[i] = wn;
            }
        }
        const Dec dr0 = decode(r0i), dr = decode(rn), dw = decode(wn);
        D.template add_row<3, false, false, true>(sh, act, r0i, rn, dr0, dr, r0i, wn, dr0, dw, rn, rn, &dr, &dr);
    }, claimed_tiles<MATS>(c) ? &wk->tile_next : nullptr, rr_rounds(c, A.nslices));
    grid_dep_launch();
    if (!finalize<3, MODE>(D, sh, wk, c))
        return;
    if (threadIdx.x == 0)
        pipe_y_tail(c, sh.dv);
}

// ---------------------------------------------------------------------------
// BiCGStab passes, staged like the p-BiCGStab passes (Algorithm 1)
// ---------------------------------------------------------------------------
// last-CTA tails shared with the unstaged passes
__device__ __forceinline__ void bicg_a_scalar(Ctl *c, double rs)
{
    c->rs = rs;
    if (c->err) {
        c->status = ST_TIMEOUT;
    } else if (!fin(rs)) {
        c->status = 3;
    } else {
        double a = __ddiv_rn(c->rho, rs);
        if (!fin(a))
            c->status = 2;
        else
            c->alpha = a;
    }
    if (c->status != ST_RUNNING)
        set_cond(c);
}

__device__ __forceinline__ void bicg_b_scalar(Ctl *c, double qy, double yy)
{
    c->qy = qy;
    c->yy = yy;
    if (c->err) {
        c->status = ST_TIMEOUT;
        set_cond(c);
    } else if (!fin(qy) || !fin(yy)) {
        c->status = 3;
        set_cond(c);
    } else {
        c->omega = (yy == 0.0) ? 0.0 : __ddiv_rn(qy, yy);
    }
}

__device__ __forceinline__ void bicg_c_scalar(Ctl *c, double rho_new, double rr)
{
    c->rho_new = rho_new;
    c->rr = rr;
    c->phase = PH_ITER;
    if (c->err) {
        c->status = ST_TIMEOUT;
    } else if (!fin(rho_new) || !fin(rr)) {
        c->status = 3;
    } else {
        c->it += 1;
        residual_step(c, rr);
    }
    set_cond(c);
}

// P(i), i >= 1: p = fma(beta, fma(-omega, s, p), r)
static __global__ void __launch_bounds__(THREADS) k_bicg_p_tma(Mat A, Vecs V, Ctl *c, Work *)
{
    grid_dep_wait();
    if (c->status != ST_RUNNING || c->it == 0)
        return;
    extern __shared__ __align__(128) uint8_t dsm[];
    const double beta = c->beta, nomega = -c->omega;
    const double *const src[3] = {V.s, V.p, V.r};
    tile_loop<3, false>(A, src, 3, nullptr, c, dsm, [&](const TilePipe<3, false> &P, int k, int tile, int warp, int lane) {
        const int sl = tile * TILE_SLICES + warp;
        const int i = sl * 32 + lane;
        const int o = warp * 32 + lane;
        if (sl < A.nslices && i < A.n)
            V.p[i] = __fma_rn(beta, __fma_rn(nomega, P.vec(k, 0)[o], P.vec(k, 1)[o]), P.vec(k, 2)[o]);
    });
    grid_dep_launch();
}

// A(i): s = A p; dot (r0, s); alpha_i
template <int MODE, bool MATS>
__global__ void __launch_bounds__(THREADS, PBCG_MINB(MODE, MATS))
    k_bicg_a_tma(Mat A, Vecs V, Ctl *c, Work *wk)
{
    extern __shared__ __align__(128) uint8_t dsm[];
    __shared__ Shm<1> sh;
    shm_init<1, MODE>(sh);
    grid_dep_wait();
    if (c->status != ST_RUNNING)
        return;
    DotSet<1, MODE> D;
    D.init();
    const double *const src[1] = {V.r0};
    tile_loop<1, MATS>(A, src, 1, V.p, c, dsm, [&](const TilePipe<1, MATS> &P, int k, int tile, int warp, int lane) {
        const int sl = tile * TILE_SLICES + warp;
        const int i = sl * 32 + lane;
        const bool act = sl < A.nslices && i < A.n;
        const int o = warp * 32 + lane;
        double si = 0.0, r0i = 0.0;
        if (sl < A.nslices) {
            si = P.spmv(k, A, warp, lane, V.p);
            r0i = P.vec(k, 0)[o];
            if (act)
                V.s[i] = si;
        }
        const Dec dr = decode(r0i), ds = decode(si);
        D.template add2<false>(sh, 0, r0i, si, dr, ds, act);
    }, claimed_tiles<MATS>(c) ? &wk->tile_next : nullptr, rr_rounds(c, A.nslices));
    grid_dep_launch();
    if (!finalize<1, MODE>(D, sh, wk, c))
        return;
    if (threadIdx.x == 0)
        bicg_a_scalar(c, sh.dv[0]);
}

// Q(i): q = r - alpha s, formed once per row as fma(-alpha, s_j, r_j), for
// pass B to gather and for passes B and C to read (alpha is known only after
// pass A).  Elementwise, two rows per thread per step.
static __global__ void __launch_bounds__(THREADS) k_bicg_q(Mat A, Vecs V, const Ctl *c)
{
    grid_dep_wait();
    grid_dep_launch();               // pass B's CTAs may become resident as these leave
    if (c->status != ST_RUNNING)
        return;
    const double nalpha = -c->alpha;
    const int n = A.n;
    const int stride = 2 * (int)(gridDim.x * blockDim.x);
    for (int i = 2 * (int)(blockIdx.x * blockDim.x + threadIdx.x); i < n; i += stride) {
        // (vectors are 16-byte aligned and padded to whole tiles: i + 1 is in the allocation)
        const double2 sv = *reinterpret_cast<const double2 *>(V.s + i);
        const double2 rv = *reinterpret_cast<const double2 *>(V.r + i);
        if (i + 1 < n) {
            *reinterpret_cast<double2 *>(V.q + i) = make_double2(__fma_rn(nalpha, sv.x, rv.x), __fma_rn(nalpha, sv.y, rv.y));
        } else {
            V.q[i] = __fma_rn(nalpha, sv.x, rv.x);
        }
    }
}

// B(i): y = A q (q from pass Q); dots (q,y), (y,y); omega_i
template <int MODE, bool MATS>
__global__ void __launch_bounds__(THREADS, PBCG_MINB(MODE, MATS))
    k_bicg_b_tma(Mat A, Vecs V, Ctl *c, Work *wk)
{
    extern __shared__ __align__(128) uint8_t dsm[];
    __shared__ Shm<2> sh;
    shm_init<2, MODE>(sh);
    grid_dep_wait();
    if (c->status != ST_RUNNING)
        return;
    DotSet<2, MODE> D;
    D.init();
    const double *const src[1] = {V.q};
    tile_loop<1, MATS>(A, src, 1, V.q, c, dsm, [&](const TilePipe<1, MATS> &P, int k, int tile, int warp, int lane) {
        const int sl = tile * TILE_SLICES + warp;
        const int i = sl * 32 + lane;
        const bool act = sl < A.nslices && i < A.n;
        const int o = warp * 32 + lane;
        double qi = 0.0, yi = 0.0;
        if (sl < A.nslices) {
            yi = P.spmv(k, A, warp, lane, V.q);
            qi = P.vec(k, 0)[o];
            if (act)
                V.y[i] = yi;
        }
        const Dec dq = decode(qi), dy = decode(yi);
        D.template add_row<2, false, true>(sh, act, qi, yi, dq, dy, yi, yi, dy, dy);
    }, claimed_tiles<MATS>(c) ? &wk->tile_next : nullptr, rr_rounds(c, A.nslices));
    grid_dep_launch();
    if (!finalize<2, MODE>(D, sh, wk, c))
        return;
    if (threadIdx.x == 0)
        bicg_b_scalar(c, sh.dv[0], sh.dv[1]);
}

// C(i): x, r updates; dots (r0,r), (r,r); beta_i, stop test
template <int MODE>
__global__ void __launch_bounds__(THREADS, MODE ? PBCG_MINB_EXACT : PBCG_MINB_PLAIN)
    k_bicg_c_tma(Mat A, Vecs V, Ctl *c, Work *wk)
{
    extern __shared__ __align__(128) uint8_t dsm[];
    __shared__ Shm<2> sh;
    shm_init<2, MODE>(sh);
    grid_dep_wait();
    if (c->status != ST_RUNNING)
        return;
    const double alpha = c->alpha, omega = c->omega;
    const double nomega = -omega;
    DotSet<2, MODE> D;
    D.init();
    // stage slots: 0 q, 1 p, 2 x, 3 y, 4 r0
    const double *const src[5] = {V.q, V.p, V.x, V.y, V.r0};
    tile_loop<5, false>(A, src, 5, nullptr, c, dsm, [&](const TilePipe<5, false> &P, int k, int tile, int warp, int lane) {
        const int sl = tile * TILE_SLICES + warp;
        const int i = sl * 32 + lane;
        const bool act = sl < A.nslices && i < A.n;
        const int o = warp * 32 + lane;
        double rn = 0.0, r0i = 0.0;
        if (act) {
            const double q = P.vec(k, 0)[o];
            V.x[i] = __fma_rn(omega, q, __fma_rn(alpha, P.vec(k, 1)[o], P.vec(k, 2)[o]));
            rn = __fma_rn(nomega, P.vec(k, 3)[o], q);
            V.r[i] = rn;
            r0i = P.vec(k, 4)[o];
        }
        const Dec dr0 = decode(r0i), dr = decode(rn);
        D.template add_row<2, false, true>(sh, act, r0i, rn, dr0, dr, rn, rn, dr, dr);
    });
    grid_dep_launch();
    if (!finalize<2, MODE>(D, sh, wk, c))
        return;
    if (threadIdx.x == 0)
        bicg_c_scalar(c, sh.dv[0], sh.dv[1]);
}

}  // namespace pbcg
