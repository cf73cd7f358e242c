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
#pragma once
#include "exdot.cuh"

namespace pbcg {

constexpr int THREADS = 256;
constexpr int WARPS = THREADS / 32;
constexpr int MAXD = 4;                 // most dots merged in one pass

enum : int { ST_RUNNING = 100, ST_CANDIDATE = 101 };
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
    int alg, use_cond, pad_i0, pad_i1;
    unsigned long long cond;            // cudaGraphConditionalHandle of the loop
    double *hist;
    int hist_cap, pad_i2;
};

// grid-wide merge workspace
struct Work {
    GAcc g[MAXD];
    unsigned int ticket;
    int maxgrid;
    double *part;                        // plain partials [MAXD][maxgrid]
};

struct Csr {
    int n;
    const int *__restrict__ rp;
    const int *__restrict__ ci;
    const double *__restrict__ va;
};

struct Vecs {
    double *x, *b, *r0, *r, *w, *t, *p, *s, *z, *v, *y;
};

__device__ __forceinline__ bool fin(double v)
{
    return ((unsigned long long)__double_as_longlong(v) & 0x7ff0000000000000ull) != 0x7ff0000000000000ull;
}

// SpMV row: acc = +0; acc = fma(val_k, x[col_k], acc) in stored order
__device__ __forceinline__ double spmv_row(const Csr &A, const double *__restrict__ x, int i)
{
    int k0 = __ldg(A.rp + i), k1 = __ldg(A.rp + i + 1);
    double acc = 0.0;
    for (int k = k0; k < k1; k++)
        acc = __fma_rn(__ldg(A.va + k), __ldg(x + __ldg(A.ci + k)), acc);
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
    Win win[ND];
    double s[ND];
    bool nf[ND];

    __device__ __forceinline__ void init()
    {
#pragma unroll
        for (int d = 0; d < ND; d++) {
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
};

template <int ND, int MODE>
__device__ __forceinline__ void shm_init(Shm<ND> &sh)
{
    if (MODE == 1)
        cta_acc_init<ND>(sh.acc);
    if (threadIdx.x == 0)
        sh.last = 0;
}

// Merge the CTA's dots grid-wide.  Returns true in the last CTA, whose
// sh.dv[] then holds the finished dot values.  Called by every thread.
template <int ND, int MODE>
__device__ bool finalize(DotSet<ND, MODE> &D, Shm<ND> &sh, Work *wk)
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
#pragma unroll
        for (int d = 0; d < ND; d++) {
            double v = D.s[d];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
                v = __dadd_rn(v, __shfl_xor_sync(0xffffffffu, v, o));
            if (lane == 0)
                sh.wpart[d][warp] = v;
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
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int t = atomicAdd(&wk->ticket, 1u);
        sh.last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!sh.last)
        return false;
    __threadfence();
    if (MODE == 1) {
        if (threadIdx.x < ND)
            sh.dv[threadIdx.x] = gacc_round_reset(&wk->g[threadIdx.x], sh.scratch[threadIdx.x]);
    } else if (warp < ND) {
        const double *pp = wk->part + warp * wk->maxgrid;
        double v = 0.0;
        for (int c = lane; c < (int)gridDim.x; c += 32)
            v = __dadd_rn(v, __ldcg(pp + c));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            v = __dadd_rn(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (lane == 0)
            sh.dv[warp] = v;
    }
    if (threadIdx.x == 0)
        wk->ticket = 0u;
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
__device__ void post_stop(Ctl *c)
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
__device__ void residual_step(Ctl *c, double rr)
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
__device__ void setup_scalar(Ctl *c, double bb, double rho, double rw)
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

// ---------------------------------------------------------------------------
// grid mapping: warp-uniform 32-row tiles, strided over all warps of the grid
// ---------------------------------------------------------------------------
#define PBCG_TILE_LOOP(n)                                                                    \
    const int lane_ = threadIdx.x & 31;                                                      \
    const int gwarp_ = (blockIdx.x * THREADS + threadIdx.x) >> 5;                            \
    const int nwarps_ = (gridDim.x * THREADS) >> 5;                                          \
    const int ntiles_ = ((n) + 31) >> 5;                                                     \
    for (int tile_ = gwarp_; tile_ < ntiles_; tile_ += nwarps_)

#define PBCG_ROW (tile_ * 32 + lane_)

// ---------------------------------------------------------------------------
// setup passes
// ---------------------------------------------------------------------------
// S1: r0 = b - A x0, r = r0 (and p = r0 for BiCGStab); dots (b,b), (r0,r0)
template <int MODE>
__global__ void __launch_bounds__(THREADS) k_setup1(Csr A, Vecs V, Ctl *c, Work *wk)
{
    __shared__ Shm<2> sh;
    shm_init<2, MODE>(sh);
    __syncthreads();
    const bool bicg = c->alg == ALG_BICGSTAB;
    DotSet<2, MODE> D;
    D.init();
    PBCG_TILE_LOOP(A.n)
    {
        int i = PBCG_ROW;
        bool act = i < A.n;
        double bi = 0.0, r0i = 0.0;
        if (act) {
            bi = V.b[i];
            r0i = __dsub_rn(bi, spmv_row(A, V.x, i));
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
__global__ void __launch_bounds__(THREADS) k_setup2(Csr A, Vecs V, Ctl *c, Work *wk)
{
    __shared__ Shm<1> sh;
    shm_init<1, MODE>(sh);
    __syncthreads();
    DotSet<1, MODE> D;
    D.init();
    PBCG_TILE_LOOP(A.n)
    {
        int i = PBCG_ROW;
        bool act = i < A.n;
        double r0i = 0.0, wi = 0.0;
        if (act) {
            r0i = V.r0[i];
            wi = spmv_row(A, V.r0, i);
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
__global__ void __launch_bounds__(THREADS) k_setup3(Csr A, Vecs V, const Ctl *c)
{
    if (c->status != ST_RUNNING && c->status != ST_CANDIDATE)
        return;
    PBCG_TILE_LOOP(A.n)
    {
        int i = PBCG_ROW;
        if (i < A.n)
            V.t[i] = spmv_row(A, V.w, i);
    }
}

// ---------------------------------------------------------------------------
// p-BiCGStab passes
// ---------------------------------------------------------------------------
// X(i): t_i = A w_i (i >= 1), p_i, s_i, z_i, q_i, y_i; dots (q,y), (y,y), (r0,s), (r0,z); omega_i
template <int MODE>
__global__ void __launch_bounds__(THREADS) k_pipe_x(Csr A, Vecs V, Ctl *c, Work *wk)
{
    if (c->status != ST_RUNNING)
        return;
    __shared__ Shm<4> sh;
    shm_init<4, MODE>(sh);
    __syncthreads();
    const bool first = (c->it == 0);
    const double alpha = c->alpha, beta = c->beta, omega = c->omega;
    const double nalpha = -alpha, nomega = -omega;
    DotSet<4, MODE> D;
    D.init();
    PBCG_TILE_LOOP(A.n)
    {
        int i = PBCG_ROW;
        bool act = i < A.n;
        double q = 0.0, y = 0.0, r0i = 0.0, si = 0.0, zi = 0.0;
        if (act) {
            double ri = V.r[i], wi = V.w[i];
            double pi, ti;
            r0i = V.r0[i];
            if (first) {
                ti = V.t[i];
                pi = ri;
                si = wi;
                zi = ti;
            } else {
                ti = spmv_row(A, V.w, i);
                pi = __fma_rn(beta, __fma_rn(nomega, V.s[i], V.p[i]), ri);
                si = __fma_rn(beta, __fma_rn(nomega, V.z[i], V.s[i]), wi);
                zi = __fma_rn(beta, __fma_rn(nomega, V.v[i], V.z[i]), ti);
                V.t[i] = ti;
            }
            V.p[i] = pi;
            V.s[i] = si;
            V.z[i] = zi;
            q = __fma_rn(nalpha, si, ri);
            y = __fma_rn(nalpha, zi, wi);
        }
        D.add(sh, 0, q, y, act);
        D.add(sh, 1, y, y, act);
        D.add(sh, 2, r0i, si, act);
        D.add(sh, 3, r0i, zi, act);
    }
    if (!finalize<4, MODE>(D, sh, wk))
        return;
    if (threadIdx.x == 0) {
        double qy = sh.dv[0], yy = sh.dv[1];
        c->qy = qy;
        c->yy = yy;
        c->rs = sh.dv[2];
        c->rz = sh.dv[3];
        if (!fin(qy) || !fin(yy)) {
            c->status = 3;
            set_cond(c);
        } else {
            c->omega = (yy == 0.0) ? 0.0 : __ddiv_rn(qy, yy);
        }
    }
}

// Y(i): v_i = A z_i, x_{i+1}, r_{i+1}, w_{i+1}; dots (r0,r), (r0,w), (r,r); beta_i, alpha_{i+1}, stop test
template <int MODE>
__global__ void __launch_bounds__(THREADS) k_pipe_y(Csr A, Vecs V, Ctl *c, Work *wk)
{
    if (c->status != ST_RUNNING)
        return;
    __shared__ Shm<3> sh;
    shm_init<3, MODE>(sh);
    __syncthreads();
    const double alpha = c->alpha, omega = c->omega;
    const double nalpha = -alpha, nomega = -omega;
    DotSet<3, MODE> D;
    D.init();
    PBCG_TILE_LOOP(A.n)
    {
        int i = PBCG_ROW;
        bool act = i < A.n;
        double rn = 0.0, wn = 0.0, r0i = 0.0;
        if (act) {
            double vi = spmv_row(A, V.z, i);
            double ri = V.r[i], si = V.s[i], wi = V.w[i], zi = V.z[i];
            double q = __fma_rn(nalpha, si, ri);
            double y = __fma_rn(nalpha, zi, wi);
            V.x[i] = __fma_rn(omega, q, __fma_rn(alpha, V.p[i], V.x[i]));
            rn = __fma_rn(nomega, y, q);
            wn = __fma_rn(nomega, __fma_rn(nalpha, vi, V.t[i]), y);
            r0i = V.r0[i];
            V.v[i] = vi;
            V.r[i] = rn;
            V.w[i] = wn;
        }
        D.add(sh, 0, r0i, rn, act);
        D.add(sh, 1, r0i, wn, act);
        D.add(sh, 2, rn, rn, act);
    }
    if (!finalize<3, MODE>(D, sh, wk))
        return;
    if (threadIdx.x == 0) {
        double rho_new = sh.dv[0], rw = sh.dv[1], rr = sh.dv[2];
        c->rho_new = rho_new;
        c->rw = rw;
        c->rr = rr;
        c->phase = PH_ITER;
        if (!fin(rho_new) || !fin(rw) || !fin(c->rs) || !fin(c->rz) || !fin(rr)) {
            c->status = 3;
        } else {
            c->it += 1;
            residual_step(c, rr);
        }
        set_cond(c);
    }
}

// ---------------------------------------------------------------------------
// BiCGStab passes
// ---------------------------------------------------------------------------
// P(i), i >= 1: p = fma(beta, fma(-omega, s, p), r)
__global__ void __launch_bounds__(THREADS) k_bicg_p(Csr A, Vecs V, const Ctl *c)
{
    if (c->status != ST_RUNNING || c->it == 0)
        return;
    const double beta = c->beta, nomega = -c->omega;
    PBCG_TILE_LOOP(A.n)
    {
        int i = PBCG_ROW;
        if (i < A.n)
            V.p[i] = __fma_rn(beta, __fma_rn(nomega, V.s[i], V.p[i]), V.r[i]);
    }
}

// A(i): s = A p; dot (r0, s); alpha_i
template <int MODE>
__global__ void __launch_bounds__(THREADS) k_bicg_a(Csr A, Vecs V, Ctl *c, Work *wk)
{
    if (c->status != ST_RUNNING)
        return;
    __shared__ Shm<1> sh;
    shm_init<1, MODE>(sh);
    __syncthreads();
    DotSet<1, MODE> D;
    D.init();
    PBCG_TILE_LOOP(A.n)
    {
        int i = PBCG_ROW;
        bool act = i < A.n;
        double si = 0.0, r0i = 0.0;
        if (act) {
            si = spmv_row(A, V.p, i);
            V.s[i] = si;
            r0i = V.r0[i];
        }
        D.add(sh, 0, r0i, si, act);
    }
    if (!finalize<1, MODE>(D, sh, wk))
        return;
    if (threadIdx.x == 0) {
        double rs = sh.dv[0];
        c->rs = rs;
        if (!fin(rs)) {
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
}

// B(i): y = A q with q_j = fma(-alpha, s_j, r_j) formed in the gather; dots (q,y), (y,y); omega_i
template <int MODE>
__global__ void __launch_bounds__(THREADS) k_bicg_b(Csr A, Vecs V, Ctl *c, Work *wk)
{
    if (c->status != ST_RUNNING)
        return;
    __shared__ Shm<2> sh;
    shm_init<2, MODE>(sh);
    __syncthreads();
    const double nalpha = -c->alpha;
    DotSet<2, MODE> D;
    D.init();
    PBCG_TILE_LOOP(A.n)
    {
        int i = PBCG_ROW;
        bool act = i < A.n;
        double qi = 0.0, yi = 0.0;
        if (act) {
            int k0 = __ldg(A.rp + i), k1 = __ldg(A.rp + i + 1);
            double acc = 0.0;
            for (int k = k0; k < k1; k++) {
                int j = __ldg(A.ci + k);
                double qj = __fma_rn(nalpha, __ldg(V.s + j), __ldg(V.r + j));
                acc = __fma_rn(__ldg(A.va + k), qj, acc);
            }
            yi = acc;
            qi = __fma_rn(nalpha, V.s[i], V.r[i]);
            V.y[i] = yi;
        }
        D.add(sh, 0, qi, yi, act);
        D.add(sh, 1, yi, yi, act);
    }
    if (!finalize<2, MODE>(D, sh, wk))
        return;
    if (threadIdx.x == 0) {
        double qy = sh.dv[0], yy = sh.dv[1];
        c->qy = qy;
        c->yy = yy;
        if (!fin(qy) || !fin(yy)) {
            c->status = 3;
            set_cond(c);
        } else {
            c->omega = (yy == 0.0) ? 0.0 : __ddiv_rn(qy, yy);
        }
    }
}

// C(i): x, r updates; dots (r0,r), (r,r); beta_i, stop test
template <int MODE>
__global__ void __launch_bounds__(THREADS) k_bicg_c(Csr A, Vecs V, Ctl *c, Work *wk)
{
    if (c->status != ST_RUNNING)
        return;
    __shared__ Shm<2> sh;
    shm_init<2, MODE>(sh);
    __syncthreads();
    const double alpha = c->alpha, omega = c->omega;
    const double nalpha = -alpha, nomega = -omega;
    DotSet<2, MODE> D;
    D.init();
    PBCG_TILE_LOOP(A.n)
    {
        int i = PBCG_ROW;
        bool act = i < A.n;
        double rn = 0.0, r0i = 0.0;
        if (act) {
            double q = __fma_rn(nalpha, V.s[i], V.r[i]);
            V.x[i] = __fma_rn(omega, q, __fma_rn(alpha, V.p[i], V.x[i]));
            rn = __fma_rn(nomega, V.y[i], q);
            V.r[i] = rn;
            r0i = V.r0[i];
        }
        D.add(sh, 0, r0i, rn, act);
        D.add(sh, 1, rn, rn, act);
    }
    if (!finalize<2, MODE>(D, sh, wk))
        return;
    if (threadIdx.x == 0) {
        double rho_new = sh.dv[0], rr = sh.dv[1];
        c->rho_new = rho_new;
        c->rr = rr;
        c->phase = PH_ITER;
        if (!fin(rho_new) || !fin(rr)) {
            c->status = 3;
        } else {
            c->it += 1;
            residual_step(c, rr);
        }
        set_cond(c);
    }
}

// ---------------------------------------------------------------------------
// true residual ||b - A x|| / ||b|| with exact dots; resolves a candidate stop
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(THREADS) k_true_res(Csr A, Vecs V, Ctl *c, Work *wk)
{
    __shared__ Shm<2> sh;
    shm_init<2, 1>(sh);
    __syncthreads();
    DotSet<2, 1> D;
    D.init();
    PBCG_TILE_LOOP(A.n)
    {
        int i = PBCG_ROW;
        bool act = i < A.n;
        double ri = 0.0, bi = 0.0;
        if (act) {
            bi = V.b[i];
            ri = __dsub_rn(bi, spmv_row(A, V.x, i));
        }
        D.add(sh, 0, ri, ri, act);
        D.add(sh, 1, bi, bi, act);
    }
    if (!finalize<2, 1>(D, sh, wk))
        return;
    if (threadIdx.x == 0) {
        double nb = __dsqrt_rn(sh.dv[1]);
        if (nb == 0.0)
            nb = 1.0;
        double tr = __ddiv_rn(__dsqrt_rn(sh.dv[0]), nb);
        c->trueres = tr;
        c->bbx = sh.dv[1];
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
}

// ---------------------------------------------------------------------------
// standalone kernels: dot and SpMV
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
    const long long gw = ((long long)blockIdx.x * THREADS + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * THREADS) >> 5;
    const long long nt = (n + 31) >> 5;
    for (long long t = gw; t < nt; t += nw) {
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

__global__ void __launch_bounds__(THREADS) k_spmv(Csr A, const double *x, double *y)
{
    PBCG_TILE_LOOP(A.n)
    {
        int i = PBCG_ROW;
        if (i < A.n)
            y[i] = spmv_row(A, x, i);
    }
}

}  // namespace pbcg
