// dist.cuh -- device side of the row-partitioned solve.
//
// Section 2 of arXiv 2404.13216 runs BiCGStab and p-BiCGStab over MPI
// processes that each own a block of rows; the dots are global reductions,
// and with ExBLAS their results (hence the iteration counts, Tables 2 and 3)
// do not depend on the number of processes.  Here each rank is one GPU grid
// running the ordinary passes on its row block.  At every reduction point the
// passes' last CTA leaves the rank's share in the merge workspace (exact: the
// integer digits of the superaccumulator; plain: the rank's partial sums,
// finalize() with Work::dist set), the host adds the ranks' shares with one
// collective, and k_dist_finish rounds the total once -- the same integer sum
// a single grid would have formed, so every rank rounds to the same double --
// and takes the scalar step of that point.  SpMV inputs owned by other ranks
// (the halo) are copied in before each pass that gathers them; k_halo_pack
// gathers the entries this rank sends.
#pragma once
#include "kernels.cuh"

namespace pbcg {

// which scalar step follows a reduction point of a partitioned solve
enum : int {
    FIN_SETUP1_P = 0,   // p-BiCGStab setup 1: (b,b), (r0,r0) stored
    FIN_SETUP1_B = 1,   // BiCGStab setup: (b,b), (r0,r0), stop test
    FIN_SETUP2 = 2,     // p-BiCGStab setup 2: (r0,w0), alpha_0, stop test
    FIN_X = 3,          // p-BiCGStab pass X: omega
    FIN_Y = 4,          // p-BiCGStab pass Y: beta, alpha, stop test
    FIN_BA = 5,         // BiCGStab pass A: alpha
    FIN_BB = 6,         // BiCGStab pass B: omega
    FIN_BC = 7,         // BiCGStab pass C: beta, stop test
    FIN_TRUE = 8        // true residual: resolves a candidate stop
};

// Reduction buffer of one point, int64 words, as the host hands it over:
//   red[0]: number of ranks whose bounded waits expired;
//   exact: then, per dot d < nd, NDIG digits (the ranks' carry-save digits
//          added as integers) and the count of ranks that saw a NaN or Inf;
//   plain: then nranks * nd doubles (bit patterns), rank r's dot d at r*nd + d.
constexpr int RED_EXACT_STRIDE = NDIG + 1;

// One CTA.  The total of each dot is written into the (otherwise cleared)
// global accumulator and rounded by the same routine a single grid uses, or,
// in plain mode, the ranks' sums are added in rank order; thread 0 then takes
// the scalar step `which`.
template <int MODE>
__global__ void __launch_bounds__(THREADS) k_dist_finish(Ctl *c, Work *wk, const long long *red, int nd, int nranks,
                                                         int which)
{
    __shared__ Shm<MAXD> sh;
    __shared__ int lo[MAXD], hi[MAXD];
    if (MODE == 1) {
        if (threadIdx.x < MAXD) {
            lo[threadIdx.x] = NDIG;
            hi[threadIdx.x] = -1;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < MAXD * NDIG; i += THREADS) {
            const int d = i / NDIG, k = i % NDIG;
            const long long v = d < nd ? red[1 + d * RED_EXACT_STRIDE + k] : 0ll;
            wk->g[d].dig[k] = (unsigned long long)v;
            if (v != 0ll) {
                atomicMin(&lo[d], k);
                atomicMax(&hi[d], k);
            }
        }
        __syncthreads();
        if (threadIdx.x < MAXD) {
            const int d = threadIdx.x;
            wk->g[d].kmin = lo[d];
            wk->g[d].kmax = hi[d];
            wk->g[d].nf = (d < nd && red[1 + d * RED_EXACT_STRIDE + NDIG] != 0ll) ? 1 : 0;
        }
        __threadfence_block();
        gacc_round_reset_cta<MAXD>(wk->g, sh.acc, sh.scratch, sh.dv);
    } else {
        if (threadIdx.x < nd) {
            double v = 0.0;
            for (int r = 0; r < nranks; r++)
                v = __dadd_rn(v, __longlong_as_double(red[1 + r * nd + threadIdx.x]));
            sh.dv[threadIdx.x] = v;
        }
        __syncthreads();
    }
    if (threadIdx.x != 0)
        return;
    if (red[0] != 0ll)
        c->err = 1;
    const double *dv = sh.dv;
    switch (which) {
    case FIN_SETUP1_P:
        c->bb = dv[0];
        c->rho = dv[1];
        break;
    case FIN_SETUP1_B:
        setup_scalar(c, dv[0], dv[1], 0.0);
        break;
    case FIN_SETUP2:
        setup_scalar(c, c->bb, c->rho, dv[0]);
        break;
    case FIN_X:
        pipe_x_tail(c, dv);
        break;
    case FIN_Y:
        pipe_y_tail(c, dv);
        break;
    case FIN_BA:
        bicg_a_scalar(c, dv[0]);
        break;
    case FIN_BB:
        bicg_b_scalar(c, dv[0], dv[1]);
        break;
    case FIN_BC:
        bicg_c_scalar(c, dv[0], dv[1]);
        break;
    default:
        true_res_tail(c, dv);
        break;
    }
    if (c->err && c->status == ST_RUNNING)
        c->status = ST_TIMEOUT;
}

// out[j] = v[idx[j]]: the entries of a solver vector that other ranks gather
static __global__ void k_halo_pack(int m, const int *__restrict__ idx, const double *__restrict__ v, double *out)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x)
        out[j] = v[idx[j]];
}

}  // namespace pbcg
