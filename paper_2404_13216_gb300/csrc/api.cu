// api.cu -- host driver and C ABI of libpbcg (declared in include/pbcg.h).
//
// A solve is: setup passes (r_0, w_0, t_0 and their dots), then the loop of
// Algorithm 1 or 2 as a CUDA graph whose body, inside a conditional WHILE
// node, is LOOP_UNROLL iterations of the fused passes; the last CTA of each
// iteration sets the node's condition, so the device iterates without host
// round trips.  The host wakes up only
// when the device proposes to stop (residual below target), runs the
// true-residual pass, and either finishes or relaunches the loop.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <set>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>
#include "../../include/pbcg.h"
#include "batched.cuh"
#include "cluster.cuh"
#include "dist.cuh"

using namespace pbcg;

namespace {

enum { V_X, V_B, V_R0, V_R, V_W, V_T, V_P, V_S, V_Z, V_V, V_Y, V_Q, V_TMP, V_COUNT };

struct LoopGraph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphConditionalHandle handle = 0;
    int alg = -1, mode = -1, n = -1;
    bool jac = false;                  // built on the Jacobi-scaled entries
    const void *mat = nullptr;
    int var = -1;                      // launch variant it was built for (staged, order, CTAs per SM)
    int unroll = 1;                    // iterations per execution of the WHILE body
};

struct Workspace {
    long long n_cap = 0;
    int hist_cap = 0;
    double *vec[V_COUNT] = {};
    Ctl *ctl = nullptr;
    Work *wk = nullptr;
    double *part = nullptr;
    double *hist = nullptr;
    double *dot_out = nullptr;
    bool base_ready = false;       // ctl, wk, part, dot_out allocated and wk initialised
    LoopGraph loop;
};

}  // namespace

// NVTX range around a public call or a host-driven launch (a no-op unless a
// profiler is attached)
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

struct pbcg_mat {
    int n;
    int ncols;             // columns: n, or n plus the halo of a partition block
    long long nnz;
    int nslices;
    long long padded;      // stored SELL-32 entries (nnz plus padding)
    int *sl_off;           // [nslices + 1]
    int *rlen;             // [nslices * 32]
    int *ci;               // [padded], solver-order column indices
    double *va;            // [padded]
    int *perm;             // [n] solver row p holds caller row perm[p]; NULL when rows keep their order
    uint16_t *lci;         // [padded] local column indices into a tile's staged gather blocks
    int *tmeta;            // [ntiles * TMETA] per tile: first and end entry, gather blocks (-1: none / too many)
    bool narrow;           // every 256-row tile spans at most MCAP SELL entries (staged in shared memory)
    double *diag = nullptr;    // [n] solver-order diagonal for Jacobi preconditioning (built on first use)
    double *va_jac = nullptr;  // [padded] entries of A M^-1, M = diag(A)
    std::vector<int32_t> h_rp, h_ci;   // host copy of the CSR (for per-batch layouts)
    std::vector<int> h_sloff;          // [nslices + 1] host copy of sl_off
    std::vector<double> h_va;
    struct BatchLayout *bl;            // tile-aligned layout of the last batched solve, or NULL
    // launch variant of pbcg_solve's passes (pbcg_set_variant / pbcg_tune); none changes exact results
    int v_staged = 1;                  // stage tiles in shared memory when they fit (narrow matrices)
    int v_order = 0;                   // tile order: 0 default, 1 round-robin, 2 claimed, 3 round-robin + claimed tail
    int v_ctas = 0;                    // resident CTAs per SM of the passes (0: as many as fit)
    int b_ctas = 0;                    // same, batched passes
    double v_us = 0.0;                 // time per iteration pbcg_tune measured for it
};

// a block-diagonal matrix laid out with every system padded to whole 256-row tiles
struct BatchLayout {
    std::vector<int32_t> key;          // the sys_row_ptr it was built for
    int nsys = 0, n_int = 0, nslices = 0, ntiles = 0;
    int *sl_off = nullptr, *rlen = nullptr, *ci = nullptr;
    double *va = nullptr;
    int *map = nullptr;                // [n_int] caller row of each internal row, -1 for padding
    int *tile_sys = nullptr, *sys_t0 = nullptr;
    bool jac = false;                  // entries of A M^-1 (Jacobi)
    double *diag = nullptr;            // [n_int] internal-order diagonal when jac (1 on padding rows)
};

struct pbcg_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int num_sms = 0;
    int maxgrid = 0;
    std::string err;
    Workspace ws;
    std::set<pbcg_mat *> mats;
    std::vector<double> hist;          // last single solve
    bool have_hist = false;
    Ctl *h_ctl = nullptr;              // pinned mirror of the control block
    std::map<const void *, int> occ;   // resident CTAs per SM of each kernel
    int rr_period = 50;                // residual replacement period of PBCG_ALG_PIPELINED_RR
    int precond = PBCG_PRECOND_NONE;   // preconditioner of pbcg_solve
    int small_cluster = 1;             // Algorithm 2 on small systems as one cluster launch
    int batch_graph = 1;               // batched solves loop in a CUDA graph (0: host-driven launches)
    std::map<long long, bool> cl_ok;   // cluster shapes (kernel, CTAs, shared memory) that can be resident
    // batched solves
    struct {
        long long n_cap = 0;
        int nsys_cap = 0, ntiles_cap = 0;
        long long hist_cap = 0;
        double *vec[13] = {};
        Ctl *ctl = nullptr;
        GAcc *acc = nullptr;
        double *part = nullptr;
        unsigned *done = nullptr;
        int *flag = nullptr;
        double *hist = nullptr;
        double *io = nullptr;          // caller-order staging of b and x
        long long io_cap = 0;
        cudaGraphExec_t exec = nullptr;
        cudaGraph_t graph = nullptr;
        const void *g_layout = nullptr;
        int g_alg = -1, g_mode = -1, g_ctas = 0;
        std::vector<Ctl> last;         // per-system control blocks of the last batched solve
        int hist_stride = 0;
    } b;
    bool last_batched = false;
};

namespace {

int fail(pbcg_ctx *c, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c)
        c->err = buf;
    return code;
}

#define CK(call)                                                                                     \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess)                                                                       \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? PBCG_ERR_OOM : PBCG_ERR_CUDA,          \
                        "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

Mat mat_of(const pbcg_mat *m)
{
    Mat A;
    A.n = m->n;
    A.ncols = m->ncols;
    A.nslices = m->nslices;
    A.sl_off = m->sl_off;
    A.rlen = m->rlen;
    A.ci = m->ci;
    A.va = m->va;
    A.sl_w = nullptr;
    A.lci = m->lci;
    A.tmeta = m->tmeta;
    return A;
}

void layout_release(BatchLayout *L)
{
    if (!L)
        return;
    cudaFree(L->sl_off);
    cudaFree(L->rlen);
    cudaFree(L->ci);
    cudaFree(L->va);
    cudaFree(L->map);
    cudaFree(L->tile_sys);
    cudaFree(L->sys_t0);
    delete L;
}

void mat_release(pbcg_mat *m)
{
    layout_release(m->bl);
    cudaFree(m->sl_off);
    cudaFree(m->rlen);
    cudaFree(m->ci);
    cudaFree(m->va);
    cudaFree(m->perm);
    cudaFree(m->lci);
    cudaFree(m->tmeta);
    cudaFree(m->diag);
    cudaFree(m->va_jac);
    delete m;
}

Vecs vecs_of(Workspace &ws)
{
    Vecs V;
    V.x = ws.vec[V_X];
    V.b = ws.vec[V_B];
    V.r0 = ws.vec[V_R0];
    V.r = ws.vec[V_R];
    V.w = ws.vec[V_W];
    V.t = ws.vec[V_T];
    V.p = ws.vec[V_P];
    V.s = ws.vec[V_S];
    V.z = ws.vec[V_Z];
    V.v = ws.vec[V_V];
    V.y = ws.vec[V_Y];
    V.q = ws.vec[V_Q];
    return V;
}

// persistent grid: every CTA resident (occupancy of this kernel x SMs), at least one slice per warp
int grid_for(pbcg_ctx *ctx, const void *fn, long long nslices, size_t smem = 0, int cap = 0)
{
    int per_sm = 0;
    auto it = ctx->occ.find(fn);
    if (it != ctx->occ.end()) {
        per_sm = it->second;
    } else {
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, THREADS, smem) != cudaSuccess || per_sm < 1)
            per_sm = 1;
        cudaGetLastError();
        ctx->occ[fn] = per_sm;
    }
    if (cap > 0 && cap < per_sm)
        per_sm = cap;
    long long g = (long long)per_sm * ctx->num_sms;
    long long need = (nslices + WARPS - 1) / WARPS;
    if (g > need)
        g = need;
    if (g > ctx->maxgrid)
        g = ctx->maxgrid;
    if (g < 1)
        g = 1;
    return (int)g;
}

void free_loop(LoopGraph &L)
{
    if (L.exec)
        cudaGraphExecDestroy(L.exec);
    if (L.graph)
        cudaGraphDestroy(L.graph);
    L = LoopGraph();
}

void free_ws(Workspace &ws)
{
    free_loop(ws.loop);
    for (auto &p : ws.vec) {
        if (p)
            cudaFree(p);
        p = nullptr;
    }
    if (ws.ctl)
        cudaFree(ws.ctl);
    if (ws.wk)
        cudaFree(ws.wk);
    if (ws.part)
        cudaFree(ws.part);
    if (ws.hist)
        cudaFree(ws.hist);
    if (ws.dot_out)
        cudaFree(ws.dot_out);
    ws = Workspace();
}

// make sure workspace ws holds n-vectors and a history of hist_cap entries
int ensure_ws_in(pbcg_ctx *ctx, Workspace &ws, long long n, int hist_cap)
{
    if (!ws.base_ready) {
        // each buffer is taken only if missing, so a call after an allocation
        // failure completes the set instead of running with a null one
        if (!ws.ctl)
            CK(cudaMalloc(&ws.ctl, sizeof(Ctl)));
        if (!ws.wk)
            CK(cudaMalloc(&ws.wk, sizeof(Work)));
        if (!ws.part)
            CK(cudaMalloc(&ws.part, sizeof(double) * MAXD * ctx->maxgrid));
        if (!ws.dot_out)
            CK(cudaMalloc(&ws.dot_out, sizeof(double)));
        Work h;
        memset(&h, 0, sizeof h);
        for (int d = 0; d < MAXD; d++) {
            h.g[d].kmin = NDIG;
            h.g[d].kmax = -1;
        }
        h.ticket = 0;
        h.maxgrid = ctx->maxgrid;
        h.part = ws.part;
        CK(cudaMemcpy(ws.wk, &h, sizeof h, cudaMemcpyHostToDevice));
        ws.base_ready = true;
    }
    if (n > ws.n_cap) {
        free_loop(ws.loop);
        for (auto &p : ws.vec) {
            if (p)
                cudaFree(p);
            p = nullptr;
        }
        ws.n_cap = 0;
        const size_t npad = (size_t)((n + TILE_ROWS - 1) / TILE_ROWS) * TILE_ROWS;
        for (auto &p : ws.vec) {
            CK(cudaMalloc(&p, sizeof(double) * npad));
            CK(cudaMemset(p, 0, sizeof(double) * npad));
        }
        ws.n_cap = n;
    }
    if (hist_cap > ws.hist_cap) {
        if (ws.hist)
            cudaFree(ws.hist);
        ws.hist = nullptr;
        ws.hist_cap = 0;
        CK(cudaMalloc(&ws.hist, sizeof(double) * (size_t)hist_cap));
        ws.hist_cap = hist_cap;
    }
    return 0;
}

int ensure_ws(pbcg_ctx *ctx, long long n, int hist_cap)
{
    return ensure_ws_in(ctx, ctx->ws, n, hist_cap);
}

// SELL-32 layout of a CSR matrix (host side), with an optional row order
// sorted by length when that saves padding.  Up to SELL_GLOBAL rows (their
// gathered vectors fit easily in L2) the sort is global, so the longest rows
// open the first tiles and slices, and the passes' round-robin assignment of
// tiles to CTAs (and slices to warps) deals the heavy ones out evenly; larger
// matrices are sorted inside windows of SELL_SIGMA rows to keep locality.
constexpr int SELL_SIGMA = 4096;
constexpr int SELL_GLOBAL = 1 << 23;

struct Sell {
    int nslices = 0;
    long long padded = 0;
    bool permuted = false;
    bool narrow = true;
    std::vector<int> sl_off, rlen, ci, perm, tmeta;
    std::vector<uint16_t> lci;          // local column index into a tile's staged gather blocks
    std::vector<double> va;
};

// ncols > n: a rectangular matrix whose columns n .. ncols - 1 keep their
// index (the halo of a row-partitioned solve); rows and the first n columns
// share the solver order
bool build_sell(int n, const int32_t *rp, const int32_t *col, const double *val, Sell &S, int ncols = 0)
{
    int ns = (n + 31) / 32;
    S.nslices = ns;
    std::vector<int> len(n);
    long long nnz = rp[n];
    for (int i = 0; i < n; i++)
        len[i] = rp[i + 1] - rp[i];
    S.perm.resize(n);
    for (int i = 0; i < n; i++)
        S.perm[i] = i;
    auto padded_of = [&](const std::vector<int> &pm) {
        long long tot = 0;
        for (int s = 0; s < ns; s++) {
            int w = 0;
            for (int l = 0; l < 32; l++) {
                int p = s * 32 + l;
                if (p < n && len[pm[p]] > w)
                    w = len[pm[p]];
            }
            tot += 32ll * w;
        }
        return tot;
    };
    long long pad0 = padded_of(S.perm);
    if ((double)pad0 > 1.10 * (double)nnz + 32.0 * ns) {
        const int sigma = n <= SELL_GLOBAL ? n : SELL_SIGMA;
        for (int w0 = 0; w0 < n; w0 += sigma) {
            int w1 = std::min(n, w0 + sigma);
            std::stable_sort(S.perm.begin() + w0, S.perm.begin() + w1,
                             [&](int a, int b) { return len[a] > len[b]; });
        }
        S.permuted = true;
    }
    std::vector<int> inv((size_t)std::max(n, ncols));
    for (int p = 0; p < n; p++)
        inv[S.perm[p]] = p;
    for (int c = n; c < ncols; c++)
        inv[(size_t)c] = c;
    S.sl_off.assign(ns + 1, 0);
    long long off = 0;
    for (int s = 0; s < ns; s++) {
        int w = 0;
        for (int l = 0; l < 32; l++) {
            int p = s * 32 + l;
            if (p < n && len[S.perm[p]] > w)
                w = len[S.perm[p]];
        }
        if (off > INT32_MAX)
            return false;
        S.sl_off[s] = (int)off;
        off += 32ll * w;
    }
    if (off > INT32_MAX)
        return false;
    S.sl_off[ns] = (int)off;
    S.padded = off;
    // pad to whole 256-row tiles so that tile copies stay inside the arrays
    const int ntiles = (ns + TILE_SLICES - 1) / TILE_SLICES;
    S.sl_off.resize((size_t)ntiles * TILE_SLICES + SLOFF_STAGE, (int)off);
    S.narrow = true;
    for (int t = 0; t < ntiles; t++) {
        int a = S.sl_off[(size_t)t * TILE_SLICES], b = S.sl_off[std::min(ns, (t + 1) * TILE_SLICES)];
        if (b - a > MCAP)
            S.narrow = false;
    }
    S.ci.assign((size_t)off, 0);
    S.va.assign((size_t)off, 0.0);
    S.rlen.assign((size_t)((ns + TILE_SLICES - 1) / TILE_SLICES) * TILE_ROWS, 0);
    for (int p = 0; p < n; p++) {
        int i = S.perm[p], s = p / 32, l = p % 32;
        S.rlen[p] = len[i];
        long long base = S.sl_off[s] + l;
        for (int j = 0; j < len[i]; j++) {
            S.ci[(size_t)(base + 32ll * j)] = inv[col[rp[i] + j]];
            S.va[(size_t)(base + 32ll * j)] = val[rp[i] + j];
        }
    }
    if (!S.permuted)
        S.perm.clear();
    // per tile: its entry range, the 256-row blocks of the gathered vector its
    // columns fall in (at most GMAX, else -1), and each entry's index into
    // those staged blocks
    const int ntl = (ns + TILE_SLICES - 1) / TILE_SLICES;
    S.tmeta.assign((size_t)ntl * TMETA, -1);
    S.lci.assign(S.ci.size(), 0);
    for (int t = 0; t < ntl; t++) {
        const int sa = t * TILE_SLICES, sb = std::min(ns, sa + TILE_SLICES);
        S.tmeta[(size_t)t * TMETA + 0] = S.sl_off[sa];
        S.tmeta[(size_t)t * TMETA + 1] = S.sl_off[sb];
        std::vector<int> blocks;
        bool ok = true;
        for (long long e = S.sl_off[sa]; e < S.sl_off[sb] && ok; e++) {
            int b = S.ci[(size_t)e] / TILE_ROWS;
            if (std::find(blocks.begin(), blocks.end(), b) == blocks.end()) {
                if ((int)blocks.size() == GMAX)
                    ok = false;
                else
                    blocks.push_back(b);
            }
        }
        if (!ok || blocks.empty())
            continue;
        std::sort(blocks.begin(), blocks.end());
        for (size_t g = 0; g < blocks.size(); g++)
            S.tmeta[(size_t)t * TMETA + 2 + g] = blocks[g];
        for (long long e = S.sl_off[sa]; e < S.sl_off[sb]; e++) {
            int b = S.ci[(size_t)e] / TILE_ROWS;
            int g = (int)(std::lower_bound(blocks.begin(), blocks.end(), b) - blocks.begin());
            S.lci[(size_t)e] = (uint16_t)(g * TILE_ROWS + S.ci[(size_t)e] % TILE_ROWS);
        }
    }
    return true;
}

int validate_csr_host(pbcg_ctx *ctx, int32_t n, int64_t nnz, const int32_t *rp, const int32_t *ci)
{
    if (n < 1)
        return fail(ctx, PBCG_ERR_INVALID, "n must be >= 1 (got %d)", n);
    if (nnz < 0 || nnz >= (1ll << 31))
        return fail(ctx, PBCG_ERR_INVALID, "nnz out of range (got %lld)", (long long)nnz);
    if (rp[0] != 0)
        return fail(ctx, PBCG_ERR_INVALID, "row_ptr[0] must be 0");
    for (int32_t i = 0; i < n; i++)
        if (rp[i + 1] < rp[i])
            return fail(ctx, PBCG_ERR_INVALID, "row_ptr decreases at row %d", i);
    if ((int64_t)rp[n] != nnz)
        return fail(ctx, PBCG_ERR_INVALID, "row_ptr[n] = %d differs from nnz = %lld", rp[n], (long long)nnz);
    for (int64_t k = 0; k < nnz; k++)
        if (ci[k] < 0 || ci[k] >= n)
            return fail(ctx, PBCG_ERR_INVALID, "col_idx[%lld] = %d outside [0, %d)", (long long)k, ci[k], n);
    return 0;
}

template <int NV, bool MATS>
constexpr size_t stage_bytes()
{
    return StageLayout<NV, MATS>::TOTAL;
}

template <int MODE>
struct Kern {
    static void *pipe_x_tma(bool mats) { return mats ? (void *)k_pipe_x_tma<MODE, true> : (void *)k_pipe_x_tma<MODE, false>; }
    static void *pipe_y_tma(bool mats) { return mats ? (void *)k_pipe_y_tma<MODE, true> : (void *)k_pipe_y_tma<MODE, false>; }
    static void *setup1() { return (void *)k_setup1<MODE>; }
    static void *setup2() { return (void *)k_setup2<MODE>; }
    static void *bicg_a(bool mats) { return mats ? (void *)k_bicg_a_tma<MODE, true> : (void *)k_bicg_a_tma<MODE, false>; }
    static void *bicg_b(bool mats) { return mats ? (void *)k_bicg_b_tma<MODE, true> : (void *)k_bicg_b_tma<MODE, false>; }
    static void *bicg_c() { return (void *)k_bicg_c_tma<MODE>; }
};

// kernel list of one loop body
struct BodyKernel {
    void *fn;
    const char *name;
    int has_work;    // kernel takes (Mat, Vecs, Ctl*, Work*) rather than (Mat, Vecs, const Ctl*)
    size_t smem;     // dynamic shared memory
    int prog = 0;    // follows the kernel before it over a programmatic edge (it waits in
                     // grid_dep_wait; the one before triggers after its tile loop)
};

// narrow: the passes stage tiles in shared memory (the matrix's tiles fit and
// the launch variant stages)
std::vector<BodyKernel> body_kernels(int alg, int mode, bool narrow)
{
    std::vector<BodyKernel> k;
    if (alg == PBCG_ALG_PIPELINED_RR) {
        k.push_back({(void *)k_rr1, "rr1", 0, 0});
        k.push_back({(void *)k_rr2, "rr2", 0, 0});
        k.push_back({(void *)k_rr3, "rr3", 0, 0});
        k.push_back({(void *)k_rr4, "rr4", 0, 0});
    }
    if (alg == PBCG_ALG_PIPELINED || alg == PBCG_ALG_PIPELINED_RR) {
        size_t sx = narrow ? stage_bytes<7, true>() : stage_bytes<7, false>();
        size_t sy = narrow ? stage_bytes<6, true>() : stage_bytes<6, false>();
        k.push_back({mode ? Kern<1>::pipe_x_tma(narrow) : Kern<0>::pipe_x_tma(narrow),
                     mode ? "pipe_x_exact" : "pipe_x_plain", 1, sx, 1});
        k.push_back({mode ? Kern<1>::pipe_y_tma(narrow) : Kern<0>::pipe_y_tma(narrow),
                     mode ? "pipe_y_exact" : "pipe_y_plain", 1, sy, 1});
    } else {
        const size_t sa = narrow ? stage_bytes<1, true>() : stage_bytes<1, false>();
        const size_t sb = narrow ? stage_bytes<1, true>() : stage_bytes<1, false>();
        k.push_back({(void *)k_bicg_p_tma, "bicg_p", 1, stage_bytes<3, false>(), 1});
        k.push_back({mode ? Kern<1>::bicg_a(narrow) : Kern<0>::bicg_a(narrow), mode ? "bicg_a_exact" : "bicg_a_plain", 1,
                     sa, 1});
        k.push_back({(void *)k_bicg_q, "bicg_q", 0, 0, 1});
        k.push_back({mode ? Kern<1>::bicg_b(narrow) : Kern<0>::bicg_b(narrow), mode ? "bicg_b_exact" : "bicg_b_plain", 1,
                     sb, 1});
        k.push_back({mode ? Kern<1>::bicg_c() : Kern<0>::bicg_c(), mode ? "bicg_c_exact" : "bicg_c_plain", 1,
                     stage_bytes<5, false>(), 1});
    }
    return k;
}

int launch_kernel(pbcg_ctx *ctx, void *fn, Mat &A, Vecs &V, Ctl *c, Work *wk, int has_work, size_t smem, int cap = 0)
{
    void *args4[4] = {&A, &V, &c, &wk};
    void *args3[3] = {&A, &V, &c};
    int grid = grid_for(ctx, fn, A.nslices, smem, cap);
    CK(cudaLaunchKernel(fn, dim3(grid), dim3(THREADS), has_work ? args4 : args3, smem, ctx->stream));
    return 0;
}

// Iterations per execution of the loop graph's WHILE body.  Each execution of
// the body costs about 6.5 us of conditional-node overhead at 128^3, and the
// passes inside one body follow each other over programmatic edges; after a
// stop every later pass of the body returns at its first check of the
// status, so a stop costs at most LOOP_UNROLL - 1 such empty iterations.
constexpr int LOOP_UNROLL = 16;

// build (or reuse) the WHILE-node loop graph for this matrix / algorithm / mode
int get_loop(pbcg_ctx *ctx, const pbcg_mat *m, int alg, int mode, bool jac, LoopGraph **out)
{
    LoopGraph &L = ctx->ws.loop;
    const int unroll = LOOP_UNROLL;
    const int var = m->v_staged | (m->v_order << 1) | (m->v_ctas << 4);
    if (L.exec && L.mat == m && L.alg == alg && L.mode == mode && L.n == m->n && L.jac == jac && L.var == var) {
        *out = &L;
        return 0;
    }
    free_loop(L);
    CK(cudaGraphCreate(&L.graph, 0));
    CK(cudaGraphConditionalHandleCreate(&L.handle, L.graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = L.handle;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cnode;
    CK(cudaGraphAddNode(&cnode, L.graph, nullptr, nullptr, 0, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    // kernel parameter values are copied into the nodes when they are added
    Mat A = mat_of(m);
    if (jac)
        A.va = m->va_jac;
    Vecs V = vecs_of(ctx->ws);
    Ctl *c = ctx->ws.ctl;
    Work *wk = ctx->ws.wk;
    cudaGraphNode_t prev = nullptr;
    const auto bks = body_kernels(alg, mode, m->narrow && m->v_staged);
    for (int u = 0; u < unroll; u++)
    for (auto &bk : bks) {
        void *args4[4] = {&A, &V, &c, &wk};
        void *args3[3] = {&A, &V, &c};
        cudaGraphNodeParams np = {};
        np.type = cudaGraphNodeTypeKernel;
        np.kernel.func = bk.fn;
        np.kernel.gridDim = dim3(grid_for(ctx, bk.fn, A.nslices, bk.smem, bk.has_work ? m->v_ctas : 0));
        np.kernel.blockDim = dim3(THREADS);
        np.kernel.sharedMemBytes = (unsigned)bk.smem;
        np.kernel.kernelParams = bk.has_work ? args4 : args3;
        // a pass behind a programmatic edge takes the SMs the CTAs of the pass
        // before it leave while that pass's last CTA merges (it waits in
        // grid_dep_wait before its first global read)
        cudaGraphEdgeData ed = {};
        const bool prog = prev && bk.prog;
        if (prog) {
            ed.from_port = cudaGraphKernelNodePortProgrammatic;
            ed.type = cudaGraphDependencyTypeProgrammatic;
        }
        cudaGraphNode_t node;
        CK(cudaGraphAddNode(&node, body, prev ? &prev : nullptr, prog ? &ed : nullptr, prev ? 1 : 0, &np));
        prev = node;
    }
    CK(cudaGraphInstantiate(&L.exec, L.graph, 0));
    L.alg = alg;
    L.mode = mode;
    L.jac = jac;
    L.var = var;
    L.unroll = unroll;
    L.mat = m;
    L.n = m->n;
    *out = &L;
    return 0;
}

int read_ctl(pbcg_ctx *ctx, const Ctl *dev_ctl = nullptr)
{
    CK(cudaMemcpyAsync(ctx->h_ctl, dev_ctl ? dev_ctl : ctx->ws.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return 0;
}

// profiling support: events around launches, accumulated per kernel name
struct Prof {
    std::vector<std::string> names;
    std::vector<double> ms;
    std::vector<int> count;
    std::vector<cudaEvent_t> ev;
    std::vector<int> which;
    void add(const std::string &n, float t)
    {
        for (size_t i = 0; i < names.size(); i++)
            if (names[i] == n) {
                ms[i] += t;
                count[i]++;
                return;
            }
        names.push_back(n);
        ms.push_back(t);
        count.push_back(1);
    }
};

// launch with optional timing
struct Launcher {
    pbcg_ctx *ctx;
    Prof *prof;
    long long launches = 0;
    std::vector<std::pair<std::string, std::pair<cudaEvent_t, cudaEvent_t>>> pending;

    int go(const char *name, void *fn, Mat &A, Vecs &V, Ctl *c, Work *wk, int has_work, size_t smem = 0, int cap = 0)
    {
        NvtxRange trace(name);
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (prof) {
            CK(cudaEventCreate(&e0));
            CK(cudaEventCreate(&e1));
            CK(cudaEventRecord(e0, ctx->stream));
        }
        int rc = launch_kernel(ctx, fn, A, V, c, wk, has_work, smem, cap);
        if (rc)
            return rc;
        launches++;
        if (prof) {
            CK(cudaEventRecord(e1, ctx->stream));
            pending.push_back({name, {e0, e1}});
        }
        return 0;
    }
    int flush()
    {
        for (auto &p : pending) {
            CK(cudaEventSynchronize(p.second.second));
            float t = 0.f;
            CK(cudaEventElapsedTime(&t, p.second.first, p.second.second));
            prof->add(p.first, t);
            cudaEventDestroy(p.second.first);
            cudaEventDestroy(p.second.second);
        }
        pending.clear();
        return 0;
    }
};

// caller-order vector (host or device) -> solver-order device vector
// Jacobi preconditioning data of a matrix: d_i = sum, in stored order, of row
// i's entries in column i (zero, non-finite or absent: INVALID), in solver
// order, and the entries of A M^-1 (v / d_col, one IEEE division each)
int host_diagonal(pbcg_ctx *ctx, const pbcg_mat *m, std::vector<double> &d)
{
    const int n = m->n;
    d.assign((size_t)n, 0.0);
    for (int i = 0; i < n; i++) {
        bool found = false;
        double s = 0.0;
        for (int k = m->h_rp[i]; k < m->h_rp[i + 1]; k++)
            if (m->h_ci[k] == i) {
                s = found ? s + m->h_va[k] : m->h_va[k];
                found = true;
            }
        if (!found || s == 0.0 || !std::isfinite(s))
            return fail(ctx, PBCG_ERR_INVALID, "Jacobi preconditioning needs a finite nonzero diagonal (row %d)", i);
        d[(size_t)i] = s;
    }
    return 0;
}

int ensure_jacobi(pbcg_ctx *ctx, pbcg_mat *m)
{
    if (m->va_jac)
        return 0;
    const int n = m->n;
    std::vector<double> d;
    if (int rc = host_diagonal(ctx, m, d))
        return rc;
    std::vector<int> perm;
    if (m->perm) {
        perm.resize((size_t)n);
        CK(cudaMemcpy(perm.data(), m->perm, sizeof(int) * (size_t)n, cudaMemcpyDeviceToHost));
    }
    std::vector<double> ds((size_t)n);
    for (int p = 0; p < n; p++)
        ds[(size_t)p] = d[(size_t)(m->perm ? perm[(size_t)p] : p)];
    const size_t P = (size_t)(m->padded ? m->padded : 1);
    // built aside and attached only once scaled, so a failed call leaves the
    // matrix as it was and a later call starts over
    double *dd = nullptr, *vs = nullptr;
    cudaError_t e = cudaMalloc(&dd, sizeof(double) * (size_t)n);
    if (e == cudaSuccess)
        e = cudaMalloc(&vs, sizeof(double) * P);
    if (e == cudaSuccess)
        e = cudaMemcpy(dd, ds.data(), sizeof(double) * (size_t)n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        long long ne = m->padded;
        const int *ci = m->ci;
        const double *va = m->va, *ddc = dd;
        void *args[5] = {&ne, (void *)&ci, (void *)&va, (void *)&ddc, &vs};
        e = cudaLaunchKernel((void *)k_jacobi_scale, dim3(ctx->num_sms * 8), dim3(256), args, 0, ctx->stream);
    }
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        cudaFree(dd);
        cudaFree(vs);
        return fail(ctx, e == cudaErrorMemoryAllocation ? PBCG_ERR_OOM : PBCG_ERR_CUDA, "Jacobi scaling: %s",
                    cudaGetErrorString(e));
    }
    m->diag = dd;
    m->va_jac = vs;
    return 0;
}

// y = x * d or x = y / d on a solver-order device vector
int jacobi_vec(pbcg_ctx *ctx, const pbcg_mat *m, double *x, bool to_scaled)
{
    int n = m->n;
    const double *dd = m->diag;
    void *args[3] = {&n, (void *)&dd, &x};
    CK(cudaLaunchKernel(to_scaled ? (void *)k_vmul : (void *)k_vdiv, dim3(ctx->num_sms * 4), dim3(256), args, 0,
                        ctx->stream));
    return 0;
}

int vec_in(pbcg_ctx *ctx, const pbcg_mat *m, const double *src, double *dst, double *tmp = nullptr)
{
    size_t bytes = sizeof(double) * (size_t)m->n;
    if (!m->perm) {
        CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, ctx->stream));
        return 0;
    }
    if (!tmp)
        tmp = ctx->ws.vec[V_TMP];
    CK(cudaMemcpyAsync(tmp, src, bytes, cudaMemcpyDefault, ctx->stream));
    int n = m->n;
    const int *pm = m->perm;
    void *args[4] = {&n, &pm, &tmp, &dst};
    CK(cudaLaunchKernel((void *)k_gather, dim3(ctx->num_sms * 4), dim3(256), args, 0, ctx->stream));
    return 0;
}

// solver-order device vector -> caller-order vector (host or device)
int vec_out(pbcg_ctx *ctx, const pbcg_mat *m, const double *src, double *dst, double *tmp = nullptr)
{
    size_t bytes = sizeof(double) * (size_t)m->n;
    if (!m->perm) {
        CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, ctx->stream));
        return 0;
    }
    if (!tmp)
        tmp = ctx->ws.vec[V_TMP];
    int n = m->n;
    const int *pm = m->perm;
    void *args[4] = {&n, &pm, &src, &tmp};
    CK(cudaLaunchKernel((void *)k_scatter, dim3(ctx->num_sms * 4), dim3(256), args, 0, ctx->stream));
    CK(cudaMemcpyAsync(dst, tmp, bytes, cudaMemcpyDefault, ctx->stream));
    return 0;
}

// Launch shape of k_pipe_cluster for a small system.
struct ClusterShape {
    int ctas, rpt, lg, emax;
    size_t smem;
};

cudaLaunchConfig_t cluster_config(pbcg_ctx *ctx, const ClusterShape &S, cudaLaunchAttribute *at)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(S.ctas);
    cfg.blockDim = dim3(THREADS);
    cfg.dynamicSmemBytes = S.smem;
    cfg.stream = ctx->stream;
    *at = cudaLaunchAttribute{};
    at->id = cudaLaunchAttributeClusterDimension;
    at->val.clusterDim.x = S.ctas;
    at->val.clusterDim.y = 1;
    at->val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cfg;
}

// The cluster shape of a small system: the fewest rows per thread (1, 2 or 4)
// that fit the system in one cluster of at most 16 CTAs, with every CTA's
// rows of the vectors and matrix in its shared memory; false when there is
// none (too many rows, rows too wide, or no such cluster can be resident).
const void *cluster_fn(int alg, int mode)
{
    if (alg == PBCG_ALG_BICGSTAB)
        return mode ? (const void *)k_bicg_cluster<1> : (const void *)k_bicg_cluster<0>;
    return mode ? (const void *)k_pipe_cluster<1> : (const void *)k_pipe_cluster<0>;
}

bool cluster_shape(pbcg_ctx *ctx, const pbcg_mat *m, int alg, int mode, ClusterShape *out)
{
    const void *fn = cluster_fn(alg, mode);
    if (m->n < 1 || m->h_sloff.size() != (size_t)m->nslices + 1)
        return false;
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device);
    for (int rpt = 1; rpt <= CLUSTER_MAX_RPT; rpt *= 2) {
        const int rows = rpt * THREADS, nsl = rows / 32;
        const long long ctas = ((long long)m->n + rows - 1) / rows;
        if (ctas > CLUSTER_MAX_CTAS)
            continue;
        int emax = 0;
        for (long long b = 0; b < ctas; b++) {
            const int s0 = (int)std::min<long long>(b * nsl, m->nslices);
            const int s1 = (int)std::min<long long>(b * nsl + nsl, m->nslices);
            emax = std::max(emax, m->h_sloff[(size_t)s1] - m->h_sloff[(size_t)s0]);
        }
        ClusterShape S{(int)ctas, rpt, 31 - __builtin_clz((unsigned)rows), emax, cluster_smem_bytes(rows, emax)};
        if (S.smem + fa.sharedSizeBytes > (size_t)optin)
            return false;                                   // more rows per thread only needs more
        const long long key = ((long long)(alg * 2 + mode) << 56) | ((long long)S.ctas << 48) | (long long)S.smem;
        auto it = ctx->cl_ok.find(key);
        bool ok;
        if (it != ctx->cl_ok.end()) {
            ok = it->second;
        } else {
            ok = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess &&
                 cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S.smem) == cudaSuccess;
            if (ok) {
                cudaLaunchAttribute at;
                cudaLaunchConfig_t cfg = cluster_config(ctx, S, &at);
                int num = 0;
                ok = cudaOccupancyMaxActiveClusters(&num, fn, &cfg) == cudaSuccess && num >= 1;
            }
            cudaGetLastError();
            ctx->cl_ok[key] = ok;
        }
        if (!ok)
            return false;
        *out = S;
        return true;
    }
    return false;
}

int launch_cluster(pbcg_ctx *ctx, int alg, int mode, Mat &A, Vecs &V, Ctl *c, const ClusterShape &S)
{
    const void *fn = cluster_fn(alg, mode);
    CK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S.smem));
    cudaLaunchAttribute at;
    cudaLaunchConfig_t cfg = cluster_config(ctx, S, &at);
    int rpt = S.rpt, lg = S.lg, emax = S.emax;
    void *args[6] = {&A, &V, &c, &rpt, &lg, &emax};
    CK(cudaLaunchKernelExC(&cfg, fn, args));
    return 0;
}

int solve_impl(pbcg_ctx *ctx, const pbcg_mat *m, const double *b, double *x, double tol, int32_t maxit, int alg,
               int mode, pbcg_result *out, Prof *prof)
{
    auto t0 = std::chrono::steady_clock::now();
    if (!ctx)
        return PBCG_ERR_INVALID;
    if (!m || !ctx->mats.count(const_cast<pbcg_mat *>(m)))
        return fail(ctx, PBCG_ERR_INVALID, "unknown matrix handle");
    if (!b || !x)
        return fail(ctx, PBCG_ERR_INVALID, "b and x must not be NULL");
    if (!(tol > 0.0))
        return fail(ctx, PBCG_ERR_INVALID, "tol must be > 0");
    if (maxit < 0 || maxit == INT32_MAX)      // the history holds maxit + 1 entries
        return fail(ctx, PBCG_ERR_INVALID, "maxit must be in 0 .. 2^31 - 2");
    if (alg != PBCG_ALG_BICGSTAB && alg != PBCG_ALG_PIPELINED && alg != PBCG_ALG_PIPELINED_RR)
        return fail(ctx, PBCG_ERR_INVALID, "unknown algorithm %d", alg);
    if (mode != PBCG_DOT_PLAIN && mode != PBCG_DOT_EXACT)
        return fail(ctx, PBCG_ERR_INVALID, "unknown dot mode %d", mode);
    CK(cudaSetDevice(ctx->device));
    int n = m->n;
    int rc = ensure_ws(ctx, n, maxit + 1);
    if (rc)
        return rc;
    Workspace &ws = ctx->ws;
    const bool jac = ctx->precond == PBCG_PRECOND_JACOBI;
    if (jac && (rc = ensure_jacobi(ctx, const_cast<pbcg_mat *>(m))))
        return rc;
    if ((rc = vec_in(ctx, m, b, ws.vec[V_B])) || (rc = vec_in(ctx, m, x, ws.vec[V_X])))
        return rc;
    if (jac && (rc = jacobi_vec(ctx, m, ws.vec[V_X], true)))     // y0 = d x0
        return rc;
    Ctl h;
    memset(&h, 0, sizeof h);
    h.it = 0;
    h.maxit = maxit;
    h.status = ST_RUNNING;
    h.tol = tol;
    h.target = tol;
    h.alg = (alg == PBCG_ALG_BICGSTAB) ? ALG_BICGSTAB : ALG_PIPELINED;
    h.rr_period = (alg == PBCG_ALG_PIPELINED_RR) ? ctx->rr_period : 0;
    h.use_cond = 0;
    h.order = m->v_order;
    h.hist = ws.hist;
    h.hist_cap = maxit + 1;
    h.trueres = __builtin_nan("");
    *ctx->h_ctl = h;
    CK(cudaMemcpyAsync(ws.ctl, ctx->h_ctl, sizeof(Ctl), cudaMemcpyHostToDevice, ctx->stream));

    Mat A = mat_of(m);
    if (jac)
        A.va = m->va_jac;                                         // A M^-1
    Vecs V = vecs_of(ws);
    Launcher L{ctx, prof, 0, {}};
    if (alg != PBCG_ALG_BICGSTAB) {
        rc = L.go("setup1", mode ? Kern<1>::setup1() : Kern<0>::setup1(), A, V, ws.ctl, ws.wk, 1);
        if (!rc)
            rc = L.go("setup2", mode ? Kern<1>::setup2() : Kern<0>::setup2(), A, V, ws.ctl, ws.wk, 1);
        if (!rc)
            rc = L.go("setup3", (void *)k_setup3, A, V, ws.ctl, ws.wk, 0);
    } else {
        rc = L.go("setup1", mode ? Kern<1>::setup1() : Kern<0>::setup1(), A, V, ws.ctl, ws.wk, 1);
    }
    if (rc)
        return rc;
    bool cond_on = false;
    bool true_done = false;
    auto body = body_kernels(alg, mode, m->narrow && m->v_staged);
    bool fresh = false;      // h_ctl already mirrors the device after a graph launch
    for (;;) {
        if (prof && (rc = L.flush()))
            return rc;
        if (!fresh && (rc = read_ctl(ctx)))
            return rc;
        fresh = false;
        int st = ctx->h_ctl->status;
        if (st == ST_CANDIDATE) {
            rc = L.go("true_res", (void *)k_true_res, A, V, ws.ctl, ws.wk, 1);
            if (rc)
                return rc;
            true_done = true;
            continue;
        }
        if (st != ST_RUNNING)
            break;
        true_done = false;
        ClusterShape cs;
        if (prof) {
            // host-driven iteration, one kernel at a time
            for (auto &bk : body)
                if ((rc = L.go(bk.name, bk.fn, A, V, ws.ctl, ws.wk, bk.has_work, bk.smem,
                               bk.has_work ? m->v_ctas : 0)))
                    return rc;
        } else if (alg != PBCG_ALG_PIPELINED_RR && ctx->small_cluster && cluster_shape(ctx, m, alg, mode, &cs)) {
            // small system: every iteration up to the next stop in one cluster launch
            if ((rc = launch_cluster(ctx, alg, mode, A, V, ws.ctl, cs)))
                return rc;
            L.launches += 1;
        } else {
            LoopGraph *G = nullptr;
            if ((rc = get_loop(ctx, m, alg, mode, jac, &G)))
                return rc;
            if (!cond_on) {
                int one = 1;
                unsigned long long hv = (unsigned long long)G->handle;
                CK(cudaMemcpyAsync(&ws.ctl->cond, &hv, sizeof hv, cudaMemcpyHostToDevice, ctx->stream));
                CK(cudaMemcpyAsync(&ws.ctl->use_cond, &one, sizeof one, cudaMemcpyHostToDevice, ctx->stream));
                cond_on = true;
            }
            int it_before = ctx->h_ctl->it;
            CK(cudaGraphLaunch(G->exec, ctx->stream));
            if ((rc = read_ctl(ctx)))
                return rc;
            // every body execution launches all body kernels (LOOP_UNROLL
            // iterations of them, those after a stop returning at once); a stop
            // inside an iteration (non-finite dot, breakdown) still ran that
            // iteration's kernels
            long long bodies = ctx->h_ctl->it - it_before;
            int s2 = ctx->h_ctl->status;
            if (s2 == 2 || s2 == 3)
                bodies += 1;
            bodies = (bodies + G->unroll - 1) / G->unroll;
            L.launches += bodies * (long long)G->unroll * (long long)body.size();
            fresh = true;
            continue;
        }
    }
    if (!true_done) {
        if ((rc = L.go("true_res", (void *)k_true_res, A, V, ws.ctl, ws.wk, 1)))
            return rc;
        if (prof && (rc = L.flush()))
            return rc;
        if ((rc = read_ctl(ctx)))
            return rc;
    }
    if (cond_on) {
        int zero = 0;
        CK(cudaMemcpyAsync(&ws.ctl->use_cond, &zero, sizeof zero, cudaMemcpyHostToDevice, ctx->stream));
    }
    Ctl fin_ctl = *ctx->h_ctl;
    if (fin_ctl.err || fin_ctl.status == ST_TIMEOUT)
        return fail(ctx, PBCG_ERR_TIMEOUT, "a bounded device wait expired (bulk copy did not complete)");
    if (jac && (rc = jacobi_vec(ctx, m, ws.vec[V_X], false)))    // x = y / d
        return rc;
    if ((rc = vec_out(ctx, m, ws.vec[V_X], x)))
        return rc;
    int hl = fin_ctl.it + 1;
    if (hl > maxit + 1)
        hl = maxit + 1;
    ctx->hist.assign(hl, 0.0);
    CK(cudaMemcpyAsync(ctx->hist.data(), ws.hist, sizeof(double) * hl, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->have_hist = true;
    ctx->last_batched = false;
    if (out) {
        out->iters = fin_ctl.it;
        out->status = fin_ctl.status;
        out->relres_recursive = fin_ctl.res;
        out->relres_true = fin_ctl.trueres;
        out->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        out->launches = (int32_t)L.launches;
        out->reserved = 0;
    }
    return fin_ctl.status;
}


// ---------------------------------------------------------------------------
// batched solves
// ---------------------------------------------------------------------------
void free_batch_graph(pbcg_ctx *ctx);

int build_layout(pbcg_ctx *ctx, pbcg_mat *m, const std::vector<int32_t> &srp, const std::vector<double> *dj)
{
    if (m->bl && m->bl->key == srp && m->bl->jac == (dj != nullptr))
        return 0;
    if (m->bl && ctx->b.g_layout == (const void *)m->bl)
        free_batch_graph(ctx);             // its nodes point into the layout being replaced
    layout_release(m->bl);
    m->bl = nullptr;
    const int nsys = (int)srp.size() - 1;
    std::vector<int> ib(nsys + 1, 0), t0(nsys + 1, 0);
    for (int k = 0; k < nsys; k++) {
        long long ns = srp[k + 1] - srp[k];
        long long np = (ns + TILE_ROWS - 1) / TILE_ROWS * TILE_ROWS;
        if ((long long)ib[k] + np > INT32_MAX / 2)
            return fail(ctx, PBCG_ERR_INVALID, "batched layout too large");
        ib[k + 1] = ib[k] + (int)np;
        t0[k + 1] = t0[k] + (int)(np / TILE_ROWS);
    }
    const int n_int = ib[nsys], ntiles = t0[nsys], ns = n_int / 32;
    std::vector<int> map(n_int, -1), tile_sys(ntiles), len(n_int, 0);
    for (int k = 0; k < nsys; k++) {
        for (int i = srp[k]; i < srp[k + 1]; i++) {
            int p = ib[k] + (i - srp[k]);
            map[p] = i;
            len[p] = m->h_rp[i + 1] - m->h_rp[i];
            for (int e = m->h_rp[i]; e < m->h_rp[i + 1]; e++) {
                int j = m->h_ci[e];
                if (j < srp[k] || j >= srp[k + 1])
                    return fail(ctx, PBCG_ERR_INVALID, "row %d has column %d outside its system %d", i, j, k);
            }
        }
        for (int t = t0[k]; t < t0[k + 1]; t++)
            tile_sys[t] = k;
    }
    std::vector<int> sl_off((size_t)ns + 1 + SLOFF_STAGE, 0);
    long long off = 0;
    for (int sl = 0; sl < ns; sl++) {
        int w = 0;
        for (int l = 0; l < 32; l++)
            w = std::max(w, len[sl * 32 + l]);
        sl_off[sl] = (int)off;
        off += 32ll * w;
        if (off > INT32_MAX)
            return fail(ctx, PBCG_ERR_INVALID, "padded matrix exceeds 2^31 entries");
    }
    for (size_t q = ns; q < sl_off.size(); q++)
        sl_off[q] = (int)off;
    std::vector<int> ci((size_t)std::max<long long>(off, 1), 0);
    std::vector<double> va((size_t)std::max<long long>(off, 1), 0.0);
    for (int k = 0; k < nsys; k++) {
        for (int i = srp[k]; i < srp[k + 1]; i++) {
            int p = ib[k] + (i - srp[k]);
            long long base = sl_off[p / 32] + (p % 32);
            int j0 = m->h_rp[i];
            for (int e = 0; e < len[p]; e++) {
                ci[(size_t)(base + 32ll * e)] = ib[k] + (m->h_ci[j0 + e] - srp[k]);
                va[(size_t)(base + 32ll * e)] =
                    dj ? m->h_va[j0 + e] / (*dj)[(size_t)m->h_ci[j0 + e]] : m->h_va[j0 + e];   // A M^-1
            }
        }
    }
    BatchLayout *L = new BatchLayout();
    L->key = srp;
    L->jac = dj != nullptr;
    L->nsys = nsys;
    L->n_int = n_int;
    L->nslices = ns;
    L->ntiles = ntiles;
    cudaError_t e = cudaMalloc(&L->sl_off, sizeof(int) * sl_off.size());
    if (e == cudaSuccess) e = cudaMalloc(&L->rlen, sizeof(int) * (size_t)n_int);
    if (e == cudaSuccess) e = cudaMalloc(&L->ci, sizeof(int) * ci.size());
    if (e == cudaSuccess) e = cudaMalloc(&L->va, sizeof(double) * va.size());
    if (e == cudaSuccess) e = cudaMalloc(&L->map, sizeof(int) * (size_t)n_int);
    if (e == cudaSuccess) e = cudaMalloc(&L->tile_sys, sizeof(int) * (size_t)ntiles);
    if (e == cudaSuccess) e = cudaMalloc(&L->sys_t0, sizeof(int) * (size_t)(nsys + 1));
    if (e == cudaSuccess) e = cudaMemcpy(L->sl_off, sl_off.data(), sizeof(int) * sl_off.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(L->rlen, len.data(), sizeof(int) * (size_t)n_int, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(L->ci, ci.data(), sizeof(int) * ci.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(L->va, va.data(), sizeof(double) * va.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(L->map, map.data(), sizeof(int) * (size_t)n_int, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(L->tile_sys, tile_sys.data(), sizeof(int) * (size_t)ntiles, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(L->sys_t0, t0.data(), sizeof(int) * (size_t)(nsys + 1), cudaMemcpyHostToDevice);
    if (dj && e == cudaSuccess) {
        std::vector<double> dl((size_t)n_int, 1.0);          // padding rows keep x = 0
        for (int p = 0; p < n_int; p++)
            if (map[(size_t)p] >= 0)
                dl[(size_t)p] = (*dj)[(size_t)map[(size_t)p]];
        e = cudaMalloc(&L->diag, sizeof(double) * (size_t)n_int);
        if (e == cudaSuccess)
            e = cudaMemcpy(L->diag, dl.data(), sizeof(double) * (size_t)n_int, cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        layout_release(L);
        return fail(ctx, e == cudaErrorMemoryAllocation ? PBCG_ERR_OOM : PBCG_ERR_CUDA, "batched layout: %s",
                    cudaGetErrorString(e));
    }
    m->bl = L;
    return 0;
}

#define BW ctx->b

void free_batch_graph(pbcg_ctx *ctx)
{
    if (BW.exec)
        cudaGraphExecDestroy(BW.exec);
    if (BW.graph)
        cudaGraphDestroy(BW.graph);
    BW.exec = nullptr;
    BW.graph = nullptr;
    BW.g_layout = nullptr;
}

int ensure_batch_ws(pbcg_ctx *ctx, const BatchLayout *L, long long n_caller, int maxit)
{
    if (L->n_int > BW.n_cap) {
        free_batch_graph(ctx);
        for (auto &p : BW.vec) {
            cudaFree(p);
            p = nullptr;
        }
        BW.n_cap = 0;
        for (auto &p : BW.vec) {
            CK(cudaMalloc(&p, sizeof(double) * (size_t)L->n_int));
            CK(cudaMemset(p, 0, sizeof(double) * (size_t)L->n_int));
        }
        BW.n_cap = L->n_int;
    }
    if (L->nsys > BW.nsys_cap) {
        free_batch_graph(ctx);
        cudaFree(BW.ctl);
        cudaFree(BW.acc);
        cudaFree(BW.done);
        BW.ctl = nullptr;
        BW.acc = nullptr;
        BW.done = nullptr;
        BW.nsys_cap = 0;
        CK(cudaMalloc(&BW.ctl, sizeof(Ctl) * (size_t)L->nsys));
        CK(cudaMalloc(&BW.acc, sizeof(GAcc) * MAXD * (size_t)L->nsys));
        CK(cudaMalloc(&BW.done, sizeof(unsigned) * (size_t)L->nsys));
        BW.nsys_cap = L->nsys;
    }
    if (L->ntiles > BW.ntiles_cap) {
        free_batch_graph(ctx);
        cudaFree(BW.part);
        BW.part = nullptr;
        BW.ntiles_cap = 0;
        CK(cudaMalloc(&BW.part, sizeof(double) * MAXD * (size_t)L->ntiles));
        BW.ntiles_cap = L->ntiles;
    }
    if (!BW.flag)
        CK(cudaMalloc(&BW.flag, sizeof(int)));
    long long hneed = (long long)L->nsys * (maxit + 1);
    if (hneed > BW.hist_cap) {
        cudaFree(BW.hist);
        BW.hist = nullptr;
        BW.hist_cap = 0;
        CK(cudaMalloc(&BW.hist, sizeof(double) * (size_t)hneed));
        BW.hist_cap = hneed;
    }
    if (n_caller > BW.io_cap) {
        cudaFree(BW.io);
        BW.io = nullptr;
        BW.io_cap = 0;
        CK(cudaMalloc(&BW.io, sizeof(double) * (size_t)n_caller));
        BW.io_cap = n_caller;
    }
    return 0;
}

Mat layout_mat(const BatchLayout *L)
{
    Mat A;
    A.n = L->n_int;
    A.ncols = L->n_int;
    A.nslices = L->nslices;
    A.sl_off = L->sl_off;
    A.rlen = L->rlen;
    A.ci = L->ci;
    A.va = L->va;
    A.sl_w = nullptr;
    A.lci = nullptr;
    A.tmeta = nullptr;
    return A;
}

Batch batch_of(pbcg_ctx *ctx, const BatchLayout *L)
{
    Batch B;
    B.nsys = L->nsys;
    B.ntiles = L->ntiles;
    B.tile_sys = L->tile_sys;
    B.sys_t0 = L->sys_t0;
    B.sys_t1 = L->sys_t0 + 1;
    B.ctl = BW.ctl;
    B.acc = BW.acc;
    B.part = BW.part;
    B.done = BW.done;
    B.flag = BW.flag;
    B.lv_n = B.lv_pre = B.lv_t0 = nullptr;
    return B;
}

Vecs batch_vecs(pbcg_ctx *ctx)
{
    Vecs V;
    V.x = BW.vec[V_X];
    V.b = BW.vec[V_B];
    V.r0 = BW.vec[V_R0];
    V.r = BW.vec[V_R];
    V.w = BW.vec[V_W];
    V.t = BW.vec[V_T];
    V.p = BW.vec[V_P];
    V.s = BW.vec[V_S];
    V.z = BW.vec[V_Z];
    V.v = BW.vec[V_V];
    V.y = BW.vec[V_Y];
    V.q = BW.vec[V_Q];
    return V;
}

struct BKernel {
    void *fn;
    const char *name;
    size_t smem;     // dynamic shared memory (staged passes), 0 otherwise
};

template <int MODE>
std::vector<BKernel> batch_body(int alg)
{
    std::vector<BKernel> k;
    k.push_back({(void *)k_batched<1, StepTrueRes<false>>, "b_true_res", 0});
    if (alg == PBCG_ALG_PIPELINED_RR) {
        k.push_back({(void *)k_batched<0, StepRR<1>>, "b_rr1", 0});
        k.push_back({(void *)k_batched<0, StepRR<2>>, "b_rr2", 0});
        k.push_back({(void *)k_batched<0, StepRR<3>>, "b_rr3", 0});
        k.push_back({(void *)k_batched<0, StepRR<4>>, "b_rr4", 0});
    }
    if (alg == PBCG_ALG_PIPELINED || alg == PBCG_ALG_PIPELINED_RR) {
        k.push_back({(void *)k_bstaged<MODE, BPipeX>, MODE ? "b_pipe_x_exact" : "b_pipe_x_plain",
                     StageLayout<BPipeX::NV, true, false>::TOTAL});
        k.push_back({(void *)k_bstaged<MODE, BPipeY>, MODE ? "b_pipe_y_exact" : "b_pipe_y_plain",
                     StageLayout<BPipeY::NV, true, false>::TOTAL});
    } else {
        k.push_back({(void *)k_batched<MODE, StepBicgP>, "b_bicg_p", 0});
        k.push_back({(void *)k_batched<MODE, StepBicgA>, MODE ? "b_bicg_a_exact" : "b_bicg_a_plain", 0});
        k.push_back({(void *)k_batched<MODE, StepBicgB>, MODE ? "b_bicg_b_exact" : "b_bicg_b_plain", 0});
        k.push_back({(void *)k_batched<MODE, StepBicgC>, MODE ? "b_bicg_c_exact" : "b_bicg_c_plain", 0});
    }
    return k;
}

int bgrid(pbcg_ctx *ctx, const void *fn, int ntiles, size_t smem = 0, int cap = 0)
{
    return grid_for(ctx, fn, (long long)ntiles * TILE_SLICES, smem, cap);
}

int blaunch(pbcg_ctx *ctx, void *fn, Mat &A, Vecs &V, Batch &B)
{
    void *args[3] = {&A, &V, &B};
    CK(cudaLaunchKernel(fn, dim3(bgrid(ctx, fn, B.ntiles)), dim3(THREADS), args, 0, ctx->stream));
    return 0;
}

int solve_batched_impl(pbcg_ctx *ctx, const pbcg_mat *Ac, int32_t nsys, const int32_t *sys_row_ptr, const double *b,
                       double *x, const double *tol, int32_t maxit, int alg, int mode, pbcg_result *out)
{
    auto t0 = std::chrono::steady_clock::now();
    if (!ctx)
        return PBCG_ERR_INVALID;
    pbcg_mat *m = const_cast<pbcg_mat *>(Ac);
    if (!m || !ctx->mats.count(m))
        return fail(ctx, PBCG_ERR_INVALID, "unknown matrix handle");
    if (nsys < 1 || !sys_row_ptr || !b || !x || !tol || !out)
        return fail(ctx, PBCG_ERR_INVALID, "bad batched arguments");
    if (maxit < 0 || maxit == INT32_MAX)      // the history holds maxit + 1 entries
        return fail(ctx, PBCG_ERR_INVALID, "maxit must be in 0 .. 2^31 - 2");
    if (alg != PBCG_ALG_BICGSTAB && alg != PBCG_ALG_PIPELINED && alg != PBCG_ALG_PIPELINED_RR)
        return fail(ctx, PBCG_ERR_INVALID, "unknown algorithm %d", alg);
    if (mode != PBCG_DOT_PLAIN && mode != PBCG_DOT_EXACT)
        return fail(ctx, PBCG_ERR_INVALID, "unknown dot mode %d", mode);
    CK(cudaSetDevice(ctx->device));
    std::vector<int32_t> srp((size_t)nsys + 1);
    std::vector<double> htol((size_t)nsys);
    CK(cudaMemcpy(srp.data(), sys_row_ptr, sizeof(int32_t) * srp.size(), cudaMemcpyDefault));
    CK(cudaMemcpy(htol.data(), tol, sizeof(double) * htol.size(), cudaMemcpyDefault));
    if (srp[0] != 0 || srp[nsys] != m->n)
        return fail(ctx, PBCG_ERR_INVALID, "sys_row_ptr must start at 0 and end at n");
    for (int k = 0; k < nsys; k++) {
        if (srp[k + 1] <= srp[k])
            return fail(ctx, PBCG_ERR_INVALID, "sys_row_ptr must be strictly increasing (system %d)", k);
        if (!(htol[k] > 0.0))
            return fail(ctx, PBCG_ERR_INVALID, "tol[%d] must be > 0", k);
    }
    const bool jac = ctx->precond == PBCG_PRECOND_JACOBI;
    std::vector<double> dj;
    int rc = jac ? host_diagonal(ctx, m, dj) : 0;
    if (rc)
        return rc;
    if ((rc = build_layout(ctx, m, srp, jac ? &dj : nullptr)))
        return rc;
    const BatchLayout *L = m->bl;
    if ((rc = ensure_batch_ws(ctx, L, m->n, maxit)))
        return rc;
    Mat A = layout_mat(L);
    Vecs V = batch_vecs(ctx);
    Batch B = batch_of(ctx, L);
    const int np = L->n_int;
    // inputs into the padded order
    {
        CK(cudaMemcpyAsync(BW.io, b, sizeof(double) * (size_t)m->n, cudaMemcpyDefault, ctx->stream));
        int *mp = L->map;
        double *src = BW.io, *dst = V.b;
        void *a1[4] = {(void *)&np, &mp, &src, &dst};
        CK(cudaLaunchKernel((void *)k_bgather, dim3(ctx->num_sms * 4), dim3(256), a1, 0, ctx->stream));
        CK(cudaMemcpyAsync(BW.io, x, sizeof(double) * (size_t)m->n, cudaMemcpyDefault, ctx->stream));
        dst = V.x;
        void *a2[4] = {(void *)&np, &mp, &src, &dst};
        CK(cudaLaunchKernel((void *)k_bgather, dim3(ctx->num_sms * 4), dim3(256), a2, 0, ctx->stream));
        if (jac) {                                            // y0 = d x0
            const double *dd = L->diag;
            void *a4[3] = {(void *)&np, (void *)&dd, &dst};
            CK(cudaLaunchKernel((void *)k_vmul, dim3(ctx->num_sms * 4), dim3(256), a4, 0, ctx->stream));
        }
    }
    std::vector<Ctl> hc((size_t)nsys);
    for (int k = 0; k < nsys; k++) {
        Ctl &c = hc[k];
        memset(&c, 0, sizeof c);
        c.maxit = maxit;
        c.status = ST_RUNNING;
        c.tol = htol[k];
        c.target = htol[k];
        c.alg = (alg == PBCG_ALG_BICGSTAB) ? ALG_BICGSTAB : ALG_PIPELINED;
        c.rr_period = (alg == PBCG_ALG_PIPELINED_RR) ? ctx->rr_period : 0;
        c.use_cond = 0;
        c.hist = BW.hist + (size_t)k * (maxit + 1);
        c.hist_cap = maxit + 1;
        c.trueres = __builtin_nan("");
    }
    CK(cudaMemcpyAsync(BW.ctl, hc.data(), sizeof(Ctl) * hc.size(), cudaMemcpyHostToDevice, ctx->stream));
    {
        std::vector<GAcc> ga((size_t)nsys * MAXD);
        for (auto &g : ga) {
            memset(&g, 0, sizeof g);
            g.kmin = NDIG;
            g.kmax = -1;
        }
        CK(cudaMemcpyAsync(BW.acc, ga.data(), sizeof(GAcc) * ga.size(), cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaMemsetAsync(BW.done, 0, sizeof(unsigned) * (size_t)nsys, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));   // ga, hc go out of scope
    }
    long long launches = 0;
    if ((rc = blaunch(ctx, mode ? (void *)k_batched<1, StepSetup1> : (void *)k_batched<0, StepSetup1>, A, V, B)))
        return rc;
    launches++;
    if (alg != PBCG_ALG_BICGSTAB) {
        if ((rc = blaunch(ctx, mode ? (void *)k_batched<1, StepSetup2> : (void *)k_batched<0, StepSetup2>, A, V, B)))
            return rc;
        if ((rc = blaunch(ctx, (void *)k_batched<0, StepSetup3>, A, V, B)))
            return rc;
        launches += 2;
    }
    // the loop: WHILE(some system running or awaiting its check) { true-res, passes, control }
    std::vector<BKernel> body = mode ? batch_body<1>(alg) : batch_body<0>(alg);
    if (!ctx->batch_graph) {
        // host-driven loop, one kernel launch at a time (for profilers), ending
        // when the control kernel reports no live system; bounded by maxit + 4
        // bodies (every system stops at maxit)
        int any = 1;
        for (long long it = 0; any && it <= (long long)maxit + 4; it++) {
            for (auto &bk : body) {
                void *args[3] = {&A, &V, &B};
                CK(cudaLaunchKernel(bk.fn, dim3(bgrid(ctx, bk.fn, B.ntiles, bk.smem, m->b_ctas)), dim3(THREADS),
                                    args, bk.smem, ctx->stream));
            }
            unsigned long long hv = 0ull;
            int zero = 0;
            void *cargs[3] = {&B, &hv, &zero};
            CK(cudaLaunchKernel((void *)k_batch_ctl, dim3(1), dim3(1024), cargs, 0, ctx->stream));
            CK(cudaMemcpyAsync(&any, B.flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
            CK(cudaStreamSynchronize(ctx->stream));
        }
    } else if (!(BW.exec && BW.g_layout == (const void *)L && BW.g_alg == alg && BW.g_mode == mode &&
                 BW.g_ctas == m->b_ctas)) {
        free_batch_graph(ctx);
        CK(cudaGraphCreate(&BW.graph, 0));
        cudaGraphConditionalHandle h;
        CK(cudaGraphConditionalHandleCreate(&h, BW.graph, 1, cudaGraphCondAssignDefault));
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t cnode;
        CK(cudaGraphAddNode(&cnode, BW.graph, nullptr, nullptr, 0, &cp));
        cudaGraph_t g = cp.conditional.phGraph_out[0];
        cudaGraphNode_t prev = nullptr;
        for (auto &bk : body) {
            void *args[3] = {&A, &V, &B};
            cudaKernelNodeParams kp{};
            kp.func = bk.fn;
            kp.gridDim = dim3(bgrid(ctx, bk.fn, B.ntiles, bk.smem, m->b_ctas));
            kp.blockDim = dim3(THREADS);
            kp.sharedMemBytes = (unsigned)bk.smem;
            kp.kernelParams = args;
            cudaGraphNode_t node;
            CK(cudaGraphAddKernelNode(&node, g, prev ? &prev : nullptr, prev ? 1 : 0, &kp));
            prev = node;
        }
        unsigned long long hv = (unsigned long long)h;
        int one = 1;
        void *cargs[3] = {&B, &hv, &one};
        cudaKernelNodeParams kp{};
        kp.func = (void *)k_batch_ctl;
        kp.gridDim = dim3(1);
        kp.blockDim = dim3(1024);
        kp.kernelParams = cargs;
        cudaGraphNode_t node;
        CK(cudaGraphAddKernelNode(&node, g, prev ? &prev : nullptr, prev ? 1 : 0, &kp));
        CK(cudaGraphInstantiate(&BW.exec, BW.graph, 0));
        BW.g_layout = L;
        BW.g_alg = alg;
        BW.g_mode = mode;
        BW.g_ctas = m->b_ctas;
    }
    if (ctx->batch_graph)
        CK(cudaGraphLaunch(BW.exec, ctx->stream));
    // final true residual of every system, then results
    if ((rc = blaunch(ctx, (void *)k_batched<1, StepTrueRes<true>>, A, V, B)))
        return rc;
    launches++;
    BW.last.resize((size_t)nsys);
    CK(cudaMemcpyAsync(BW.last.data(), BW.ctl, sizeof(Ctl) * (size_t)nsys, cudaMemcpyDeviceToHost, ctx->stream));
    {
        int *mp = L->map;
        double *src = V.x, *dst = BW.io;
        if (jac) {                                            // x = y / d
            const double *dd = L->diag;
            void *a4[3] = {(void *)&np, (void *)&dd, &src};
            CK(cudaLaunchKernel((void *)k_vdiv, dim3(ctx->num_sms * 4), dim3(256), a4, 0, ctx->stream));
        }
        void *a3[4] = {(void *)&np, &mp, &src, &dst};
        CK(cudaLaunchKernel((void *)k_bscatter, dim3(ctx->num_sms * 4), dim3(256), a3, 0, ctx->stream));
        CK(cudaMemcpyAsync(x, BW.io, sizeof(double) * (size_t)m->n, cudaMemcpyDefault, ctx->stream));
    }
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->last_batched = true;
    BW.hist_stride = maxit + 1;
    int maxit_it = 0, worst = 0;
    for (int k = 0; k < nsys; k++)
        maxit_it = std::max(maxit_it, BW.last[k].it);
    launches += (long long)(maxit_it + 1) * (long long)(body.size() + 1);
    double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    for (int k = 0; k < nsys; k++) {
        const Ctl &c = BW.last[k];
        if (c.err)
            return fail(ctx, PBCG_ERR_TIMEOUT, "a bounded device wait expired");
        out[k].iters = c.it;
        out[k].status = c.status;
        out[k].relres_recursive = c.res;
        out[k].relres_true = c.trueres;
        out[k].seconds = secs;
        out[k].launches = (int32_t)std::min<long long>(launches, INT32_MAX);
        out[k].reserved = 0;
        worst = std::max(worst, c.status);
    }
    return worst;
}

#undef BW


// ---------------------------------------------------------------------------
// pools: continuous batching of independent systems
//
// A pool owns one block-diagonal layout of fixed capacity.  Each resident
// system (a slot) holds a range of whole 256-row tiles and a range of SELL-32
// entries.  Admission uploads on the pool's copy stream into ranges that no
// running step reads (free tiles are skipped by the sweep, and a retired
// slot's tiles stay skipped because its status is final), then a small kernel
// on the solve stream makes the slot live.  A step is one graph launch of up
// to K iterations of every live slot; after it the control blocks are copied
// into a ring of pinned snapshots, so polling never waits for the GPU.
// ---------------------------------------------------------------------------
// first-fit allocator of [start, start + len) ranges
struct RangeAlloc {
    std::map<long long, long long> fr;     // start -> end of free ranges
    void init(long long cap)
    {
        fr.clear();
        if (cap > 0)
            fr[0] = cap;
    }
    long long take(long long len)
    {
        for (auto it = fr.begin(); it != fr.end(); ++it) {
            if (it->second - it->first >= len) {
                long long a = it->first, e = it->second;
                fr.erase(it);
                if (a + len < e)
                    fr[a + len] = e;
                return a;
            }
        }
        return -1;
    }
    void give(long long a, long long len)
    {
        if (len <= 0)
            return;
        long long e = a + len;
        auto nx = fr.lower_bound(a);
        if (nx != fr.end() && nx->first == e) {
            e = nx->second;
            fr.erase(nx);
        }
        auto pv = fr.lower_bound(a);
        if (pv != fr.begin()) {
            --pv;
            if (pv->second == a) {
                a = pv->first;
                fr.erase(pv);
            }
        }
        fr[a] = e;
    }
    long long largest() const
    {
        long long m = 0;
        for (auto &kv : fr)
            m = std::max(m, kv.second - kv.first);
        return m;
    }
};

struct PoolSlot {
    bool used = false, reported = false;
    int gen = 0;
    int tile0 = 0, ntiles = 0, n = 0;
    long long e0 = 0, ne = 0;
    Ctl last;                          // control block at the snapshot that reported it
};

constexpr int POOL_RING = 4;

}  // namespace

struct pbcg_pool {
    pbcg_ctx *ctx = nullptr;
    pbcg_pool_config cfg = {};
    int max_tiles = 0;
    cudaStream_t cstream = nullptr;    // uploads and result copies
    cudaEvent_t up_ev = nullptr;
    cudaEvent_t ev[POOL_RING] = {};
    Ctl *snap[POOL_RING] = {};         // pinned
    long long issued = 0;              // steps launched
    int *meta = nullptr;               // pinned: rp | sl_w | sl_off of one request
    int *sl_off = nullptr, *sl_w = nullptr, *rlen = nullptr, *ci = nullptr, *tile_sys = nullptr;
    int *t0 = nullptr, *t1 = nullptr, *left = nullptr, *flag = nullptr, *bad = nullptr;
    int *lv_n = nullptr, *lv_pre = nullptr, *lv_t0 = nullptr;    // live-tile list
    int *st_rp = nullptr, *st_ci = nullptr, *st_meta = nullptr;   // staging of one request
    double *st_va = nullptr;
    double *va = nullptr, *hist = nullptr;
    double *diag = nullptr;            // Jacobi: d of every resident row (arena order), or NULL
    double *vec[V_COUNT] = {};
    Ctl *ctl = nullptr;
    GAcc *acc = nullptr;
    double *part = nullptr;
    unsigned *done = nullptr;
    RangeAlloc tiles, entries;
    std::vector<PoolSlot> slots;
    int next_gen = 1;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int body_kernels = 0;
};

namespace {

void pool_release(pbcg_pool *P)
{
    if (!P)
        return;
    if (P->exec)
        cudaGraphExecDestroy(P->exec);
    if (P->graph)
        cudaGraphDestroy(P->graph);
    void *ptrs[] = {P->sl_off, P->sl_w, P->rlen,  P->ci,      P->tile_sys, P->t0,   P->t1,   P->left,
                    P->flag,   P->bad,  P->st_rp, P->st_ci,   P->st_meta,  P->st_va, P->va,  P->hist,
                    P->ctl,    P->acc,  P->part,  P->done,     P->lv_n, P->lv_pre, P->lv_t0, P->diag};
    for (void *q : ptrs)
        cudaFree(q);
    for (auto &v : P->vec)
        cudaFree(v);
    for (auto &h : P->snap)
        cudaFreeHost(h);
    cudaFreeHost(P->meta);
    for (auto &e : P->ev)
        if (e)
            cudaEventDestroy(e);
    if (P->up_ev)
        cudaEventDestroy(P->up_ev);
    if (P->cstream)
        cudaStreamDestroy(P->cstream);
    delete P;
}

Mat pool_mat(const pbcg_pool *P)
{
    Mat A;
    A.n = P->max_tiles * TILE_ROWS;
    A.ncols = A.n;
    A.nslices = P->max_tiles * TILE_SLICES;
    A.sl_off = P->sl_off;
    A.sl_w = P->sl_w;
    A.rlen = P->rlen;
    A.ci = P->ci;
    A.va = P->va;
    A.lci = nullptr;
    A.tmeta = nullptr;
    return A;
}

Vecs pool_vecs(const pbcg_pool *P)
{
    Vecs V;
    V.x = P->vec[V_X];
    V.b = P->vec[V_B];
    V.r0 = P->vec[V_R0];
    V.r = P->vec[V_R];
    V.w = P->vec[V_W];
    V.t = P->vec[V_T];
    V.p = P->vec[V_P];
    V.s = P->vec[V_S];
    V.z = P->vec[V_Z];
    V.v = P->vec[V_V];
    V.y = P->vec[V_Y];
    V.q = P->vec[V_Q];
    return V;
}

Batch pool_batch(const pbcg_pool *P)
{
    Batch B;
    B.nsys = P->cfg.max_slots;
    B.ntiles = P->max_tiles;
    B.tile_sys = P->tile_sys;
    B.sys_t0 = P->t0;
    B.sys_t1 = P->t1;
    B.ctl = P->ctl;
    B.acc = P->acc;
    B.part = P->part;
    B.done = P->done;
    B.flag = P->flag;
    B.lv_n = P->lv_n;
    B.lv_pre = P->lv_pre;
    B.lv_t0 = P->lv_t0;
    return B;
}

template <int MODE>
std::vector<BKernel> pool_body(int alg)
{
    std::vector<BKernel> k;
    k.push_back({(void *)k_batched<MODE, PoolSetup1>, "pool_setup1", 0});
    if (alg != PBCG_ALG_BICGSTAB) {
        k.push_back({(void *)k_batched<MODE, PoolSetup2>, "pool_setup2", 0});
        k.push_back({(void *)k_batched<0, PoolSetup3>, "pool_setup3", 0});
    }
    k.push_back({(void *)k_batched<1, StepTrueRes<false>>, "pool_true_res", 0});
    if (alg == PBCG_ALG_PIPELINED_RR) {
        k.push_back({(void *)k_batched<0, StepRR<1>>, "pool_rr1", 0});
        k.push_back({(void *)k_batched<0, StepRR<2>>, "pool_rr2", 0});
        k.push_back({(void *)k_batched<0, StepRR<3>>, "pool_rr3", 0});
        k.push_back({(void *)k_batched<0, StepRR<4>>, "pool_rr4", 0});
    }
    if (alg == PBCG_ALG_BICGSTAB) {
        k.push_back({(void *)k_batched<MODE, StepBicgP>, "pool_bicg_p", 0});
        k.push_back({(void *)k_batched<MODE, StepBicgA>, "pool_bicg_a", 0});
        k.push_back({(void *)k_batched<MODE, StepBicgB>, "pool_bicg_b", 0});
        k.push_back({(void *)k_batched<MODE, StepBicgC>, "pool_bicg_c", 0});
    } else {
        k.push_back({(void *)k_bstaged<MODE, BPipeX>, "pool_pipe_x", StageLayout<BPipeX::NV, true, false>::TOTAL});
        k.push_back({(void *)k_bstaged<MODE, BPipeY>, "pool_pipe_y", StageLayout<BPipeY::NV, true, false>::TOTAL});
    }
    return k;
}

// graph: list the live tiles, then WHILE { setup passes of new slots, true
// residual of candidates, [replacement passes], the iteration's passes, step
// control (which lists the live tiles again) }
int pool_build_graph(pbcg_ctx *ctx, pbcg_pool *P)
{
    CK(cudaGraphCreate(&P->graph, 0));
    cudaGraphConditionalHandle h;
    CK(cudaGraphConditionalHandleCreate(&h, P->graph, 1, cudaGraphCondAssignDefault));
    Mat A = pool_mat(P);
    Vecs V = pool_vecs(P);
    Batch B = pool_batch(P);
    unsigned long long hv = (unsigned long long)h;
    int *lvn = P->lv_n, *lvp = P->lv_pre, *lvt = P->lv_t0, *left = P->left;
    auto ctl_node = [&](cudaGraph_t g, cudaGraphNode_t *dep, int first, cudaGraphNode_t *node) -> int {
        int f = first;
        void *cargs[] = {&B, &lvn, &lvp, &lvt, &left, &hv, &f};
        cudaKernelNodeParams kp{};
        kp.func = (void *)k_pool_ctl;
        kp.gridDim = dim3(1);
        kp.blockDim = dim3(1024);
        kp.kernelParams = cargs;
        CK(cudaGraphAddKernelNode(node, g, dep, dep ? 1 : 0, &kp));
        return 0;
    };
    cudaGraphNode_t list0;
    int rc = ctl_node(P->graph, nullptr, 1, &list0);
    if (rc)
        return rc;
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cnode;
    CK(cudaGraphAddNode(&cnode, P->graph, &list0, nullptr, 1, &cp));
    cudaGraph_t g = cp.conditional.phGraph_out[0];
    std::vector<BKernel> body = P->cfg.dot_mode ? pool_body<1>(P->cfg.alg) : pool_body<0>(P->cfg.alg);
    cudaGraphNode_t prev = nullptr;
    for (auto &bk : body) {
        void *args[3] = {&A, &V, &B};
        cudaKernelNodeParams kp{};
        kp.func = bk.fn;
        kp.gridDim = dim3(bgrid(ctx, bk.fn, B.ntiles, bk.smem));
        kp.blockDim = dim3(THREADS);
        kp.sharedMemBytes = (unsigned)bk.smem;
        kp.kernelParams = args;
        cudaGraphNode_t node;
        CK(cudaGraphAddKernelNode(&node, g, prev ? &prev : nullptr, prev ? 1 : 0, &kp));
        prev = node;
    }
    cudaGraphNode_t last;
    rc = ctl_node(g, &prev, 0, &last);
    if (rc)
        return rc;
    CK(cudaGraphInstantiate(&P->exec, P->graph, 0));
    P->body_kernels = (int)body.size() + 1;
    return 0;
}

// SELL-32 device copy of a validated host CSR matrix with n rows (ncols > n:
// the columns n .. ncols - 1 are a halo, see build_sell); not registered in
// ctx->mats
int make_mat(pbcg_ctx *ctx, int n, int ncols, std::vector<int32_t> &&hrp, std::vector<int32_t> &&hci,
             std::vector<double> &&hva, pbcg_mat **out)
{
    const long long nnz = (long long)hci.size();
    Sell S;
    if (!build_sell(n, hrp.data(), hci.data(), hva.data(), S, ncols))
        return fail(ctx, PBCG_ERR_INVALID, "padded matrix exceeds 2^31 entries");
    pbcg_mat *m = new pbcg_mat();
    m->n = n;
    m->ncols = ncols > n ? ncols : n;
    m->nnz = nnz;
    m->nslices = S.nslices;
    m->padded = S.padded;
    m->sl_off = m->rlen = m->ci = m->perm = m->tmeta = nullptr;
    m->lci = nullptr;
    m->va = nullptr;
    m->narrow = S.narrow;
    m->bl = nullptr;
    m->h_sloff.assign(S.sl_off.begin(), S.sl_off.begin() + (S.nslices + 1));
    m->h_rp = std::move(hrp);
    m->h_ci = std::move(hci);
    m->h_va = std::move(hva);
    size_t P = (size_t)(S.padded ? S.padded : 1);
    cudaError_t e = cudaMalloc(&m->sl_off, sizeof(int) * S.sl_off.size());
    if (e == cudaSuccess)
        e = cudaMalloc(&m->rlen, sizeof(int) * S.rlen.size());
    if (e == cudaSuccess)
        e = cudaMalloc(&m->ci, sizeof(int) * P);
    if (e == cudaSuccess)
        e = cudaMalloc(&m->va, sizeof(double) * P);
    if (e == cudaSuccess && S.permuted)
        e = cudaMalloc(&m->perm, sizeof(int) * (size_t)n);
    if (e == cudaSuccess)
        e = cudaMalloc(&m->lci, sizeof(uint16_t) * P);
    if (e == cudaSuccess)
        e = cudaMalloc(&m->tmeta, sizeof(int) * S.tmeta.size());
    if (e == cudaSuccess && S.padded)
        e = cudaMemcpy(m->lci, S.lci.data(), sizeof(uint16_t) * (size_t)S.padded, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(m->tmeta, S.tmeta.data(), sizeof(int) * S.tmeta.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(m->sl_off, S.sl_off.data(), sizeof(int) * S.sl_off.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(m->rlen, S.rlen.data(), sizeof(int) * S.rlen.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && S.padded)
        e = cudaMemcpy(m->ci, S.ci.data(), sizeof(int) * (size_t)S.padded, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && S.padded)
        e = cudaMemcpy(m->va, S.va.data(), sizeof(double) * (size_t)S.padded, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && S.permuted)
        e = cudaMemcpy(m->perm, S.perm.data(), sizeof(int) * (size_t)n, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        mat_release(m);
        return fail(ctx, e == cudaErrorMemoryAllocation ? PBCG_ERR_OOM : PBCG_ERR_CUDA, "matrix upload: %s",
                    cudaGetErrorString(e));
    }
    *out = m;
    return 0;
}

// ---------------------------------------------------------------------------
// launch variants and the autotuner (pbcg_tune)
// ---------------------------------------------------------------------------
pbcg_variant variant_of(const pbcg_mat *m)
{
    pbcg_variant v;
    v.staged = m->v_staged;
    v.order = m->v_order;
    v.ctas_per_sm = m->v_ctas;
    v.batched_ctas_per_sm = m->b_ctas;
    v.us_per_iter = m->v_us;
    return v;
}

bool variant_ok(const pbcg_variant &v)
{
    return (v.staged == 0 || v.staged == 1) && v.order >= 0 && v.order <= 3 && v.ctas_per_sm >= 0 &&
           v.ctas_per_sm <= 32 && v.batched_ctas_per_sm >= 0 && v.batched_ctas_per_sm <= 32;
}

void apply_variant(pbcg_mat *m, const pbcg_variant &v)
{
    m->v_staged = v.staged;
    m->v_order = v.order;
    m->v_ctas = v.ctas_per_sm;
    m->b_ctas = v.batched_ctas_per_sm;
    m->v_us = v.us_per_iter;
}

// FNV-1a over 64-bit words
struct Fnv {
    unsigned long long h = 1469598103934665603ull;
    void add(unsigned long long v)
    {
        for (int k = 0; k < 8; k++) {
            h ^= (v >> (8 * k)) & 0xffull;
            h *= 1099511628211ull;
        }
    }
};

std::string tune_key(const pbcg_ctx *ctx, const pbcg_mat *m, int alg, int mode, int nsys, const int32_t *srp)
{
    // row-length histogram: how many rows have each length (sparse, by length)
    std::map<int, long long> hist;
    for (int i = 0; i < m->n; i++)
        hist[m->h_rp[(size_t)i + 1] - m->h_rp[(size_t)i]]++;
    Fnv f;
    for (auto &e : hist) {
        f.add((unsigned long long)e.first);
        f.add((unsigned long long)e.second);
    }
    Fnv g;
    for (int k = 0; nsys > 0 && k <= nsys; k++)
        g.add((unsigned long long)(unsigned)srp[k]);
    char buf[256];
    snprintf(buf, sizeof buf, "n=%d;nnz=%lld;rows=%016llx;nsys=%d;sys=%016llx;alg=%d;mode=%d;sms=%d", m->n, m->nnz, f.h,
             nsys, nsys > 0 ? g.h : 0ull, alg, mode, ctx->num_sms);
    return buf;
}

// the variant recorded for `key` in a JSON-lines cache file, if any
bool cache_find(const char *path, const std::string &key, pbcg_variant *v)
{
    FILE *f = path ? fopen(path, "r") : nullptr;
    if (!f)
        return false;
    char line[1024];
    bool found = false;
    const std::string want = "\"key\": \"" + key + "\"";
    while (fgets(line, sizeof line, f)) {
        if (!strstr(line, want.c_str()))
            continue;
        pbcg_variant t{};
        const char *p;
        if ((p = strstr(line, "\"staged\": ")) && sscanf(p + 10, "%d", &t.staged) == 1 &&
            (p = strstr(line, "\"order\": ")) && sscanf(p + 9, "%d", &t.order) == 1 &&
            (p = strstr(line, "\"ctas_per_sm\": ")) && sscanf(p + 15, "%d", &t.ctas_per_sm) == 1 &&
            (p = strstr(line, "\"batched_ctas_per_sm\": ")) && sscanf(p + 23, "%d", &t.batched_ctas_per_sm) == 1 &&
            (p = strstr(line, "\"us_per_iter\": ")) && sscanf(p + 15, "%lf", &t.us_per_iter) == 1 && variant_ok(t)) {
            *v = t;                  // the last record of a key wins
            found = true;
        }
    }
    fclose(f);
    return found;
}

void cache_add(const char *path, const std::string &key, const pbcg_variant &v)
{
    FILE *f = path ? fopen(path, "a") : nullptr;
    if (!f)
        return;
    fprintf(f,
            "{\"key\": \"%s\", \"staged\": %d, \"order\": %d, \"ctas_per_sm\": %d, \"batched_ctas_per_sm\": %d, "
            "\"us_per_iter\": %.4f}\n",
            key.c_str(), v.staged, v.order, v.ctas_per_sm, v.batched_ctas_per_sm, v.us_per_iter);
    fclose(f);
}

int tune_impl(pbcg_ctx *ctx, pbcg_mat *m, int alg, int mode, int32_t nsys, const int32_t *srp, int32_t iters,
              const char *cache_path, pbcg_variant *chosen, pbcg_variant *tried, int32_t cap, int32_t *ntried)
{
    if (!m || !ctx->mats.count(m))
        return fail(ctx, PBCG_ERR_INVALID, "unknown matrix handle");
    if (alg != PBCG_ALG_BICGSTAB && alg != PBCG_ALG_PIPELINED && alg != PBCG_ALG_PIPELINED_RR)
        return fail(ctx, PBCG_ERR_INVALID, "unknown algorithm %d", alg);
    if (mode != PBCG_DOT_PLAIN && mode != PBCG_DOT_EXACT)
        return fail(ctx, PBCG_ERR_INVALID, "unknown dot mode %d", mode);
    if (iters < 1 || iters > 30000 || nsys < 0 || (nsys > 0 && !srp) || cap < 0 || (cap > 0 && !tried))
        return fail(ctx, PBCG_ERR_INVALID, "bad tuning arguments");
    if (nsys > 0) {
        if (srp[0] != 0 || srp[nsys] != m->n)
            return fail(ctx, PBCG_ERR_INVALID, "sys_row_ptr must run from 0 to n");
        for (int k = 0; k < nsys; k++)
            if (srp[k + 1] <= srp[k])
                return fail(ctx, PBCG_ERR_INVALID, "sys_row_ptr must increase strictly");
    }
    if (ntried)
        *ntried = 0;
    CK(cudaSetDevice(ctx->device));
    const std::string key = tune_key(ctx, m, alg, mode, nsys, srp);
    pbcg_variant base = variant_of(m);
    pbcg_variant got;
    if (cache_find(cache_path, key, &got)) {
        // the part of the variant this key tunes; the rest stays
        if (nsys > 0) {
            base.batched_ctas_per_sm = got.batched_ctas_per_sm;
        } else {
            base.staged = got.staged;
            base.order = got.order;
            base.ctas_per_sm = got.ctas_per_sm;
        }
        base.us_per_iter = got.us_per_iter;
        got = base;
        apply_variant(m, got);
        if (chosen)
            *chosen = got;
        return 0;
    }
    // candidates, the default first
    std::vector<pbcg_variant> cand;
    pbcg_variant d = base;
    if (nsys > 0) {
        for (int c : {0, 1}) {
            d.batched_ctas_per_sm = c;
            cand.push_back(d);
        }
    } else {
        ClusterShape cs;
        const bool cluster = alg != PBCG_ALG_PIPELINED_RR && ctx->small_cluster && cluster_shape(ctx, m, alg, mode, &cs);
        for (int st : {1, 0}) {
            if (st == 0 && (!m->narrow || cluster))
                continue;           // nothing to stage either way
            for (int alt : {0, 1, 2}) {
                if (alt && cluster)
                    continue;
                for (int c : {0, 1}) {
                    if (c && cluster)
                        continue;
                    d.staged = st;
                    // this staging's default order, the other pure order, round-robin with a claimed tail
                    d.order = alt == 0 ? 0 : alt == 1 ? ((m->narrow && st) ? 2 : 1) : 3;
                    d.ctas_per_sm = c;
                    cand.push_back(d);
                }
            }
        }
    }
    // trial system: b = A * ones, x0 = 0, no stop (tol far below any residual)
    struct Buf {
        double *p = nullptr;
        ~Buf() { if (p) cudaFree(p); }
    } one, bb, xx;
    const size_t n = (size_t)m->n;
    CK(cudaMalloc(&one.p, sizeof(double) * n));
    CK(cudaMalloc(&bb.p, sizeof(double) * n));
    CK(cudaMalloc(&xx.p, sizeof(double) * n));
    {
        std::vector<double> h(n, 1.0);
        CK(cudaMemcpy(one.p, h.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
    }
    int rc;
    if ((rc = pbcg_spmv(ctx, m, one.p, bb.p)))
        return rc;
    std::vector<double> tols((size_t)std::max(nsys, 1), 1e-300);
    std::vector<pbcg_result> res((size_t)std::max(nsys, 1));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    struct Ev {
        cudaEvent_t a, b;
        ~Ev() { cudaEventDestroy(a); cudaEventDestroy(b); }
    } ev{e0, e1};
    // one trial solve of `its` iterations; *ms its CUDA-event time (NULL: untimed)
    auto trial = [&](int its, float *ms) -> int {
        CK(cudaMemsetAsync(xx.p, 0, sizeof(double) * n, ctx->stream));
        if (ms)
            CK(cudaEventRecord(e0, ctx->stream));
        int r = nsys > 0 ? solve_batched_impl(ctx, m, nsys, srp, bb.p, xx.p, tols.data(), its, alg, mode, res.data())
                         : solve_impl(ctx, m, bb.p, xx.p, 1e-300, its, alg, mode, res.data(), nullptr);
        if (r < 0)
            return r;
        if (ms) {
            CK(cudaEventRecord(e1, ctx->stream));
            CK(cudaEventSynchronize(e1));
            CK(cudaEventElapsedTime(ms, e0, e1));
        }
        return 0;
    };
    pbcg_variant best = base;
    double best_us = 1e300;
    int k = 0;
    for (auto &c : cand) {
        apply_variant(m, c);
        // iterations iters+1 .. 3 iters: the difference of two timed trials
        // (setup, the first iterations and the true-residual check drop out)
        float t1 = 0.f, t3 = 0.f;
        if ((rc = trial(iters, nullptr)) || (rc = trial(iters, &t1)) || (rc = trial(3 * iters, &t3))) {
            apply_variant(m, base);
            return rc;
        }
        const double us = 1e3 * (double)(t3 - t1) / (2.0 * iters);
        c.us_per_iter = us;
        if (tried && k < cap)
            tried[k] = c;
        k++;
        if (us < best_us) {
            best_us = us;
            best = c;
        }
    }
    if (ntried)
        *ntried = k;
    apply_variant(m, best);
    cache_add(cache_path, key, best);
    if (chosen)
        *chosen = best;
    return 0;
}

// ---------------------------------------------------------------------------
// row-partitioned solves (one rank's block; see pbcg_part_* in pbcg.h)
// ---------------------------------------------------------------------------
// Host plan of one block: its halo (external columns, ascending, hence grouped
// by owner), how many of them each rank owns, and every entry's local column.
int part_plan_host(int nranks, int rank, const int32_t *rs, long long nnz, const int32_t *rp, const int32_t *ci,
                   std::vector<int32_t> &halo, std::vector<int32_t> &recv_counts, std::vector<int32_t> *local,
                   std::string &why)
{
    char buf[200];
    if (nranks < 1 || rank < 0 || rank >= nranks) {
        why = "need 1 <= nranks and 0 <= rank < nranks";
        return PBCG_ERR_INVALID;
    }
    if (rs[0] != 0) {
        why = "row_starts[0] must be 0";
        return PBCG_ERR_INVALID;
    }
    for (int k = 0; k < nranks; k++)
        if (rs[k + 1] < rs[k]) {
            snprintf(buf, sizeof buf, "row_starts decreases at rank %d", k);
            why = buf;
            return PBCG_ERR_INVALID;
        }
    const int row0 = rs[rank], nloc = rs[rank + 1] - rs[rank], nglob = rs[nranks];
    if (nloc < 1 || nloc > INT32_MAX / 2) {
        why = "the rank's block must hold 1 .. 2^30 - 1 rows";
        return PBCG_ERR_INVALID;
    }
    if (nnz < 0 || nnz >= (1ll << 31) || rp[0] != 0 || (long long)rp[nloc] != nnz) {
        why = "row_ptr must start at 0 and end at nnz < 2^31";
        return PBCG_ERR_INVALID;
    }
    for (int i = 0; i < nloc; i++)
        if (rp[i + 1] < rp[i]) {
            snprintf(buf, sizeof buf, "row_ptr decreases at local row %d", i);
            why = buf;
            return PBCG_ERR_INVALID;
        }
    for (long long k = 0; k < nnz; k++)
        if (ci[k] < 0 || ci[k] >= nglob) {
            snprintf(buf, sizeof buf, "col_idx[%lld] = %d outside [0, %d)", k, ci[k], nglob);
            why = buf;
            return PBCG_ERR_INVALID;
        }
    halo.clear();
    for (long long k = 0; k < nnz; k++)
        if (ci[k] < row0 || ci[k] >= row0 + nloc)
            halo.push_back(ci[k]);
    std::sort(halo.begin(), halo.end());
    halo.erase(std::unique(halo.begin(), halo.end()), halo.end());
    if ((long long)nloc + (long long)halo.size() > INT32_MAX / 2) {
        why = "rows plus halo exceed 2^30 - 1";
        return PBCG_ERR_INVALID;
    }
    recv_counts.assign((size_t)nranks, 0);
    int owner = 0;
    for (int32_t c : halo) {
        while (c >= rs[owner + 1])
            owner++;
        recv_counts[(size_t)owner]++;
    }
    if (local) {
        local->resize((size_t)nnz);
        for (long long k = 0; k < nnz; k++) {
            const int32_t c = ci[k];
            (*local)[(size_t)k] = (c >= row0 && c < row0 + nloc)
                                      ? c - row0
                                      : nloc + (int32_t)(std::lower_bound(halo.begin(), halo.end(), c) - halo.begin());
        }
    }
    return 0;
}

}  // namespace

struct pbcg_part {
    pbcg_ctx *ctx = nullptr;
    pbcg_comm comm{};
    int nranks = 1, rank = 0, row0 = 0, nloc = 0, nhalo = 0, nsend = 0;
    pbcg_mat *m = nullptr;                       // rows nloc, columns nloc + nhalo (local numbering)
    Workspace ws;                                // vectors hold the halo after the block's rows
    std::vector<int64_t> sb, sd, rb, rd;         // alltoallv byte counts and offsets of a halo exchange
    int *d_send_idx = nullptr;                   // [nsend] solver-order rows the other ranks gather
    double *d_send = nullptr;                    // [nsend]
    double *h_send = nullptr, *h_recv = nullptr; // pinned
    long long *h_red = nullptr, *d_red = nullptr;
    GAcc *h_g = nullptr;                         // pinned copy of the block's global accumulators
    double *h_loc = nullptr;
    int *h_err = nullptr;
    int red_cap = 0;
};

namespace {

void part_release(pbcg_part *P)
{
    if (!P)
        return;
    if (P->m)
        mat_release(P->m);
    free_ws(P->ws);
    cudaFree(P->d_send_idx);
    cudaFree(P->d_send);
    cudaFree(P->d_red);
    cudaFreeHost(P->h_send);
    cudaFreeHost(P->h_recv);
    cudaFreeHost(P->h_red);
    cudaFreeHost(P->h_g);
    cudaFreeHost(P->h_loc);
    cudaFreeHost(P->h_err);
    delete P;
}

// every rank's flag summed: nonzero when any rank reported a problem
int comm_any(pbcg_ctx *ctx, const pbcg_comm &cm, long long flag, long long *sum)
{
    int64_t v = flag;
    if (cm.allreduce_sum_i64(cm.user, &v, 1) != 0)
        return fail(ctx, PBCG_ERR_COMM, "allreduce callback failed");
    *sum = v;
    return 0;
}

// copy the entries of solver vector v that other ranks need to them, and
// theirs into v's halo (after the block's rows)
int part_halo(pbcg_part *P, double *v)
{
    pbcg_ctx *ctx = P->ctx;
    if (P->nranks == 1)
        return 0;
    if (P->nsend > 0) {
        int m = P->nsend;
        const int *idx = P->d_send_idx;
        double *out = P->d_send;
        void *args[4] = {&m, (void *)&idx, &v, &out};
        CK(cudaLaunchKernel((void *)k_halo_pack, dim3(std::min(ctx->num_sms * 4, (m + 255) / 256)), dim3(256), args,
                            0, ctx->stream));
        CK(cudaMemcpyAsync(P->h_send, P->d_send, sizeof(double) * (size_t)m, cudaMemcpyDeviceToHost, ctx->stream));
    }
    CK(cudaStreamSynchronize(ctx->stream));
    if (P->comm.alltoallv(P->comm.user, P->h_send, P->sb.data(), P->sd.data(), P->h_recv, P->rb.data(),
                          P->rd.data()) != 0)
        return fail(ctx, PBCG_ERR_COMM, "alltoallv callback failed (halo exchange)");
    if (P->nhalo > 0)
        CK(cudaMemcpyAsync(v + P->nloc, P->h_recv, sizeof(double) * (size_t)P->nhalo, cudaMemcpyHostToDevice,
                           ctx->stream));
    return 0;
}

// the reduction point after a pass with nd dots: add the ranks' shares and
// run k_dist_finish (rounding and the scalar step `which`)
int part_reduce(pbcg_part *P, int nd, int mode, int which)
{
    pbcg_ctx *ctx = P->ctx;
    Work *wk = P->ws.wk;
    if (mode)
        CK(cudaMemcpyAsync(P->h_g, wk->g, sizeof(GAcc) * (size_t)nd, cudaMemcpyDeviceToHost, ctx->stream));
    else
        CK(cudaMemcpyAsync(P->h_loc, wk->loc, sizeof(double) * (size_t)nd, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(P->h_err, &P->ws.ctl->err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    const int words = mode ? 1 + nd * RED_EXACT_STRIDE : 1 + P->nranks * nd;
    long long *r = P->h_red;
    memset(r, 0, sizeof(long long) * (size_t)words);
    r[0] = *P->h_err ? 1 : 0;
    if (mode) {
        for (int d = 0; d < nd; d++) {
            const GAcc &g = P->h_g[d];
            for (int k = 0; k < NDIG; k++)
                r[1 + d * RED_EXACT_STRIDE + k] = (k >= g.kmin && k <= g.kmax) ? (long long)g.dig[k] : 0ll;
            r[1 + d * RED_EXACT_STRIDE + NDIG] = g.nf ? 1 : 0;
        }
    } else {
        for (int d = 0; d < nd; d++) {
            long long bits;
            memcpy(&bits, &P->h_loc[d], sizeof bits);
            r[1 + P->rank * nd + d] = bits;
        }
    }
    if (P->nranks > 1 && P->comm.allreduce_sum_i64(P->comm.user, reinterpret_cast<int64_t *>(r), words) != 0)
        return fail(ctx, PBCG_ERR_COMM, "allreduce callback failed (dot products)");
    CK(cudaMemcpyAsync(P->d_red, r, sizeof(long long) * (size_t)words, cudaMemcpyHostToDevice, ctx->stream));
    Ctl *c = P->ws.ctl;
    const long long *red = P->d_red;
    int nranks = P->nranks;
    void *args[6] = {&c, &wk, (void *)&red, &nd, &nranks, &which};
    CK(cudaLaunchKernel(mode ? (void *)k_dist_finish<1> : (void *)k_dist_finish<0>, dim3(1), dim3(THREADS), args, 0,
                        ctx->stream));
    return 0;
}

int part_solve_impl(pbcg_part *P, const double *b, double *x, double tol, int32_t maxit, int alg, int mode,
                    pbcg_result *out)
{
    auto t0 = std::chrono::steady_clock::now();
    pbcg_ctx *ctx = P->ctx;
    // arguments checked here and agreed over the ranks before any exchange
    long long bad = 0;
    if (!b || !x)
        fail(ctx, PBCG_ERR_INVALID, "b and x must not be NULL"), bad = 1;
    else if (!(tol > 0.0))
        fail(ctx, PBCG_ERR_INVALID, "tol must be > 0"), bad = 1;
    else if (maxit < 0 || maxit == INT32_MAX)
        fail(ctx, PBCG_ERR_INVALID, "maxit must be in 0 .. 2^31 - 2"), bad = 1;
    else if (alg != PBCG_ALG_BICGSTAB && alg != PBCG_ALG_PIPELINED)
        fail(ctx, PBCG_ERR_INVALID, "a partitioned solve runs PBCG_ALG_BICGSTAB or PBCG_ALG_PIPELINED"), bad = 1;
    else if (mode != PBCG_DOT_PLAIN && mode != PBCG_DOT_EXACT)
        fail(ctx, PBCG_ERR_INVALID, "unknown dot mode %d", mode), bad = 1;
    int rc = 0;
    if (!bad && cudaSetDevice(ctx->device) != cudaSuccess)
        fail(ctx, PBCG_ERR_CUDA, "cudaSetDevice failed"), bad = 1;
    if (!bad && (rc = ensure_ws_in(ctx, P->ws, std::max<long long>(P->nloc, (long long)P->nloc + P->nhalo),
                                   maxit + 1)))
        bad = 1;
    if (!bad) {
        // this workspace's merges belong to a partitioned solve
        int one = 1;
        if (cudaMemcpy(&P->ws.wk->dist, &one, sizeof one, cudaMemcpyHostToDevice) != cudaSuccess)
            fail(ctx, PBCG_ERR_CUDA, "workspace setup failed"), bad = 1;
    }
    long long anybad = 0;
    if (P->nranks > 1) {
        if ((rc = comm_any(ctx, P->comm, bad, &anybad)))
            return rc;
    } else {
        anybad = bad;
    }
    if (anybad) {
        if (bad)
            return rc ? rc : PBCG_ERR_INVALID;
        return fail(ctx, PBCG_ERR_INVALID, "another rank refused the solve's arguments");
    }
    Workspace &ws = P->ws;
    const pbcg_mat *m = P->m;
    double *tmp = ws.vec[V_TMP];
    if ((rc = vec_in(ctx, m, b, ws.vec[V_B], tmp)) || (rc = vec_in(ctx, m, x, ws.vec[V_X], tmp)))
        return rc;
    Ctl h;
    memset(&h, 0, sizeof h);
    h.maxit = maxit;
    h.status = ST_RUNNING;
    h.tol = tol;
    h.target = tol;
    h.alg = (alg == PBCG_ALG_BICGSTAB) ? ALG_BICGSTAB : ALG_PIPELINED;
    h.hist = ws.hist;
    h.hist_cap = maxit + 1;
    h.trueres = __builtin_nan("");
    *ctx->h_ctl = h;
    CK(cudaMemcpyAsync(ws.ctl, ctx->h_ctl, sizeof(Ctl), cudaMemcpyHostToDevice, ctx->stream));
    Mat A = mat_of(m);
    Vecs V = vecs_of(ws);
    Ctl *c = ws.ctl;
    Work *wk = ws.wk;
    Launcher L{ctx, nullptr, 0, {}};
    auto status = [&](int *st) -> int {
        int r = read_ctl(ctx, c);
        *st = ctx->h_ctl->status;
        return r;
    };
    const bool pipe = alg == PBCG_ALG_PIPELINED;
    // setup: r0 = b - A x0 (and w0 = A r0, t0 = A w0)
    if ((rc = part_halo(P, V.x)) || (rc = L.go("setup1", mode ? Kern<1>::setup1() : Kern<0>::setup1(), A, V, c, wk, 1)) ||
        (rc = part_reduce(P, 2, mode, pipe ? FIN_SETUP1_P : FIN_SETUP1_B)))
        return rc;
    if (pipe) {
        int st = 0;
        if ((rc = part_halo(P, V.r0)) ||
            (rc = L.go("setup2", mode ? Kern<1>::setup2() : Kern<0>::setup2(), A, V, c, wk, 1)) ||
            (rc = part_reduce(P, 1, mode, FIN_SETUP2)) || (rc = status(&st)))
            return rc;
        if (st == ST_RUNNING || st == ST_CANDIDATE)
            if ((rc = part_halo(P, V.w)) || (rc = L.go("setup3", (void *)k_setup3, A, V, c, wk, 0)))
                return rc;
    }
    auto body = body_kernels(alg, mode, m->narrow);
    bool true_done = false;
    for (;;) {
        int st = 0;
        if ((rc = status(&st)))
            return rc;
        if (st == ST_CANDIDATE) {
            if ((rc = part_halo(P, V.x)) || (rc = L.go("true_res", (void *)k_true_res, A, V, c, wk, 1)) ||
                (rc = part_reduce(P, 2, 1, FIN_TRUE)))
                return rc;
            true_done = true;
            continue;
        }
        if (st != ST_RUNNING)
            break;
        true_done = false;
        if (pipe) {
            const BodyKernel &bx = body[0], &by = body[1];
            if ((rc = part_halo(P, V.w)) || (rc = L.go(bx.name, bx.fn, A, V, c, wk, 1, bx.smem)) ||
                (rc = part_reduce(P, 4, mode, FIN_X)) || (rc = status(&st)))
                return rc;
            if (st != ST_RUNNING)
                continue;
            if ((rc = part_halo(P, V.z)) || (rc = L.go(by.name, by.fn, A, V, c, wk, 1, by.smem)) ||
                (rc = part_reduce(P, 3, mode, FIN_Y)))
                return rc;
        } else {
            const BodyKernel &kp = body[0], &ka = body[1], &kq = body[2], &kb = body[3], &kc = body[4];
            if ((rc = L.go(kp.name, kp.fn, A, V, c, wk, 1, kp.smem)) || (rc = part_halo(P, V.p)) ||
                (rc = L.go(ka.name, ka.fn, A, V, c, wk, 1, ka.smem)) || (rc = part_reduce(P, 1, mode, FIN_BA)) ||
                (rc = status(&st)))
                return rc;
            if (st != ST_RUNNING)
                continue;
            if ((rc = L.go(kq.name, kq.fn, A, V, c, wk, 0)) || (rc = part_halo(P, V.q)) ||
                (rc = L.go(kb.name, kb.fn, A, V, c, wk, 1, kb.smem)) || (rc = part_reduce(P, 2, mode, FIN_BB)) ||
                (rc = status(&st)))
                return rc;
            if (st != ST_RUNNING)
                continue;
            if ((rc = L.go(kc.name, kc.fn, A, V, c, wk, 1, kc.smem)) || (rc = part_reduce(P, 2, mode, FIN_BC)))
                return rc;
        }
    }
    if (!true_done) {
        if ((rc = part_halo(P, V.x)) || (rc = L.go("true_res", (void *)k_true_res, A, V, c, wk, 1)) ||
            (rc = part_reduce(P, 2, 1, FIN_TRUE)) || (rc = read_ctl(ctx, c)))
            return rc;
    }
    Ctl fin_ctl = *ctx->h_ctl;
    if (fin_ctl.err || fin_ctl.status == ST_TIMEOUT)
        return fail(ctx, PBCG_ERR_TIMEOUT, "a bounded device wait expired on some rank");
    if ((rc = vec_out(ctx, m, ws.vec[V_X], x, tmp)))
        return rc;
    int hl = std::min(fin_ctl.it + 1, maxit + 1);
    ctx->hist.assign((size_t)hl, 0.0);
    CK(cudaMemcpyAsync(ctx->hist.data(), ws.hist, sizeof(double) * (size_t)hl, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->have_hist = true;
    ctx->last_batched = false;
    if (out) {
        out->iters = fin_ctl.it;
        out->status = fin_ctl.status;
        out->relres_recursive = fin_ctl.res;
        out->relres_true = fin_ctl.trueres;
        out->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        out->launches = (int32_t)L.launches;
        out->reserved = 0;
    }
    return fin_ctl.status;
}

bool final_status(const Ctl &c)
{
    return (c.status >= 0 && c.status <= 3) || c.status == ST_INVALID || c.status == ST_TIMEOUT || c.err;
}

}  // namespace


extern "C" {

int pbcg_create(pbcg_ctx **out, int device, void *cuda_stream)
{
    if (!out)
        return PBCG_ERR_INVALID;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return PBCG_ERR_INVALID;
    pbcg_ctx *ctx = new pbcg_ctx();
    ctx->device = device;
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) {
        delete ctx;
        return PBCG_ERR_CUDA;
    }
    cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    ctx->maxgrid = ctx->num_sms * (2048 / THREADS);
    if (cuda_stream) {
        ctx->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete ctx;
            return PBCG_ERR_CUDA;
        }
        ctx->own_stream = true;
    }
    if (cudaMallocHost(&ctx->h_ctl, sizeof(Ctl)) != cudaSuccess) {
        if (ctx->own_stream)
            cudaStreamDestroy(ctx->stream);
        delete ctx;
        return PBCG_ERR_OOM;
    }
    *out = ctx;
    return 0;
}

void pbcg_destroy(pbcg_ctx *ctx)
{
    if (!ctx)
        return;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    for (auto *m : ctx->mats)
        mat_release(m);
    ctx->mats.clear();
    free_ws(ctx->ws);
    free_batch_graph(ctx);
    for (auto &p : ctx->b.vec)
        cudaFree(p);
    cudaFree(ctx->b.ctl);
    cudaFree(ctx->b.acc);
    cudaFree(ctx->b.part);
    cudaFree(ctx->b.done);
    cudaFree(ctx->b.flag);
    cudaFree(ctx->b.hist);
    cudaFree(ctx->b.io);
    if (ctx->h_ctl)
        cudaFreeHost(ctx->h_ctl);
    if (ctx->own_stream)
        cudaStreamDestroy(ctx->stream);
    delete ctx;
}

const char *pbcg_last_error(pbcg_ctx *ctx)
{
    return ctx ? ctx->err.c_str() : "no context";
}

int pbcg_csr_upload(pbcg_ctx *ctx, int32_t n, int64_t nnz, const int32_t *row_ptr, const int32_t *col_idx,
                    const double *vals, int ptrs_on_device, pbcg_mat **out)
{
    (void)ptrs_on_device;
    if (!ctx)
        return PBCG_ERR_INVALID;
    if (!out || !row_ptr || (nnz > 0 && (!col_idx || !vals)))
        return fail(ctx, PBCG_ERR_INVALID, "NULL argument");
    *out = nullptr;
    // rows padded to whole 256-row tiles are indexed in int32 by the kernels
    if (n < 1 || n > INT32_MAX / 2)
        return fail(ctx, PBCG_ERR_INVALID, "n must be in 1 .. 2^30 - 1 (got %d)", n);
    if (nnz < 0 || nnz >= (1ll << 31))
        return fail(ctx, PBCG_ERR_INVALID, "nnz out of range (got %lld)", (long long)nnz);
    CK(cudaSetDevice(ctx->device));
    // bring the CSR arrays to the host (validation and layout conversion)
    std::vector<int32_t> hrp((size_t)n + 1), hci((size_t)nnz);
    std::vector<double> hva((size_t)nnz);
    CK(cudaMemcpy(hrp.data(), row_ptr, sizeof(int32_t) * ((size_t)n + 1), cudaMemcpyDefault));
    if (nnz) {
        CK(cudaMemcpy(hci.data(), col_idx, sizeof(int32_t) * (size_t)nnz, cudaMemcpyDefault));
        CK(cudaMemcpy(hva.data(), vals, sizeof(double) * (size_t)nnz, cudaMemcpyDefault));
    }
    int rc = validate_csr_host(ctx, n, nnz, hrp.data(), hci.data());
    if (rc)
        return rc;
    pbcg_mat *m = nullptr;
    if ((rc = make_mat(ctx, n, 0, std::move(hrp), std::move(hci), std::move(hva), &m)))
        return rc;
    ctx->mats.insert(m);
    *out = m;
    return 0;
}

int pbcg_mat_free(pbcg_ctx *ctx, pbcg_mat *m)
{
    if (!ctx)
        return PBCG_ERR_INVALID;
    if (!m)
        return 0;
    if (!ctx->mats.count(m))
        return fail(ctx, PBCG_ERR_INVALID, "unknown matrix handle");
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    if (ctx->ws.loop.mat == m)
        free_loop(ctx->ws.loop);
    if (m->bl && ctx->b.g_layout == (const void *)m->bl)
        free_batch_graph(ctx);             // its nodes point into this matrix's layout
    ctx->mats.erase(m);
    mat_release(m);
    return 0;
}

int pbcg_solve(pbcg_ctx *ctx, const pbcg_mat *A, const double *b, double *x, double tol, int32_t maxit, int alg,
               int dot_mode, pbcg_result *out)
{
    NvtxRange trace("pbcg_solve");
    return solve_impl(ctx, A, b, x, tol, maxit, alg, dot_mode, out, nullptr);
}

int pbcg_profile_solve(pbcg_ctx *ctx, const pbcg_mat *A, const double *b, double *x, double tol, int32_t maxit,
                       int alg, int dot_mode, pbcg_result *out, char (*names)[32], double *ms, int32_t *launches,
                       int32_t cap, int32_t *count)
{
    NvtxRange trace("pbcg_profile_solve");
    Prof prof;
    int rc = solve_impl(ctx, A, b, x, tol, maxit, alg, dot_mode, out, &prof);
    if (rc < 0)
        return rc;
    int k = (int)prof.names.size();
    if (count)
        *count = k;
    for (int i = 0; i < k && i < cap; i++) {
        if (names) {
            strncpy(names[i], prof.names[i].c_str(), 31);
            names[i][31] = '\0';
        }
        if (ms)
            ms[i] = prof.ms[i];
        if (launches)
            launches[i] = prof.count[i];
    }
    return rc;
}

int pbcg_set_option(pbcg_ctx *ctx, int option, int64_t value)
{
    if (!ctx)
        return PBCG_ERR_INVALID;
    if (option == PBCG_OPT_RR_PERIOD) {
        if (value < 1 || value > INT32_MAX)
            return fail(ctx, PBCG_ERR_INVALID, "residual replacement period must be >= 1");
        ctx->rr_period = (int)value;
        return 0;
    }
    if (option == PBCG_OPT_BATCH_GRAPH) {
        if (value != 0 && value != 1)
            return fail(ctx, PBCG_ERR_INVALID, "PBCG_OPT_BATCH_GRAPH takes 0 or 1");
        ctx->batch_graph = (int)value;
        return 0;
    }
    if (option == PBCG_OPT_SMALL_CLUSTER) {
        if (value != 0 && value != 1)
            return fail(ctx, PBCG_ERR_INVALID, "PBCG_OPT_SMALL_CLUSTER takes 0 or 1");
        ctx->small_cluster = (int)value;
        return 0;
    }
    if (option == PBCG_OPT_PRECOND) {
        if (value != PBCG_PRECOND_NONE && value != PBCG_PRECOND_JACOBI)
            return fail(ctx, PBCG_ERR_INVALID, "unknown preconditioner %lld", (long long)value);
        ctx->precond = (int)value;
        return 0;
    }
    return fail(ctx, PBCG_ERR_INVALID, "unknown option %d", option);
}

int pbcg_residual_history(pbcg_ctx *ctx, int32_t sys, double *out, int32_t cap, int32_t *len)
{
    if (!ctx)
        return PBCG_ERR_INVALID;
    if (ctx->last_batched) {
        if (sys < 0 || sys >= (int32_t)ctx->b.last.size())
            return fail(ctx, PBCG_ERR_INVALID, "no residual history for system %d", sys);
        int32_t Lb = std::min(ctx->b.last[sys].it + 1, ctx->b.hist_stride);
        if (len)
            *len = Lb;
        if (out && cap > 0) {
            CK(cudaMemcpy(out, ctx->b.hist + (size_t)sys * ctx->b.hist_stride, sizeof(double) * (size_t)std::min(cap, Lb),
                          cudaMemcpyDeviceToHost));
        }
        return 0;
    }
    if (sys != 0 || !ctx->have_hist)
        return fail(ctx, PBCG_ERR_INVALID, "no residual history for system %d", sys);
    int32_t L = (int32_t)ctx->hist.size();
    if (len)
        *len = L;
    if (out && cap > 0)
        memcpy(out, ctx->hist.data(), sizeof(double) * (size_t)(cap < L ? cap : L));
    return 0;
}

int pbcg_dot(pbcg_ctx *ctx, int64_t n, const double *a, const double *b, int dot_mode, double *out)
{
    if (!ctx)
        return PBCG_ERR_INVALID;
    if (n < 0 || (n > 0 && (!a || !b)) || !out)
        return fail(ctx, PBCG_ERR_INVALID, "bad dot arguments");
    if (dot_mode != PBCG_DOT_PLAIN && dot_mode != PBCG_DOT_EXACT)
        return fail(ctx, PBCG_ERR_INVALID, "unknown dot mode %d", dot_mode);
    CK(cudaSetDevice(ctx->device));
    int rc = ensure_ws(ctx, 0, 0);
    if (rc)
        return rc;
    // host operands are staged in buffers freed on every return
    struct Staging {
        double *p = nullptr;
        ~Staging() { if (p) cudaFree(p); }
    } sa, sb;
    double *&da = sa.p, *&db = sb.p;
    cudaPointerAttributes pa, pb;
    bool a_dev = n > 0 && cudaPointerGetAttributes(&pa, a) == cudaSuccess && pa.type == cudaMemoryTypeDevice;
    bool b_dev = n > 0 && cudaPointerGetAttributes(&pb, b) == cudaSuccess && pb.type == cudaMemoryTypeDevice;
    cudaGetLastError();
    if (n > 0 && !a_dev) {
        CK(cudaMalloc(&da, sizeof(double) * (size_t)n));
        CK(cudaMemcpyAsync(da, a, sizeof(double) * (size_t)n, cudaMemcpyDefault, ctx->stream));
    }
    if (n > 0 && !b_dev) {
        CK(cudaMalloc(&db, sizeof(double) * (size_t)n));
        CK(cudaMemcpyAsync(db, b, sizeof(double) * (size_t)n, cudaMemcpyDefault, ctx->stream));
    }
    const double *pa_ = a_dev ? a : da, *pb_ = b_dev ? b : db;
    int grid = grid_for(ctx, dot_mode ? (void *)k_dot<1> : (void *)k_dot<0>, (n + 31) / 32);
    long long nn = n;
    double *o = ctx->ws.dot_out;
    Work *wk = ctx->ws.wk;
    void *args[5] = {&nn, &pa_, &pb_, &o, &wk};
    CK(cudaLaunchKernel(dot_mode ? (void *)k_dot<1> : (void *)k_dot<0>, dim3(grid), dim3(THREADS), args, 0,
                        ctx->stream));
    CK(cudaMemcpyAsync(out, o, sizeof(double), cudaMemcpyDefault, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return 0;
}

int pbcg_check_wait(pbcg_ctx *ctx, int32_t probes, int32_t *expired, double *seconds)
{
    if (!ctx)
        return PBCG_ERR_INVALID;
    if (probes < 1 || (unsigned)probes > MBAR_CHECK_MAX || !expired || !seconds)
        return fail(ctx, PBCG_ERR_INVALID, "pbcg_check_wait: probes must be in 1 .. 2^22 and outputs non-NULL");
    CK(cudaSetDevice(ctx->device));
    unsigned *d = nullptr;
    CK(cudaMalloc(&d, 3 * sizeof(unsigned)));
    unsigned h[3] = {0u, 0u, 0u};
    cudaError_t e = cudaMemsetAsync(d, 0, 3 * sizeof(unsigned), ctx->stream);
    if (e == cudaSuccess) {
        unsigned pr = (unsigned)probes;
        void *args[2] = {&pr, &d};
        e = cudaLaunchKernel((void *)k_check_wait, dim3(1), dim3(32), args, 0, ctx->stream);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h, d, sizeof h, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(ctx->stream);
    cudaFree(d);
    if (e != cudaSuccess)
        return fail(ctx, PBCG_ERR_CUDA, "pbcg_check_wait: %s", cudaGetErrorString(e));
    int clk = 0;
    cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, ctx->device);     // kHz
    const unsigned long long cyc = ((unsigned long long)h[2] << 32) | h[1];
    *expired = (int32_t)h[0];
    *seconds = clk > 0 ? (double)cyc / ((double)clk * 1e3) : 0.0;
    return 0;
}

int pbcg_spmv(pbcg_ctx *ctx, const pbcg_mat *m, const double *x, double *y)
{
    if (!ctx)
        return PBCG_ERR_INVALID;
    if (!m || !ctx->mats.count(const_cast<pbcg_mat *>(m)))
        return fail(ctx, PBCG_ERR_INVALID, "unknown matrix handle");
    if (!x || !y)
        return fail(ctx, PBCG_ERR_INVALID, "x and y must not be NULL");
    CK(cudaSetDevice(ctx->device));
    int rc = ensure_ws(ctx, m->n, 0);
    if (rc)
        return rc;
    double *dx = ctx->ws.vec[V_P], *dy = ctx->ws.vec[V_S];
    if ((rc = vec_in(ctx, m, x, dx)))
        return rc;
    Mat A = mat_of(m);
    void *args[3] = {&A, &dx, &dy};
    CK(cudaLaunchKernel((void *)k_spmv, dim3(grid_for(ctx, (void *)k_spmv, A.nslices)), dim3(THREADS), args, 0,
                        ctx->stream));
    if ((rc = vec_out(ctx, m, dy, y)))
        return rc;
    CK(cudaStreamSynchronize(ctx->stream));
    return 0;
}

int pbcg_solve_batched(pbcg_ctx *ctx, const pbcg_mat *A, int32_t nsys, const int32_t *sys_row_ptr, const double *b,
                       double *x, const double *tol, int32_t maxit, int alg, int dot_mode, pbcg_result *out)
{
    NvtxRange trace("pbcg_solve_batched");
    return solve_batched_impl(ctx, A, nsys, sys_row_ptr, b, x, tol, maxit, alg, dot_mode, out);
}


int pbcg_pool_create(pbcg_ctx *ctx, const pbcg_pool_config *cfg, pbcg_pool **out)
{
    if (!ctx)
        return PBCG_ERR_INVALID;
    if (!cfg || !out)
        return fail(ctx, PBCG_ERR_INVALID, "NULL argument");
    *out = nullptr;
    const pbcg_pool_config c = *cfg;
    if (c.max_rows < 1 || c.max_entries < 1 || c.max_slots < 1 || c.maxit < 0 || c.maxit == INT32_MAX ||
        c.max_request_rows < 1 ||
        c.max_request_nnz < 0)
        return fail(ctx, PBCG_ERR_INVALID, "pool sizes must be positive (maxit 0 .. 2^31 - 2)");
    if (c.alg != PBCG_ALG_BICGSTAB && c.alg != PBCG_ALG_PIPELINED && c.alg != PBCG_ALG_PIPELINED_RR)
        return fail(ctx, PBCG_ERR_INVALID, "unknown algorithm %d", c.alg);
    if (c.dot_mode != PBCG_DOT_PLAIN && c.dot_mode != PBCG_DOT_EXACT)
        return fail(ctx, PBCG_ERR_INVALID, "unknown dot mode %d", c.dot_mode);
    if ((c.precond != PBCG_PRECOND_NONE && c.precond != PBCG_PRECOND_JACOBI) || c.reserved != 0)
        return fail(ctx, PBCG_ERR_INVALID, "unknown preconditioner %d (or reserved not 0)", c.precond);
    const long long tiles = (c.max_rows + TILE_ROWS - 1) / TILE_ROWS;
    if (tiles * TILE_ROWS > INT32_MAX / 2 || c.max_entries > INT32_MAX || c.max_request_rows > INT32_MAX / 2 ||
        c.max_request_nnz >= (1ll << 31) || c.max_slots > (1 << 20))
        return fail(ctx, PBCG_ERR_INVALID, "pool too large");
    CK(cudaSetDevice(ctx->device));
    pbcg_pool *P = new pbcg_pool();
    P->ctx = ctx;
    P->cfg = c;
    P->max_tiles = (int)tiles;
    const size_t rows = (size_t)tiles * TILE_ROWS, nsl = (size_t)tiles * TILE_SLICES;
    const size_t req_tiles = (size_t)((c.max_request_rows + TILE_ROWS - 1) / TILE_ROWS);
    const size_t meta_ints = (size_t)c.max_request_rows + 1 + 2 * req_tiles * TILE_SLICES;
    const size_t ns = (size_t)c.max_slots;
    cudaError_t e = cudaSuccess;
    auto dev = [&](void **q, size_t bytes) {
        if (e == cudaSuccess)
            e = cudaMalloc(q, std::max<size_t>(bytes, 16));
    };
    dev((void **)&P->sl_off, sizeof(int) * (nsl + SLOFF_STAGE));
    dev((void **)&P->sl_w, sizeof(int) * nsl);
    dev((void **)&P->rlen, sizeof(int) * rows);
    dev((void **)&P->ci, sizeof(int) * (size_t)c.max_entries);
    dev((void **)&P->va, sizeof(double) * (size_t)c.max_entries);
    dev((void **)&P->tile_sys, sizeof(int) * (size_t)tiles);
    dev((void **)&P->t0, sizeof(int) * ns);
    dev((void **)&P->t1, sizeof(int) * ns);
    dev((void **)&P->left, sizeof(int));
    dev((void **)&P->flag, sizeof(int));
    dev((void **)&P->bad, sizeof(int) * ns);
    dev((void **)&P->lv_n, sizeof(int) * 2);
    dev((void **)&P->lv_pre, sizeof(int) * (ns + 1));
    dev((void **)&P->lv_t0, sizeof(int) * ns);
    dev((void **)&P->st_meta, sizeof(int) * meta_ints);
    dev((void **)&P->st_ci, sizeof(int) * (size_t)c.max_request_nnz);
    dev((void **)&P->st_va, sizeof(double) * (size_t)c.max_request_nnz);
    dev((void **)&P->hist, sizeof(double) * ns * ((size_t)c.maxit + 1));
    dev((void **)&P->ctl, sizeof(Ctl) * ns);
    dev((void **)&P->acc, sizeof(GAcc) * MAXD * ns);
    dev((void **)&P->part, sizeof(double) * MAXD * (size_t)tiles);
    dev((void **)&P->done, sizeof(unsigned) * ns);
    if (c.precond == PBCG_PRECOND_JACOBI)
        dev((void **)&P->diag, sizeof(double) * rows);
    for (auto &v : P->vec)
        dev((void **)&v, sizeof(double) * rows);
    for (auto &h : P->snap)
        if (e == cudaSuccess)
            e = cudaMallocHost((void **)&h, sizeof(Ctl) * ns);
    if (e == cudaSuccess)
        e = cudaMallocHost((void **)&P->meta, sizeof(int) * meta_ints);
    for (auto &ev : P->ev)
        if (e == cudaSuccess)
            e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess)
        e = cudaEventCreateWithFlags(&P->up_ev, cudaEventDisableTiming);
    if (e == cudaSuccess)
        e = cudaStreamCreateWithFlags(&P->cstream, cudaStreamNonBlocking);
    // zeroed state: every tile free, every slot final (skipped), accumulators empty
    if (e == cudaSuccess)
        e = cudaMemset(P->tile_sys, 0xff, sizeof(int) * (size_t)tiles);
    if (e == cudaSuccess)
        e = cudaMemset(P->sl_off, 0, sizeof(int) * (nsl + SLOFF_STAGE));
    if (e == cudaSuccess)
        e = cudaMemset(P->sl_w, 0, sizeof(int) * nsl);
    if (e == cudaSuccess)
        e = cudaMemset(P->rlen, 0, sizeof(int) * rows);
    if (e == cudaSuccess)
        e = cudaMemset(P->done, 0, sizeof(unsigned) * ns);
    if (e == cudaSuccess)
        e = cudaMemset(P->bad, 0, sizeof(int) * ns);
    if (e == cudaSuccess)
        e = cudaMemset(P->st_meta, 0, sizeof(int) * meta_ints);
    for (auto &v : P->vec)
        if (e == cudaSuccess)
            e = cudaMemset(v, 0, sizeof(double) * rows);
    if (e == cudaSuccess) {
        std::vector<Ctl> hc(ns);
        for (auto &q : hc) {
            memset(&q, 0, sizeof q);
            q.status = ST_FREE;
        }
        e = cudaMemcpy(P->ctl, hc.data(), sizeof(Ctl) * ns, cudaMemcpyHostToDevice);
        std::vector<GAcc> ga(ns * MAXD);
        for (auto &g : ga) {
            memset(&g, 0, sizeof g);
            g.kmin = NDIG;
            g.kmax = -1;
        }
        if (e == cudaSuccess)
            e = cudaMemcpy(P->acc, ga.data(), sizeof(GAcc) * ga.size(), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        pool_release(P);
        return fail(ctx, e == cudaErrorMemoryAllocation ? PBCG_ERR_OOM : PBCG_ERR_CUDA, "pool: %s",
                    cudaGetErrorString(e));
    }
    P->tiles.init(tiles);
    P->entries.init(c.max_entries);
    P->slots.assign(ns, PoolSlot());
    int rc = pool_build_graph(ctx, P);
    if (rc) {
        pool_release(P);
        return rc;
    }
    *out = P;
    return 0;
}

void pbcg_pool_destroy(pbcg_pool *P)
{
    if (!P)
        return;
    cudaSetDevice(P->ctx->device);
    cudaStreamSynchronize(P->ctx->stream);
    cudaStreamSynchronize(P->cstream);
    pool_release(P);
}

int pbcg_pool_admit(pbcg_pool *P, int32_t n, int64_t nnz, const int32_t *row_ptr, const int32_t *col_idx,
                    const double *vals, const double *b, const double *x0, double tol, int32_t maxit, int32_t *slot)
{
    NvtxRange trace("pbcg_pool_admit");
    if (!P)
        return PBCG_ERR_INVALID;
    pbcg_ctx *ctx = P->ctx;
    if (!slot || !row_ptr || !b || (nnz > 0 && (!col_idx || !vals)))
        return fail(ctx, PBCG_ERR_INVALID, "NULL argument");
    *slot = -1;
    if (n < 1 || n > P->cfg.max_request_rows || nnz < 0 || nnz > P->cfg.max_request_nnz)
        return fail(ctx, PBCG_ERR_INVALID, "request size n = %d, nnz = %lld beyond the pool's limits (%lld, %lld)",
                    n, (long long)nnz, (long long)P->cfg.max_request_rows, (long long)P->cfg.max_request_nnz);
    if (!(tol > 0.0) || maxit < 0 || maxit > P->cfg.maxit)
        return fail(ctx, PBCG_ERR_INVALID, "tol must be > 0 and 0 <= maxit <= %d", P->cfg.maxit);
    CK(cudaSetDevice(ctx->device));
    const int ntl = (n + TILE_ROWS - 1) / TILE_ROWS, nsl = ntl * TILE_SLICES, rows = ntl * TILE_ROWS;
    int *hrp = P->meta, *hw = P->meta + (n + 1), *hoff = hw + nsl;
    {
        // row pointers to the host without touching the legacy default stream
        cudaPointerAttributes pa;
        bool host = true;
        if (cudaPointerGetAttributes(&pa, row_ptr) == cudaSuccess)
            host = pa.type == cudaMemoryTypeHost || pa.type == cudaMemoryTypeUnregistered;
        else
            cudaGetLastError();
        if (host) {
            memcpy(hrp, row_ptr, sizeof(int32_t) * ((size_t)n + 1));
        } else {
            CK(cudaMemcpyAsync(hrp, row_ptr, sizeof(int32_t) * ((size_t)n + 1), cudaMemcpyDefault, P->cstream));
            CK(cudaStreamSynchronize(P->cstream));
        }
    }
    if (hrp[0] != 0)
        return fail(ctx, PBCG_ERR_INVALID, "row_ptr[0] must be 0");
    if ((int64_t)hrp[n] != nnz)
        return fail(ctx, PBCG_ERR_INVALID, "row_ptr[n] = %d differs from nnz = %lld", hrp[n], (long long)nnz);
    long long ne = 0;
    for (int sl = 0; sl < nsl; sl++) {
        int w = 0;
        for (int i = sl * 32; i < std::min(sl * 32 + 32, n); i++) {
            const int len = hrp[i + 1] - hrp[i];
            if (len < 0)
                return fail(ctx, PBCG_ERR_INVALID, "row_ptr decreases at row %d", i);
            w = std::max(w, len);
        }
        hw[sl] = w;
        hoff[sl] = (int)ne;
        ne += 32ll * w;
    }
    // room: a free slot, a tile range and an entry range (1 = no room now)
    int sid = -1;
    for (int k = 0; k < P->cfg.max_slots; k++)
        if (!P->slots[k].used) {
            sid = k;
            break;
        }
    if (sid < 0)
        return 1;
    const long long tA = P->tiles.take(ntl);
    if (tA < 0)
        return 1;
    const long long eA = ne ? P->entries.take(ne) : 0;
    if (eA < 0) {
        P->tiles.give(tA, ntl);
        return 1;
    }
    for (int sl = 0; sl < nsl; sl++)
        hoff[sl] += (int)eA;
    const int row0 = (int)tA * TILE_ROWS;
    const size_t sl0 = (size_t)tA * TILE_SLICES;
    cudaStream_t cs = P->cstream;
    // uploads on the copy stream into ranges that no step reads
    CK(cudaMemcpyAsync(P->st_meta, P->meta, sizeof(int) * ((size_t)n + 1 + 2 * (size_t)nsl), cudaMemcpyHostToDevice,
                       cs));
    CK(cudaMemcpyAsync(P->sl_w + sl0, P->st_meta + (n + 1), sizeof(int) * nsl, cudaMemcpyDeviceToDevice, cs));
    CK(cudaMemcpyAsync(P->sl_off + sl0, P->st_meta + (n + 1) + nsl, sizeof(int) * nsl, cudaMemcpyDeviceToDevice, cs));
    if (nnz) {
        CK(cudaMemcpyAsync(P->st_ci, col_idx, sizeof(int32_t) * (size_t)nnz, cudaMemcpyDefault, cs));
        CK(cudaMemcpyAsync(P->st_va, vals, sizeof(double) * (size_t)nnz, cudaMemcpyDefault, cs));
    }
    CK(cudaMemsetAsync(P->bad + sid, 0, sizeof(int), cs));
    {
        int nn = n, nr = rows, r0 = row0;
        const int *rp_d = P->st_meta, *ci_d = P->st_ci, *so = P->sl_off + sl0, *sw = P->sl_w + sl0;
        const double *va_d = P->st_va;
        int *rl = P->rlen, *co = P->ci, *bd = P->bad + sid;
        double *vo = P->va;
        void *args[] = {&nn, &nr, &r0, (void *)&rp_d, (void *)&ci_d, (void *)&va_d, (void *)&so, (void *)&sw,
                        &rl, &co, &vo, &bd};
        const int g = std::min((rows + 255) / 256, ctx->num_sms * 8);
        CK(cudaLaunchKernel((void *)k_pool_scatter, dim3(g), dim3(256), args, 0, cs));
        if (P->diag) {
            // Jacobi: d from the staged CSR, then the slot's entries become those of A M^-1
            double *dg = P->diag;
            void *a1[] = {&nn, &nr, &r0, (void *)&rp_d, (void *)&ci_d, (void *)&va_d, &dg, &bd};
            CK(cudaLaunchKernel((void *)k_pool_diag, dim3(g), dim3(256), a1, 0, cs));
            const int *rl_c = rl, *co_c = co;
            const double *dg_c = dg;
            void *a2[] = {&nr, &r0, (void *)&so, (void *)&rl_c, (void *)&co_c, &vo, (void *)&dg_c};
            CK(cudaLaunchKernel((void *)k_pool_jscale, dim3(g), dim3(256), a2, 0, cs));
        }
    }
    CK(cudaMemsetAsync(P->vec[V_B] + row0, 0, sizeof(double) * rows, cs));
    CK(cudaMemsetAsync(P->vec[V_X] + row0, 0, sizeof(double) * rows, cs));
    CK(cudaMemcpyAsync(P->vec[V_B] + row0, b, sizeof(double) * n, cudaMemcpyDefault, cs));
    if (x0) {
        CK(cudaMemcpyAsync(P->vec[V_X] + row0, x0, sizeof(double) * n, cudaMemcpyDefault, cs));
        if (P->diag) {                                        // y0 = x0 * d
            int nn = n;
            const double *dd = P->diag + row0;
            double *xx = P->vec[V_X] + row0;
            void *a3[] = {&nn, (void *)&dd, &xx};
            CK(cudaLaunchKernel((void *)k_vmul, dim3(std::min((n + 255) / 256, ctx->num_sms * 4)), dim3(256), a3, 0,
                                cs));
        }
    }
    CK(cudaEventRecord(P->up_ev, cs));
    // the slot goes live on the solve stream once its uploads are in
    CK(cudaStreamWaitEvent(ctx->stream, P->up_ev, 0));
    PoolSlot &S = P->slots[sid];
    S = PoolSlot();
    S.used = true;
    S.gen = P->next_gen++;
    S.tile0 = (int)tA;
    S.ntiles = ntl;
    S.n = n;
    S.e0 = eA;
    S.ne = ne;
    Ctl init;
    memset(&init, 0, sizeof init);
    init.maxit = maxit;
    init.status = ST_SETUP1;
    init.tol = tol;
    init.target = tol;
    init.alg = (P->cfg.alg == PBCG_ALG_BICGSTAB) ? ALG_BICGSTAB : ALG_PIPELINED;
    init.rr_period = (P->cfg.alg == PBCG_ALG_PIPELINED_RR) ? ctx->rr_period : 0;
    init.hist = P->hist + (size_t)sid * (size_t)(P->cfg.maxit + 1);
    init.hist_cap = P->cfg.maxit + 1;
    init.trueres = __builtin_nan("");
    init.gen = S.gen;
    {
        int *ts = P->tile_sys, *a0 = P->t0, *a1 = P->t1;
        Ctl *cl = P->ctl;
        int s_ = sid, t_ = (int)tA, k_ = ntl;
        const int *bd = P->bad;
        unsigned *dn = P->done;
        GAcc *ac = P->acc;
        void *args[] = {&ts, &a0, &a1, &cl, &s_, &t_, &k_, &init, (void *)&bd, &dn, &ac};
        CK(cudaLaunchKernel((void *)k_pool_activate, dim3(1), dim3(256), args, 0, ctx->stream));
    }
    // the caller's arrays and the pinned row pointers are consumed when this returns
    CK(cudaStreamSynchronize(cs));
    *slot = sid;
    return 0;
}

int pbcg_pool_step(pbcg_pool *P, int32_t iters)
{
    NvtxRange trace("pbcg_pool_step");
    if (!P)
        return PBCG_ERR_INVALID;
    pbcg_ctx *ctx = P->ctx;
    if (iters < 1)
        return fail(ctx, PBCG_ERR_INVALID, "iters must be >= 1");
    CK(cudaSetDevice(ctx->device));
    const int k = (int)(P->issued % POOL_RING);
    // the snapshot buffer about to be reused must not still be in flight
    CK(cudaEventSynchronize(P->ev[k]));
    {
        int *l = P->left;
        int it = iters;
        void *args[] = {&l, &it};
        CK(cudaLaunchKernel((void *)k_pool_arm, dim3(1), dim3(1), args, 0, ctx->stream));
    }
    CK(cudaGraphLaunch(P->exec, ctx->stream));
    CK(cudaMemcpyAsync(P->snap[k], P->ctl, sizeof(Ctl) * (size_t)P->cfg.max_slots, cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaEventRecord(P->ev[k], ctx->stream));
    P->issued++;
    return 0;
}

int pbcg_pool_poll(pbcg_pool *P, int wait, int32_t *done_slots, int32_t cap, int32_t *count, int32_t *pending)
{
    if (!P)
        return PBCG_ERR_INVALID;
    pbcg_ctx *ctx = P->ctx;
    if (!count || cap < 0 || (cap > 0 && !done_slots))
        return fail(ctx, PBCG_ERR_INVALID, "bad output arguments");
    CK(cudaSetDevice(ctx->device));
    *count = 0;
    long long newest = -1;
    const long long lo = std::max(0ll, P->issued - POOL_RING);
    for (long long j = P->issued - 1; j >= lo; --j) {
        cudaEvent_t ev = P->ev[j % POOL_RING];
        if (wait && j == P->issued - 1)
            CK(cudaEventSynchronize(ev));
        cudaError_t q = cudaEventQuery(ev);
        if (q == cudaSuccess) {
            newest = j;
            break;
        }
        if (q != cudaErrorNotReady)
            CK(q);
    }
    if (pending)
        *pending = (int32_t)(P->issued - 1 - newest);
    if (newest < 0)
        return 0;
    const Ctl *sn = P->snap[newest % POOL_RING];
    int k = 0;
    for (int s = 0; s < P->cfg.max_slots; s++) {
        PoolSlot &S = P->slots[s];
        if (!S.used || S.reported || sn[s].gen != S.gen || !final_status(sn[s]))
            continue;
        S.reported = true;
        S.last = sn[s];
        if (k < cap)
            done_slots[k] = s;
        k++;
    }
    *count = k;
    return 0;
}

int pbcg_pool_result(pbcg_pool *P, int32_t slot, double *x, pbcg_result *out)
{
    if (!P)
        return PBCG_ERR_INVALID;
    pbcg_ctx *ctx = P->ctx;
    if (slot < 0 || slot >= P->cfg.max_slots || !P->slots[slot].used || !P->slots[slot].reported)
        return fail(ctx, PBCG_ERR_INVALID, "slot %d has no finished request", slot);
    CK(cudaSetDevice(ctx->device));
    PoolSlot &S = P->slots[slot];
    // a finished slot's rows are no longer written: copy without waiting for running steps
    if (x) {
        double *xs = P->vec[V_X] + (size_t)S.tile0 * TILE_ROWS;
        if (P->diag && S.last.status != ST_INVALID) {         // x = y / d (the slot is retiring)
            int nn = S.n;
            const double *dd = P->diag + (size_t)S.tile0 * TILE_ROWS;
            void *a3[] = {&nn, (void *)&dd, &xs};
            CK(cudaLaunchKernel((void *)k_vdiv, dim3(std::min((S.n + 255) / 256, ctx->num_sms * 4)), dim3(256), a3, 0,
                                P->cstream));
        }
        CK(cudaMemcpyAsync(x, xs, sizeof(double) * (size_t)S.n, cudaMemcpyDefault, P->cstream));
        CK(cudaStreamSynchronize(P->cstream));
    }
    const Ctl &c = S.last;
    const bool timeout = c.status == ST_TIMEOUT || c.err;
    const bool invalid = c.status == ST_INVALID;
    if (out) {
        out->iters = c.it;
        out->status = timeout ? PBCG_ERR_TIMEOUT : invalid ? PBCG_ERR_INVALID : c.status;
        out->relres_recursive = c.res;
        out->relres_true = c.trueres;
        out->seconds = 0.0;
        out->launches = 0;
        out->reserved = 0;
    }
    // retire: the tiles leave the sweep (ordered after running steps), the ranges return
    {
        int *ts = P->tile_sys;
        int t_ = S.tile0, k_ = S.ntiles;
        void *args[] = {&ts, &t_, &k_};
        CK(cudaLaunchKernel((void *)k_pool_clear, dim3(1), dim3(256), args, 0, ctx->stream));
    }
    P->tiles.give(S.tile0, S.ntiles);
    P->entries.give(S.e0, S.ne);
    S = PoolSlot();
    if (timeout)
        return fail(ctx, PBCG_ERR_TIMEOUT, "a bounded device wait expired");
    if (invalid)
        return fail(ctx, PBCG_ERR_INVALID,
                    "request in slot %d has a column index outside [0, n) or, with Jacobi, an unusable diagonal", slot);
    return c.status;
}

int pbcg_pool_history(pbcg_pool *P, int32_t slot, double *out, int32_t cap, int32_t *len)
{
    if (!P)
        return PBCG_ERR_INVALID;
    pbcg_ctx *ctx = P->ctx;
    if (slot < 0 || slot >= P->cfg.max_slots || !P->slots[slot].used || !P->slots[slot].reported)
        return fail(ctx, PBCG_ERR_INVALID, "slot %d has no finished request", slot);
    CK(cudaSetDevice(ctx->device));
    const Ctl &c = P->slots[slot].last;
    const int32_t L = c.status == ST_INVALID ? 0 : std::min(c.it + 1, P->cfg.maxit + 1);
    if (len)
        *len = L;
    if (out && cap > 0 && L > 0) {
        CK(cudaMemcpyAsync(out, P->hist + (size_t)slot * (size_t)(P->cfg.maxit + 1),
                           sizeof(double) * (size_t)std::min(cap, L), cudaMemcpyDeviceToHost, P->cstream));
        CK(cudaStreamSynchronize(P->cstream));
    }
    return 0;
}

int pbcg_pool_room(const pbcg_pool *P, int32_t *free_slots, int64_t *free_rows, int64_t *free_entries)
{
    if (!P)
        return PBCG_ERR_INVALID;
    int fs = 0;
    for (auto &S : P->slots)
        fs += !S.used;
    if (free_slots)
        *free_slots = fs;
    if (free_rows)
        *free_rows = P->tiles.largest() * TILE_ROWS;
    if (free_entries)
        *free_entries = P->entries.largest();
    return 0;
}

int pbcg_part_plan(int32_t nranks, int32_t rank, const int32_t *row_starts, int64_t nnz, const int32_t *row_ptr,
                   const int32_t *col_idx, int32_t *nhalo, int32_t *halo_cols, int32_t cap, int32_t *recv_counts,
                   int32_t *local_col)
{
    if (!row_starts || !row_ptr || (nnz > 0 && !col_idx) || !nhalo || cap < 0 || (cap > 0 && !halo_cols) ||
        nranks < 1 || rank < 0 || rank >= nranks)
        return PBCG_ERR_INVALID;
    std::vector<int32_t> halo, rc, loc;
    std::string why;
    int r = part_plan_host(nranks, rank, row_starts, nnz, row_ptr, col_idx, halo, rc, local_col ? &loc : nullptr,
                           why);
    if (r)
        return r;
    *nhalo = (int32_t)halo.size();
    for (int32_t i = 0; i < cap && i < (int32_t)halo.size(); i++)
        halo_cols[i] = halo[(size_t)i];
    if (recv_counts)
        for (int k = 0; k < nranks; k++)
            recv_counts[k] = rc[(size_t)k];
    if (local_col)
        std::copy(loc.begin(), loc.end(), local_col);
    return 0;
}

int pbcg_part_create(pbcg_ctx *ctx, const pbcg_comm *comm, int32_t nranks, int32_t rank, const int32_t *row_starts,
                     int64_t nnz, const int32_t *row_ptr, const int32_t *col_idx, const double *vals,
                     pbcg_part **out)
{
    if (!ctx)
        return PBCG_ERR_INVALID;
    if (!out || !comm || !comm->allreduce_sum_i64 || !comm->alltoallv || !row_starts || nranks < 1 || rank < 0 ||
        rank >= nranks)
        return fail(ctx, PBCG_ERR_INVALID, "NULL argument, communicator callback or bad rank");
    *out = nullptr;
    NvtxRange trace("pbcg_part_create");
    // local checks first, then one allreduce so that every rank fails together
    long long bad = 0;
    std::vector<int32_t> rs((size_t)nranks + 1), hrp, hci, halo, rcount, local;
    std::vector<double> hva;
    int rc = 0;
    memcpy(rs.data(), row_starts, sizeof(int32_t) * ((size_t)nranks + 1));
    const int nloc = rs[(size_t)rank + 1] - rs[(size_t)rank];
    if (cudaSetDevice(ctx->device) != cudaSuccess)
        rc = fail(ctx, PBCG_ERR_CUDA, "cudaSetDevice failed");
    else if (!row_ptr || (nnz > 0 && (!col_idx || !vals)) || nnz < 0 || nnz >= (1ll << 31) || nloc < 1 ||
             nloc > INT32_MAX / 2)
        rc = fail(ctx, PBCG_ERR_INVALID, "bad block: NULL CSR array, nnz out of range or rows outside 1 .. 2^30 - 1");
    if (!rc) {
        hrp.resize((size_t)nloc + 1);
        hci.resize((size_t)nnz);
        hva.resize((size_t)nnz);
        cudaError_t e = cudaMemcpy(hrp.data(), row_ptr, sizeof(int32_t) * hrp.size(), cudaMemcpyDefault);
        if (e == cudaSuccess && nnz)
            e = cudaMemcpy(hci.data(), col_idx, sizeof(int32_t) * (size_t)nnz, cudaMemcpyDefault);
        if (e == cudaSuccess && nnz)
            e = cudaMemcpy(hva.data(), vals, sizeof(double) * (size_t)nnz, cudaMemcpyDefault);
        if (e != cudaSuccess)
            rc = fail(ctx, PBCG_ERR_CUDA, "copying the block: %s", cudaGetErrorString(e));
    }
    if (!rc) {
        std::string why;
        if ((rc = part_plan_host(nranks, rank, rs.data(), nnz, hrp.data(), hci.data(), halo, rcount, &local, why)))
            fail(ctx, rc, "%s", why.c_str());
    }
    bad = rc ? 1 : 0;
    long long anybad = bad;
    if (nranks > 1) {
        int r2 = comm_any(ctx, *comm, bad, &anybad);
        if (r2)
            return r2;
    }
    if (anybad)
        return rc ? rc : fail(ctx, PBCG_ERR_INVALID, "another rank refused its block");
    pbcg_part *P = new pbcg_part();
    P->ctx = ctx;
    P->comm = *comm;
    P->nranks = nranks;
    P->rank = rank;
    P->row0 = rs[(size_t)rank];
    P->nloc = nloc;
    P->nhalo = (int)halo.size();
    // which of my rows each rank gathers: counts, then the global indices
    std::vector<int64_t> cnt_send((size_t)nranks), cnt_recv((size_t)nranks), b8((size_t)nranks, 8), d8((size_t)nranks);
    for (int k = 0; k < nranks; k++) {
        cnt_send[(size_t)k] = rcount[(size_t)k];
        d8[(size_t)k] = 8ll * k;
    }
    if (nranks > 1 && comm->alltoallv(comm->user, cnt_send.data(), b8.data(), d8.data(), cnt_recv.data(), b8.data(),
                                      d8.data()) != 0) {
        part_release(P);
        return fail(ctx, PBCG_ERR_COMM, "alltoallv callback failed (halo counts)");
    }
    if (nranks == 1)
        cnt_recv = cnt_send;
    std::vector<int64_t> qb((size_t)nranks), qd((size_t)nranks), ab((size_t)nranks), ad((size_t)nranks);
    long long qoff = 0, aoff = 0;
    for (int k = 0; k < nranks; k++) {
        qb[(size_t)k] = 4ll * cnt_send[(size_t)k];     // my halo columns owned by k (requests to k)
        qd[(size_t)k] = qoff;
        qoff += qb[(size_t)k];
        ab[(size_t)k] = 4ll * cnt_recv[(size_t)k];     // rows of mine that k requests
        ad[(size_t)k] = aoff;
        aoff += ab[(size_t)k];
    }
    std::vector<int32_t> wanted((size_t)(aoff / 4) + 1);
    if (nranks > 1 && comm->alltoallv(comm->user, halo.data(), qb.data(), qd.data(), wanted.data(), ab.data(),
                                      ad.data()) != 0) {
        part_release(P);
        return fail(ctx, PBCG_ERR_COMM, "alltoallv callback failed (halo indices)");
    }
    P->nsend = (int)(aoff / 4);
    bad = 0;
    for (int j = 0; j < P->nsend; j++)
        if (wanted[(size_t)j] < P->row0 || wanted[(size_t)j] >= P->row0 + nloc)
            bad = 1;
    if (bad)
        fail(ctx, PBCG_ERR_INVALID, "a rank asked for rows outside this block (row_starts differ between ranks?)");
    // the block's matrix with local columns, and the buffers of the exchanges
    if (!bad) {
        rc = make_mat(ctx, nloc, nloc + P->nhalo, std::move(hrp), std::move(local), std::move(hva), &P->m);
        if (rc)
            bad = 1;
    }
    if (!bad) {
        std::vector<int> perm;
        if (P->m->perm) {
            perm.resize((size_t)nloc);
            if (cudaMemcpy(perm.data(), P->m->perm, sizeof(int) * (size_t)nloc, cudaMemcpyDeviceToHost) != cudaSuccess)
                bad = 1;
        }
        std::vector<int> inv((size_t)nloc);
        for (int p = 0; p < nloc; p++)
            inv[(size_t)(perm.empty() ? p : perm[(size_t)p])] = p;
        std::vector<int> sidx((size_t)P->nsend + 1);
        for (int j = 0; j < P->nsend; j++)
            sidx[(size_t)j] = inv[(size_t)(wanted[(size_t)j] - P->row0)];
        P->red_cap = 1 + std::max(MAXD * RED_EXACT_STRIDE, nranks * MAXD);
        cudaError_t e = bad ? cudaErrorUnknown : cudaSuccess;
        if (e == cudaSuccess)
            e = cudaMalloc(&P->d_send_idx, sizeof(int) * sidx.size());
        if (e == cudaSuccess)
            e = cudaMalloc(&P->d_send, sizeof(double) * sidx.size());
        if (e == cudaSuccess)
            e = cudaMalloc(&P->d_red, sizeof(long long) * (size_t)P->red_cap);
        if (e == cudaSuccess)
            e = cudaMallocHost(&P->h_send, sizeof(double) * sidx.size());
        if (e == cudaSuccess)
            e = cudaMallocHost(&P->h_recv, sizeof(double) * ((size_t)P->nhalo + 1));
        if (e == cudaSuccess)
            e = cudaMallocHost(&P->h_red, sizeof(long long) * (size_t)P->red_cap);
        if (e == cudaSuccess)
            e = cudaMallocHost(&P->h_g, sizeof(GAcc) * MAXD);
        if (e == cudaSuccess)
            e = cudaMallocHost(&P->h_loc, sizeof(double) * MAXD);
        if (e == cudaSuccess)
            e = cudaMallocHost(&P->h_err, sizeof(int));
        if (e == cudaSuccess)
            e = cudaMemcpy(P->d_send_idx, sidx.data(), sizeof(int) * sidx.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            rc = fail(ctx, e == cudaErrorMemoryAllocation ? PBCG_ERR_OOM : PBCG_ERR_CUDA, "block buffers: %s",
                      cudaGetErrorString(e));
            bad = 1;
        }
    }
    if (!bad) {
        P->sb.resize((size_t)nranks);
        P->sd.resize((size_t)nranks);
        P->rb.resize((size_t)nranks);
        P->rd.resize((size_t)nranks);
        for (int k = 0; k < nranks; k++) {
            P->sb[(size_t)k] = 2 * ab[(size_t)k];       // doubles where the requests were int32
            P->sd[(size_t)k] = 2 * ad[(size_t)k];
            P->rb[(size_t)k] = 2 * qb[(size_t)k];
            P->rd[(size_t)k] = 2 * qd[(size_t)k];
        }
    }
    anybad = bad;
    if (nranks > 1) {
        int r2 = comm_any(ctx, *comm, bad, &anybad);
        if (r2) {
            part_release(P);
            return r2;
        }
    }
    if (anybad) {
        part_release(P);
        return bad ? (rc ? rc : PBCG_ERR_INVALID) : fail(ctx, PBCG_ERR_INVALID, "another rank failed to set up");
    }
    *out = P;
    return 0;
}

int pbcg_part_solve(pbcg_part *part, const double *b, double *x, double tol, int32_t maxit, int alg, int dot_mode,
                    pbcg_result *out)
{
    if (!part)
        return PBCG_ERR_INVALID;
    NvtxRange trace("pbcg_part_solve");
    return part_solve_impl(part, b, x, tol, maxit, alg, dot_mode, out);
}

void pbcg_part_destroy(pbcg_part *part)
{
    if (!part)
        return;
    cudaSetDevice(part->ctx->device);
    cudaStreamSynchronize(part->ctx->stream);
    part_release(part);
}

int pbcg_set_variant(pbcg_ctx *ctx, pbcg_mat *m, const pbcg_variant *v)
{
    if (!ctx)
        return PBCG_ERR_INVALID;
    if (!m || !ctx->mats.count(m))
        return fail(ctx, PBCG_ERR_INVALID, "unknown matrix handle");
    pbcg_variant d{1, 0, 0, 0, 0.0};
    if (v && !variant_ok(*v))
        return fail(ctx, PBCG_ERR_INVALID, "variant field out of range");
    apply_variant(m, v ? *v : d);
    if (v)
        m->v_us = 0.0;
    return 0;
}

int pbcg_get_variant(pbcg_ctx *ctx, const pbcg_mat *m, pbcg_variant *out)
{
    if (!ctx)
        return PBCG_ERR_INVALID;
    if (!m || !out || !ctx->mats.count(const_cast<pbcg_mat *>(m)))
        return fail(ctx, PBCG_ERR_INVALID, "unknown matrix handle or NULL output");
    *out = variant_of(m);
    return 0;
}

int pbcg_tune(pbcg_ctx *ctx, pbcg_mat *A, int alg, int dot_mode, int32_t nsys, const int32_t *sys_row_ptr,
              int32_t iters, const char *cache_path, pbcg_variant *chosen, pbcg_variant *tried, int32_t cap,
              int32_t *ntried)
{
    if (!ctx)
        return PBCG_ERR_INVALID;
    NvtxRange trace("pbcg_tune");
    return tune_impl(ctx, A, alg, dot_mode, nsys, sys_row_ptr, iters, cache_path, chosen, tried, cap, ntried);
}

int pbcg_check_word(pbcg_ctx *ctx, int reset, int32_t *enabled, uint64_t *word)
{
    if (!ctx)
        return PBCG_ERR_INVALID;
    if (!enabled || !word)
        return fail(ctx, PBCG_ERR_INVALID, "NULL output");
    *enabled = PBCG_CHECKS;
    *word = 0;
#if PBCG_CHECKS
    CK(cudaSetDevice(ctx->device));
    CK(cudaStreamSynchronize(ctx->stream));
    unsigned long long w = 0;
    CK(cudaMemcpyFromSymbol(&w, g_check_word, sizeof w));
    *word = (uint64_t)w;
    if (reset) {
        const unsigned long long z = 0;
        CK(cudaMemcpyToSymbol(g_check_word, &z, sizeof z));
    }
#else
    (void)reset;
#endif
    return 0;
}

int pbcg_mat_check(pbcg_ctx *ctx, const pbcg_mat *m, uint64_t *word)
{
    if (!ctx)
        return PBCG_ERR_INVALID;
    if (!m || !word || !ctx->mats.count(const_cast<pbcg_mat *>(m)))
        return fail(ctx, PBCG_ERR_INVALID, "unknown matrix handle or NULL output");
    CK(cudaSetDevice(ctx->device));
    unsigned long long *d = nullptr;
    CK(cudaMalloc(&d, sizeof(unsigned long long)));
    Mat A = mat_of(m);
    long long padded = m->padded;
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof(unsigned long long), ctx->stream);
    if (e == cudaSuccess) {
        void *args[3] = {&A, &padded, &d};
        e = cudaLaunchKernel((void *)k_mat_check, dim3(ctx->num_sms * 4), dim3(256), args, 0, ctx->stream);
    }
    unsigned long long h = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&h, d, sizeof h, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(ctx->stream);
    cudaFree(d);
    if (e != cudaSuccess)
        return fail(ctx, PBCG_ERR_CUDA, "pbcg_mat_check: %s", cudaGetErrorString(e));
    *word = (uint64_t)h;
    return 0;
}

int pbcg_debug_set_col(pbcg_ctx *ctx, pbcg_mat *m, int64_t entry, int32_t col)
{
    if (!ctx)
        return PBCG_ERR_INVALID;
#if PBCG_CHECKS
    if (!m || !ctx->mats.count(m) || entry < 0 || entry >= m->padded)
        return fail(ctx, PBCG_ERR_INVALID, "unknown matrix handle or entry outside the layout");
    CK(cudaSetDevice(ctx->device));
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaMemcpy(m->ci + entry, &col, sizeof col, cudaMemcpyHostToDevice));
    free_loop(ctx->ws.loop);
    return 0;
#else
    (void)m;
    (void)entry;
    (void)col;
    return fail(ctx, PBCG_ERR_INVALID, "pbcg_debug_set_col needs the checked build");
#endif
}

}  // extern "C"
