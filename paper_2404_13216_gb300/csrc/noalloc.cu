// noalloc.cu -- a dot-product entry point that allocates nothing.
//
// pbcg_dot needs a context, and a context allocates device memory (its
// workspace, pinned host memory, a stream).  Some callers cannot allocate at
// all: code running inside another allocator's arena or a memory-capped
// sandbox, code that holds a fixed memory budget agreed in advance, or a hot
// loop that must not touch the allocator (cudaMalloc can synchronise the
// device).  pbcg_dot_noalloc serves them: the caller passes device pointers
// for the inputs and the output, and the grid-wide merge state the kernel
// needs lives in one file-scope __device__ array of fixed size that every GPU
// loading this library holds until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/pbcg.h"
#include "kernels.cuh"

using namespace pbcg;

constexpr int NOALLOC_MAXGRID = 2048;                        // CTAs of one call at most
constexpr long long NOALLOC_MAX_N = (1ll << 31) - 1;         // longest vectors accepted
constexpr size_t NOALLOC_PART_OFF = (sizeof(Work) + 255) / 256 * 256;
constexpr size_t NOALLOC_BYTES = NOALLOC_PART_OFF + sizeof(double) * MAXD * NOALLOC_MAXGRID;
static_assert(NOALLOC_BYTES == 70144, "scratch size stated in include/pbcg.h");

// The merge state of every call on this device: a Work header (four exact
// accumulators, a ticket) followed by the plain partials of up to 2048 CTAs.
// In host code this name is a host-side stand-in, not a device address: the
// host passes the address cudaGetSymbolAddress returned for the device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

namespace {

constexpr int MAXDEV = 64;
std::mutex g_mu;
bool g_ready[MAXDEV];
int g_sms[MAXDEV];
int g_occ[MAXDEV][2];

// clear the merge state before each call (the array keeps the last call's contents)
__global__ void k_noalloc_init(unsigned char *base)
{
    Work *wk = reinterpret_cast<Work *>(base);
    for (int i = threadIdx.x; i < MAXD * NDIG; i += blockDim.x)
        wk->g[i / NDIG].dig[i % NDIG] = 0ull;
    if (threadIdx.x < MAXD) {
        wk->g[threadIdx.x].kmin = NDIG;
        wk->g[threadIdx.x].kmax = -1;
        wk->g[threadIdx.x].nf = 0;
    }
    if (threadIdx.x == 0) {
        wk->ticket = 0u;
        wk->tile_next = 0u;
        wk->maxgrid = NOALLOC_MAXGRID;
        wk->part = reinterpret_cast<double *>(base + NOALLOC_PART_OFF);
    }
}

// the same computation as the context's dot kernel, with the merge state in the static array
template <int MODE>
__global__ void __launch_bounds__(THREADS) k_noalloc_dot(long long n, const double *a, const double *b,
                                                         double *out, Work *wk)
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

// once per device, with that device current: the SM count and the occupancy
// of the two dot kernels (neither changes while the process runs)
int noalloc_setup(int dev)
{
    std::lock_guard<std::mutex> lock(g_mu);
    if (g_ready[dev])
        return 0;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        return PBCG_ERR_CUDA;
    for (int m = 0; m < 2; m++) {
        int o = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, m ? (const void *)k_noalloc_dot<1>
                                                                : (const void *)k_noalloc_dot<0>,
                                                          THREADS, 0) != cudaSuccess || o < 1)
            return PBCG_ERR_CUDA;
        g_occ[dev][m] = o;
    }
    g_sms[dev] = sms;
    g_ready[dev] = true;
    return 0;
}

// true when p is device (or managed) memory that device `dev` owns; the
// query allocates nothing
bool on_device(const void *p, int dev)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == dev;
}

}  // namespace

extern "C" int pbcg_dot_noalloc(int64_t n, const double *a, const double *b, int dot_mode, double *out,
                                void *cuda_stream)
{
    if (n < 0 || n > NOALLOC_MAX_N)
        return PBCG_ERR_INVALID;
    if ((n > 0 && (!a || !b)) || !out)
        return PBCG_ERR_INVALID;
    if (dot_mode != PBCG_DOT_PLAIN && dot_mode != PBCG_DOT_EXACT)
        return PBCG_ERR_INVALID;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAXDEV)
        return PBCG_ERR_CUDA;
    if ((n > 0 && (!on_device(a, dev) || !on_device(b, dev))) || !on_device(out, dev))
        return PBCG_ERR_INVALID;
    int rc = noalloc_setup(dev);
    if (rc)
        return rc;
    // the array's device address, looked up on every call (it allocates
    // nothing), so that a module reloaded after a device reset is followed
    void *sym = nullptr;
    if (cudaGetSymbolAddress(&sym, g_noalloc_scratch) != cudaSuccess || !sym) {
        cudaGetLastError();
        return PBCG_ERR_CUDA;
    }
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    long long tiles = (n + 31) / 32;
    long long need = (tiles + WARPS - 1) / WARPS;
    long long grid = (long long)g_occ[dev][dot_mode] * g_sms[dev];
    if (grid > need)
        grid = need;
    if (grid > NOALLOC_MAXGRID)
        grid = NOALLOC_MAXGRID;
    if (grid < 1)
        grid = 1;
    unsigned char *base = static_cast<unsigned char *>(sym);
    k_noalloc_init<<<1, THREADS, 0, st>>>(base);
    Work *wk = reinterpret_cast<Work *>(base);
    long long nn = n;
    if (dot_mode == PBCG_DOT_EXACT)
        k_noalloc_dot<1><<<(int)grid, THREADS, 0, st>>>(nn, a, b, out, wk);
    else
        k_noalloc_dot<0><<<(int)grid, THREADS, 0, st>>>(nn, a, b, out, wk);
    return cudaGetLastError() == cudaSuccess ? 0 : PBCG_ERR_CUDA;
}
