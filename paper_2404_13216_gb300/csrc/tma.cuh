// tma.cuh -- bulk-copy (TMA) staging of row tiles into shared memory.
//
// A CTA of 8 warps works on tiles of 8 SELL-32 slices (256 rows).  One thread
// issues 1-D bulk copies (cp.async.bulk, the non-tensor form of the Tensor
// Memory Accelerator path) of the tile's input vectors, row lengths, slice
// offsets and -- when the tile's SELL span fits -- its column indices and
// values into one of two shared-memory stages; completion is tracked by the
// stage's mbarrier with a transaction byte count.  While the warps compute on
// one stage the copies for the next tile land in the other, so DRAM latency
// is hidden behind the FP64 and integer work instead of stalling each warp.
//
// Every wait on an mbarrier is bounded: after MBAR_SPIN_LIMIT failed probes the
// waiting thread gives up and reports it, so a lost copy can never hang the GPU.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace pbcg {

constexpr int TILE_SLICES = 8;                 // = warps per CTA
constexpr int TILE_ROWS = TILE_SLICES * 32;
constexpr int NSTAGE = 2;
constexpr int MCAP = TILE_ROWS * 7;            // staged SELL entries per tile (width <= 7)
constexpr int SLOFF_STAGE = 16;                // slice offsets copied per tile (needs 9)
constexpr int GMAX = 6;                        // 256-row blocks of the gathered vector staged per tile
constexpr int TMETA = 8;                       // ints per tile record: first entry, end entry, GMAX blocks
constexpr unsigned MBAR_SPIN_LIMIT = 1u << 18;   // about 1 s of probes on GB300 (3.8 us each)
constexpr unsigned MBAR_CHECK_MAX = 1u << 22;    // largest limit pbcg_check_wait accepts

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// completes the current phase of a count-1 barrier with no bytes expected
__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0u;
}

// bounded wait: true when the phase completed, false after the spin limit
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, unsigned limit = MBAR_SPIN_LIMIT)
{
    for (unsigned i = 0; i < limit; i++)
        if (mbar_try_wait(bar, parity))
            return true;
    return false;
}

// make mbarrier initialisation visible to the asynchronous (bulk-copy) proxy
__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_async_shared()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 1-D bulk copy global -> shared, completing on `bar` (16-byte aligned, size a multiple of 16)
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Dynamic shared memory of a staged pass with NV input vectors:
// NSTAGE stages of { vec[NV][256] f64, gwin[GMAX][256] f64 (if staged with windows), va[MCAP] f64 (if staged),
// ci[MCAP] i32 or 16-bit local indices (if staged), rlen[256] i32, sl_off[16] i32, meta[TMETA] i32 }.
// meta holds the record of the tile this stage takes next, so the warp that
// refills the stage needs no global load.
// When a tile's columns fall in at most GMAX 256-row blocks, those blocks of
// the gathered vector are staged in gwin and ci holds local indices into it.
template <int NV, bool MATS, bool WIN = MATS>
struct StageLayout {
    static constexpr uint32_t VEC = NV * TILE_ROWS * 8;
    static constexpr uint32_t GWIN = (MATS && WIN) ? GMAX * TILE_ROWS * 8 : 0;
    static constexpr uint32_t VA = MATS ? MCAP * 8 : 0;
    static constexpr uint32_t CI = MATS ? MCAP * 4 : 0;
    static constexpr uint32_t RLEN = TILE_ROWS * 4;
    static constexpr uint32_t SLOFF = SLOFF_STAGE * 4;
    static constexpr uint32_t META = TMETA * 4;
    static constexpr uint32_t STAGE = VEC + GWIN + VA + CI + RLEN + SLOFF + META;
    static constexpr uint32_t TOTAL = NSTAGE * STAGE;
    static_assert(STAGE % 16 == 0, "stages must stay 16-byte aligned");
};

// bookkeeping of one stage, in static shared memory
struct StageInfo {
    int e0;          // first SELL entry of the tile
    int staged;      // 1 if the tile's ci/va are in shared memory
    int windowed;    // 1 if the gathered vector's blocks are in shared memory (ci local)
    int tile;        // the tile held
    int span;        // SELL entries of the tile (bounds checks)
    int nblk;        // gather blocks staged (bounds checks)
};

}  // namespace pbcg
