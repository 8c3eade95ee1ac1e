/*
 * Device infrastructure shared by the kernels: the workspace layout, the
 * tile-status words of the single-pass decoupled look-back scan, block-level
 * scans and the "last CTA finishes the call" protocol.
 *
 * Output offsets.  Every kernel that writes output turns per-character output
 * lengths into output offsets in one pass over the input.  The paper's
 * conclusion suggests decoding pieces of a string independently once the
 * character offsets are known; here each tile of the input computes its own
 * output length, publishes it, and learns the total of all earlier tiles by
 * looking back over their published words (Merrill & Garland, "Single-pass
 * Parallel Prefix Scan with Decoupled Look-back", 2016).
 *
 * Tiles are taken in order from a ticket counter, so a tile only ever waits
 * for tiles that started before it: no deadlock whatever the residency.  Every
 * wait is bounded; a wait that runs out records a timeout in the workspace
 * header and the call reports GPUTF_TIMEOUT.
 *
 * The workspace cleans itself: the CTA that finishes last resets the ticket
 * and done counters and the error words, and moves the epoch on.  Status
 * words carry the epoch of the call that wrote them, so words left by an
 * earlier call are never read as current and need no clearing between calls.
 */
#ifndef GPUTF_COMMON_CUH
#define GPUTF_COMMON_CUH

#include <cstdint>
#include <cuda_runtime.h>

#include "utf8_scheme.h"

namespace gputf {

constexpr unsigned FULL_MASK = 0xFFFFFFFFu;
constexpr uint64_t NONE = ~0ull;

/* Workspace header, at the start of the caller's workspace. */
struct WsHeader {
    unsigned long long ticket;    /* next tile ticket                          */
    unsigned long long done;      /* CTAs that finished                        */
    unsigned long long err_pos;   /* first flagged input position, NONE if none */
    unsigned long long cap_pos;   /* first character whose output does not fit */
    unsigned long long accum;     /* sum of a length pass                      */
    unsigned int epoch;           /* current call epoch, 1 .. EPOCH_LIMIT-1    */
    unsigned int flags;           /* FLAG_TIMEOUT                              */
    unsigned long long out_base;  /* host forms: output units of the chunks before */
    unsigned long long reserved[25];
};
static_assert(sizeof(WsHeader) == 256, "workspace header is 256 bytes");

constexpr unsigned FLAG_TIMEOUT = 1u;
constexpr size_t HEADER_BYTES = 256;

/* Epoch-tagged words (tile status words of every kernel, and the batched
 * kernel's per-string error words) all keep the epoch of the call that wrote
 * them in bits 43..63.  A word left by an earlier call, whatever kind of word
 * it was, then carries a smaller epoch and never reads as current, even when
 * a later call lays the workspace out differently.
 * Tile status word: epoch (21 bits) | spare (1) | flag (2) | value (40). */
constexpr unsigned EPOCH_BITS = 21;
constexpr unsigned EPOCH_LIMIT = 1u << EPOCH_BITS;
constexpr uint64_t VALUE_MASK = (1ull << 40) - 1;
constexpr uint64_t ST_AGGREGATE = 1;   /* value = this tile's own total            */
constexpr uint64_t ST_PREFIX = 2;      /* value = total of this tile and all before */

__device__ __forceinline__ uint64_t make_status(unsigned epoch, uint64_t flag, uint64_t value)
{
    return ((uint64_t)epoch << 43) | (flag << 40) | (value & VALUE_MASK);
}

__device__ __forceinline__ void st_release(unsigned long long *p, uint64_t v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint64_t ld_acquire(const unsigned long long *p)
{
    uint64_t v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ uint64_t ld_relaxed(const unsigned long long *p)
{
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

/* Upper bound on polls of one status word (with back-off, about a second). */
constexpr int SPIN_LIMIT = 1 << 21;

/*
 * Exclusive prefix of tile `tile` by decoupled look-back.  Called by all 32
 * lanes of one warp after the tile's aggregate has been published.  Each lane
 * reads one predecessor; the window moves back 32 tiles at a time until it
 * meets a tile that published its inclusive prefix.  A word still
 * unpublished after `limit` polls is taken as a prefix of 0 and a timeout is
 * recorded in *flags.
 */
__device__ __forceinline__ uint64_t look_back(unsigned long long *status, long long tile,
                                              unsigned epoch, unsigned *flags, int limit = SPIN_LIMIT)
{
    const int lane = threadIdx.x & 31;
    uint64_t exclusive = 0;
    long long end = tile - 1;     /* newest predecessor in the window */
    while (end >= 0) {
        long long idx = end - lane;
        uint64_t flag = ST_PREFIX, value = 0;
        if (idx >= 0) {
            int spins = 0;
            unsigned ns = 32;
            while (true) {
                uint64_t w = ld_acquire(status + idx);
                if ((unsigned)(w >> 43) == epoch && ((w >> 40) & 3) != 0) {
                    flag = (w >> 40) & 3;
                    value = w & VALUE_MASK;
                    break;
                }
                if (++spins > limit) {
                    atomicOr(flags, FLAG_TIMEOUT);
                    flag = ST_PREFIX;
                    value = 0;
                    break;
                }
                __nanosleep(ns);
                if (ns < 512) ns <<= 1;
            }
        }
        unsigned pmask = __ballot_sync(FULL_MASK, flag == ST_PREFIX);
        /* lanes up to and including the nearest inclusive prefix count */
        int stop = pmask ? __ffs(pmask) - 1 : 31;
        uint64_t v = lane <= stop ? value : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL_MASK, v, o);
        exclusive += v;
        if (pmask) break;
        end -= 32;
    }
    return exclusive;
}

/* Inclusive warp scan of 32-bit values. */
__device__ __forceinline__ uint32_t warp_inclusive(uint32_t v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(FULL_MASK, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

/*
 * Block-wide exclusive scan of one 32-bit value per thread.  `warp_sums`
 * holds at least THREADS/32 words of shared memory.  Returns the thread's
 * exclusive prefix; *total gets the block total.  Contains __syncthreads().
 */
template <int THREADS>
__device__ __forceinline__ uint32_t block_exclusive(uint32_t v, uint32_t *warp_sums, uint32_t *total)
{
    constexpr int WARPS = THREADS / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = warp_inclusive(v);
    if (lane == 31) warp_sums[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint32_t s = lane < WARPS ? warp_sums[lane] : 0;
        uint32_t si = warp_inclusive(s);
        if (lane < WARPS) warp_sums[lane] = si - s;
        if (lane == 31) warp_sums[WARPS] = si;
    }
    __syncthreads();
    *total = warp_sums[WARPS];
    return warp_sums[warp] + inc - v;
}

/* As block_exclusive, also OR-ing a flag over the block into *any.
 * `warp_sums` holds at least THREADS/32 + 2 words. */
template <int THREADS>
__device__ __forceinline__ uint32_t block_exclusive_or(uint32_t v, bool flag, uint32_t *warp_sums,
                                                       uint32_t *total, bool *any)
{
    constexpr int WARPS = THREADS / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = warp_inclusive(v);
    const unsigned f = __ballot_sync(FULL_MASK, flag);
    if (lane == 31) warp_sums[warp] = inc | (f ? 0x80000000u : 0u);
    __syncthreads();
    if (warp == 0) {
        uint32_t s = lane < WARPS ? warp_sums[lane] : 0;
        const unsigned fl = __ballot_sync(FULL_MASK, (s >> 31) != 0);
        s &= 0x7FFFFFFFu;
        uint32_t si = warp_inclusive(s);
        if (lane < WARPS) warp_sums[lane] = si - s;
        if (lane == 31) {
            warp_sums[WARPS] = si;
            warp_sums[WARPS + 1] = fl ? 1u : 0u;
        }
    }
    __syncthreads();
    *total = warp_sums[WARPS];
    *any = warp_sums[WARPS + 1] != 0;
    return warp_sums[warp] + inc - v;
}

/* Block-wide minimum of 64-bit values into *out (shared); contains syncs. */
template <int THREADS>
__device__ __forceinline__ uint64_t block_min(uint64_t v, unsigned long long *scratch)
{
    constexpr int WARPS = THREADS / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        uint64_t t = __shfl_xor_sync(FULL_MASK, v, o);
        v = t < v ? t : v;
    }
    if (lane == 0) scratch[warp] = v;
    __syncthreads();
    uint64_t m = scratch[0];
#pragma unroll
    for (int w = 1; w < WARPS; w++) m = scratch[w] < m ? scratch[w] : m;
    __syncthreads();
    return m;
}

/* Block-wide sum of 64-bit values, returned to every thread; contains syncs. */
template <int THREADS>
__device__ __forceinline__ uint64_t block_sum(uint64_t v, unsigned long long *scratch)
{
    constexpr int WARPS = THREADS / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL_MASK, v, o);
    if (lane == 0) scratch[warp] = v;
    __syncthreads();
    uint64_t m = 0;
#pragma unroll
    for (int w = 0; w < WARPS; w++) m += scratch[w];
    __syncthreads();
    return m;
}

/* Marks this CTA done; returns true (to every thread) in the CTA that
 * finished last.  Everything the CTA wrote before is visible to that CTA. */
__device__ __forceinline__ bool finish_cta(WsHeader *h, unsigned *smem_flag)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned long long prev = atomicAdd(&h->done, 1ull);
        *smem_flag = (prev == (unsigned long long)gridDim.x - 1) ? 1u : 0u;
        if (*smem_flag) __threadfence();
    }
    __syncthreads();
    return *smem_flag != 0;
}

/* Reset the header for the next call (last CTA only) and advance the epoch.
 * When the epoch would wrap, every status word is cleared first. */
__device__ __forceinline__ void reset_workspace(WsHeader *h, unsigned long long *status,
                                                uint64_t status_words)
{
    unsigned next = h->epoch + 1;
    if (next >= EPOCH_LIMIT) {
        for (uint64_t i = threadIdx.x; i < status_words; i += blockDim.x) status[i] = 0;
        next = 1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        h->ticket = 0;
        h->done = 0;
        h->err_pos = NONE;
        h->cap_pos = NONE;
        h->accum = 0;
        h->flags = 0;
        h->epoch = next;
        __threadfence();
    }
}

/* Non-caching 16-byte global load (streamed input). */
__device__ __forceinline__ uint4 ld_stream16(const void *p)
{
    uint4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

/* Streaming 16-byte global store. */
__device__ __forceinline__ void st_stream16(void *p, uint4 v)
{
    asm volatile("st.global.cs.v4.u32 [%0], {%1,%2,%3,%4};" ::"l"(p), "r"(v.x), "r"(v.y),
                 "r"(v.z), "r"(v.w)
                 : "memory");
}

/* ---------------------------------------------------------------------------
 * 1-D TMA bulk copies (global -> shared, completion counted on an mbarrier).
 * Copies start on 16-byte boundaries and move multiples of 16 bytes.  No
 * multicast.
 * ------------------------------------------------------------------------- */
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

/* Orders this thread's earlier shared-memory accesses before later
 * accesses by the async (TMA) proxy. */
__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned long long *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

/* Upper bound on polls of one mbarrier phase (each poll itself waits a
 * little in hardware); past it the caller records a timeout. */
constexpr int MBAR_SPIN_LIMIT = 1 << 22;

__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, uint32_t parity, int limit = MBAR_SPIN_LIMIT)
{
    for (int i = 0; i < limit; i++)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void bulk_load(void *dst_smem, const void *src_gmem, uint32_t bytes,
                                          unsigned long long *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst_smem)),
        "l"(src_gmem), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ uint32_t word_of(const uint4 &v, int k)
{
    return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w));
}

}  // namespace gputf

#endif
