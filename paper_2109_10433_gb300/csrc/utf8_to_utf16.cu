/*
 * Validating UTF-8 -> UTF-16LE (or UTF-16BE), and the UTF-8 validate-only and
 * length-only passes.
 *
 * The transcoder is a persistent kernel; each CTA takes tiles of 8 KiB in
 * ticket order and, for each:
 *   1. load: the tile (plus 16 bytes of halo on each side) arrives in a
 *      two-stage shared-memory ring by a TMA bulk copy (the tile grid is
 *      aligned to 16 bytes below the input pointer; tiles at the ends of the
 *      buffer are filled with guarded loads); each thread reads its 32
 *      consecutive bytes and the 4 bytes before them;
 *   2. classify and validate: a warp whose bytes (and the bytes just before)
 *      are all ASCII skips validation (the all-ASCII fast path of
 *      Algorithm 3); other threads run the nibble-table scheme of
 *      utf8_scheme.h four bytes at a time;
 *   3. per-byte output length: 1 unit at every byte that is not a
 *      continuation byte, 2 at a four-byte lead (Table 2: supplementary
 *      characters take a surrogate pair), summed per thread, scanned over the
 *      block and over all earlier tiles by decoupled look-back (warp 0);
 *   4. decode at every lead with the bit arithmetic of Section 3 and Figs.
 *      2-4 (gputf_utf8_decode in utf8_scheme.h; for four-byte characters
 *      subtract 0x10000 and split into 110110 / 110111 halves) into a
 *      shared-memory staging buffer at tile-local offsets, then write the
 *      tile's output range with aligned 16-byte stores, realigned by funnel
 *      shifts;
 *   5. the first flagged byte goes to an atomicMin; the CTA that finishes
 *      last turns it into the exact error start and class (scalar step of
 *      utf8_scheme.h), the output count of the valid prefix and the result.
 * Output past the caller's capacity is never written; the first character
 * that does not fit is reported as GPUTF_OUTPUT_TOO_SMALL.
 */
#include <cstdint>

#include "common.cuh"
#include "kernels.h"
#include "utf8_dfa.h"

namespace gputf {

/* One byte at extended index ex (input index ex - head), zero outside. */
__device__ __forceinline__ uint32_t byte_at(const uint8_t *base, long long ex, uint64_t head,
                                            uint64_t endx)
{
    return (ex >= (long long)head && ex < (long long)endx) ? base[ex] : 0u;
}

/* Four bytes at extended index ex (a multiple of 4), zero outside. */
__device__ __forceinline__ uint32_t word_at(const uint8_t *base, long long ex, uint64_t head,
                                            uint64_t endx)
{
    if (ex >= (long long)head && ex + 4 <= (long long)endx)
        return *reinterpret_cast<const uint32_t *>(base + ex);
    uint32_t w = 0;
#pragma unroll
    for (int k = 0; k < 4; k++) w |= byte_at(base, ex + k, head, endx) << (8 * k);
    return w;
}

/* Loads one thread's chunk of 4*WORDS bytes; returns true when it lies
 * wholly inside the input. */
template <int WORDS>
__device__ __forceinline__ bool load_chunk8(const uint8_t *base, uint64_t e0, uint64_t head,
                                            uint64_t endx, uint32_t (&w)[WORDS])
{
    const bool interior = e0 >= head && e0 + 4 * WORDS <= endx;
    if (interior) {
#pragma unroll
        for (int v = 0; v < WORDS / 4; v++) {
            uint4 q = ld_stream16(base + e0 + 16 * v);
            w[4 * v + 0] = q.x;
            w[4 * v + 1] = q.y;
            w[4 * v + 2] = q.z;
            w[4 * v + 3] = q.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < WORDS; k++) w[k] = word_at(base, (long long)(e0 + 4 * k), head, endx);
    }
    return interior;
}

/* Bit 7 of each byte of the word at extended index ex: set when the byte is
 * an input byte (head <= index < endx). */
__device__ __forceinline__ uint32_t range_mask(long long ex, uint64_t head, uint64_t endx, bool incl_end)
{
    uint32_t m = 0;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        long long e = ex + k;
        bool in = e >= (long long)head && (incl_end ? e <= (long long)endx : e < (long long)endx);
        m |= in ? (0x80u << (8 * k)) : 0u;
    }
    return m;
}

/* Byte index (0..3) of the lowest byte with bit 7 set in a nonzero mask. */
__device__ __forceinline__ int first_byte(uint32_t m) { return (__ffs(m) - 8) >> 3; }

constexpr int HALO8 = 16;   /* bytes staged on each side of a tile */

/* Stores the four units a (units 0, 1) and b (units 2, 3) at unit index u of
 * the staging buffer, in the widest stores that u's alignment allows (u is
 * the same modulo 4 across the warp). */
__device__ __forceinline__ void put_units4(uint16_t *o16, uint32_t u, uint32_t a, uint32_t b)
{
    if ((u & 3) == 0) {
        *reinterpret_cast<uint2 *>(o16 + u) = make_uint2(a, b);
    } else if ((u & 1) == 0) {
        *reinterpret_cast<uint32_t *>(o16 + u) = a;
        *reinterpret_cast<uint32_t *>(o16 + u + 2) = b;
    } else {
        o16[u] = (uint16_t)a;
        o16[u + 1] = (uint16_t)(a >> 16);
        o16[u + 2] = (uint16_t)b;
        o16[u + 3] = (uint16_t)(b >> 16);
    }
}

/* Stores the two units a (low half first) at unit index u. */
__device__ __forceinline__ void put_units2(uint16_t *o16, uint32_t u, uint32_t a)
{
    if ((u & 1) == 0) {
        *reinterpret_cast<uint32_t *>(o16 + u) = a;
    } else {
        o16[u] = (uint16_t)a;
        o16[u + 1] = (uint16_t)(a >> 16);
    }
}

/* The 16 bytes that start 2 S bytes before the end of the first of the two
 * granules w[0..3], w[4..7]. */
template <int S>
__device__ __forceinline__ uint4 window16(const uint32_t (&w)[8])
{
    constexpr int b = 16 - 2 * S, k = b >> 2;
    if constexpr ((b & 3) == 0) {
        return make_uint4(w[k], w[k + 1], w[k + 2], w[k + 3]);
    } else {
        return make_uint4(__funnelshift_r(w[k], w[k + 1], 16), __funnelshift_r(w[k + 1], w[k + 2], 16),
                          __funnelshift_r(w[k + 2], w[k + 3], 16), __funnelshift_r(w[k + 3], w[k + 4], 16));
    }
}

template <int THREADS, int WORDS, int STAGES>
struct U8Layout {
    static constexpr int BPT = 4 * WORDS;
    static constexpr uint64_t TILE = (uint64_t)THREADS * BPT;
    static constexpr uint32_t STAGE_BYTES = (uint32_t)TILE + 2 * HALO8;
    /* a thread's count is clamped to BPT + 1 units (see phase A) and its
     * decoding writes at most 2 units a byte from there */
    static constexpr uint32_t OUT_BYTES = (uint32_t)((2 * ((BPT + 1) * THREADS + 2 * BPT) + 15) / 16 * 16);
    static constexpr size_t SMEM = (size_t)STAGES * STAGE_BYTES + OUT_BYTES;
    static_assert(STAGE_BYTES % 16 == 0 && OUT_BYTES % 16 == 0, "16-byte granules");
};

/*
 * Persistent transcoder, software-pipelined over tiles (the same schedule as
 * the UTF-16 -> UTF-8 kernel): each iteration runs phase A of the tile n
 * whose input just arrived (lengths, validation, block scan, aggregate) and
 * phase B of the tile c before it (decode into the staging buffer,
 * look-back, inclusive prefix, write-out).  Thread 0 takes a new ticket as
 * phase B starts and writes it to c's ring entry before the look-back
 * barrier; after that barrier (every thread has read c's stage) the ticket's
 * input copy starts into that stage (a two-stage ring).  Input arrives with
 * 16 bytes of halo on each side: the 3 bytes before a position validate it,
 * the 3 after complete a character that starts near the tile's end.
 *
 * Barriers per iteration: the block scan's two and the look-back barrier,
 * and a last one only when no tile follows.  The ring entry is read at the
 * top of the next iteration after the look-back barrier that follows its
 * write; the staging buffer, the G0 word and the scan and minimum scratch
 * words of this iteration are read before the next iteration's block scan,
 * whose barriers come before anything rewrites them.  Without a next tile
 * there is no scan, hence the last barrier.
 *
 * A look-back waits only for the aggregates of smaller tickets, and the
 * ticket a CTA holds unpublished during its look-back is larger than the
 * tile it looks back from, so the CTA holding the smallest unpublished
 * ticket never waits: every wait ends.
 */
template <int THREADS, int WORDS, int STAGES, bool VALIDATE, bool BE, bool CHAINED>
/* CHAINED (the host forms' chunks) is a separate instance, held to 5 CTAs
 * per SM: as a runtime flag, its output base cost the single calls 16
 * registers and a CTA per SM */
__global__ void __launch_bounds__(THREADS, CHAINED ? 5 : 0)
utf8_to_utf16_kernel(const uint8_t *__restrict__ in, uint64_t n, uint16_t *__restrict__ out,
                     uint64_t cap, WsHeader *hdr, unsigned long long *status,
                     uint64_t status_words, uint64_t tiles, DevResult *res)
{
    using Lay = U8Layout<THREADS, WORDS, STAGES>;
    constexpr int BPT = Lay::BPT;
    constexpr uint64_t TILE = Lay::TILE;
    constexpr int WARPS = THREADS / 32;
    static_assert(STAGES == 2, "tile in phase A, tile in phase B (whose stage is refilled mid-iteration)");
    extern __shared__ uint4 smem4[];
    uint8_t *stages = reinterpret_cast<uint8_t *>(smem4);
    uint4 *outw4 = smem4 + (size_t)STAGES * Lay::STAGE_BYTES / 16;
    uint16_t *out16 = reinterpret_cast<uint16_t *>(outw4);
    uint8_t *outb = reinterpret_cast<uint8_t *>(outw4);
    __shared__ unsigned long long s_bar[STAGES];
    __shared__ unsigned long long s_ring[STAGES];
    __shared__ uint32_t s_warp[WARPS + 2];
    __shared__ unsigned long long s_min[WARPS];
    __shared__ unsigned long long s_lb_g0;
    __shared__ unsigned s_flag;

    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const uint64_t head = (uintptr_t)in & 15;
    const uint8_t *base = in - head;
    const uint64_t endx = head + n;    /* extended index of the end position */
    const unsigned epoch = *(volatile unsigned *)&hdr->epoch;
    /* a host form's chunks run chained: each writes its output after the
     * units of the chunks before it, which the header holds (the previous
     * chunk's last CTA moved it on) */
    if constexpr (CHAINED) {
        const uint64_t obase = ld_relaxed(&hdr->out_base);
        out += obase;
        cap = cap > obase ? cap - obase : 0;
    }

    /* thread 0: put tile t (already in stage s's ring entry) in flight into stage s */
    auto issue = [&](unsigned long long t, int s) {
        if (t >= tiles) return;
        const uint64_t x0 = t * TILE;
        if (x0 >= head + HALO8 && x0 + TILE + HALO8 <= endx) {
            fence_proxy_async();
            mbar_arrive_expect_tx(&s_bar[s], Lay::STAGE_BYTES);
            bulk_load(stages + (size_t)s * Lay::STAGE_BYTES, base + x0 - HALO8, Lay::STAGE_BYTES, &s_bar[s]);
        } else {
            mbar_arrive(&s_bar[s]);
        }
    };

    if (tid == 0) {
        for (int s = 0; s < STAGES; s++) mbar_init(&s_bar[s], 1);
        fence_mbar_init();
        for (int s = 0; s < STAGES; s++) {
            const unsigned long long t0 = atomicAdd(&hdr->ticket, 1ull);
            s_ring[s] = t0;
            issue(t0, s);
        }
    }
    __syncthreads();

    bool have_c = false, c_interior = false;
    unsigned long long c_tile = 0;
    uint32_t c_total = 0, c_excl = 0;
    int c_stage = 0;

    for (int it = 0;; it++) {
        /* ---------------- phase A of tile n ---------------- */
        const int sn = it % STAGES;
        const unsigned long long t = s_ring[sn];
        const bool have_n = t < tiles;
        const uint64_t x0n = t * TILE;
        const bool interior = have_n && x0n >= head + HALO8 && x0n + TILE + HALO8 <= endx;
        uint32_t n_total = 0, n_excl = 0;
        if (have_n) {
            uint8_t *sb = stages + (size_t)sn * Lay::STAGE_BYTES;
            if (interior) {
                if (!mbar_wait(&s_bar[sn], (uint32_t)((it / STAGES) & 1))) atomicOr(&hdr->flags, FLAG_TIMEOUT);
            } else {
                for (int i = tid; i < (int)Lay::STAGE_BYTES; i += THREADS)
                    sb[i] = (uint8_t)byte_at(base, (long long)(x0n + i) - HALO8, head, endx);
                __syncthreads();
            }
            const int i0 = HALO8 + tid * BPT;
            const long long e0 = (long long)(x0n + (uint64_t)tid * BPT);
            uint32_t w[WORDS];
#pragma unroll
            for (int v = 0; v < WORDS / 4; v++) {
                const uint4 q = *reinterpret_cast<const uint4 *>(sb + i0 + 16 * v);
                w[4 * v + 0] = q.x;
                w[4 * v + 1] = q.y;
                w[4 * v + 2] = q.z;
                w[4 * v + 3] = q.w;
            }
            const uint32_t pw = *reinterpret_cast<const uint32_t *>(sb + i0 - 4);
            /* per-byte output units: leads (non-continuation bytes) count 1,
             * four-byte leads 2 */
            uint32_t any = pw;
#pragma unroll
            for (int k = 0; k < WORDS; k++) {
                const uint32_t x = w[k];
                any |= x;
                uint32_t lead = ~(x & ~(x << 1)) & 0x80808080u;
                uint32_t f4 = x & (x << 1) & (x << 2) & (x << 3) & 0x80808080u;
                if (!interior) {
                    const uint32_t rm = range_mask(e0 + 4 * k, head, endx, false);
                    lead &= rm;
                    f4 &= rm;
                }
                n_total += __popc(lead) + __popc(f4);
            }
            /* When a chunk's bytes up to its end are a prefix of valid UTF-8,
             * every complete character gives at most one unit a byte and a
             * 4-byte lead cut off by the chunk's end two for its one byte, so
             * the chunk counts at most BPT + 1 units.  More means an error at
             * or before the chunk's end, after which the output carries no
             * meaning (and the result's `written` is recounted from the tiles
             * before the error): the clamp bounds the staging buffer. */
            if (n_total > (uint32_t)BPT + 1) n_total = (uint32_t)BPT + 1;
            /* validation, skipped by all-ASCII warps and all-ASCII threads */
            const bool ascii = (any & 0x80808080u) == 0;
            uint64_t first_err = NONE;
            if (VALIDATE && !__all_sync(FULL_MASK, ascii) && !ascii) {
                gputf_u8state st = gputf_u8state_of(pw);
                uint32_t errs[WORDS], anyerr = 0;
#pragma unroll
                for (int k = 0; k < WORDS; k++) {
                    errs[k] = gputf_utf8_errors_step(&st, w[k]);
                    anyerr |= errs[k];
                }
                if (anyerr) {   /* the first flagged byte of the chunk */
#pragma unroll
                    for (int k = WORDS - 1; k >= 0; k--) {
                        uint32_t nz = gputf_nonzero_bytes(errs[k]);
                        if (!interior) nz &= range_mask(e0 + 4 * k, head, endx, true);
                        if (nz) first_err = (uint64_t)(e0 + 4 * k + first_byte(nz)) - head;
                    }
                }
            }
            bool any_err;
            n_excl = block_exclusive_or<THREADS>(n_total, first_err != NONE, s_warp, &n_total, &any_err);
            if (tid == 0)
                st_release(status + t, make_status(epoch, t == 0 ? ST_PREFIX : ST_AGGREGATE, n_total));
            if (any_err) {
                const uint64_t m = block_min<THREADS>(first_err, s_min);
                if (tid == 0) atomicMin(&hdr->err_pos, (unsigned long long)m);
            }
        }

        /* ---------------- look-back and phase B of tile c ---------------- */
        if (have_c) {
            const uint8_t *sb = stages + (size_t)c_stage * Lay::STAGE_BYTES;
            const int i0 = HALO8 + tid * BPT;
            const long long e0 = (long long)(c_tile * TILE + (uint64_t)tid * BPT);
            const long long lb_idx = (long long)c_tile - 1 - tid;   /* warp 0's lanes */
            const uint64_t lb_word = (tid < 32 && c_tile > 0 && lb_idx >= 0) ? ld_relaxed(status + lb_idx) : 0;
            unsigned long long tk = 0;   /* the next tile's ticket (thread 0; its latency hides behind the decoding) */
            if (tid == 0 && have_n) tk = atomicAdd(&hdr->ticket, 1ull);

            uint32_t w[WORDS];
#pragma unroll
            for (int v = 0; v < WORDS / 4; v++) {
                const uint4 q = *reinterpret_cast<const uint4 *>(sb + i0 + 16 * v);
                w[4 * v + 0] = q.x;
                w[4 * v + 1] = q.y;
                w[4 * v + 2] = q.z;
                w[4 * v + 3] = q.w;
            }
            uint32_t lead[WORDS], any = 0;
#pragma unroll
            for (int k = 0; k < WORDS; k++) {
                const uint32_t x = w[k];
                any |= x;
                lead[k] = ~(x & ~(x << 1)) & 0x80808080u;
                if (!c_interior) lead[k] &= range_mask(e0 + 4 * k, head, endx, false);
            }
            /* decode at every lead into the staging buffer, in units from the
             * tile's first output unit (Section 3 bit arithmetic; Figs. 2-4) */
            uint32_t o = c_excl;
            /* The all-ASCII and all-2-byte warp paths store cooperatively:
             * in step i lane L takes the warp's word 32 i + L, so that a
             * store instruction covers consecutive units instead of one unit
             * in each lane's own stretch (lanes 8 or 16 words apart: 8- or
             * 16-way bank conflicts).  The warp's units are consecutive from
             * its lane 0's offset; stores are as wide as that offset's
             * alignment allows. */
            const uint32_t ow = __shfl_sync(FULL_MASK, o, 0);
            const uint32_t *wsrc = reinterpret_cast<const uint32_t *>(sb + HALO8 + (size_t)wid * 32 * BPT);
            if (__all_sync(FULL_MASK, (any & 0x80808080u) == 0)) {
                if (c_interior) {   /* every byte a character: unit ow + b for the warp's byte b */
#pragma unroll
                    for (int i = 0; i < WORDS; i++) {
                        const uint32_t x = wsrc[32 * i + lane];
                        const uint32_t u = ow + 128 * i + 4 * lane;
                        put_units4(out16, u, __byte_perm(x, 0u, 0x4140), __byte_perm(x, 0u, 0x4342));
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < WORDS; k++) {
#pragma unroll
                        for (int j = 0; j < 4; j++) {
                            if (lead[k] & (0x80u << (8 * j))) out16[o++] = (uint16_t)((w[k] >> (8 * j)) & 0xFF);
                        }
                    }
                }
            } else {
                /* one bit per character start of the chunk */
                uint32_t lm = 0;
#pragma unroll
                for (int k = 0; k < WORDS; k++)
                    lm |= ((((lead[k] >> 7) & 0x01010101u) * 0x01020408u) >> 24) << (4 * k);
                const uint8_t *row = sb + i0;
                /* Uniform-pattern paths (Section 4, the fast paths in front of
                 * Algorithm 2: a block of 2-byte characters only, or of 3-byte
                 * characters only).  A chunk qualifies when no byte is ASCII,
                 * its leads come every other byte with none from 0xE0 (2-byte
                 * characters), or every third byte all in E0-EF (3-byte
                 * characters); it then holds exactly the characters those
                 * leads start, the last one ending in the bytes after the
                 * chunk.  Warp-uniform: a warp takes a path only when all its
                 * threads qualify. */
                bool two = c_interior && (lm == 0x55555555u || lm == 0xAAAAAAAAu);
                bool three = c_interior && (lm == 0x49249249u || lm == 0x92492492u || lm == 0x24924924u);
                const bool try_two = __all_sync(FULL_MASK, two), try_three = __all_sync(FULL_MASK, three);
                if (try_two || try_three) {   /* the bytes, only where the leads already fit a pattern */
                    uint32_t all = 0xFFFFFFFFu, e0 = 0, f0 = 0, lead_lt_e0 = 0;
#pragma unroll
                    for (int k = 0; k < WORDS; k++) {
                        const uint32_t x = w[k];
                        const uint32_t ge_e0 = x & (x << 1) & (x << 2) & 0x80808080u;
                        all &= x;
                        e0 |= ge_e0;
                        f0 |= ge_e0 & (x << 3);
                        lead_lt_e0 |= lead[k] & ~ge_e0;
                    }
                    const bool no_ascii = (all & 0x80808080u) == 0x80808080u;
                    two = two && no_ascii && e0 == 0;
                    three = three && no_ascii && f0 == 0 && lead_lt_e0 == 0;
                }
                if (try_two && __all_sync(FULL_MASK, two)) {
                    /* Every lane holds 16 characters, and in valid text in
                     * the same phase (a chunk's last character ends where
                     * the next chunk's first begins), so the warp's 512
                     * characters start at r + 2 m, r being lane 0's first
                     * lead: four bytes lead, continuation, lead,
                     * continuation give two units, 110xxxxx 10yyyyyy -> x:y.
                     * (Invalid text gives other units here, inside the
                     * warp's 512, after its first error.) */
                    const uint32_t r8 = __shfl_sync(FULL_MASK, (lm & 1u) ? 0u : 8u, 0);
#pragma unroll
                    for (int i = 0; i < WORDS; i++) {
                        const uint32_t q = 32 * i + lane;
                        const uint32_t x = __funnelshift_r(wsrc[q], wsrc[q + 1], r8);
                        const uint32_t u2 = ((x & 0x001F001Fu) << 6) | ((x >> 8) & 0x003F003Fu);
                        put_units2(out16, ow + 2 * q, u2);
                    }
                    lm = 0;
                } else if (try_three && __all_sync(FULL_MASK, three)) {
                    /* 10 or 11 characters from the first lead r (0, 1 or 2):
                     * each 12 bytes from r + 12m hold four, 1110xxxx 10yyyyyy
                     * 10zzzzzz -> x:y:z */
                    const uint32_t wn0 = *reinterpret_cast<const uint32_t *>(row + BPT);
                    const uint32_t wn1 = *reinterpret_cast<const uint32_t *>(row + BPT + 4);
                    const uint32_t r = (lm & 1u) ? 0u : ((lm & 2u) ? 1u : 2u);
                    const uint32_t nc = __popc(lm);
                    uint32_t ww[WORDS + 2];
#pragma unroll
                    for (int k = 0; k < WORDS; k++) ww[k] = w[k];
                    ww[WORDS] = wn0;
                    ww[WORDS + 1] = wn1;
#pragma unroll
                    for (int m = 0; m < (BPT + 11) / 12; m++) {
                        const uint32_t x0 = __funnelshift_r(ww[3 * m], ww[3 * m + 1], 8 * r);
                        const uint32_t x1 = __funnelshift_r(ww[3 * m + 1], ww[3 * m + 2], 8 * r);
                        const uint32_t x2 = __funnelshift_r(ww[3 * m + 2], ww[3 * m + 3], 8 * r);
                        const uint32_t cs[4] = {x0, __funnelshift_r(x0, x1, 24), __funnelshift_r(x1, x2, 16), x2 >> 8};
#pragma unroll
                        for (int j = 0; j < 4; j++) {
                            const uint32_t c = cs[j];
                            const uint32_t u = ((c & 0x0Fu) << 12) | ((c >> 2) & 0x0FC0u) | ((c >> 16) & 0x3Fu);
                            if (4 * m + j < (int)nc) out16[o + 4 * m + j] = (uint16_t)u;
                        }
                    }
                    lm = 0;
                }
                /* the rest: each step reads the four bytes at a character
                 * start from the stage */
                while (lm) {
                    const int p = __ffs(lm) - 1;
                    lm &= lm - 1;
                    const uint32_t *wp = reinterpret_cast<const uint32_t *>(row + (p & ~3));
                    uint32_t u0, u1;
                    const int c = gputf_utf8_decode(__funnelshift_r(wp[0], wp[1], 8 * (p & 3)), &u0, &u1);
                    out16[o] = (uint16_t)u0;
                    if (c == 2) out16[o + 1] = (uint16_t)u1;
                    o += c;
                }
            }

            /* c's exclusive output offset, by warp 0 alone: its window (the
             * 32 tiles before c) is usable when an inclusive prefix appears in
             * it and every entry before that one has been published; otherwise
             * the warp walks back, waiting (bounded) for each word.  The
             * barrier then marks the staging buffer complete and hands G0 to
             * every thread. */
            if (c_tile > 0 && wid == 0) {
                const bool in_window = lb_idx >= 0;
                const uint64_t flag = in_window ? ((lb_word >> 40) & 3) : ST_PREFIX;
                const bool ok = !in_window || ((unsigned)(lb_word >> 43) == epoch && flag != 0);
                const unsigned pmask = __ballot_sync(FULL_MASK, ok && flag == ST_PREFIX);
                const unsigned badm = __ballot_sync(FULL_MASK, !ok);
                const int stop = pmask ? __ffs(pmask) - 1 : 31;
                uint64_t v = (lane <= stop && in_window) ? (lb_word & VALUE_MASK) : 0;
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(FULL_MASK, v, off);
                if (!pmask || (badm & (stop == 31 ? FULL_MASK : ((2u << stop) - 1))))
                    v = look_back(status, (long long)c_tile, epoch, &hdr->flags);
                if (lane == 0) {
                    s_lb_g0 = v;
                    st_release(status + c_tile, make_status(epoch, ST_PREFIX, v + c_total));
                }
            }
            if (tid == 0 && have_n) s_ring[c_stage] = tk;
            __syncthreads();
            const uint64_t G0 = c_tile > 0 ? s_lb_g0 : 0;
            const unsigned long long next_t = s_ring[c_stage];
            /* every thread has read c's stage: the new ticket's tile goes in
             * flight into it */
            if (tid == 0 && have_n) issue(tk, c_stage);

            /* write the tile's units [G0, G0 + cnt), clipped to the capacity,
             * with aligned 16-byte stores: global vector i takes the staging
             * bytes [16 i - shift, 16 i - shift + 16), from the staging
             * granules i - 1 and i (whole 16-byte reads, consecutive across
             * the lanes) */
            const uint64_t cnt = G0 >= cap ? 0 : (G0 + c_total > cap ? cap - G0 : c_total);
            const uint32_t shift = (uint32_t)((uintptr_t)(out + G0) & 15);
            uint8_t *gbase = reinterpret_cast<uint8_t *>(out + G0) - shift;
            const uint32_t lim = shift + 2 * (uint32_t)cnt;
            const uint32_t vf = shift ? 1u : 0u, vl = lim >> 4;   /* the whole vectors: [vf, vl) */
            for (uint32_t i = vf + tid; i < vl; i += THREADS) {
                const uint4 cur = outw4[i];
                uint4 ov = cur;
                if (shift) {   /* i >= 1: vf = 1 */
                    const uint4 prv = outw4[i - 1];
                    const uint32_t pw[8] = {prv.x, prv.y, prv.z, prv.w, cur.x, cur.y, cur.z, cur.w};
                    switch (shift >> 1) {   /* even: units are 2 bytes */
                    case 1: ov = window16<1>(pw); break;
                    case 2: ov = window16<2>(pw); break;
                    case 3: ov = window16<3>(pw); break;
                    case 4: ov = window16<4>(pw); break;
                    case 5: ov = window16<5>(pw); break;
                    case 6: ov = window16<6>(pw); break;
                    default: ov = window16<7>(pw); break;
                    }
                }
                if (BE) {   /* UTF-16BE: each unit's two bytes the other way round (shift is even) */
                    ov.x = __byte_perm(ov.x, 0u, 0x2301);
                    ov.y = __byte_perm(ov.y, 0u, 0x2301);
                    ov.z = __byte_perm(ov.z, 0u, 0x2301);
                    ov.w = __byte_perm(ov.w, 0u, 0x2301);
                }
                st_stream16(gbase + 16 * i, ov);
            }
            {   /* the partial vectors at the two ends, a unit per thread of the last warp */
                const uint32_t head_end = 16 * vf < lim ? 16 * vf : lim;         /* bytes [shift, head_end) */
                const uint32_t tail_start = 16 * vl > head_end ? 16 * vl : head_end;   /* [tail_start, lim) */
                const int t = tid - (THREADS - 32);
                uint32_t b = ~0u;
                if (t >= 0 && t < 8) {
                    b = shift + 2 * (uint32_t)t;
                    if (b >= head_end) b = ~0u;
                } else if (t >= 8 && t < 16) {
                    b = tail_start + 2 * (uint32_t)(t - 8);
                    if (b >= lim) b = ~0u;
                }
                if (b != ~0u) {
                    const uint32_t u = *reinterpret_cast<const uint16_t *>(outb + b - shift);
                    *reinterpret_cast<uint16_t *>(gbase + b) = (uint16_t)(BE ? __byte_perm(u, 0u, 0x4401) : u);
                }
            }

            /* the first character whose units do not fit (only in the tile
             * that crosses the capacity) */
            if (G0 <= cap && G0 + c_total > cap) {
                uint64_t cap_first = NONE;
                uint64_t g = G0 + c_excl;
#pragma unroll
                for (int k = 0; k < WORDS; k++) {
#pragma unroll
                    for (int j = 0; j < 4; j++) {
                        if (lead[k] & (0x80u << (8 * j))) {
                            const uint32_t c = ((w[k] >> (8 * j)) & 0xFF) >= 0xF0 ? 2u : 1u;
                            if (g + c > cap && cap_first == NONE) cap_first = (uint64_t)(e0 + 4 * k + j) - head;
                            g += c;
                        }
                    }
                }
                const uint64_t m = block_min<THREADS>(cap_first, s_min);
                if (tid == 0 && m != NONE) atomicMin(&hdr->cap_pos, (unsigned long long)m);
            }
            /* with no tile to follow, the next iteration has no block scan:
             * this barrier keeps the staging buffer and G0 until every thread
             * has written its part out */
            if (!have_n || next_t >= tiles) __syncthreads();
        }

        if (!have_n) break;
        have_c = true;
        c_interior = interior;
        c_tile = t;
        c_total = n_total;
        c_excl = n_excl;
        c_stage = sn;
    }

    /* the CTA that finishes last writes the result */
    if (!finish_cta(hdr, &s_flag)) return;
    const uint64_t f = ld_relaxed(&hdr->err_pos);
    const uint64_t cpos = ld_relaxed(&hdr->cap_pos);
    const unsigned flags = *(volatile unsigned *)&hdr->flags;
    int32_t error = GPUTF_E_OK;
    uint64_t pos = n;
    if (flags & FLAG_TIMEOUT) {
        error = GPUTF_E_TIMEOUT;
        pos = 0;
    } else {
        uint64_t s = NONE;
        int cls = GPUTF_E_OK;
        if (f != NONE) {
            if (gputf_utf8_fixup(in, n, f, &cls, &s) != 0) cls = GPUTF_E_INTERNAL;
        }
        if (cpos != NONE && (s == NONE || cpos < s)) {
            error = GPUTF_E_OUTPUT_TOO_SMALL;
            pos = cpos;
        } else if (s != NONE) {
            error = cls;
            pos = s;
        }
    }
    uint64_t written = 0;
    if (error == GPUTF_E_OK) {
        written = ld_relaxed(status + tiles - 1) & VALUE_MASK;
    } else if (error != GPUTF_E_TIMEOUT) {
        /* output units of [0, pos): earlier tiles' total plus a recount */
        const uint64_t t = (head + pos) / TILE;
        const uint64_t before = t ? (ld_relaxed(status + t - 1) & VALUE_MASK) : 0;
        const uint64_t start = t * TILE > head ? t * TILE - head : 0;
        uint32_t c = 0;
        for (uint64_t i = start + tid; i < pos; i += THREADS) {
            const uint32_t b = in[i];
            c += ((b & 0xC0) != 0x80) + (b >= 0xF0);
        }
        uint32_t sum;
        block_exclusive<THREADS>(c, s_warp, &sum);
        written = before + sum;
    }
    if (tid == 0) {
        res->error = error;
        res->reserved = 0;
        res->position = pos;
        res->written = written;
        if constexpr (CHAINED) hdr->out_base = ld_relaxed(&hdr->out_base) + written;
    }
    reset_workspace(hdr, status, status_words);
}

/* ------------------------------------------------------------------------
 * Validate-only and length-only passes: one read of the input, no scan.
 * ---------------------------------------------------------------------- */
/* Streaming passes: a grid of resident CTAs walks the tiles (grid-stride);
 * each thread issues the loads of its chunk of the next tile before working
 * on the current one, and no barrier is taken per tile. */

/* The validate-only pass runs the automaton of utf8_dfa.h over each byte:
 * a byte's class, then the next state, both looked up in shared memory.
 * Each table is kept once per bank: entry e sits in word 32 e + lane, so
 * the 32 lanes of a warp read 32 different banks whatever they look up.
 * Class entries hold the class times 128 and transition entries the next
 * state times 128 * classes, byte offsets into the transition table, so a
 * step is a shift and a mask for the byte, two loads and one add. */
constexpr uint32_t DFA_ROW = 128;                                            /* 32 lanes x 4 bytes */
constexpr uint32_t DFA_CLASS_BYTES = 256 * DFA_ROW;
constexpr uint32_t DFA_STATE_STRIDE = GPUTF_DFA_CLASSES * DFA_ROW;
constexpr uint32_t DFA_SMEM = DFA_CLASS_BYTES + GPUTF_DFA_STATES * DFA_STATE_STRIDE;

template <int THREADS>
__device__ __forceinline__ void dfa_tables(uint32_t *t)
{
    for (uint32_t i = threadIdx.x; i < 256 * 32; i += THREADS) t[i] = gputf_dfa_class(i >> 5) * DFA_ROW;
    uint32_t *nt = t + DFA_CLASS_BYTES / 4;
    for (uint32_t i = threadIdx.x; i < GPUTF_DFA_STATES * GPUTF_DFA_CLASSES * 32; i += THREADS) {
        const uint32_t e = i >> 5;
        nt[i] = gputf_dfa_next(e / GPUTF_DFA_CLASSES, e % GPUTF_DFA_CLASSES) * DFA_STATE_STRIDE;
    }
}

/* One step: the state offset after byte j of word w. */
template <int J>
__device__ __forceinline__ uint32_t dfa_step(const char *tab, uint32_t sv, uint32_t w, uint32_t lane4)
{
    const uint32_t boff = (J == 0 ? (w << 7) : (w >> (8 * J - 7))) & 0x7F80u;   /* byte * 128 */
    const uint32_t cls = *reinterpret_cast<const uint32_t *>(tab + (boff | lane4));
    return *reinterpret_cast<const uint32_t *>(tab + DFA_CLASS_BYTES + sv + cls + lane4);
}

template <int THREADS, int WORDS>
__global__ void __launch_bounds__(THREADS)
validate_utf8_kernel(const uint8_t *__restrict__ in, uint64_t n, uint64_t tiles, WsHeader *hdr,
                     DevResult *res)
{
    constexpr int BPT = 4 * WORDS;
    constexpr uint64_t TILE = (uint64_t)THREADS * BPT;
    constexpr uint32_t SV_REJECT = GPUTF_DFA_REJECT * DFA_STATE_STRIDE;
    extern __shared__ uint4 smem4[];
    const char *tab = reinterpret_cast<const char *>(smem4);
    __shared__ unsigned long long s_min[THREADS / 32];
    __shared__ unsigned s_flag;
    dfa_tables<THREADS>(reinterpret_cast<uint32_t *>(smem4));
    __syncthreads();
    const int tid = threadIdx.x, lane = tid & 31;
    const uint32_t lane4 = 4u * (uint32_t)lane;
    const uint64_t head = (uintptr_t)in & 15;
    const uint8_t *base = in - head;
    const uint64_t endx = head + n;
    uint64_t first_err = NONE;
    uint64_t tile = blockIdx.x;
    uint32_t w[WORDS];
    /* lane 0 also needs the word before its chunk and lane 31 the word
     * after it (other warps'): loaded with the chunk, one tile ahead */
    uint32_t side = 0;
    auto side_word = [&](uint64_t e0) -> uint32_t {
        if (lane == 0) return word_at(base, (long long)e0 - 4, head, endx);
        if (lane == 31) return word_at(base, (long long)(e0 + BPT), head, endx);
        return 0u;
    };
    if (tile < tiles) {
        load_chunk8<WORDS>(base, tile * TILE + (uint64_t)tid * BPT, head, endx, w);
        side = side_word(tile * TILE + (uint64_t)tid * BPT);
    }
    while (tile < tiles) {
        const uint64_t e0 = tile * TILE + (uint64_t)tid * BPT;
        const uint64_t next = tile + gridDim.x;
        uint32_t v[WORDS], v_side = 0;
        if (next < tiles) {
            load_chunk8<WORDS>(base, next * TILE + (uint64_t)tid * BPT, head, endx, v);
            v_side = side_word(next * TILE + (uint64_t)tid * BPT);
        }
        uint32_t pw = __shfl_up_sync(FULL_MASK, w[WORDS - 1], 1);
        uint32_t nw = __shfl_down_sync(FULL_MASK, w[0], 1);
        if (lane == 0) pw = side;
        if (lane == 31) nw = side;
        uint32_t any = pw;
#pragma unroll
        for (int k = 0; k < WORDS; k++) any |= w[k];
        /* all-ASCII chunks (and the bytes before them) hold no error */
        if ((any & 0x80808080u) != 0 && first_err == NONE) {
            /* the state at the chunk: the three bytes before it replayed
             * from SYNC0; then every byte; then, while inside a character,
             * up to three bytes after the chunk (bytes outside the input
             * read as zero, so a character cut by the end rejects there) */
            /* two independent runs, over the chunk's two halves, each
             * resynchronised from the three bytes before it; the first runs
             * on into the second half while inside a character */
            constexpr int HW = WORDS / 2;
            const uint32_t inside_lo = GPUTF_DFA_NEED1 * DFA_STATE_STRIDE;
            const uint32_t inside_span = (GPUTF_DFA_AFTER_F4 - GPUTF_DFA_NEED1) * DFA_STATE_STRIDE;
            uint32_t sa = GPUTF_DFA_SYNC0 * DFA_STATE_STRIDE, sb = sa;
            sa = dfa_step<1>(tab, sa, pw, lane4);
            sb = dfa_step<1>(tab, sb, w[HW - 1], lane4);
            sa = dfa_step<2>(tab, sa, pw, lane4);
            sb = dfa_step<2>(tab, sb, w[HW - 1], lane4);
            sa = dfa_step<3>(tab, sa, pw, lane4);
            sb = dfa_step<3>(tab, sb, w[HW - 1], lane4);
#pragma unroll
            for (int k = 0; k < HW; k++) {
                sa = dfa_step<0>(tab, sa, w[k], lane4);
                sb = dfa_step<0>(tab, sb, w[HW + k], lane4);
                sa = dfa_step<1>(tab, sa, w[k], lane4);
                sb = dfa_step<1>(tab, sb, w[HW + k], lane4);
                sa = dfa_step<2>(tab, sa, w[k], lane4);
                sb = dfa_step<2>(tab, sb, w[HW + k], lane4);
                sa = dfa_step<3>(tab, sa, w[k], lane4);
                sb = dfa_step<3>(tab, sb, w[HW + k], lane4);
            }
            if (sa - inside_lo <= inside_span) sa = dfa_step<0>(tab, sa, w[HW], lane4);
            if (sb - inside_lo <= inside_span) sb = dfa_step<0>(tab, sb, nw, lane4);
            if (sa - inside_lo <= inside_span) sa = dfa_step<1>(tab, sa, w[HW], lane4);
            if (sb - inside_lo <= inside_span) sb = dfa_step<1>(tab, sb, nw, lane4);
            if (sa - inside_lo <= inside_span) sa = dfa_step<2>(tab, sa, w[HW], lane4);
            if (sb - inside_lo <= inside_span) sb = dfa_step<2>(tab, sb, nw, lane4);
            if (sa == SV_REJECT || sb == SV_REJECT) {
                /* rare: walk again, one byte at a time, to the first
                 * rejected byte (a rejection while replaying the bytes
                 * before the chunk counts at the chunk's first byte) */
                uint32_t st = GPUTF_DFA_SYNC0;
                int at = -1;
                for (int i = -3; i < BPT + 3 && at < 0; i++) {
                    const uint32_t word = i < 0 ? pw : (i < BPT ? w[(i >> 2) & (WORDS - 1)] : nw);
                    const uint32_t b = (word >> (8 * ((i + 4) & 3))) & 0xFF;
                    if (i >= BPT && !gputf_dfa_inside(st)) break;
                    st = gputf_dfa_next(st, gputf_dfa_class(b));
                    if (st == GPUTF_DFA_REJECT) at = i < 0 ? 0 : i;
                }
                if (at >= 0) {
                    const uint64_t pos = e0 + (uint64_t)at - head;
                    first_err = pos < n ? pos : n;
                }
            }
        }
#pragma unroll
        for (int k = 0; k < WORDS; k++) w[k] = v[k];
        side = v_side;
        tile = next;
    }
    if (__syncthreads_or(first_err != NONE)) {
        const uint64_t m = block_min<THREADS>(first_err, s_min);
        if (tid == 0) atomicMin(&hdr->err_pos, (unsigned long long)m);
    }
    if (!finish_cta(hdr, &s_flag)) return;
    if (tid == 0) {
        const uint64_t f = ld_relaxed(&hdr->err_pos);
        int cls = GPUTF_E_OK;
        uint64_t s = n;
        if (f != NONE && gputf_utf8_fixup(in, n, f, &cls, &s) != 0) cls = GPUTF_E_INTERNAL;
        res->error = cls;
        res->reserved = 0;
        res->position = s;
        res->written = 0;
    }
    reset_workspace(hdr, nullptr, 0);
}

template <int THREADS, int WORDS>
__global__ void __launch_bounds__(THREADS)
utf16_length_from_utf8_kernel(const uint8_t *__restrict__ in, uint64_t n, uint64_t tiles,
                              WsHeader *hdr, unsigned long long *len_out)
{
    constexpr int BPT = 4 * WORDS;
    constexpr uint64_t TILE = (uint64_t)THREADS * BPT;
    __shared__ unsigned long long s_part[THREADS / 32];
    __shared__ unsigned s_flag;
    const int tid = threadIdx.x;
    const uint64_t head = (uintptr_t)in & 15;
    const uint8_t *base = in - head;
    const uint64_t endx = head + n;
    uint64_t acc = 0;
    uint64_t tile = blockIdx.x;
    uint32_t w[WORDS];
    bool interior = false;
    if (tile < tiles) interior = load_chunk8<WORDS>(base, tile * TILE + (uint64_t)tid * BPT, head, endx, w);
    while (tile < tiles) {
        const uint64_t e0 = tile * TILE + (uint64_t)tid * BPT;
        const uint64_t next = tile + gridDim.x;
        uint32_t v[WORDS];
        bool v_interior = false;
        if (next < tiles) v_interior = load_chunk8<WORDS>(base, next * TILE + (uint64_t)tid * BPT, head, endx, v);
        uint32_t c = 0;   /* per-byte counts, at most 2 a word: 16 a byte */
#pragma unroll
        for (int k = 0; k < WORDS; k++) {
            const uint32_t x = w[k];
            uint32_t lead = ~(x & ~(x << 1)) & 0x80808080u;            /* not 10xxxxxx */
            uint32_t f4 = x & (x << 1) & (x << 2) & (x << 3) & 0x80808080u;   /* 1111xxxx */
            if (!interior) {
                const uint32_t rm = range_mask((long long)(e0 + 4 * k), head, endx, false);
                lead &= rm;
                f4 &= rm;
            }
            c += (lead >> 7) + (f4 >> 7);
        }
        acc += (c * 0x01010101u) >> 24;
#pragma unroll
        for (int k = 0; k < WORDS; k++) w[k] = v[k];
        interior = v_interior;
        tile = next;
    }
    const uint64_t sum = block_sum<THREADS>(acc, s_part);
    if (tid == 0) atomicAdd(&hdr->accum, (unsigned long long)sum);
    if (!finish_cta(hdr, &s_flag)) return;
    if (tid == 0) *len_out = ld_relaxed(&hdr->accum);
    reset_workspace(hdr, nullptr, 0);
}

/* ------------------------------------------------------------------------
 * Launchers.
 * ---------------------------------------------------------------------- */
constexpr int U8_THREADS = 256;
constexpr int U8_WORDS = 8;     /* 32 bytes per thread, 8 KiB tiles */
constexpr int U8_STAGES = 2;
using U8Lay = U8Layout<U8_THREADS, U8_WORDS, U8_STAGES>;

uint64_t utf8_to_utf16_tiles(const void *in, uint64_t n)
{
    /* tiles cover the end position n as well (a character cut short there is
     * flagged at n) */
    return ((uintptr_t)in % 16 + n + 1 + U8Lay::TILE - 1) / U8Lay::TILE;
}

template <bool VALIDATE, bool BE, bool CHAINED>
static cudaError_t launch8(const uint8_t *in, uint64_t n, uint16_t *out, uint64_t cap, void *ws,
                           uint64_t status_words, DevResult *res, int sms, cudaStream_t stream)
{
    auto kern = utf8_to_utf16_kernel<U8_THREADS, U8_WORDS, U8_STAGES, VALIDATE, BE, CHAINED>;
    static int per_sm = 0;
    if (per_sm == 0) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)U8Lay::SMEM);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, U8_THREADS, U8Lay::SMEM);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) per_sm = 1;
    }
    const uint64_t tiles = utf8_to_utf16_tiles(in, n);
    const uint64_t grid = tiles < (uint64_t)sms * per_sm ? tiles : (uint64_t)sms * per_sm;
    WsHeader *hdr = static_cast<WsHeader *>(ws);
    auto *status = reinterpret_cast<unsigned long long *>(static_cast<char *>(ws) + HEADER_BYTES);
    kern<<<(unsigned)grid, U8_THREADS, U8Lay::SMEM, stream>>>(in, n, out, cap, hdr, status, status_words,
                                                              tiles, res);
    return cudaGetLastError();
}

cudaError_t launch_utf8_to_utf16(const uint8_t *in, uint64_t n, uint16_t *out, uint64_t cap,
                                 void *ws, uint64_t status_words, DevResult *res, int sms, bool validate,
                                 bool big_endian, bool chained, cudaStream_t stream)
{
    if (chained) {   /* the host forms' chunks: validating, little-endian */
        if (!validate || big_endian) return cudaErrorInvalidValue;
        return launch8<true, false, true>(in, n, out, cap, ws, status_words, res, sms, stream);
    }
    if (big_endian)
        return validate ? launch8<true, true, false>(in, n, out, cap, ws, status_words, res, sms, stream)
                        : launch8<false, true, false>(in, n, out, cap, ws, status_words, res, sms, stream);
    return validate ? launch8<true, false, false>(in, n, out, cap, ws, status_words, res, sms, stream)
                    : launch8<false, false, false>(in, n, out, cap, ws, status_words, res, sms, stream);
}

/* Grid of a streaming pass: the CTAs that fit on the device at once (no
 * more than there are tiles). */
template <typename K>
static unsigned resident_grid8(K kern, int threads, uint64_t tiles, int sms, int *per_sm)
{
    if (*per_sm == 0) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, threads, 0) != cudaSuccess || b < 1) b = 1;
        *per_sm = b;
    }
    const uint64_t g = (uint64_t)sms * *per_sm;
    return (unsigned)(tiles < g ? (tiles ? tiles : 1) : g);
}

cudaError_t launch_validate_utf8(const uint8_t *in, uint64_t n, void *ws, DevResult *res,
                                 int sms, cudaStream_t stream)
{
    constexpr int T = 256, W = 8;
    constexpr uint64_t TILE = (uint64_t)T * 4 * W;
    const uint64_t tiles = ((uintptr_t)in % 16 + n + 1 + TILE - 1) / TILE;
    static int per_sm = 0;
    auto kern = validate_utf8_kernel<T, W>;
    if (per_sm == 0) {   /* the automaton's tables take more than the default 48 KiB of shared memory */
        const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)DFA_SMEM);
        if (e != cudaSuccess) return e;
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, T, DFA_SMEM) != cudaSuccess || b < 1) b = 1;
        per_sm = b;
    }
    kern<<<resident_grid8(kern, T, tiles, sms, &per_sm), T, DFA_SMEM, stream>>>(in, n, tiles,
                                                                                 static_cast<WsHeader *>(ws), res);
    return cudaGetLastError();
}

cudaError_t launch_utf16_length_from_utf8(const uint8_t *in, uint64_t n, void *ws,
                                          unsigned long long *len, int sms, cudaStream_t stream)
{
    constexpr int T = 256, W = 8;
    constexpr uint64_t TILE = (uint64_t)T * 4 * W;
    const uint64_t tiles = ((uintptr_t)in % 16 + n + TILE - 1) / TILE;
    static int per_sm = 0;
    auto kern = utf16_length_from_utf8_kernel<T, W>;
    kern<<<resident_grid8(kern, T, tiles, sms, &per_sm), T, 0, stream>>>(in, n, tiles, static_cast<WsHeader *>(ws),
                                                                          len);
    return cudaGetLastError();
}

}  // namespace gputf
