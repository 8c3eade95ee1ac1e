/*
 * Validating UTF-16LE (or UTF-16BE) -> UTF-8, and the UTF-16 validate-only
 * and length-only passes.
 *
 * The transcoder is a persistent kernel; each CTA takes tiles of 6144 units
 * in ticket order and, for each:
 *   1. load: the tile (plus 8 units of halo on each side) arrives in a
 *      two-stage shared-memory ring by a TMA bulk copy; each thread reads
 *      its 24 consecutive units, the unit before and the unit after;
 *   2. per-unit output bytes and validation (utf16_scheme.h, Section 3 and
 *      Table 2), four units per step on their gathered high bytes: 1, 2 or
 *      3 bytes by value, the 4 bytes of a surrogate pair on its high unit and
 *      none on its low unit, 2 for a lone surrogate; the pairing rule is
 *      checked on the way;
 *   3. offsets: a block scan of the per-thread sums and a decoupled
 *      look-back over earlier tiles (warp 0 alone);
 *   4. encode each unit (lead prefixes 110 / 1110 / 11110, continuation
 *      prefix 10 over 6-bit groups; Section 5) into a shared-memory staging
 *      buffer at tile-local offsets: warps whose units all take one length
 *      store at fixed offsets; otherwise each thread writes its units back to
 *      front, three unconditional continuation-byte stores and one predicated
 *      lead store per unit; the tile's range then goes out with aligned
 *      16-byte stores, realigned by funnel shifts;
 *   5. the first invalid unit (exact: no fix-up is needed in UTF-16) goes to
 *      an atomicMin; the CTA that finishes last writes the result.
 */
#include <cstdint>

#include "common.cuh"
#include "kernels.h"
#include "utf16_scheme.h"

namespace gputf {

__device__ __forceinline__ uint32_t unit_at(const uint16_t *base, long long ex, uint64_t head,
                                            uint64_t endx)
{
    return (ex >= (long long)head && ex < (long long)endx) ? base[ex] : 0u;
}

/* Two units at extended index ex (even), zero outside. */
__device__ __forceinline__ uint32_t pair_at(const uint16_t *base, long long ex, uint64_t head,
                                            uint64_t endx)
{
    if (ex >= (long long)head && ex + 2 <= (long long)endx)
        return *reinterpret_cast<const uint32_t *>(base + ex);
    return unit_at(base, ex, head, endx) | (unit_at(base, ex + 1, head, endx) << 16);
}

/* Loads one thread's chunk of 2*WORDS units; true when wholly inside. */
template <int WORDS>
__device__ __forceinline__ bool load_chunk16(const uint16_t *base, uint64_t e0, uint64_t head,
                                             uint64_t endx, uint32_t (&w)[WORDS])
{
    const bool interior = e0 >= head && e0 + 2 * WORDS <= endx;
    if (interior) {
#pragma unroll
        for (int v = 0; v < WORDS / 4; v++) {
            uint4 q = ld_stream16(base + e0 + 8 * v);
            w[4 * v + 0] = q.x;
            w[4 * v + 1] = q.y;
            w[4 * v + 2] = q.z;
            w[4 * v + 3] = q.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < WORDS; k++) w[k] = pair_at(base, (long long)(e0 + 2 * k), head, endx);
    }
    return interior;
}

/* Byte order: UTF-16BE input holds each unit's two bytes the other way
 * round; swapping them in registers gives the unit values. */
template <bool BE>
__device__ __forceinline__ uint32_t units_of(uint32_t w) { return BE ? __byte_perm(w, 0u, 0x2301) : w; }
template <bool BE>
__device__ __forceinline__ uint32_t unit_of(uint32_t u) { return BE ? __byte_perm(u, 0u, 0x4401) : u; }

__device__ __forceinline__ bool is_high(uint32_t u) { return (u & 0xFC00) == 0xD800; }
__device__ __forceinline__ bool is_low(uint32_t u) { return (u & 0xFC00) == 0xDC00; }

/* Sum of the four bytes of x (the sum below 256). */
__device__ __forceinline__ uint32_t byte_sum(uint32_t x) { return (x * 0x01010101u) >> 24; }

/* Byte j of x, zero-extended (one instruction for a constant j). */
__device__ __forceinline__ uint32_t byte_at(uint32_t x, int j)
{
    return j == 0 ? (x & 0xFFu) : j == 3 ? (x >> 24) : __byte_perm(x, 0u, 0x4440u + (uint32_t)j);
}

/* Output bytes of a unit by value: 1, 2 or 3, and 2 for a surrogate unit
 * (the closed form of the length pass; Table 2). */
__device__ __forceinline__ uint32_t len8(uint32_t u)
{
    return u < 0x80 ? 1u : ((u < 0x800 || (u & 0xF800) == 0xD800) ? 2u : 3u);
}

/* 0xFF in byte i of the result for each set bit i of the 4 low bits of x. */
__device__ __forceinline__ uint32_t byte_mask4(uint32_t x)
{
    return (((x & 0xFu) * 0x00204081u) & 0x01010101u) * 0xFFu;
}

/*
 * Bytes written per unit inside a tile.  A surrogate pair is written whole by
 * its high unit (4 bytes) and its low unit writes none; every other unit
 * writes its len8().  Over any run of valid text this adds up to the same
 * total as len8(), and it lets every unit write its bytes from its own value
 * and the value of the unit after it:
 *   1 byte  : u
 *   2 bytes : 110xxxxx 10xxxxxx                 (u < 0x800)
 *   3 bytes : 1110xxxx 10xxxxxx 10xxxxxx        (other BMP units)
 *   4 bytes : 11110xxx 10xxxxxx 10xxxxxx 10xxxxxx of the code point
 *             c = ((hi - 0xD800) << 10) + (lo - 0xDC00) + 0x10000
 * (Section 3 pair construction; Section 5 byte layout with lead prefixes
 * 110 / 1110 / 11110 and continuation prefix 10.)  A lone surrogate (an
 * error) writes 2 bytes of no meaning; they lie past the valid prefix.
 */
__device__ __forceinline__ void put_utf8(uint32_t sa, uint32_t u, uint32_t next, uint32_t l)
{
    const uint32_t se = sa + l;                        /* sa: shared address of the lead byte; se: one past the last */
    uint32_t lead, b1, b2, b3;
    gputf_u16_utf8_bytes(u, next, l, &lead, &b1, &b2, &b3);
    /* predicated stores: lead at o, continuation bytes at end-1, end-2, end-3
     * as far as the unit's length goes */
    asm volatile("{\n\t.reg .pred p1, p2, p3, p4;\n\t"
                 "setp.ne.u32 p1, %4, 0;\n\t"
                 "setp.ge.u32 p2, %4, 2;\n\t"
                 "setp.ge.u32 p3, %4, 3;\n\t"
                 "setp.eq.u32 p4, %4, 4;\n\t"
                 "@p1 st.shared.u8 [%0], %1;\n\t"
                 "@p2 st.shared.u8 [%5+-1], %2;\n\t"
                 "@p3 st.shared.u8 [%5+-2], %3;\n\t"
                 "@p4 st.shared.u8 [%5+-3], %6;\n\t}"
                 :: "r"(sa), "r"(lead), "r"(b1), "r"(b2), "r"(l), "r"(se), "r"(b3) : "memory");
}

/*
 * The same bytes, written back to front: the unit's bytes end at shared
 * address e (exclusive); returns its start e - l.  The continuation-byte
 * positions e-3, e-2, e-1 are stored unconditionally and the lead byte last,
 * so a unit shorter than 4 bytes leaves stray bytes below its start, in the
 * bytes of the units before it.  Units therefore go in reverse order (each
 * unit's earlier neighbours overwrite its strays), and the caller keeps e - 3
 * at or above the start of the thread's run.  Only the lead store needs a
 * predicate (a unit of 0 bytes writes nothing of its own).
 */
__device__ __forceinline__ uint32_t put_utf8_back(uint32_t e, uint32_t u, uint32_t next, uint32_t l)
{
    const uint32_t s = e - l;
    uint32_t lead, b1, b2, b3;
    gputf_u16_utf8_bytes_back(u, next, l, &lead, &b1, &b2, &b3);
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "setp.ne.u32 p, %4, 0;\n\t"
                 "st.shared.u8 [%0+-3], %3;\n\t"
                 "st.shared.u8 [%0+-2], %2;\n\t"
                 "st.shared.u8 [%0+-1], %1;\n\t"
                 "@p st.shared.u8 [%5], %6;\n\t}"
                 :: "r"(e), "r"(b1), "r"(b2), "r"(b3), "r"(l), "r"(s), "r"(lead) : "memory");
    return s;
}

constexpr int HALO16 = 8;   /* units staged on each side of a tile (16 bytes) */

template <int THREADS, int UPT, int STAGES>
struct U16Layout {
    static constexpr uint64_t TILE = (uint64_t)THREADS * UPT;
    static constexpr int STAGE_UNITS = (int)TILE + 2 * HALO16;
    static constexpr uint32_t STAGE_BYTES = (uint32_t)STAGE_UNITS * 2;
    /* a warp's staging area: at most 3 bytes a unit, plus 1 when the warp's
     * units end inside a pair, from the 16-byte phase (0..15) of its address */
    static constexpr uint32_t WARP_OUT = (uint32_t)((3 * 32 * UPT + 1 + 15 + 15) / 16 * 16);
    static constexpr uint32_t OUT_WORDS = (uint32_t)(THREADS / 32) * WARP_OUT / 4;
    static constexpr size_t SMEM = (size_t)STAGES * STAGE_BYTES + (size_t)OUT_WORDS * 4;
    static_assert(STAGE_BYTES % 16 == 0 && WARP_OUT % 16 == 0, "16-byte granules");
};

/*
 * Persistent transcoder, software-pipelined over tiles.  Each iteration of a
 * CTA's loop does, for the tile n whose input just arrived and the tile c
 * before it:
 *   phase A(n): bytes per unit, validation, block scan; publish n's aggregate
 *               (and its first error);
 *   phase B(c): c's bytes into the staging buffer at tile-local offsets;
 *               c's exclusive output offset by decoupled look-back (its
 *               status words are requested at the top of the iteration and
 *               examined after the bytes are written); the next tile's
 *               input copy starts into c's stage, now read; publish c's
 *               inclusive prefix; write the tile out with aligned 16-byte
 *               stores.
 * The ticket for that next tile is taken when its copy starts, so a tile's
 * aggregate goes out about half an iteration after its ticket, and its
 * look-back runs about one iteration after that.  A look-back waits only
 * for the aggregates of smaller tickets, and a CTA's pending look-back is
 * always for a ticket smaller than any it holds unpublished, so the CTA
 * holding the smallest unpublished ticket never waits: every wait ends.
 *
 * Input tiles (plus 8 units of halo on each side) arrive in a two-stage
 * shared-memory ring by 1-D TMA bulk copies completing on per-stage
 * mbarriers.  Tiles at the ends of the buffer (halo outside the input) are
 * filled by the threads with guarded loads instead.
 */
template <int THREADS, int UPT, int STAGES, bool VALIDATE, bool BE, bool CHAINED>
/* CHAINED (the host forms' chunks) is a separate instance, held to 5 CTAs
 * per SM: as a runtime flag, its output base cost the single calls 16
 * registers and a CTA per SM */
__global__ void __launch_bounds__(THREADS, CHAINED ? 5 : 0)
utf16_to_utf8_kernel(const uint16_t *__restrict__ in, uint64_t n, uint8_t *__restrict__ out,
                     uint64_t cap, WsHeader *hdr, unsigned long long *status,
                     uint64_t status_words, uint64_t tiles, DevResult *res)
{
    using Lay = U16Layout<THREADS, UPT, STAGES>;
    constexpr uint64_t TILE = Lay::TILE;
    constexpr int WARPS = THREADS / 32;
    constexpr int WORDS = UPT / 2;
    constexpr int NL = UPT / 4;   /* words of per-unit byte counts, one byte a unit */
    static_assert(UPT % 8 == 0 && UPT <= 32, "units per thread: a multiple of 8, at most 32");
    static_assert(STAGES == 2, "tile in phase A, tile in phase B (whose stage is refilled mid-iteration)");
    extern __shared__ uint4 smem4[];
    uint16_t *stages = reinterpret_cast<uint16_t *>(smem4);
    uint4 *outw4 = smem4 + (size_t)STAGES * Lay::STAGE_BYTES / 16;
    uint8_t *outb = reinterpret_cast<uint8_t *>(outw4);
    __shared__ unsigned long long s_bar[STAGES];
    __shared__ unsigned long long s_ring[STAGES];
    __shared__ uint32_t s_warp[WARPS + 2];
    __shared__ unsigned long long s_min[WARPS];
    __shared__ unsigned long long s_lb_g0;
    __shared__ unsigned s_flag;

    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const uint64_t head = ((uintptr_t)in & 15) / 2;
    const uint16_t *base = in - head;
    const uint64_t endx = head + n;
    const unsigned epoch = *(volatile unsigned *)&hdr->epoch;
    /* a host form's chunks run chained: each writes its output after the
     * units of the chunks before it, which the header holds (the previous
     * chunk's last CTA moved it on) */
    if constexpr (CHAINED) {
        const uint64_t obase = ld_relaxed(&hdr->out_base);
        out += obase;
        cap = cap > obase ? cap - obase : 0;
    }

    /* thread 0: put tile t in flight into stage s */
    auto issue = [&](unsigned long long t, int s) {
        s_ring[s] = t;
        if (t >= tiles) return;
        const uint64_t x0 = t * TILE;
        if (x0 >= head + HALO16 && x0 + TILE + HALO16 <= endx) {
            fence_proxy_async();
            mbar_arrive_expect_tx(&s_bar[s], Lay::STAGE_BYTES);
            bulk_load(stages + (size_t)s * Lay::STAGE_UNITS, base + x0 - HALO16, Lay::STAGE_BYTES, &s_bar[s]);
        } else {
            mbar_arrive(&s_bar[s]);
        }
    };

    if (tid == 0) {
        for (int s = 0; s < STAGES; s++) mbar_init(&s_bar[s], 1);
        fence_mbar_init();
        issue(atomicAdd(&hdr->ticket, 1ull), 0);
        issue(atomicAdd(&hdr->ticket, 1ull), 1);
    }
    __syncthreads();

    /* state of tile c (phase A done, phase B pending) */
    bool have_c = false;
    unsigned long long c_tile = 0;
    uint32_t c_total = 0, c_end = 0, c_len[NL];   /* c_end: end of the thread's bytes, from the tile's first byte */
#pragma unroll
    for (int j = 0; j < NL; j++) c_len[j] = 0;
    int c_stage = 0;
    bool c_whole = false;   /* every unit of tile c lies inside the input */

#define UNIT(k) ((w[(k) / 2] >> (16 * ((k) & 1))) & 0xFFFFu)
    for (int it = 0;; it++) {
        /* the look-back window of tile c (the tiles before it) is requested
         * first: its words arrive while phase A of tile n and the encoding
         * of tile c run, and are examined after them */
        const long long lb_idx = (long long)c_tile - 1 - tid;   /* warp 0's lanes */
        const uint64_t lb_word = (tid < 32 && have_c && c_tile > 0 && lb_idx >= 0) ? ld_relaxed(status + lb_idx) : 0;
        /* ---------------- phase A of tile n ---------------- */
        const int sn = it % STAGES;
        const unsigned long long t = s_ring[sn];
        const bool have_n = t < tiles;
        uint32_t n_total = 0, n_end = 0, n_len[NL];
#pragma unroll
        for (int j = 0; j < NL; j++) n_len[j] = 0;
        if (have_n) {
            const uint64_t x0 = t * TILE;
            uint16_t *sb = stages + (size_t)sn * Lay::STAGE_UNITS;
            const bool interior = x0 >= head + HALO16 && x0 + TILE + HALO16 <= endx;
            if (interior) {
                if (!mbar_wait(&s_bar[sn], (uint32_t)((it / STAGES) & 1))) atomicOr(&hdr->flags, FLAG_TIMEOUT);
            } else {
                for (int i = tid; i < Lay::STAGE_UNITS; i += THREADS)
                    sb[i] = (uint16_t)unit_at(base, (long long)(x0 + i) - HALO16, head, endx);
                __syncthreads();
            }
            const int i0 = HALO16 + tid * UPT;
            uint32_t w[WORDS];
#pragma unroll
            for (int v = 0; v < WORDS / 4; v++) {
                const uint4 q = *reinterpret_cast<const uint4 *>(sb + i0 + 8 * v);
                w[4 * v + 0] = units_of<BE>(q.x);
                w[4 * v + 1] = units_of<BE>(q.y);
                w[4 * v + 2] = units_of<BE>(q.z);
                w[4 * v + 3] = units_of<BE>(q.w);
            }
            const uint32_t pu = unit_of<BE>(sb[i0 - 1]), nu = unit_of<BE>(sb[i0 + UPT]);
            const long long e0 = (long long)(x0 + (uint64_t)tid * UPT);
            /* bytes per unit (utf16_scheme.h: Table 2, with a surrogate pair
             * written whole by its high unit, so no tile needs more than 3
             * bytes a unit, plus one for a pair cut by the tile's end), four
             * units per step; Section 3's pairing rule checked on the way */
            uint32_t lens = 0, bad = 0;
            uint32_t hprev = is_high(pu) ? 0x80000000u : 0u;
            uint32_t p_c3 = 0, p_hi = 0, p_lo = 0, p_N = 0, p_A = 0;   /* the group before */
#pragma unroll
            for (int g = 0; g <= NL; g++) {
                uint32_t c3 = 0, hi = 0, lo = is_low(nu) ? 0x80u : 0u, N = 0, A = 0;
                if (g < NL) gputf_u16_classify(w[2 * g], w[2 * g + 1], &hprev, &bad, &c3, &hi, &lo, &N, &A);
                if (g > 0) {   /* finish group g-1 */
                    const uint32_t L = gputf_u16_counts(p_c3, p_hi, p_lo, p_N, p_A, lo);
                    n_len[g - 1] = L;
                    lens += L;
                }
                p_c3 = c3;
                p_hi = hi;
                p_lo = lo;
                p_N = N;
                p_A = A;
            }
            if (VALIDATE) bad |= gputf_u16_end_mismatch(hprev, nu);
            else bad = 0;
            n_total = byte_sum(lens);
            uint32_t inr = 0xFFFFFFFFu;
            if (!interior) {   /* units outside the input write nothing */
                inr = 0;
#pragma unroll
                for (int k = 0; k < UPT; k++)
                    inr |= (e0 + k >= (long long)head && e0 + k < (long long)endx) ? (1u << k) : 0u;
                n_total = 0;
#pragma unroll
                for (int j = 0; j < NL; j++) {
                    n_len[j] &= byte_mask4(inr >> (4 * j));
                    n_total += byte_sum(n_len[j]);
                }
            }
            uint64_t first_err = NONE;
            if (VALIDATE && bad) {   /* some pair breaks the rule: find the first invalid unit of the chunk */
                uint32_t prev = pu;
#pragma unroll
                for (int k = 0; k < UPT; k++) {
                    const uint32_t u = UNIT(k);
                    const uint32_t nx = k + 1 < UPT ? UNIT(k + 1) : nu;
                    const bool e = (is_high(u) && !is_low(nx)) || (is_low(u) && !is_high(prev));
                    if (e && ((inr >> k) & 1) && first_err == NONE) first_err = (uint64_t)(e0 + k) - head;
                    prev = u;
                }
            }
            bool any_err;
            n_end = n_total + block_exclusive_or<THREADS>(n_total, first_err != NONE, s_warp, &n_total, &any_err);
            if (tid == 0)
                st_release(status + t, make_status(epoch, t == 0 ? ST_PREFIX : ST_AGGREGATE, n_total));
            if (any_err) {
                const uint64_t m = block_min<THREADS>(first_err, s_min);
                if (tid == 0) atomicMin(&hdr->err_pos, (unsigned long long)m);
            }
        }

        /* ---------------- look-back and phase B of tile c ---------------- */
        if (have_c) {
            const uint16_t *sb = stages + (size_t)c_stage * Lay::STAGE_UNITS;
            const int i0 = HALO16 + tid * UPT;

            uint32_t w[WORDS];
#pragma unroll
            for (int v = 0; v < WORDS / 4; v++) {
                const uint4 q = *reinterpret_cast<const uint4 *>(sb + i0 + 8 * v);
                w[4 * v + 0] = units_of<BE>(q.x);
                w[4 * v + 1] = units_of<BE>(q.y);
                w[4 * v + 2] = units_of<BE>(q.z);
                w[4 * v + 3] = units_of<BE>(q.w);
            }
            const uint32_t nu = unit_of<BE>(sb[i0 + UPT]);
            /* c's exclusive output offset, by warp 0 alone: its window (the
             * 32 tiles before c, requested at the top of the iteration, so
             * its words have arrived while phase A of n ran) is usable when an
             * inclusive prefix appears in it and every entry before that one
             * has been published; otherwise the warp walks back, waiting
             * (bounded) for each word.  The barrier then hands G0 to every
             * thread (all of them have read c's stage by then). */
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
            __syncthreads();
            const uint64_t G0 = c_tile > 0 ? s_lb_g0 : 0;
            /* every thread has read c's stage: a new ticket's tile goes in
             * flight into it (a ticket taken this late keeps the tiles in
             * flight close together, so look-backs seldom wait) */
            if (tid == 0 && have_n) issue(atomicAdd(&hdr->ticket, 1ull), c_stage);

            /* this warp's part of the tile's output, bytes [ws, we) from the
             * tile's first byte, is staged in the warp's own area at the
             * 16-byte phase of its global address, so that it leaves as whole
             * 16-byte vectors copied as they are (plus at most 15 bytes at
             * each end), without waiting for the other warps */
            uint32_t own = 0;
#pragma unroll
            for (int j = 0; j < NL; j++) own += byte_sum(c_len[j]);
            const uint32_t ws = __shfl_sync(FULL_MASK, c_end - own, 0), we = __shfl_sync(FULL_MASK, c_end, 31);
            const uint32_t a = (uint32_t)(((uintptr_t)out + G0 + ws) & 15);
            uint8_t *wb = outb + (size_t)wid * Lay::WARP_OUT;
            const uint32_t cpos = a + (c_end - ws);   /* end of this thread's bytes in the warp's area */
            /* each unit's bytes, in this warp's staging area.
             * Uniform-class fast paths: when every unit of every thread of
             * the warp takes 3 bytes (BMP from U+0800, no surrogate), or 1,
             * or 2, the bytes go to fixed offsets with no per-unit length
             * work (the same bytes the general path writes). */
            uint32_t len_and = c_len[0], len_or = c_len[0];
#pragma unroll
            for (int j = 1; j < NL; j++) {
                len_and &= c_len[j];
                len_or |= c_len[j];
            }
            if (__all_sync(FULL_MASK, len_and == 0x03030303u && len_or == 0x03030303u)) {
                uint8_t *dst = wb + cpos - 3 * UPT;
#pragma unroll
                for (int k = 0; k < UPT; k++) {
                    const uint32_t u = UNIT(k);
                    dst[3 * k] = (uint8_t)(0xE0 | (u >> 12));
                    dst[3 * k + 1] = (uint8_t)(0x80 | ((u >> 6) & 0x3F));
                    dst[3 * k + 2] = (uint8_t)(0x80 | (u & 0x3F));
                }
            } else if (__all_sync(FULL_MASK, len_and == 0x01010101u && len_or == 0x01010101u)) {
                uint8_t *dst = wb + cpos - UPT;
#pragma unroll
                for (int k = 0; k < UPT; k++) dst[k] = (uint8_t)UNIT(k);
            } else if (__all_sync(FULL_MASK, len_and == 0x02020202u && len_or == 0x02020202u)) {
                uint8_t *dst = wb + cpos - 2 * UPT;
#pragma unroll
                for (int k = 0; k < UPT; k++) {
                    const uint32_t u = UNIT(k);
                    dst[2 * k] = (uint8_t)(0xC0 | (u >> 6));
                    dst[2 * k + 1] = (uint8_t)(0x80 | (u & 0x3F));
                }
            } else if (c_whole) {
                /* every unit of the tile is inside the input: units 3.. go
                 * back to front with unconditional stores, then units 2, 1, 0
                 * exactly.  The strays stay inside the thread's run because
                 * units 0-3 take at least 3 bytes: only the low half of a
                 * pair takes none, and if that is unit 1, 2 or 3, its high
                 * half is unit 0, 1 or 2 and takes 4. */
                uint32_t e = smem_u32(wb) + cpos;
#pragma unroll
                for (int k = UPT - 1; k >= 3; k--)
                    e = put_utf8_back(e, UNIT(k), k + 1 < UPT ? UNIT(k + 1) : nu,
                                      byte_at(c_len[k / 4], k % 4));
#pragma unroll
                for (int k = 2; k >= 0; k--) {
                    const uint32_t l = byte_at(c_len[k / 4], k % 4);
                    e -= l;
                    put_utf8(e, UNIT(k), UNIT(k + 1), l);
                }
            } else {
                uint32_t e = smem_u32(wb) + cpos;
#pragma unroll
                for (int k = UPT - 1; k >= 0; k--) {
                    const uint32_t l = byte_at(c_len[k / 4], k % 4);
                    e -= l;
                    put_utf8(e, UNIT(k), k + 1 < UPT ? UNIT(k + 1) : nu, l);
                }
            }

            __syncwarp();
            {   /* write-out of [G0 + ws, G0 + we), clipped to the capacity */
                const uint64_t g = G0 + ws;
                const uint64_t cnt = g >= cap ? 0 : (g + (we - ws) > cap ? cap - g : (uint64_t)(we - ws));
                uint8_t *gbase = out + g - a;   /* 16-byte aligned; global byte j <-> staged byte j */
                const uint32_t lim = a + (uint32_t)cnt;
                const uint32_t vf = a ? 1u : 0u, vl = lim >> 4;   /* the whole vectors: [vf, vl) */
                for (uint32_t i = vf + lane; i < vl; i += 32)
                    st_stream16(gbase + 16 * i, *reinterpret_cast<const uint4 *>(wb + 16 * i));
                const uint32_t head_end = a ? (16 < lim ? 16u : lim) : 0u;          /* bytes [a, head_end) */
                const uint32_t tail_start = 16 * vl > head_end ? 16 * vl : head_end;   /* bytes [tail_start, lim) */
                if (lane < 16) {
                    const uint32_t b = a + (uint32_t)lane;
                    if (b < head_end) gbase[b] = wb[b];
                } else {
                    const uint32_t b = tail_start + (uint32_t)(lane - 16);
                    if (b < lim) gbase[b] = wb[b];
                }
            }

            /* the first character whose bytes do not fit (only in the tile
             * that crosses the capacity): a unit that writes bytes starts a
             * character, and a pair needs all four */
            if (G0 <= cap && G0 + c_total > cap) {
                const long long e0 = (long long)(c_tile * TILE + (uint64_t)tid * UPT);
                uint64_t cap_first = NONE;
                uint64_t g = G0 + c_end - own;
#pragma unroll
                for (int k = 0; k < UPT; k++) {
                    const uint32_t l = byte_at(c_len[k / 4], k % 4);
                    if (l && g + l > cap && cap_first == NONE) cap_first = (uint64_t)(e0 + k) - head;
                    g += l;
                }
                const uint64_t m = block_min<THREADS>(cap_first, s_min);
                if (tid == 0 && m != NONE) atomicMin(&hdr->cap_pos, (unsigned long long)m);
            }
            /* this barrier also orders thread 0's ring entry for the tile
             * now in flight (written by issue() above) before every thread
             * reads it at the top of the next iteration */
            __syncthreads();
        }

        /* tile n becomes c */
        if (!have_n) break;
        have_c = true;
        c_tile = t;
        c_total = n_total;
        c_end = n_end;
        c_whole = t * TILE >= head && t * TILE + TILE <= endx;
#pragma unroll
        for (int j = 0; j < NL; j++) c_len[j] = n_len[j];
        c_stage = sn;
    }
#undef UNIT

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
    } else if (cpos != NONE && (f == NONE || cpos < f)) {
        error = GPUTF_E_OUTPUT_TOO_SMALL;
        pos = cpos;
    } else if (f != NONE) {
        error = GPUTF_E_SURROGATE;
        pos = f;
    }
    uint64_t written = 0;
    if (error == GPUTF_E_OK) {
        written = ld_relaxed(status + tiles - 1) & VALUE_MASK;
    } else if (error != GPUTF_E_TIMEOUT) {
        /* bytes of [0, pos): the tiles before pos's tile, then a recount
         * with the kernel's per-unit convention (a pair's 4 bytes on its high
         * unit, 2 for a lone surrogate, which only the non-validating call
         * can meet before pos) */
        const uint64_t t = (head + pos) / TILE;
        const uint64_t before = t ? (ld_relaxed(status + t - 1) & VALUE_MASK) : 0;
        const uint64_t start = t * TILE > head ? t * TILE - head : 0;
        uint32_t c = 0;
        for (uint64_t i = start + tid; i < pos; i += THREADS) {
            const uint32_t u = unit_of<BE>(in[i]);
            if (is_high(u)) c += (i + 1 < n && is_low(unit_of<BE>(in[i + 1]))) ? 4u : 2u;
            else if (is_low(u)) c += (i > 0 && is_high(unit_of<BE>(in[i - 1]))) ? 0u : 2u;
            else c += len8(u);
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
 * Validate-only and length-only passes.
 *
 * Streaming kernels: a grid of resident CTAs walks the tiles (grid-stride);
 * each thread holds its chunk of the current tile in registers and issues the
 * loads of its chunk of the next tile before working on the current one, so
 * that a tile's memory latency hides behind the previous tile's arithmetic.
 * No barrier is taken per tile.
 * ---------------------------------------------------------------------- */

/* Section 3's surrogate rule over a chunk: a high surrogate must be followed
 * by a low one and a low one must follow a high one, i.e. for every two
 * adjacent units, "the first is high" equals "the second is low".  Returns a
 * nonzero word when some pair in the chunk (including the unit before it,
 * pu, and the one after it, nu) breaks the rule. */
template <int WORDS>
__device__ __forceinline__ uint32_t surrogate_mismatch(const uint32_t (&w)[WORDS], uint32_t pu, uint32_t nu)
{
    static_assert(WORDS % 2 == 0, "four units per step");
    uint32_t bad = 0;
    uint32_t hprev = is_high(pu) ? 0x80000000u : 0u;   /* byte 3: the unit before the group is high */
#pragma unroll
    for (int g = 0; g < WORDS / 2; g++) bad |= gputf_u16_mismatch4(w[2 * g], w[2 * g + 1], &hprev);
    return bad | gputf_u16_end_mismatch(hprev, nu);
}

template <int THREADS, int WORDS, bool BE>
__global__ void __launch_bounds__(THREADS)
validate_utf16_kernel(const uint16_t *__restrict__ in, uint64_t n, uint64_t tiles, WsHeader *hdr,
                      DevResult *res)
{
    constexpr int UPT = 2 * WORDS;
    constexpr uint64_t TILE = (uint64_t)THREADS * UPT;
    __shared__ unsigned long long s_min[THREADS / 32];
    __shared__ unsigned s_flag;
    const int tid = threadIdx.x, lane = tid & 31;
    const uint64_t head = ((uintptr_t)in & 15) / 2;
    const uint16_t *base = in - head;
    const uint64_t endx = head + n;
    uint64_t first_err = NONE;
    uint64_t tile = blockIdx.x;
    uint32_t w[WORDS];
    /* lanes 0 and 31 also need the unit before / after their warp's span
     * (another warp's): loaded with the chunk, one tile ahead like the rest */
    uint32_t side = 0;
    auto side_unit = [&](uint64_t e0) -> uint32_t {
        if (lane == 0) return unit_at(base, (long long)e0 - 1, head, endx);
        if (lane == 31) return unit_at(base, (long long)(e0 + UPT), head, endx);
        return 0u;
    };
    if (tile < tiles) {
        load_chunk16<WORDS>(base, tile * TILE + (uint64_t)tid * UPT, head, endx, w);
        side = side_unit(tile * TILE + (uint64_t)tid * UPT);
    }
    while (tile < tiles) {
        const uint64_t e0 = tile * TILE + (uint64_t)tid * UPT;
        const uint64_t next = tile + gridDim.x;
        uint32_t v[WORDS], v_side = 0;
        if (next < tiles) {
            load_chunk16<WORDS>(base, next * TILE + (uint64_t)tid * UPT, head, endx, v);
            v_side = side_unit(next * TILE + (uint64_t)tid * UPT);
        }
#pragma unroll
        for (int k = 0; k < WORDS; k++) w[k] = units_of<BE>(w[k]);
        uint32_t pu = __shfl_up_sync(FULL_MASK, w[WORDS - 1] >> 16, 1);
        uint32_t nu = __shfl_down_sync(FULL_MASK, w[0] & 0xFFFF, 1);
        if (lane == 0) pu = unit_of<BE>(side);
        if (lane == 31) nu = unit_of<BE>(side);
        /* units outside the input read as zero, which is no surrogate, so a
         * broken pair always has an input unit to blame */
        if (surrogate_mismatch<WORDS>(w, pu, nu) && first_err == NONE) {
            uint32_t prev = pu;
#pragma unroll
            for (int k = 0; k < UPT; k++) {
                const uint32_t u = (w[k / 2] >> (16 * (k & 1))) & 0xFFFF;
                const uint32_t nx = k + 1 < UPT ? (w[(k + 1) / 2] >> (16 * ((k + 1) & 1))) & 0xFFFF : nu;
                const bool bad = (is_high(u) && !is_low(nx)) || (is_low(u) && !is_high(prev));
                const long long ex = (long long)(e0 + k);
                if (bad && ex >= (long long)head && ex < (long long)endx && first_err == NONE)
                    first_err = e0 + k - head;
                prev = u;
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
        res->error = f == NONE ? GPUTF_E_OK : GPUTF_E_SURROGATE;
        res->reserved = 0;
        res->position = f == NONE ? n : f;
        res->written = 0;
    }
    reset_workspace(hdr, nullptr, 0);
}

/* UTF-8 length (Table 2): n + #(u >= 0x80) + #(u >= 0x800 and not a
 * surrogate), the counts taken four units at a time on their gathered high
 * and low bytes.  A unit outside the input reads as zero and adds nothing. */
template <int THREADS, int WORDS, bool BE>
__global__ void __launch_bounds__(THREADS)
utf8_length_from_utf16_kernel(const uint16_t *__restrict__ in, uint64_t n, uint64_t tiles,
                              WsHeader *hdr, unsigned long long *len_out)
{
    constexpr int UPT = 2 * WORDS;
    constexpr uint64_t TILE = (uint64_t)THREADS * UPT;
    __shared__ unsigned long long s_part[THREADS / 32];
    __shared__ unsigned s_flag;
    const int tid = threadIdx.x;
    const uint64_t head = ((uintptr_t)in & 15) / 2;
    const uint16_t *base = in - head;
    const uint64_t endx = head + n;
    uint64_t acc = 0;
    uint64_t tile = blockIdx.x;
    uint32_t w[WORDS];
    if (tile < tiles) load_chunk16<WORDS>(base, tile * TILE + (uint64_t)tid * UPT, head, endx, w);
    while (tile < tiles) {
        const uint64_t next = tile + gridDim.x;
        uint32_t v[WORDS];
        if (next < tiles) load_chunk16<WORDS>(base, next * TILE + (uint64_t)tid * UPT, head, endx, v);
        uint32_t up = 0;   /* per-byte counts of the extra bytes, at most 2 per group */
#pragma unroll
        for (int g = 0; g < WORDS / 2; g++)
            up += gputf_u16_utf8_extra4(units_of<BE>(w[2 * g]), units_of<BE>(w[2 * g + 1]));
        acc += byte_sum(up);
#pragma unroll
        for (int k = 0; k < WORDS; k++) w[k] = v[k];
        tile = next;
    }
    const uint64_t sum = block_sum<THREADS>(acc, s_part);
    if (tid == 0) atomicAdd(&hdr->accum, (unsigned long long)sum);
    if (!finish_cta(hdr, &s_flag)) return;
    if (tid == 0) *len_out = ld_relaxed(&hdr->accum) + n;
    reset_workspace(hdr, nullptr, 0);
}

/* ------------------------------------------------------------------------
 * Launchers.
 * ---------------------------------------------------------------------- */
constexpr int U16_THREADS = 256;
constexpr int U16_UPT = 24;     /* 6144-unit tiles */
constexpr int U16_STAGES = 2;
using U16Lay = U16Layout<U16_THREADS, U16_UPT, U16_STAGES>;

uint64_t utf16_to_utf8_tiles(const void *in, uint64_t n)
{
    return (((uintptr_t)in % 16) / 2 + n + U16Lay::TILE) / U16Lay::TILE;   /* at least one tile */
}

template <bool VALIDATE, bool BE, bool CHAINED>
static cudaError_t launch16(const uint16_t *in, uint64_t n, uint8_t *out, uint64_t cap, void *ws,
                            uint64_t status_words, DevResult *res, int sms, cudaStream_t stream)
{
    auto kern = utf16_to_utf8_kernel<U16_THREADS, U16_UPT, U16_STAGES, VALIDATE, BE, CHAINED>;
    static int per_sm = 0;     /* resident CTAs per SM (same for every sm_103 device) */
    if (per_sm == 0) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)U16Lay::SMEM);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, U16_THREADS, U16Lay::SMEM);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) per_sm = 1;
    }
    const uint64_t tiles = utf16_to_utf8_tiles(in, n);
    const uint64_t grid = tiles < (uint64_t)sms * per_sm ? tiles : (uint64_t)sms * per_sm;
    WsHeader *hdr = static_cast<WsHeader *>(ws);
    auto *status = reinterpret_cast<unsigned long long *>(static_cast<char *>(ws) + HEADER_BYTES);
    kern<<<(unsigned)grid, U16_THREADS, U16Lay::SMEM, stream>>>(in, n, out, cap, hdr, status,
                                                                 status_words, tiles, res);
    return cudaGetLastError();
}

cudaError_t launch_utf16_to_utf8(const uint16_t *in, uint64_t n, uint8_t *out, uint64_t cap,
                                 void *ws, uint64_t status_words, DevResult *res, int sms, bool validate,
                                 bool big_endian, bool chained, cudaStream_t stream)
{
    if (chained) {   /* the host forms' chunks: validating, little-endian */
        if (!validate || big_endian) return cudaErrorInvalidValue;
        return launch16<true, false, true>(in, n, out, cap, ws, status_words, res, sms, stream);
    }
    if (big_endian)
        return validate ? launch16<true, true, false>(in, n, out, cap, ws, status_words, res, sms, stream)
                        : launch16<false, true, false>(in, n, out, cap, ws, status_words, res, sms, stream);
    return validate ? launch16<true, false, false>(in, n, out, cap, ws, status_words, res, sms, stream)
                    : launch16<false, false, false>(in, n, out, cap, ws, status_words, res, sms, stream);
}

/* Grid of a streaming pass: the CTAs that fit on the device at once (no
 * more than there are tiles). */
template <typename K>
static unsigned resident_grid(K kern, int threads, uint64_t tiles, int sms, int *per_sm)
{
    if (*per_sm == 0) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, threads, 0) != cudaSuccess || b < 1) b = 1;
        *per_sm = b;
    }
    const uint64_t g = (uint64_t)sms * *per_sm;
    return (unsigned)(tiles < g ? (tiles ? tiles : 1) : g);
}

cudaError_t launch_validate_utf16(const uint16_t *in, uint64_t n, void *ws, DevResult *res,
                                  int sms, bool big_endian, cudaStream_t stream)
{
    constexpr int T = 256, W = 8;
    constexpr uint64_t TILE = (uint64_t)T * 2 * W;
    const uint64_t tiles = (((uintptr_t)in % 16) / 2 + n + TILE - 1) / TILE;
    static int per_sm[2] = {0, 0};
    if (big_endian) {
        auto kern = validate_utf16_kernel<T, W, true>;
        kern<<<resident_grid(kern, T, tiles, sms, &per_sm[1]), T, 0, stream>>>(in, n, tiles,
                                                                               static_cast<WsHeader *>(ws), res);
    } else {
        auto kern = validate_utf16_kernel<T, W, false>;
        kern<<<resident_grid(kern, T, tiles, sms, &per_sm[0]), T, 0, stream>>>(in, n, tiles,
                                                                               static_cast<WsHeader *>(ws), res);
    }
    return cudaGetLastError();
}

cudaError_t launch_utf8_length_from_utf16(const uint16_t *in, uint64_t n, void *ws,
                                          unsigned long long *len, int sms, bool big_endian,
                                          cudaStream_t stream)
{
    constexpr int T = 256, W = 8;
    constexpr uint64_t TILE = (uint64_t)T * 2 * W;
    const uint64_t tiles = (((uintptr_t)in % 16) / 2 + n + TILE - 1) / TILE;
    static int per_sm[2] = {0, 0};
    if (big_endian) {
        auto kern = utf8_length_from_utf16_kernel<T, W, true>;
        kern<<<resident_grid(kern, T, tiles, sms, &per_sm[1]), T, 0, stream>>>(in, n, tiles,
                                                                               static_cast<WsHeader *>(ws), len);
    } else {
        auto kern = utf8_length_from_utf16_kernel<T, W, false>;
        kern<<<resident_grid(kern, T, tiles, sms, &per_sm[0]), T, 0, stream>>>(in, n, tiles,
                                                                               static_cast<WsHeader *>(ws), len);
    }
    return cudaGetLastError();
}

}  // namespace gputf
