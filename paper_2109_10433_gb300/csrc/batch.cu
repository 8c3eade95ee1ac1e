/*
 * Batched transcoding: many strings of uneven lengths, given as CSR offsets,
 * in one launch whose tiles cross string boundaries.
 *
 * For each direction, the strings are the consecutive pieces of one input
 * buffer, in_offsets[s] .. in_offsets[s + 1], and string s writes its output
 * into out[out_offsets[s] .. out_offsets[s + 1]) (its capacity) and its
 * result into results[s].  Tiles of that buffer are taken in ticket order by
 * one grid that serves both directions (UTF-8 tiles first).
 *
 * Output offsets inside each string come from a segmented scan: per tile,
 * the block scans (starts-a-string, sum) pairs, and the tile's carry into
 * the string it begins inside comes from a segmented decoupled look-back
 * (a walk back that stops at an inclusive prefix or at a tile in which a
 * string starts).  Validation follows the strings' edges: a string's first
 * units do not see the units before it, and a UTF-8 character cut short by
 * the string's end is flagged at the end.  The tile that holds a string's
 * last unit writes its result; errors and overflowing capacities are then
 * finished by that thread with the scalar steps of the single-buffer path.
 */
#include <cstdint>

#include "common.cuh"
#include "batch_piece.h"
#include "kernels.h"

namespace gputf {

/* Segmented status word: epoch (21) | starts-a-string (1) | flag (2) | value (40). */
constexpr unsigned SEG_EPOCH_BITS = 21;
constexpr unsigned SEG_EPOCH_MASK = (1u << SEG_EPOCH_BITS) - 1;

__device__ __forceinline__ uint64_t seg_status(unsigned epoch, uint64_t flag, bool start, uint64_t value)
{
    return ((uint64_t)(epoch & SEG_EPOCH_MASK) << 43) | ((uint64_t)start << 42) | (flag << 40) |
           (value & VALUE_MASK);
}

/* Per-string error words: (epoch << 43) | (VALUE_MASK - position), combined
 * with atomicMax, so the smallest position of the current call wins and
 * words from earlier calls (smaller epochs) never read as current. */
__device__ __forceinline__ void record_string_error(unsigned long long *errw, uint64_t s, unsigned epoch,
                                                    uint64_t pos)
{
    atomicMax(errw + s, ((unsigned long long)epoch << 43) | (VALUE_MASK - pos));
}

__device__ __forceinline__ uint64_t string_error(const unsigned long long *errw, uint64_t s, unsigned epoch)
{
    const uint64_t w = ld_relaxed(errw + s);
    return (unsigned)(w >> 43) == epoch ? VALUE_MASK - (w & VALUE_MASK) : NONE;
}

constexpr int BATCH_OFF_CACHE = 512;   /* string offsets cached per tile */

struct BatchShared {
    unsigned long long off[BATCH_OFF_CACHE];
    unsigned long long s_first;
    unsigned n_cached;
    uint32_t warp_f[33];
    unsigned long long warp_v[33];
    unsigned long long lb_sum[32];
    unsigned long long carry;
};

/* in_off[s], from the tile's cache when it holds it. */
__device__ __forceinline__ uint64_t off_at(const BatchDir &d, const BatchShared &sm, uint64_t s)
{
    const uint64_t j = s - sm.s_first;
    return j < sm.n_cached ? sm.off[j] : d.in_off[s];
}

/* Output units of a string before absolute position x (st <= x <= en):
 * the published status words of the string's whole tiles before x's tile,
 * walked back like the look-back (to a PREFIX word or the string's first
 * tile), plus len(j) summed over the units of x's own tile before x.  The
 * words are all published by the time the string's last tile runs its
 * phase B.  Cost: the string's tile count plus one tile, not its length.
 * Returns false if a word is not published (a broken invariant). */
template <uint64_t TILE, typename LenFn>
__device__ bool string_prefix(const BatchDir &d, unsigned epoch, uint64_t st, uint64_t x, LenFn len,
                              uint64_t *out)
{
    const uint64_t xs = x / TILE * TILE;
    uint64_t sum = 0;
    for (uint64_t j = st > xs ? st : xs; j < x; j++) sum += len(j);
    if (st < xs) {
        for (long long k = (long long)(x / TILE) - 1; k >= 0; k--) {
            const uint64_t w = ld_acquire(d.status + k);
            const uint64_t fl = (w >> 40) & 3;
            if ((unsigned)(w >> 43) != (epoch & SEG_EPOCH_MASK) || fl == 0) return false;
            sum += w & VALUE_MASK;
            if (fl == ST_PREFIX || ((w >> 42) & 1)) break;
        }
    }
    *out = sum;
    return true;
}

/* The first unit q of a string with len(q) > 0 whose output does not fit
 * the capacity cap (g(q) <= cap < g(q) + len(q), g = output before q), with
 * g(q): the tile holding it is found from the status words (output through
 * each tile), then that tile is scanned.  Same cost bound as above.
 * Returns false if there is no such unit or a word is not published. */
template <uint64_t TILE, typename LenFn>
__device__ bool string_crossing(const BatchDir &d, unsigned epoch, uint64_t st, uint64_t en, uint64_t cap,
                                LenFn len, uint64_t *q, uint64_t *gq)
{
    const uint64_t t0 = st / TILE, t1 = (en - 1) / TILE;
    uint64_t before = 0, k = t0;
    for (; k < t1; k++) {
        const uint64_t w = ld_acquire(d.status + k);
        const uint64_t fl = (w >> 40) & 3;
        if ((unsigned)(w >> 43) != (epoch & SEG_EPOCH_MASK) || fl == 0) return false;
        const uint64_t v = w & VALUE_MASK;
        const uint64_t through = (fl == ST_PREFIX || k == t0) ? v : before + v;
        if (through > cap) break;
        before = through;
    }
    uint64_t g = before;
    const uint64_t a = st > k * TILE ? st : k * TILE, b = en < (k + 1) * TILE ? en : (k + 1) * TILE;
    for (uint64_t j = a; j < b; j++) {
        const uint64_t l = len(j);
        if (l && g + l > cap) {
            *q = j;
            *gq = g;
            return true;
        }
        g += l;
    }
    return false;
}

/* Warp 0: the last string s with in_off[s] <= x (the one containing unit x
 * when it is not empty), then the offsets from there to the first one at or
 * past x_end: the first BATCH_OFF_CACHE go into the cache, and every empty
 * string starting in [x, x_end) gets its result here. */
__device__ void find_strings(const BatchDir &d, BatchShared &sm, uint64_t x, uint64_t x_end)
{
    const int lane = threadIdx.x & 31;
    uint64_t lo = 0, hi = d.count;   /* answer in [lo, hi]; in_off[lo] <= x */
    while (hi - lo > 31) {
        const uint64_t step = (hi - lo + 31) / 32;
        const uint64_t probe = lo + step * lane;
        const bool le = probe <= hi && d.in_off[probe] <= x;
        const unsigned m = __ballot_sync(FULL_MASK, le);
        const uint64_t nlo = lo + step * (31 - __clz(m));
        hi = nlo + step < hi ? nlo + step : hi;
        lo = nlo;
    }
    {
        const uint64_t probe = lo + lane;
        const bool le = probe <= hi && d.in_off[probe] <= x;
        const unsigned m = __ballot_sync(FULL_MASK, le);
        lo = lo + (31 - __clz(m));
    }
    const uint64_t s_first = lo < d.count ? lo : (d.count ? d.count - 1 : 0);
    if (lane == 0) sm.s_first = s_first;
    uint64_t n = 0;
    for (;;) {
        const uint64_t s = s_first + n + lane;
        const bool have = s <= d.count;
        const uint64_t v = have ? d.in_off[s] : ~0ull;
        if (have && n + lane < BATCH_OFF_CACHE) sm.off[n + lane] = v;
        if (have && s < d.count && v >= x && v < x_end && d.in_off[s + 1] == v) {
            d.res[s].error = GPUTF_E_OK;
            d.res[s].reserved = 0;
            d.res[s].position = 0;
            d.res[s].written = 0;
        }
        const unsigned beyond = __ballot_sync(FULL_MASK, !have || v >= x_end);
        const unsigned havem = __ballot_sync(FULL_MASK, have);
        if (beyond) {
            const int fb = __ffs(beyond) - 1;
            n += fb + ((havem >> fb) & 1u);   /* keep the first offset at or past x_end */
            break;
        }
        n += 32;
    }
    if (lane == 0) sm.n_cached = (unsigned)(n < BATCH_OFF_CACHE ? n : BATCH_OFF_CACHE);
}

/* Segmented block scan: each thread gives (f = a string starts in its
 * chunk, v = sum after its last start, or its whole sum).  Returns the
 * thread's exclusive pair within the tile, and the tile's aggregate. */
template <int THREADS>
__device__ void block_seg_scan(bool f, uint64_t v, BatchShared &sm, bool *ef, uint64_t *ev, bool *tf, uint64_t *tv)
{
    constexpr int WARPS = THREADS / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    bool fi = f;
    uint64_t vi = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const bool fo = __shfl_up_sync(FULL_MASK, (int)fi, o);
        const uint64_t vo = __shfl_up_sync(FULL_MASK, vi, o);
        if (lane >= o) {
            vi = fi ? vi : vo + vi;
            fi = fi || fo;
        }
    }
    /* lane's exclusive within the warp */
    bool fx = __shfl_up_sync(FULL_MASK, (int)fi, 1);
    uint64_t vx = __shfl_up_sync(FULL_MASK, vi, 1);
    if (lane == 0) {
        fx = false;
        vx = 0;
    }
    if (lane == 31) {
        sm.warp_f[warp] = fi;
        sm.warp_v[warp] = vi;
    }
    __syncthreads();
    if (warp == 0) {
        bool wf = lane < WARPS ? sm.warp_f[lane] != 0 : false;
        uint64_t wv = lane < WARPS ? sm.warp_v[lane] : 0;
        bool pf = wf;
        uint64_t pv = wv;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const bool fo = __shfl_up_sync(FULL_MASK, (int)pf, o);
            const uint64_t vo = __shfl_up_sync(FULL_MASK, pv, o);
            if (lane >= o) {
                pv = pf ? pv : vo + pv;
                pf = pf || fo;
            }
        }
        /* exclusive per warp, and the tile's inclusive total */
        bool xf = __shfl_up_sync(FULL_MASK, (int)pf, 1);
        uint64_t xv = __shfl_up_sync(FULL_MASK, pv, 1);
        if (lane == 0) {
            xf = false;
            xv = 0;
        }
        if (lane < WARPS) {
            sm.warp_f[lane] = xf;
            sm.warp_v[lane] = xv;
        }
        if (lane == WARPS - 1) {
            sm.warp_f[32] = pf;
            sm.warp_v[32] = pv;
        }
    }
    __syncthreads();
    const bool wf = sm.warp_f[warp] != 0;
    const uint64_t wv = sm.warp_v[warp];
    /* combine the warp's exclusive with the lane's */
    *ev = fx ? vx : wv + vx;
    *ef = wf || fx;
    *tf = sm.warp_f[32] != 0;
    *tv = sm.warp_v[32];
    __syncthreads();
}

/* Segmented look-back: the sum carried into tile t from the string it
 * begins inside.  Warp 0 reads the status words of the 32 tiles before t
 * (lane L: tile t - 1 - L) and stops at the nearest tile that published an
 * inclusive prefix or holds a string start (usually the tile just before),
 * once every tile nearer than that one has published its aggregate; tiles
 * beyond the stop are not waited for.  With no stop among 32 published
 * words it moves 32 tiles back.  The polls are bounded; the other warps
 * only wait for the result.  Called by all threads; returns the value to
 * every thread. */
template <int THREADS>
__device__ uint64_t block_seg_look_back(unsigned long long *status, long long tile, unsigned epoch,
                                        unsigned *flags, BatchShared &sm)
{
    const int lane = threadIdx.x & 31;
    if (threadIdx.x < 32) {
        uint64_t carry = 0;
        long long end = tile - 1;
        int spins = 0;
        while (end >= 0) {
            const long long idx = end - lane;
            unsigned ns = 32;
            uint64_t value = 0;
            unsigned pmask;
            bool timed_out = false;
            for (;;) {
                bool ok = true, stop = true;   /* before tile 0: the start, adding nothing */
                value = 0;
                if (idx >= 0) {
                    const uint64_t w = ld_acquire(status + idx);
                    const uint64_t fl = (w >> 40) & 3;
                    ok = (unsigned)(w >> 43) == (epoch & SEG_EPOCH_MASK) && fl != 0;
                    stop = ok && (fl == ST_PREFIX || ((w >> 42) & 1));
                    value = w & VALUE_MASK;
                }
                pmask = __ballot_sync(FULL_MASK, stop);
                const unsigned umask = __ballot_sync(FULL_MASK, !ok);
                const unsigned nearer = pmask ? (pmask & (0u - pmask)) - 1u : FULL_MASK;   /* lanes before the stop */
                if ((umask & nearer) == 0) break;
                if (++spins > SPIN_LIMIT) {
                    timed_out = true;
                    break;
                }
                __nanosleep(ns);
                if (ns < 256) ns <<= 1;
            }
            if (timed_out) {
                if (lane == 0) atomicOr(flags, FLAG_TIMEOUT);
                carry = 0;
                break;
            }
            const int st = pmask ? __ffs(pmask) - 1 : 31;
            uint64_t v = (lane <= st && idx >= 0) ? value : 0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL_MASK, v, o);
            carry += v;
            if (pmask) break;
            end -= 32;
        }
        if (lane == 0) sm.lb_sum[0] = carry;
    }
    __syncthreads();
    return sm.lb_sum[0];
}

/* Position x relative to a thread's first unit c0, clamped to [-8, lim]:
 * exact wherever the per-unit loops compare it (string starts within 8
 * units before the chunk, ends up to lim). */
__device__ __forceinline__ int rel_pos(uint64_t x, uint64_t c0, int lim)
{
    const long long r = (long long)(x - c0);
    return r < -8 ? -8 : (r > lim ? lim : (int)r);
}

/* Stages input elements [x0 - halo, x0 + count - halo) of a direction (bytes
 * `esize` each; zeros outside [0, units)): whole 16-byte vectors when the
 * span lies inside the input and starts 16-byte aligned, else element by
 * element. */
template <typename T, int THREADS>
__device__ __forceinline__ void stage_fill(T *stage, const T *in, uint64_t x0, uint64_t units, int halo, int count)
{
    const int tid = threadIdx.x;
    const bool whole = x0 >= (uint64_t)halo && x0 - halo + count <= units &&
                       ((uintptr_t)(in + (x0 - halo)) & 15) == 0 && (count * sizeof(T)) % 16 == 0;
    if (whole) {
        const uint4 *src = reinterpret_cast<const uint4 *>(in + (x0 - halo));
        uint4 *dst = reinterpret_cast<uint4 *>(stage);
        const int nv = count * (int)sizeof(T) / 16;
        for (int i = tid; i < nv; i += THREADS) dst[i] = src[i];
    } else {
        for (int i = tid; i < count; i += THREADS) {
            const long long x = (long long)x0 + i - halo;
            stage[i] = (x >= 0 && (uint64_t)x < units) ? in[x] : T(0);
        }
    }
}

/* ------------------------------------------------------------------------
 * UTF-16 -> UTF-8 tiles.
 * ---------------------------------------------------------------------- */
__device__ __forceinline__ bool is_hi16(uint32_t u) { return (u & 0xFC00) == 0xD800; }
__device__ __forceinline__ bool is_lo16(uint32_t u) { return (u & 0xFC00) == 0xDC00; }
__device__ __forceinline__ uint32_t len8_of(uint32_t u)
{
    return u < 0x80 ? 1u : ((u < 0x800 || (u & 0xF800) == 0xD800) ? 2u : 3u);
}

/* Bytes unit i of a string writes (string-local neighbours prev / next,
 * 0 outside the string): a pair is written whole by its high unit. */
__device__ __forceinline__ uint32_t bytes16(uint32_t u, uint32_t prev, uint32_t next)
{
    if (is_lo16(u) && is_hi16(prev)) return 0;
    if (is_hi16(u) && is_lo16(next)) return 4;
    return len8_of(u);
}

__device__ __forceinline__ void put_bytes16(uint8_t *dst, uint32_t u, uint32_t next, uint32_t l)
{
    if (l == 1) {
        dst[0] = (uint8_t)u;
    } else if (l == 2) {
        dst[0] = (uint8_t)(0xC0 | ((u >> 6) & 0x1F));
        dst[1] = (uint8_t)(0x80 | (u & 0x3F));
    } else if (l == 3) {
        dst[0] = (uint8_t)(0xE0 | (u >> 12));
        dst[1] = (uint8_t)(0x80 | ((u >> 6) & 0x3F));
        dst[2] = (uint8_t)(0x80 | (u & 0x3F));
    } else if (l == 4) {
        const uint32_t c = (u << 10) + next - 0x35FDC00u;
        dst[0] = (uint8_t)(0xF0 | (c >> 18));
        dst[1] = (uint8_t)(0x80 | ((c >> 12) & 0x3F));
        dst[2] = (uint8_t)(0x80 | ((c >> 6) & 0x3F));
        dst[3] = (uint8_t)(0x80 | (c & 0x3F));
    }
}

/* Result of string s when it has an error or overflows its capacity, by
 * one thread of the tile holding its last unit.  The error at unit p (the
 * first unit flagged) wins unless output before it already overflows; then
 * the result is OUTPUT_TOO_SMALL at the first unit that does not fit.
 * `total` is the string's whole output.  Bounded work (string_prefix,
 * string_crossing). */
template <uint64_t TILE>
__device__ void finish_string16(const BatchDir &d, unsigned epoch, uint64_t s, uint64_t first_err, uint64_t total)
{
    const uint16_t *in = static_cast<const uint16_t *>(d.in);
    const uint64_t st = d.in_off[s], en = d.in_off[s + 1];
    const uint64_t cap = d.out ? d.out_off[s + 1] - d.out_off[s] : ~0ull;   /* no limit when validating */
    auto len = [&](uint64_t j) -> uint64_t {
        const uint32_t prev = j > st ? in[j - 1] : 0u;
        const uint32_t next = j + 1 < en ? in[j + 1] : 0u;
        return bytes16(in[j], prev, next);
    };
    int32_t error = GPUTF_E_OK;
    uint64_t pos = en - st, written = total;
    bool ok = true;
    bool crossing = first_err == NONE;
    if (first_err != NONE) {
        uint64_t gp = 0;
        ok = string_prefix<TILE>(d, epoch, st, st + first_err, len, &gp);
        if (gp <= cap) {
            error = GPUTF_E_SURROGATE;
            pos = first_err;
            written = gp;
        } else {
            crossing = true;
        }
    }
    if (ok && crossing && total > cap) {
        uint64_t q = 0, gq = 0;
        ok = string_crossing<TILE>(d, epoch, st, en, cap, len, &q, &gq);
        error = GPUTF_E_OUTPUT_TOO_SMALL;
        pos = q - st;
        written = gq;
    }
    if (!ok) {
        error = GPUTF_E_INTERNAL;
        pos = 0;
        written = 0;
    }
    d.res[s].error = error;
    d.res[s].reserved = 0;
    d.res[s].position = pos;
    d.res[s].written = d.out ? written : 0;
}

template <int THREADS, int UPT>
__device__ void batch16_tile(const BatchDir &d, uint64_t t, unsigned epoch, WsHeader *hdr, BatchShared &sm,
                             uint16_t *stage)
{
    constexpr uint64_t TILE = (uint64_t)THREADS * UPT;
    constexpr int HALO = 8;
    const uint16_t *in = static_cast<const uint16_t *>(d.in);
    uint8_t *out = static_cast<uint8_t *>(d.out);
    const int tid = threadIdx.x;
    const uint64_t x0 = t * TILE;
    const uint64_t x1 = x0 + TILE < d.units ? x0 + TILE : d.units;

    if (tid < 32) find_strings(d, sm, x0, t + 1 == d.tiles ? ~0ull : x1);
    stage_fill<uint16_t, THREADS>(stage, in, x0, d.units, HALO, (int)TILE + 2 * HALO);
    __syncthreads();

    /* this thread's units [c0, c1) and the string holding c0 */
    const uint64_t c0 = x0 + (uint64_t)tid * UPT;
    const uint64_t c1 = c0 + UPT < x1 ? c0 + UPT : (x1 > c0 ? x1 : c0);
    uint64_t s;
    {
        /* binary search among the cached offsets (the walk steps on past
         * the cache through in_off when a tile holds more strings) */
        uint64_t lo = 0, hi = sm.n_cached;
        while (hi - lo > 1) {
            const uint64_t mid = (lo + hi) / 2;
            if (sm.off[mid] <= c0) lo = mid;
            else hi = mid;
        }
        s = sm.s_first + lo;
    }
#define U16AT(x) ((uint32_t)stage[(x) - x0 + HALO])
    /* phase A, one string piece of the chunk at a time (positions j
     * relative to c0): bytes, starts, errors, from bit masks over the
     * chunk's units (batch_piece.h: Table 2's closed form corrected where a
     * pair crosses the chunk's edge; the pairing rule with nothing before a
     * string's first unit or after its last) */
    const int base = tid * UPT + HALO;   /* stage index of c0 */
    const int nloc = (int)(c1 - c0);
    bool f = false;
    uint64_t v = 0;
    if (nloc > 0) {
        uint32_t w[UPT / 2];
#pragma unroll
        for (int q = 0; q < UPT / 8; q++) {
            const uint4 x = *reinterpret_cast<const uint4 *>(stage + base + 8 * q);
            w[4 * q + 0] = x.x;
            w[4 * q + 1] = x.y;
            w[4 * q + 2] = x.z;
            w[4 * q + 3] = x.w;
        }
        uint32_t m80 = 0, m3 = 0, hi = 0, lo = 0;   /* bit k: unit c0 + k */
#pragma unroll
        for (int g4 = 0; g4 < UPT / 4; g4++) {
            uint32_t a, b, h, l;
            gputf_u16_unit_bits4(w[2 * g4], w[2 * g4 + 1], &a, &b, &h, &l);
            m80 |= a << (4 * g4);
            m3 |= b << (4 * g4);
            hi |= h << (4 * g4);
            lo |= l << (4 * g4);
        }
        const bool pu_hi = is_hi16(stage[base - 1]), nu_lo = is_lo16(stage[base + nloc]);
        uint64_t ss = s, st = off_at(d, sm, ss), en = off_at(d, sm, ss + 1);
        int stl = rel_pos(st, c0, UPT + 8), enl = rel_pos(en, c0, UPT + 8);
        uint64_t err_s = NONE;
        int j = 0;
        while (j < nloc) {
            while (j >= enl) {
                ss++;
                st = en;
                stl = enl;
                en = off_at(d, sm, ss + 1);
                enl = rel_pos(en, c0, UPT + 8);
            }
            const int pe = enl < nloc ? enl : nloc;   /* the piece [j, pe) */
            if (j == stl) {
                f = true;
                v = 0;
            }
            /* a piece starts at its string's start or at the chunk's start,
             * and ends at its string's end or at the chunk's end */
            const bool ph = j != stl && pu_hi;   /* the unit before the piece is high */
            const bool nl = pe != enl && nu_lo;   /* the unit after the piece is low */
            uint32_t bad;
            v += gputf_u16_piece(m80, m3, hi, lo, j, pe, ph, nl, &bad);
            if (bad && err_s != ss) {
                record_string_error(d.errw, ss, epoch, c0 + (__ffs(bad) - 1) - st);
                err_s = ss;
            }
            j = pe;
        }
    }
    /* The look-back also orders the error words: a string's result is read
     * only after every tile from its first on has published, so it runs
     * when validating only (out == NULL) too. */
    const bool wr = d.out != nullptr;
    bool ef, tf;
    uint64_t ev, tv;
    block_seg_scan<THREADS>(f, v, sm, &ef, &ev, &tf, &tv);
    if (tid == 0) {
        __threadfence();
        st_release(d.status + t, seg_status(epoch, t == 0 ? ST_PREFIX : ST_AGGREGATE, tf, tv));
    }
    uint64_t carry = 0;
    if (t > 0) carry = block_seg_look_back<THREADS>(d.status, (long long)t, epoch, &hdr->flags, sm);
    if (tid == 0 && t > 0) st_release(d.status + t, seg_status(epoch, ST_PREFIX, false, tf ? tv : carry + tv));
    /* No fence here: the error words a string's result reads were written
     * by the tiles from the string's first on.  Those tiles' aggregates (or
     * an inclusive prefix published after their look-back) were read with
     * acquire loads in the look-back, whose closing barrier hands that
     * ordering to every thread; this tile's own writes are ordered by the
     * scan's barriers. */

    /* phase B: bytes out, results of strings ending here */
    if (nloc > 0) {
        uint64_t ss = s, st = off_at(d, sm, ss), en = off_at(d, sm, ss + 1);
        int stl = rel_pos(st, c0, UPT + 8), enl = rel_pos(en, c0, UPT + 8);
        uint64_t g = ef ? ev : carry + ev;   /* output position within the string */
        uint64_t ob = wr ? d.out_off[ss] : 0, oc = wr ? d.out_off[ss + 1] - ob : ~0ull;
        uint32_t prev = stl < 0 ? (uint32_t)stage[base - 1] : 0u, u = stage[base];
        for (int j = 0; j < nloc; j++) {
            while (j >= enl) {
                ss++;
                st = en;
                stl = enl;
                en = off_at(d, sm, ss + 1);
                enl = rel_pos(en, c0, UPT + 8);
                ob = wr ? d.out_off[ss] : 0;
                oc = wr ? d.out_off[ss + 1] - ob : ~0ull;
            }
            if (j == stl) {
                g = 0;
                prev = 0;
            }
            const uint32_t nx = stage[base + j + 1];
            const uint32_t next = j + 1 < enl ? nx : 0u;
            const uint32_t l = bytes16(u, prev, next);
            if (wr && l && g + l <= oc) put_bytes16(out + ob + g, u, next, l);
            g += l;
            if (j + 1 == enl) {   /* the string's last unit: its result */
                const uint64_t e = string_error(d.errw, ss, epoch);
                if (e == NONE && g <= oc) {
                    d.res[ss].error = GPUTF_E_OK;
                    d.res[ss].reserved = 0;
                    d.res[ss].position = en - st;
                    d.res[ss].written = wr ? g : 0;
                } else {
                    finish_string16<TILE>(d, epoch, ss, e, g);
                }
            }
            prev = u;
            u = nx;
        }
    }
#undef U16AT
    __syncthreads();
}

/* ------------------------------------------------------------------------
 * UTF-8 -> UTF-16 tiles.
 * ---------------------------------------------------------------------- */

/* Error flag at byte i of a string whose bytes start at position st of the
 * stage (bytes before st and from en on read as zero; i may equal en, the
 * string's end position). */
__device__ __forceinline__ bool flag_at(const uint8_t *stage, long long i, long long st, long long en)
{
    uint32_t p = 0, w = 0;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const long long a = i - 7 + k, b = i - 3 + k;
        p |= (a >= st && a < en ? (uint32_t)stage[a] : 0u) << (8 * k);
        w |= (b >= st && b < en ? (uint32_t)stage[b] : 0u) << (8 * k);
    }
    return (gputf_utf8_errors(p, w) >> 24) != 0;
}

__device__ __forceinline__ uint32_t len16_of(uint32_t b) { return ((b & 0xC0) != 0x80) + (b >= 0xF0); }

/* Result of string s when it has an error or overflows its capacity, by
 * one thread of the tile holding its last unit: the exact error start p and
 * class come from the first flagged byte (gputf_utf8_fixup, a few bytes of
 * work); the error wins unless output before p already overflows, and then
 * the result is OUTPUT_TOO_SMALL at the first lead that does not fit.
 * Bounded work (string_prefix, string_crossing). */
template <uint64_t TILE>
__device__ void finish_string8(const BatchDir &d, unsigned epoch, uint64_t s, uint64_t flag, uint64_t total)
{
    const uint8_t *in = static_cast<const uint8_t *>(d.in);
    const uint64_t st = d.in_off[s], en = d.in_off[s + 1];
    const uint64_t n = en - st;
    const uint64_t cap = d.out ? d.out_off[s + 1] - d.out_off[s] : ~0ull;   /* no limit when validating */
    auto len = [&](uint64_t j) -> uint64_t { return len16_of(in[j]); };
    int32_t error = GPUTF_E_OK;
    uint64_t pos = n, written = total;
    bool ok = true;
    bool crossing = flag == NONE;
    if (flag != NONE) {
        uint64_t err_pos = NONE;
        int cls = GPUTF_E_OK;
        ok = gputf_utf8_fixup(in + st, n, flag, &cls, &err_pos) == 0 && err_pos != NONE && err_pos <= n;
        uint64_t gp = 0;
        if (ok) ok = string_prefix<TILE>(d, epoch, st, st + err_pos, len, &gp);
        if (ok && gp <= cap) {
            error = cls;
            pos = err_pos;
            written = gp;
        } else {
            crossing = true;
        }
    }
    if (ok && crossing && total > cap) {
        uint64_t q = 0, gq = 0;
        ok = string_crossing<TILE>(d, epoch, st, en, cap, len, &q, &gq);
        error = GPUTF_E_OUTPUT_TOO_SMALL;
        pos = q - st;
        written = gq;
    }
    if (!ok) {
        error = GPUTF_E_INTERNAL;
        pos = 0;
        written = 0;
    }
    d.res[s].error = error;
    d.res[s].reserved = 0;
    d.res[s].position = pos;
    d.res[s].written = d.out ? written : 0;
}

template <int THREADS, int BPT>
__device__ void batch8_tile(const BatchDir &d, uint64_t t, unsigned epoch, WsHeader *hdr, BatchShared &sm,
                            uint8_t *stage)
{
    constexpr uint64_t TILE = (uint64_t)THREADS * BPT;
    constexpr int HALO = 16;
    static_assert(BPT % 4 == 0 && BPT <= 32, "whole words per thread, one flag bit per byte");
    const uint8_t *in = static_cast<const uint8_t *>(d.in);
    uint16_t *out = static_cast<uint16_t *>(d.out);
    const int tid = threadIdx.x;
    const uint64_t x0 = t * TILE;
    const uint64_t x1 = x0 + TILE < d.units ? x0 + TILE : d.units;

    if (tid < 32) find_strings(d, sm, x0, t + 1 == d.tiles ? ~0ull : x1);
    stage_fill<uint8_t, THREADS>(stage, in, x0, d.units, HALO, (int)TILE + 2 * HALO);
    __syncthreads();

    const uint64_t c0 = x0 + (uint64_t)tid * BPT;
    const uint64_t c1 = c0 + BPT < x1 ? c0 + BPT : (x1 > c0 ? x1 : c0);
    uint64_t s;
    {
        uint64_t lo = 0, hi = sm.n_cached;
        while (hi - lo > 1) {
            const uint64_t mid = (lo + hi) / 2;
            if (sm.off[mid] <= c0) lo = mid;
            else hi = mid;
        }
        s = sm.s_first + lo;
    }
#define SIDX(x) ((long long)((x) - x0) + HALO)
    /* per byte of the chunk (bit j: byte c0 + j): error flags, each checked
     * against the three bytes before it whatever string they belong to
     * (exact for every byte at least three past its string's start);
     * leads (not 10xxxxxx: one unit each); 4-byte leads (one more) */
    uint32_t fl = 0, lb = 0, fb = 0;
    if (c0 < c1) {
        const uint32_t *sw = reinterpret_cast<const uint32_t *>(stage + SIDX(c0));
        gputf_u8state u8s = gputf_u8state_of(sw[-1]);
#pragma unroll
        for (int k = 0; k < BPT / 4; k++) {
            const uint32_t x = sw[k];
            const uint32_t nz = gputf_nonzero_bytes(gputf_utf8_errors_step(&u8s, x));
            fl |= ((((nz >> 7) & 0x01010101u) * 0x01020408u) >> 24) << (4 * k);
            uint32_t l4, f4;
            gputf_u8_lead_bits(x, &l4, &f4);
            lb |= l4 << (4 * k);
            fb |= f4 << (4 * k);
        }
    }
    /* phase A, one string piece of the chunk at a time (positions j
     * relative to c0): units, starts, the first flagged byte per string */
    const int base = tid * BPT + HALO;   /* stage index of c0 */
    const int nloc = (int)(c1 - c0);
    bool f = false;
    uint64_t v = 0;
    if (nloc > 0) {
        uint64_t ss = s, st = off_at(d, sm, ss), en = off_at(d, sm, ss + 1);
        int stl = rel_pos(st, c0, BPT + 8), enl = rel_pos(en, c0, BPT + 8);
        uint64_t flagged = NONE;
        int j = 0;
        while (j < nloc) {
            while (j >= enl) {
                ss++;
                st = en;
                stl = enl;
                en = off_at(d, sm, ss + 1);
                enl = rel_pos(en, c0, BPT + 8);
            }
            const int pe = enl < nloc ? enl : nloc;   /* the piece [j, pe) */
            const uint32_t pm = gputf_bit_range(j, pe);
            if (j == stl) {
                f = true;
                v = 0;
            }
            v += gputf_u8_piece_units(lb, fb, j, pe);
            /* the string's first three bytes see only its own bytes before
             * them (zeros before its start): their flags are taken exactly */
            uint32_t fm = fl & pm;
            const int e3 = stl + 3 < pe ? stl + 3 : pe;
            for (int k = stl > j ? stl : j; k < e3; k++) {
                if (flag_at(stage, base + k, base + stl, base + enl)) fm |= 1u << k;
                else fm &= ~(1u << k);
            }
            if (flagged != ss && fm) {
                record_string_error(d.errw, ss, epoch, c0 + (__ffs(fm) - 1) - st);
                flagged = ss;
            }
            if (pe == enl && flagged != ss && flag_at(stage, base + enl, base + stl, base + enl)) {   /* cut short at its end */
                record_string_error(d.errw, ss, epoch, en - st);
                flagged = ss;
            }
            j = pe;
        }
    }
    /* The look-back also orders the error words: a string's result is read
     * only after every tile from its first on has published, so it runs
     * when validating only (out == NULL) too. */
    const bool wr = d.out != nullptr;
    bool ef, tf;
    uint64_t ev, tv;
    block_seg_scan<THREADS>(f, v, sm, &ef, &ev, &tf, &tv);
    if (tid == 0) {
        __threadfence();
        st_release(d.status + t, seg_status(epoch, t == 0 ? ST_PREFIX : ST_AGGREGATE, tf, tv));
    }
    uint64_t carry = 0;
    if (t > 0) carry = block_seg_look_back<THREADS>(d.status, (long long)t, epoch, &hdr->flags, sm);
    if (tid == 0 && t > 0) st_release(d.status + t, seg_status(epoch, ST_PREFIX, false, tf ? tv : carry + tv));
    /* No fence here: the error words a string's result reads were written
     * by the tiles from the string's first on.  Those tiles' aggregates (or
     * an inclusive prefix published after their look-back) were read with
     * acquire loads in the look-back, whose closing barrier hands that
     * ordering to every thread; this tile's own writes are ordered by the
     * scan's barriers. */

    /* phase B, one string piece at a time: units out at each lead (its
     * four bytes from two stage words, those past the string's end
     * cleared), results of strings ending here */
    if (nloc > 0) {
        uint64_t ss = s, st = off_at(d, sm, ss), en = off_at(d, sm, ss + 1);
        int stl = rel_pos(st, c0, BPT + 8), enl = rel_pos(en, c0, BPT + 8);
        uint64_t g = ef ? ev : carry + ev;
        uint64_t ob = wr ? d.out_off[ss] : 0, oc = wr ? d.out_off[ss + 1] - ob : ~0ull;
        int j = 0;
        while (j < nloc) {
            while (j >= enl) {
                ss++;
                st = en;
                stl = enl;
                en = off_at(d, sm, ss + 1);
                enl = rel_pos(en, c0, BPT + 8);
                ob = wr ? d.out_off[ss] : 0;
                oc = wr ? d.out_off[ss + 1] - ob : ~0ull;
            }
            if (j == stl) g = 0;
            const int pe = enl < nloc ? enl : nloc;
            if (wr) {
                uint32_t lm = lb & gputf_bit_range(j, pe);
                while (lm) {
                    const int k = __ffs(lm) - 1;
                    lm &= lm - 1;
                    const int p = base + k;
                    const uint32_t *wp = reinterpret_cast<const uint32_t *>(stage + (p & ~3));
                    uint32_t q = __funnelshift_r(wp[0], wp[1], 8 * (p & 3));
                    const int rem = enl - k;   /* bytes of the string from this lead on, at least 1 */
                    if (rem < 4) q &= (1u << (8 * rem)) - 1u;
                    const uint32_t b0 = q & 0xFF;
                    const uint32_t two = ((b0 & 0x1F) << 6) | ((q >> 8) & 0x3F);
                    const uint32_t three = ((b0 & 0x0F) << 12) | ((q >> 2) & 0x0FC0) | ((q >> 16) & 0x3F);
                    const uint32_t four = ((b0 & 0x07) << 18) | ((q << 4) & 0x3F000) | ((q >> 10) & 0x0FC0) |
                                          ((q >> 24) & 0x3F);
                    const uint32_t x = four - 0x10000;
                    const uint32_t l = len16_of(b0);
                    if (g + l <= oc) {
                        if (l == 2) {
                            out[ob + g] = (uint16_t)(0xD800 | ((x >> 10) & 0x3FF));
                            out[ob + g + 1] = (uint16_t)(0xDC00 | (x & 0x3FF));
                        } else {
                            out[ob + g] = (uint16_t)(b0 < 0x80 ? b0 : (b0 < 0xE0 ? two : three));
                        }
                    }
                    g += l;
                }
            }
            if (pe == enl) {   /* the string's last byte is here: its result */
                const uint64_t e = string_error(d.errw, ss, epoch);
                if (e == NONE && g <= oc) {
                    d.res[ss].error = GPUTF_E_OK;
                    d.res[ss].reserved = 0;
                    d.res[ss].position = en - st;
                    d.res[ss].written = wr ? g : 0;
                } else {
                    finish_string8<TILE>(d, epoch, ss, e, g);
                }
            }
            j = pe;
        }
    }
#undef SIDX
    __syncthreads();
}

/* ------------------------------------------------------------------------
 * The batched kernel: tickets [0, d8.tiles) are UTF-8 tiles, the rest
 * UTF-16 tiles, taken in ticket order.  Two forms: one tile per CTA (the
 * hardware's block scheduler hands out the CTAs), or persistent (a grid of
 * resident CTAs, each taking tickets until none is left).  Either way a
 * CTA waits only for tiles of smaller tickets, which running CTAs hold.
 * ---------------------------------------------------------------------- */
template <int THREADS, int UPT8, int UPT16, bool PERSIST>
__global__ void __launch_bounds__(THREADS)
batch_kernel(BatchDir d8, BatchDir d16, WsHeader *hdr, unsigned long long *ws_words, uint64_t ws_nwords)
{
    __shared__ BatchShared sm;
    __shared__ unsigned s_tile_flag;
    __shared__ unsigned long long s_ticket;
    extern __shared__ uint4 smem4[];
    const unsigned epoch = *(volatile unsigned *)&hdr->epoch;
    if constexpr (!PERSIST) {
        if (threadIdx.x == 0) s_ticket = atomicAdd(&hdr->ticket, 1ull);
        __syncthreads();
        const uint64_t t = s_ticket;
        if (t < d8.tiles)
            batch8_tile<THREADS, UPT8>(d8, t, epoch, hdr, sm, reinterpret_cast<uint8_t *>(smem4));
        else if (t - d8.tiles < d16.tiles)
            batch16_tile<THREADS, UPT16>(d16, t - d8.tiles, epoch, hdr, sm, reinterpret_cast<uint16_t *>(smem4));
    } else {
        for (;;) {
            if (threadIdx.x == 0) s_ticket = atomicAdd(&hdr->ticket, 1ull);
            __syncthreads();
            const uint64_t t = s_ticket;
            if (t < d8.tiles)
                batch8_tile<THREADS, UPT8>(d8, t, epoch, hdr, sm, reinterpret_cast<uint8_t *>(smem4));
            else if (t - d8.tiles < d16.tiles)
                batch16_tile<THREADS, UPT16>(d16, t - d8.tiles, epoch, hdr, sm,
                                             reinterpret_cast<uint16_t *>(smem4));
            else
                break;   /* every thread read the same ticket */
            /* the tile functions end with a barrier: every thread has read
             * s_ticket before thread 0 takes the next one */
        }
    }
    if (!finish_cta(hdr, &s_tile_flag)) return;
    reset_workspace(hdr, ws_words, ws_nwords);
}

/* ------------------------------------------------------------------------
 * Launch: configurations chosen by the autotuner, by index.
 * ---------------------------------------------------------------------- */
/* The workspace holds one status word per tile, counted for tiles of this
 * many units (gputf_batch_workspace_bytes): no shape may have smaller ones. */
constexpr uint64_t BATCH_MIN_TILE_UNITS = 128 * 8;

template <int T, int U8, int U16, bool PERSIST>
static cudaError_t launch_cfg(const BatchDir &a8, const BatchDir &a16, void *ws, uint64_t ws_nwords,
                              cudaStream_t stream)
{
    static_assert((uint64_t)T * U8 >= BATCH_MIN_TILE_UNITS && (uint64_t)T * U16 >= BATCH_MIN_TILE_UNITS,
                  "tiles smaller than the workspace sizing assumes");
    BatchDir d8 = a8, d16 = a16;
    d8.tiles = (d8.units + (uint64_t)T * U8 - 1) / ((uint64_t)T * U8);
    d16.tiles = (d16.units + (uint64_t)T * U16 - 1) / ((uint64_t)T * U16);
    if (d8.count && !d8.tiles) d8.tiles = 1;     /* a batch of empty strings still needs a tile */
    if (d16.count && !d16.tiles) d16.tiles = 1;
    auto *words = reinterpret_cast<unsigned long long *>(static_cast<char *>(ws) + HEADER_BYTES);
    d8.status = words;
    d16.status = d8.status + d8.tiles;
    d8.errw = d16.status + d16.tiles;
    d16.errw = d8.errw + d8.count;
    uint64_t grid = d8.tiles + d16.tiles;
    if (grid == 0) return cudaSuccess;
    const size_t smem = ((uint64_t)T * U16 + 16) * 2 > (uint64_t)T * U8 + 32 ? ((uint64_t)T * U16 + 16) * 2
                                                                             : (uint64_t)T * U8 + 32;
    auto kern = batch_kernel<T, U8, U16, PERSIST>;
    if (PERSIST) {   /* the CTAs that fit on the device at once */
        static int resident = 0;   /* per configuration (a template instance); same for every sm_103 device */
        if (resident == 0) {
            int dev = 0, sms = 0, per_sm = 0;
            cudaError_t e = cudaGetDevice(&dev);
            if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, T, smem);
            if (e != cudaSuccess) return e;
            resident = sms * (per_sm > 0 ? per_sm : 1);
        }
        if (grid > (uint64_t)resident) grid = (uint64_t)resident;
    }
    kern<<<(unsigned)grid, T, smem, stream>>>(d8, d16, static_cast<WsHeader *>(ws), words, ws_nwords);
    return cudaGetLastError();
}

int batch_config_count() { return 18; }

uint64_t batch_min_tile_units() { return BATCH_MIN_TILE_UNITS; }

cudaError_t launch_batch(int cfg, const BatchDir &d8, const BatchDir &d16, void *ws, uint64_t ws_nwords,
                         cudaStream_t stream)
{
    /* threads x UTF-8 bytes x UTF-16 units per thread; 0-3, 8-9 and 12-14:
     * one tile per CTA; 4-7, 10-11 and 15-17: the same shapes, persistent */
    switch (cfg) {
    case 0: return launch_cfg<256, 16, 16, false>(d8, d16, ws, ws_nwords, stream);
    case 1: return launch_cfg<256, 8, 8, false>(d8, d16, ws, ws_nwords, stream);
    case 2: return launch_cfg<128, 16, 16, false>(d8, d16, ws, ws_nwords, stream);
    case 3: return launch_cfg<128, 8, 8, false>(d8, d16, ws, ws_nwords, stream);
    case 4: return launch_cfg<256, 16, 16, true>(d8, d16, ws, ws_nwords, stream);
    case 5: return launch_cfg<256, 8, 8, true>(d8, d16, ws, ws_nwords, stream);
    case 6: return launch_cfg<128, 16, 16, true>(d8, d16, ws, ws_nwords, stream);
    case 7: return launch_cfg<128, 8, 8, true>(d8, d16, ws, ws_nwords, stream);
    case 8: return launch_cfg<128, 32, 8, false>(d8, d16, ws, ws_nwords, stream);
    case 9: return launch_cfg<64, 16, 16, false>(d8, d16, ws, ws_nwords, stream);
    case 10: return launch_cfg<128, 32, 8, true>(d8, d16, ws, ws_nwords, stream);
    case 11: return launch_cfg<64, 16, 16, true>(d8, d16, ws, ws_nwords, stream);
    case 12: return launch_cfg<128, 32, 16, false>(d8, d16, ws, ws_nwords, stream);
    case 13: return launch_cfg<256, 32, 8, false>(d8, d16, ws, ws_nwords, stream);
    case 14: return launch_cfg<64, 32, 16, false>(d8, d16, ws, ws_nwords, stream);
    case 15: return launch_cfg<128, 32, 16, true>(d8, d16, ws, ws_nwords, stream);
    case 16: return launch_cfg<256, 32, 8, true>(d8, d16, ws, ws_nwords, stream);
    case 17: return launch_cfg<64, 32, 16, true>(d8, d16, ws, ws_nwords, stream);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace gputf
