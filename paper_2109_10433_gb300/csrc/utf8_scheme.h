/*
 * Per-byte UTF-8 validation with three 16-entry nibble tables, four bytes at
 * a time, plus the scalar decoder that pins the exact error class and start.
 *
 * The same source compiles for the GPU (nvcc) and for the host (gcc), so the
 * host test suite can prove the scheme exhaustively on short strings.
 *
 * Scheme (validation rules 1-6 of Section 3 of the paper, as pair terms):
 *   for byte c with previous byte p,
 *     E = T1[p >> 4] & T2[p & 15] & T3[c >> 4]          (tables: utf8_tables.h)
 *   c is flagged when a bit of E other than TWO_CONTS is set, or when the
 *   TWO_CONTS bit (p and c both continuation bytes) differs from "a lead of
 *   three or four bytes sits two or three bytes before c" (must23).
 * The end of the input is checked by running one zero byte past it: a
 * character cut short there is flagged at the end position n.
 *
 * The flags are not the error report: the first flagged position f lies in
 * [s, s + 3] where s is the start of the first invalid character, and the
 * scalar step gputf_utf8_fixup() walks forward from just before f to find s
 * and the class, in decoding order.
 *
 * Lookups use PRMT: a 16-entry byte table is two 8-byte halves; a selector
 * nibble with bit 3 set selects "replicate the sign bit", which also gives a
 * cheap per-byte mask of "index >= 8".
 */
#ifndef GPUTF_UTF8_SCHEME_H
#define GPUTF_UTF8_SCHEME_H

#include <stdint.h>
#include "utf8_tables.h"

#if defined(__CUDACC__)
#define GPUTF_HD static __host__ __device__ __forceinline__
#else
#define GPUTF_HD static inline
#endif

/* Error classes of the public interface. */
#define GPUTF_E_OK 0
#define GPUTF_E_HEADER_BITS 1
#define GPUTF_E_TOO_SHORT 2
#define GPUTF_E_TOO_LONG 3
#define GPUTF_E_OVERLONG 4
#define GPUTF_E_TOO_LARGE 5
#define GPUTF_E_SURROGATE 6
#define GPUTF_E_OUTPUT_TOO_SMALL 7
#define GPUTF_E_TIMEOUT 8
#define GPUTF_E_INTERNAL 9

/* PTX prmt.b32 default mode: result byte k is byte (sel_k & 7) of {b:a}
 * (a = bytes 0-3, b = bytes 4-7); if sel_k & 8 the sign bit of that byte is
 * replicated instead.  sel_k is bits 4k..4k+3 of sel. */
GPUTF_HD uint32_t gputf_prmt(uint32_t a, uint32_t b, uint32_t sel)
{
#if defined(__CUDA_ARCH__)
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
    return d;
#else
    uint64_t v = (uint64_t)a | ((uint64_t)b << 32);
    uint32_t d = 0;
    for (int k = 0; k < 4; k++) {
        uint32_t s = (sel >> (4 * k)) & 0xF;
        uint32_t byte = (uint32_t)(v >> (8 * (s & 7))) & 0xFF;
        if (s & 8) byte = (byte & 0x80) ? 0xFF : 0x00;
        d |= byte << (8 * k);
    }
    return d;
#endif
}

/* High 32 bits of (hi:lo) << s, 0 < s < 32. */
GPUTF_HD uint32_t gputf_fshl(uint32_t lo, uint32_t hi, uint32_t s)
{
#if defined(__CUDA_ARCH__)
    return __funnelshift_l(lo, hi, s);
#else
    return (hi << s) | (lo >> (32 - s));
#endif
}

/* Low 32 bits of (hi:lo) >> s, 0 <= s < 32. */
GPUTF_HD uint32_t gputf_fshr(uint32_t lo, uint32_t hi, uint32_t s)
{
#if defined(__CUDA_ARCH__)
    return __funnelshift_r(lo, hi, s);
#else
    s &= 31;   /* the shift count taken modulo 32, as the device instruction takes it */
    return s ? (lo >> s) | (hi << (32 - s)) : lo;
#endif
}

/* Byte permute with plain selectors (no sign-replicate mode): the compiler's
 * intrinsic on the GPU, which it can schedule and combine, the PTX model on
 * the host. */
GPUTF_HD uint32_t gputf_bperm(uint32_t a, uint32_t b, uint32_t sel)
{
#if defined(__CUDA_ARCH__)
    return __byte_perm(a, b, sel);
#else
    return gputf_prmt(a, b, sel);
#endif
}

/* x << s and x >> s for any s, 0 once s >= 32 (the GPU's clamped shifts). */
GPUTF_HD uint32_t gputf_shl(uint32_t x, uint32_t s)
{
#if defined(__CUDA_ARCH__)
    return __funnelshift_lc(0u, x, s);
#else
    return s >= 32 ? 0u : x << s;
#endif
}
GPUTF_HD uint32_t gputf_shr(uint32_t x, uint32_t s)
{
#if defined(__CUDA_ARCH__)
    return __funnelshift_rc(x, 0u, s);
#else
    return s >= 32 ? 0u : x >> s;
#endif
}

/* Leading zero bits of x (32 for 0). */
GPUTF_HD uint32_t gputf_clz(uint32_t x)
{
#if defined(__CUDA_ARCH__)
    return (uint32_t)__clz(x);
#else
    return x ? (uint32_t)__builtin_clz(x) : 32u;
#endif
}

/* Pack the four nibbles held in the low halves of the bytes of x into a
 * 16-bit PRMT selector (nibble k = byte k); bits 16-31 are zero. */
GPUTF_HD uint32_t gputf_pack_nibbles(uint32_t x)
{
    uint32_t y = x | (x >> 4);
    return gputf_prmt(y, 0, 0x4420);
}

/* 16-entry table lookup: sel = packed indexes, m = 0xFF in each byte whose
 * index is >= 8. */
GPUTF_HD uint32_t gputf_lut16(uint32_t sel, uint32_t m, uint32_t q0, uint32_t q1,
                              uint32_t q2, uint32_t q3)
{
    uint32_t lo = gputf_prmt(q0, q1, sel);
    uint32_t hi = gputf_prmt(q2, q3, sel ^ 0x8888);
    return (hi & m) | (lo & ~m);
}

#if GPUTF_T1_W0 != GPUTF_T1_W1 || GPUTF_T3_W0 != GPUTF_T3_W1 || \
    (GPUTF_T1_W0 & 0xFF) * 0x01010101u != GPUTF_T1_W0 || (GPUTF_T3_W0 & 0xFF) * 0x01010101u != GPUTF_T3_W0
#error "T1 and T3 must be constant over indexes 0-7 (one PRMT per lookup below)"
#endif

/* What the check of a word needs from the word before it: the word, its
 * bytes' high and low nibbles packed as PRMT selectors, and bit 7 of each
 * byte set where the byte is >= 0xE0 (e0) or >= 0xF0 (f0). */
typedef struct gputf_u8state {
    uint32_t w, hi, lo, e0, f0;
} gputf_u8state;

GPUTF_HD gputf_u8state gputf_u8state_of(uint32_t w)
{
    gputf_u8state s;
    s.w = w;
    s.hi = gputf_pack_nibbles((w >> 4) & 0x0F0F0F0Fu);
    s.lo = gputf_pack_nibbles(w & 0x0F0F0F0Fu);
    s.e0 = w & (w << 1) & (w << 2);
    s.f0 = s.e0 & (w << 3);
    return s;
}

/* Error flags of the four bytes of w (nonzero byte k: byte k of w flagged)
 * given the state of the four bytes just before w; the state moves on to
 * w.  Byte k is checked against the byte before it through the three
 * nibble tables (T1[p >> 4] & T2[p & 15] & T3[c >> 4]); bit 7 of the
 * result (the two-continuations term) is then compared with "two bytes back
 * >= 0xE0 or three bytes back >= 0xF0".  The selectors and the >= masks of
 * the bytes before w are w's own, shifted by one nibble or byte with the
 * previous word's carried in.  T1 and T3 are constant over indexes 0-7, so
 * each takes one PRMT over entries 8-15. */
GPUTF_HD uint32_t gputf_utf8_errors_step(gputf_u8state *st, uint32_t w)
{
    const gputf_u8state c = gputf_u8state_of(w);
    const uint32_t prev1 = gputf_fshl(st->w, w, 8);            /* byte k: the byte before w.k */
    const uint32_t sel_p_hi = (c.hi << 4) | (st->hi >> 12);
    const uint32_t sel_p_lo = (c.lo << 4) | (st->lo >> 12);
    const uint32_t m_p_hi = gputf_prmt(prev1, 0, 0xBA98);       /* p >> 4 >= 8  */
    const uint32_t m_p_lo = gputf_prmt(prev1 << 4, 0, 0xBA98);  /* p & 15 >= 8  */
    const uint32_t m_c_hi = gputf_prmt(w, 0, 0xBA98);           /* c >> 4 >= 8  */
    const uint32_t t1 = (gputf_prmt(GPUTF_T1_W2, GPUTF_T1_W3, sel_p_hi ^ 0x8888) & m_p_hi) | (GPUTF_T1_W0 & ~m_p_hi);
    const uint32_t t2 = gputf_lut16(sel_p_lo, m_p_lo, GPUTF_T2_W0, GPUTF_T2_W1, GPUTF_T2_W2, GPUTF_T2_W3);
    const uint32_t t3 = (gputf_prmt(GPUTF_T3_W2, GPUTF_T3_W3, c.hi ^ 0x8888) & m_c_hi) | (GPUTF_T3_W0 & ~m_c_hi);
    /* bit 7 of each byte: byte two back >= 0xE0, or three back >= 0xF0 */
    const uint32_t must23 = (gputf_fshl(st->e0, c.e0, 16) | gputf_fshl(st->f0, c.f0, 24)) & 0x80808080u;
    *st = c;
    return (t1 & t2 & t3) ^ must23;
}

/* Error flags of the four bytes of w given p, the four bytes just before w. */
GPUTF_HD uint32_t gputf_utf8_errors(uint32_t p, uint32_t w)
{
    gputf_u8state st = gputf_u8state_of(p);
    return gputf_utf8_errors_step(&st, w);
}

/* Bit 7 of each byte set iff that byte of x is nonzero. */
GPUTF_HD uint32_t gputf_nonzero_bytes(uint32_t x)
{
    return (((x & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | x) & 0x80808080u;
}

/* One UTF-8 character at in[p], p < n: returns its class and, when valid,
 * its length.  Classes in decoding order: the lead byte (stray continuation,
 * or 0xF8..0xFF), then missing continuation bytes, then the ranges of the
 * second byte that give overlong, too large and surrogate values. */
GPUTF_HD int gputf_utf8_char(const uint8_t *in, uint64_t n, uint64_t p, int *len)
{
    uint32_t b = in[p];
    if (b < 0x80) {
        *len = 1;
        return GPUTF_E_OK;
    }
    if (b < 0xC0) return GPUTF_E_TOO_LONG;
    if (b >= 0xF8) return GPUTF_E_HEADER_BITS;
    int L = b >= 0xF0 ? 4 : (b >= 0xE0 ? 3 : 2);
    for (int k = 1; k < L; k++) {
        if (p + (uint64_t)k >= n || (in[p + k] & 0xC0) != 0x80) return GPUTF_E_TOO_SHORT;
    }
    uint32_t b1 = in[p + 1];
    if (L == 2 && b < 0xC2) return GPUTF_E_OVERLONG;
    if (L == 3 && b == 0xE0 && b1 < 0xA0) return GPUTF_E_OVERLONG;
    if (L == 3 && b == 0xED && b1 >= 0xA0) return GPUTF_E_SURROGATE;
    if (L == 4 && b == 0xF0 && b1 < 0x90) return GPUTF_E_OVERLONG;
    if (L == 4 && (b > 0xF4 || (b == 0xF4 && b1 >= 0x90))) return GPUTF_E_TOO_LARGE;
    *len = L;
    return GPUTF_E_OK;
}

/* From the first flagged position f (0 <= f <= n, n > 0), find the start and
 * class of the first invalid character.  The scan starts at most three bytes
 * before f, backed up over at most four continuation bytes to a character
 * start of the valid prefix.  Returns 0 when it finds the error, -1 if the
 * flags and the decoder disagree (which the scheme's proof rules out). */
GPUTF_HD int gputf_utf8_fixup(const uint8_t *in, uint64_t n, uint64_t f, int *cls,
                              uint64_t *start)
{
    uint64_t q = f >= 3 ? f - 3 : 0;
    for (int k = 0; k < 4 && q > 0 && (in[q] & 0xC0) == 0x80; k++) q--;
    uint64_t p = q;
    for (int it = 0; it < 8 && p < n; it++) {
        int L = 1;
        int c = gputf_utf8_char(in, n, p, &L);
        if (c != GPUTF_E_OK) {
            *cls = c;
            *start = p;
            return 0;
        }
        p += (uint64_t)L;
    }
    *cls = GPUTF_E_OK;
    *start = p;
    return -1;
}

#if !defined(__CUDACC__)
/* Host-side mirror of what the kernels compute over a whole buffer: the first
 * flagged position (<= n), or UINT64_MAX when nothing is flagged.  Bytes
 * before the buffer and from n on read as zero. */
GPUTF_HD uint64_t gputf_utf8_first_flag(const uint8_t *in, uint64_t n)
{
    gputf_u8state st = gputf_u8state_of(0);
    for (uint64_t base = 0; base <= n; base += 4) {
        uint32_t w = 0;
        for (int k = 0; k < 4; k++)
            if (base + k < n) w |= (uint32_t)in[base + k] << (8 * k);
        uint32_t nz = gputf_nonzero_bytes(gputf_utf8_errors_step(&st, w));
        while (nz) {
            int k = (int)((__builtin_ctz(nz) - 7) / 8);
            if (base + (uint64_t)k <= n) return base + (uint64_t)k;
            nz &= nz - 1;
        }
    }
    return UINT64_MAX;
}
#endif

/*
 * UTF-16 of the character whose lead is byte 0 of q (bytes 1..3 follow);
 * returns the unit count, *u0 and *u1 the units.  With the bytes in
 * big-endian order, the sequence length n is the number of leading ones of
 * the lead (taken as 1 for ASCII); shifting left and back by n clears the
 * lead's prefix, masking with 3F clears the continuation prefixes, and two
 * shift-and-mask steps pack the four 6-bit groups (Section 3; Figs. 2-4)
 * into b0 << 18 | b1 << 12 | b2 << 6 | b3, whose top 6n bits are the scalar
 * value.  Four-byte characters give v - 0x10000 split under 110110 / 110111
 * (Fig. 4).  Any lead byte >= 0xF0 counts two units, as the length pass
 * counts it; the units of an invalid sequence are unspecified.
 */
GPUTF_HD int gputf_utf8_decode(uint32_t q, uint32_t *u0, uint32_t *u1)
{
    const uint32_t r = gputf_bperm(q, 0u, 0x0123);   /* lead in bits 24-31 */
    const uint32_t clo = gputf_clz(~r);
    const uint32_t n = clo > 1 ? clo : 1u;
    const uint32_t v = gputf_shr(gputf_shl(r, n), n) & 0x7F3F3F3Fu;
    const uint32_t t = ((v >> 2) & 0x3FC03FC0u) | (v & 0x00FF00FFu);     /* two 12-bit halves */
    const uint32_t code = gputf_shr(((t >> 4) & 0x0FFFF000u) | (t & 0xFFFu), 24u - 6u * n);
    const uint32_t x = code - 0x10000u;
    const int pair = n >= 4;
    *u0 = pair ? (0xD800u | ((x >> 10) & 0x3FFu)) : code;
    *u1 = 0xDC00u | (x & 0x3FFu);
    return pair ? 2 : 1;
}

#endif
