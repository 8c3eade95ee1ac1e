/*
 * UTF-16 classification four units at a time: the per-unit output byte
 * counts of the UTF-16 -> UTF-8 transcoder and the check of the surrogate
 * pairing rule (Section 3: a high surrogate D800-DBFF must be followed by a
 * low surrogate DC00-DFFF, and a low one must follow a high one).
 *
 * The same source compiles for the GPU (nvcc) and for the host (gcc), so the
 * host test suite can check it against the oracle exhaustively.
 *
 * Count convention (Table 2, arranged so that every unit writes its own
 * bytes): 1 below U+0080, 2 below U+0800, 3 for the rest of the BMP; a high
 * surrogate followed by a low one writes the pair's 4 bytes and that low one
 * writes 0; a lone surrogate counts 2.  Over any stretch that does not cut a
 * pair this adds up to the UTF-8 length of Table 2, and no unit counts more
 * than 3 except the high half of a pair (4, with 0 right after it), so a run
 * of units never needs more than 3 bytes a unit, plus one when it ends
 * between the two halves of a pair.
 *
 * Four units per step: a byte permute gathers their high bytes (and low
 * bytes) into one word, exact per-byte tests classify them, and three flags
 * at bit 7 of each byte give the counts:
 *   N: not the low half of a pair (counts 1),
 *   A: counts one more (2-byte units, and surrogates other than a pair's
 *      low half),
 *   B: counts two more (3-byte units, and a pair's high half).
 * B needs the "next unit is low" flags of the group after, so each step
 * finishes the group before it.
 */
#ifndef GPUTF_UTF16_SCHEME_H
#define GPUTF_UTF16_SCHEME_H

#include <stdint.h>
#include "utf8_scheme.h"   /* GPUTF_HD, gputf_bperm, gputf_fshr */

GPUTF_HD int gputf_is_high(uint32_t u) { return (u & 0xFC00) == 0xD800; }
GPUTF_HD int gputf_is_low(uint32_t u) { return (u & 0xFC00) == 0xDC00; }

/* Bit 7 of each byte: set when that byte of x is zero (exact per byte: no
 * carry crosses a byte). */
GPUTF_HD uint32_t gputf_zero_bytes(uint32_t x)
{
    return ~(((x & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | x) & 0x80808080u;
}

/*
 * Classifies four units (w0: units 0 and 1, w1: units 2 and 3, low half
 * first): sets their flags, at bit 7 of each byte, in *c3 (3-byte unit),
 * *hi / *lo (high / low surrogate), *N and *A (above); *hprev carries bit 31
 * = "the unit before the group is high" from group to group, and *bad
 * collects the pairs of adjacent units that break the pairing rule.
 */
GPUTF_HD void gputf_u16_classify(uint32_t w0, uint32_t w1, uint32_t *hprev, uint32_t *bad, uint32_t *c3,
                                 uint32_t *hi, uint32_t *lo, uint32_t *N, uint32_t *A)
{
    const uint32_t H = gputf_bperm(w0, w1, 0x7531);    /* high bytes */
    const uint32_t Lo = gputf_bperm(w0, w1, 0x6420);   /* low bytes */
    const uint32_t hz = gputf_zero_bytes(H);
    const uint32_t ge08 = (((H & 0x78787878u) + 0x78787878u) | H) & 0x80808080u;   /* >= U+0800 */
    const uint32_t sur = gputf_zero_bytes((H & 0xF8F8F8F8u) ^ 0xD8D8D8D8u);        /* D800-DFFF */
    const uint32_t t = H << 5;   /* bit 2 of each high byte (a low surrogate) to bit 7 */
    *hi = sur & ~t;
    *lo = sur & t;
    const uint32_t ph = gputf_bperm(*hprev, *hi, 0x6543);   /* the unit before each unit is high */
    *bad |= ph ^ *lo;
    *hprev = *hi;
    *c3 = ge08 & ~sur;
    *N = ~(*lo & ph) & 0x80808080u;
    *A = ~(hz & ~Lo) & ~*c3 & *N;                          /* neither ASCII nor 3-byte */
}

/* The four count bytes (byte k: unit k) of a group with flags c3, hi, lo, N,
 * A, given the "is low" flags of the group after it (bit 7 of byte 0 is what
 * matters; for the last group, 0x80 when the unit after the run is low). */
GPUTF_HD uint32_t gputf_u16_counts(uint32_t c3, uint32_t hi, uint32_t lo, uint32_t N, uint32_t A,
                                   uint32_t next_lo)
{
    const uint32_t nl = gputf_fshr(lo, next_lo, 8);   /* each unit's next unit is low */
    const uint32_t B = c3 | (hi & nl);
    return (N >> 7) + (A >> 7) + (B >> 6);
}

/*
 * The UTF-8 bytes of one unit u that writes l bytes (its count above),
 * followed by the unit `next`: the lead byte and the last three bytes, b1
 * the last, b2 the one before, b3 the one before that.  l = 4 (the high
 * half of a pair, `next` its low half) encodes the code point
 *   c = ((u - 0xD800) << 10) + (next - 0xDC00) + 0x10000     (Section 3),
 * l = 1, 2, 3 encode u itself: the lead carries the prefix 0 / 110 / 1110 /
 * 11110 and the top bits, each continuation byte the prefix 10 and one
 * 6-bit group (Section 5, Table 2).  Only the low byte of *lead counts; bytes
 * beyond a unit's length carry no meaning (a lone surrogate's 2 bytes
 * neither).  Two forms of the same bytes, for the kernel's two store orders:
 * front to back (lead prefix by a shift of the four prefixes) and back to
 * front (lead prefix by a byte permute; b3 always from c, whose bits 12-17
 * are the third byte of a pair's encoding).
 */
GPUTF_HD void gputf_u16_utf8_bytes(uint32_t u, uint32_t next, uint32_t l, uint32_t *lead, uint32_t *b1,
                                   uint32_t *b2, uint32_t *b3)
{
    const uint32_t c = (u << 10) + next - 0x35FDC00u;
    const uint32_t y = l == 4 ? c : u;
    *lead = gputf_fshr(y, 0u, 6 * l - 6) | gputf_fshr(0xF0E0C000u, 0u, 8 * l - 8);
    *b1 = (y & 0x3F) | 0x80;
    *b2 = ((y >> 6) & 0x3F) | 0x80;
    *b3 = ((y >> 12) & 0x3F) | 0x80;
}

GPUTF_HD void gputf_u16_utf8_bytes_back(uint32_t u, uint32_t next, uint32_t l, uint32_t *lead, uint32_t *b1,
                                        uint32_t *b2, uint32_t *b3)
{
    const uint32_t c = (u << 10) + next - 0x35FDC00u;
    const uint32_t y = l == 4 ? c : u;
    *lead = gputf_fshr(y, 0u, 6 * l - 6) | gputf_bperm(0xE0C00000u, 0xF0u, l);
    *b1 = (y & 0x3F) | 0x80;
    *b2 = ((y >> 6) & 0x3F) | 0x80;
    *b3 = ((c >> 12) & 0x3F) | 0x80;
}

/* The pairing check across the end of a run: the last unit's "is high" (bit
 * 31 of hprev after the last group) against "the unit after is low". */
GPUTF_HD uint32_t gputf_u16_end_mismatch(uint32_t hprev, uint32_t nu)
{
    return (hprev >> 31) ^ (gputf_is_low(nu) ? 1u : 0u);
}

/* The validate-only pass: the pairing check of four units (w0, w1 as for
 * gputf_u16_classify), nonzero when two adjacent units break the rule;
 * *hprev carries the "unit before is high" flag as there. */
GPUTF_HD uint32_t gputf_u16_mismatch4(uint32_t w0, uint32_t w1, uint32_t *hprev)
{
    const uint32_t H = gputf_bperm(w0, w1, 0x7531);
    const uint32_t sur = gputf_zero_bytes((H & 0xF8F8F8F8u) ^ 0xD8D8D8D8u);
    const uint32_t t = H << 5;
    const uint32_t hi = sur & ~t, lo = sur & t;
    const uint32_t bad = gputf_bperm(*hprev, hi, 0x6543) ^ lo;
    *hprev = hi;
    return bad;
}

/* The length-only pass (Table 2's closed form, no pairing): for each of four
 * units a byte holding its UTF-8 length minus one, [u >= U+0080] + [u >=
 * U+0800 and not a surrogate], so that a surrogate unit counts 2 bytes. */
GPUTF_HD uint32_t gputf_u16_utf8_extra4(uint32_t w0, uint32_t w1)
{
    const uint32_t H = gputf_bperm(w0, w1, 0x7531), Lo = gputf_bperm(w0, w1, 0x6420);
    const uint32_t ge80 = ~(gputf_zero_bytes(H) & ~Lo) & 0x80808080u;                  /* >= U+0080 */
    const uint32_t ge08 = (((H & 0x78787878u) + 0x78787878u) | H) & 0x80808080u;     /* >= U+0800 */
    const uint32_t c3 = ge08 & ~gputf_zero_bytes((H & 0xF8F8F8F8u) ^ 0xD8D8D8D8u);   /* and no surrogate */
    return (ge80 >> 7) + (c3 >> 7);
}

#endif
