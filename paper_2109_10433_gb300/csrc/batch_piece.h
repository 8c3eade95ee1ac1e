/*
 * The batched kernel's per-piece arithmetic: a thread's chunk of one
 * direction is worked one string piece at a time (the part of the chunk that
 * lies in one string), from bit masks over the chunk (bit k: unit or byte k
 * of the chunk, at most 32).  Compiled for the GPU (batch.cu) and for the
 * host, so the host tests can check it against the oracle.
 *
 * UTF-8 -> UTF-16: a piece's output units are its leads (bytes that are not
 * 10xxxxxx) plus its 4-byte leads (0xF0 and above), Table 2.
 *
 * UTF-16 -> UTF-8: a piece's bytes are Table 2's closed form per unit (1
 * below U+0080, 2 below U+0800 and for a surrogate, else 3), so a surrogate
 * pair inside the piece gives its 4.  Where a pair crosses the piece's edge,
 * its bytes sit on its high half (the batched kernel's per-unit convention,
 * as in the single-buffer transcoder): the low half opening the piece writes
 * none (2 less), the high half closing it writes all 4 (2 more).  A unit
 * breaks Section 3's pairing rule when it is high and the next unit of its
 * string is not low, or low and the unit before in its string is not high.
 */
#ifndef GPUTF_BATCH_PIECE_H
#define GPUTF_BATCH_PIECE_H

#include <stdint.h>
#include "utf16_scheme.h"

GPUTF_HD uint32_t gputf_popc(uint32_t x)
{
#if defined(__CUDA_ARCH__)
    return (uint32_t)__popc(x);
#else
    return (uint32_t)__builtin_popcount(x);
#endif
}

/* Bit 7 of each byte of m gathered into bits 0-3 (byte k -> bit k). */
GPUTF_HD uint32_t gputf_bit7_nibble(uint32_t m)
{
    return (((m >> 7) & 0x01010101u) * 0x01020408u) >> 24;
}

/* Bits [a, b) of a word, 0 <= a < b <= 32. */
GPUTF_HD uint32_t gputf_bit_range(int a, int b)
{
    return (b >= 32 ? 0u : (1u << b)) - (1u << a);
}

/* The four bytes of x (byte k -> bit k): leads, and 4-byte leads. */
GPUTF_HD void gputf_u8_lead_bits(uint32_t x, uint32_t *lead, uint32_t *lead4)
{
    *lead = gputf_bit7_nibble(~(x & ~(x << 1)) & 0x80808080u);
    *lead4 = gputf_bit7_nibble(x & (x << 1) & (x << 2) & (x << 3) & 0x80808080u);
}

/* Output units of the UTF-8 piece [j, pe) of a chunk with lead bits lb and
 * 4-byte-lead bits fb. */
GPUTF_HD uint32_t gputf_u8_piece_units(uint32_t lb, uint32_t fb, int j, int pe)
{
    const uint32_t pm = gputf_bit_range(j, pe);
    return gputf_popc(lb & pm) + gputf_popc(fb & pm);
}

/* Four UTF-16 units (w0: units 0, 1; w1: units 2, 3; low half first) into
 * bits 0-3: at least U+0080, at least U+0800 and not a surrogate, high
 * surrogate, low surrogate; tested on their gathered high and low bytes. */
GPUTF_HD void gputf_u16_unit_bits4(uint32_t w0, uint32_t w1, uint32_t *m80, uint32_t *m3, uint32_t *hi,
                                   uint32_t *lo)
{
    const uint32_t H = gputf_bperm(w0, w1, 0x7531);   /* high bytes */
    const uint32_t L = gputf_bperm(w0, w1, 0x6420);   /* low bytes */
    const uint32_t ge80 = ~(gputf_zero_bytes(H) & ~L) & 0x80808080u;
    const uint32_t ge08 = (((H & 0x78787878u) + 0x78787878u) | H) & 0x80808080u;
    const uint32_t sur = gputf_zero_bytes((H & 0xF8F8F8F8u) ^ 0xD8D8D8D8u);
    const uint32_t t = H << 5;   /* bit 2 of the high byte: a low surrogate */
    *m80 = gputf_bit7_nibble(ge80);
    *m3 = gputf_bit7_nibble(ge08 & ~sur);
    *hi = gputf_bit7_nibble(sur & ~t);
    *lo = gputf_bit7_nibble(sur & t);
}

/* The UTF-16 piece [j, pe) of a chunk with unit bits m80, m3, hi, lo: its
 * UTF-8 bytes, and in *bad its units that break the pairing rule.  ph: the
 * unit before the piece is a high surrogate of the same string (the piece
 * opens the chunk, inside a string); nl: the unit after the piece is a low
 * surrogate of the same string (the piece closes the chunk, inside a
 * string). */
GPUTF_HD uint32_t gputf_u16_piece(uint32_t m80, uint32_t m3, uint32_t hi, uint32_t lo, int j, int pe, int ph,
                                  int nl, uint32_t *bad)
{
    const uint32_t pm = gputf_bit_range(j, pe), fb = 1u << j, lb = 1u << (pe - 1);
    uint32_t bytes = gputf_popc(pm) + gputf_popc(m80 & pm) + gputf_popc(m3 & pm);
    if ((lo & fb) && ph) bytes -= 2;
    if ((hi & lb) && nl) bytes += 2;
    const uint32_t prevhi = ((hi << 1) & ~fb) | (ph ? fb : 0u);
    const uint32_t nextlo = ((lo >> 1) & ~lb) | (nl ? lb : 0u);
    *bad = ((hi & ~nextlo) | (lo & ~prevhi)) & pm;
    return bytes;
}

#endif
