/*
 * Test harness: runs the CUDA path's UTF-8 character decoder
 * (gputf_utf8_decode in utf8_scheme.h, compiled for the host from the same
 * header the UTF-8 -> UTF-16 kernel uses) beside the CPU oracle.  Test
 * infrastructure only.
 *   decode_check_scalars: for every scalar value, its UTF-8 bytes from the
 *     oracle, followed by each of `nfill` filler patterns, must decode to the
 *     oracle's UTF-16 units with the right unit count;
 *   decode_check_counts: for every lead byte and every second byte, with the
 *     remaining bytes from a filler set, the unit count must be 1 + [lead >=
 *     0xF0] (the length pass's count, which places the output).
 * Each returns the number of failures and the first failing input word.
 */
#include <stdint.h>

#include "oracle.c"
#include "utf8_scheme.h"

uint64_t decode_check_scalars(const uint32_t *fill, int nfill, uint32_t *first_bad)
{
    uint64_t bad = 0;
    *first_bad = 0;
    for (uint32_t cp = 0; cp <= 0x10FFFF; cp++) {
        if (cp >= 0xD800 && cp <= 0xDFFF) continue;
        uint8_t b[4];
        uint16_t want[2];
        const int nb = oracle_encode_utf8(cp, b);
        const int nu = oracle_encode_utf16(cp, want);
        for (int f = 0; f < nfill; f++) {
            uint32_t q = fill[f];
            for (int k = 0; k < nb; k++) q = (q & ~(0xFFu << (8 * k))) | ((uint32_t)b[k] << (8 * k));
            uint32_t u0, u1;
            const int c = gputf_utf8_decode(q, &u0, &u1);
            const int ok = c == nu && u0 == want[0] && (nu == 1 || u1 == want[1]);
            if (!ok) {
                if (!bad) *first_bad = q;
                bad++;
            }
        }
    }
    return bad;
}

uint64_t decode_check_counts(const uint32_t *fill, int nfill, uint32_t *first_bad)
{
    uint64_t bad = 0;
    *first_bad = 0;
    for (uint32_t b0 = 0; b0 < 256; b0++)
        for (uint32_t b1 = 0; b1 < 256; b1++)
            for (int f = 0; f < nfill; f++) {
                const uint32_t q = (fill[f] & 0xFFFF0000u) | (b1 << 8) | b0;
                uint32_t u0, u1;
                const int c = gputf_utf8_decode(q, &u0, &u1);
                if (c != 1 + (b0 >= 0xF0)) {
                    if (!bad) *first_bad = q;
                    bad++;
                }
            }
    return bad;
}
