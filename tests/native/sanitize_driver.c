/*
 * Test harness: drives the CPU oracle and the host-compiled kernel headers
 * over many short and random inputs, every buffer allocated at exactly the
 * size the call is given, for a build with AddressSanitizer and
 * UndefinedBehaviorSanitizer.  Any read or write outside a buffer, any shift
 * by the width or more, any signed overflow ends the process with an error
 * report; a clean run prints the number of calls and exits 0.  The results
 * themselves are checked by the other host tests; here only the absence of
 * undefined behaviour is.  Test infrastructure only.
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.c"
#include "batch_piece.h"    /* includes utf16_scheme.h and utf8_scheme.h */

static uint64_t rng_state = 0x9E3779B97F4A7C15ull;

/* xorshift64*: a test-input generator, nothing of the method's arithmetic */
static uint64_t next_rand(void)
{
    rng_state ^= rng_state >> 12;
    rng_state ^= rng_state << 25;
    rng_state ^= rng_state >> 27;
    return rng_state * 0x2545F4914F6CDD1Dull;
}

static uint64_t calls;

/* A copy of src in a buffer of exactly n bytes (NULL for n = 0). */
static void *exact_copy(const void *src, size_t n)
{
    if (n == 0) return NULL;
    void *p = malloc(n);
    memcpy(p, src, n);
    return p;
}

static void drive_utf8(const uint8_t *src, uint64_t n)
{
    uint8_t *in = exact_copy(src, n);
    oracle_result r;
    /* capacities: none, a few, the exact need, and ample */
    uint64_t need = oracle_utf16_length_from_utf8(in, n);
    uint64_t caps[4] = {0, n / 3, need, n};
    for (int c = 0; c < 4; c++) {
        uint16_t *out = caps[c] ? malloc(caps[c] * sizeof(uint16_t)) : NULL;
        oracle_utf8_to_utf16(in, n, out, caps[c], &r);
        free(out);
        calls++;
    }
    oracle_validate_utf8(in, n, &r);
#ifdef PLANT_OVERREAD
    if (n) oracle_validate_utf8(in, n + 1, &r);   /* one byte past the buffer: the run must fail */
#endif
    /* the kernels' scheme over the same bytes, and its fix-up */
    if (n > 0) {
        uint64_t f = gputf_utf8_first_flag(in, n);
        if (f != UINT64_MAX) {
            int cls;
            uint64_t start;
            (void)gputf_utf8_fixup(in, n, f, &cls, &start);
        }
    }
    /* the decoder on every window of four bytes */
    for (uint64_t p = 0; p + 4 <= n; p++) {
        uint32_t q = (uint32_t)in[p] | (uint32_t)in[p + 1] << 8 | (uint32_t)in[p + 2] << 16 |
                     (uint32_t)in[p + 3] << 24, u0, u1;
        (void)gputf_utf8_decode(q, &u0, &u1);
    }
    calls += 3;
    free(in);
}

static void drive_utf16(const uint16_t *src, uint64_t n)
{
    uint16_t *in = exact_copy(src, n * sizeof(uint16_t));
    oracle_result r;
    uint64_t need = oracle_utf8_length_from_utf16(in, n);
    uint64_t caps[4] = {0, n, need, 3 * n};
    for (int c = 0; c < 4; c++) {
        uint8_t *out = caps[c] ? malloc(caps[c]) : NULL;
        oracle_utf16_to_utf8(in, n, out, caps[c], &r);
        free(out);
        calls++;
    }
    oracle_validate_utf16(in, n, &r);
    /* the kernels' classification and byte arithmetic, four units per step */
    uint32_t hprev = 0, bad = 0;
    for (uint64_t g = 0; g + 4 <= n; g += 4) {
        uint32_t c3, hi, lo, N, A;
        const uint32_t w0 = in[g] | (uint32_t)in[g + 1] << 16, w1 = in[g + 2] | (uint32_t)in[g + 3] << 16;
        gputf_u16_classify(w0, w1, &hprev, &bad, &c3, &hi, &lo, &N, &A);
        const uint32_t L = gputf_u16_counts(c3, hi, lo, N, A, 0);
        uint32_t h2 = 0;
        (void)gputf_u16_mismatch4(w0, w1, &h2);
        (void)gputf_u16_utf8_extra4(w0, w1);
        for (int k = 0; k < 4; k++) {
            uint32_t lead, b1, b2, b3;
            const uint32_t next = g + k + 1 < n ? in[g + k + 1] : 0u;
            gputf_u16_utf8_bytes(in[g + k], next, (L >> (8 * k)) & 0xFF, &lead, &b1, &b2, &b3);
            gputf_u16_utf8_bytes_back(in[g + k], next, (L >> (8 * k)) & 0xFF, &lead, &b1, &b2, &b3);
        }
    }
    (void)gputf_u16_end_mismatch(hprev, n ? in[n - 1] : 0);
    calls += 2;
    free(in);
}

int main(void)
{
    uint8_t b[256];
    uint16_t u[256];

    /* every string of 0, 1 and 2 bytes */
    drive_utf8(b, 0);
    for (int x = 0; x < 256; x++) {
        b[0] = (uint8_t)x;
        drive_utf8(b, 1);
        for (int y = 0; y < 256; y += 3) {
            b[1] = (uint8_t)y;
            drive_utf8(b, 2);
        }
    }
    /* every scalar value (and the values around the valid range) encoded
     * and decoded back, into buffers of exactly its length */
    for (uint32_t cp = 0; cp <= 0x110010; cp += (cp < 0x11000 ? 1 : 61)) {
        uint8_t e8[4];
        uint16_t e16[2];
        int l8 = oracle_encode_utf8(cp, e8), l16 = oracle_encode_utf16(cp, e16);
        if (l8) drive_utf8(e8, (uint64_t)l8);
        if (l16) drive_utf16(e16, (uint64_t)l16);
    }
    /* random bytes and units, biased towards the interesting classes */
    for (int t = 0; t < 20000; t++) {
        const uint64_t n = next_rand() % 97;
        for (uint64_t k = 0; k < n; k++) {
            const uint64_t r = next_rand();
            switch (r % 4) {
            case 0: b[k] = (uint8_t)(r >> 8); break;
            case 1: b[k] = (uint8_t)(0x80 | ((r >> 8) & 0x3F)); break;
            case 2: b[k] = (uint8_t)(0xC0 | ((r >> 8) & 0x3F)); break;
            default: b[k] = (uint8_t)((r >> 8) & 0x7F); break;
            }
            u[k] = (r >> 16) % 3 == 0 ? (uint16_t)(0xD800 | ((r >> 20) & 0x7FF)) : (uint16_t)(r >> 32);
        }
        drive_utf8(b, n);
        drive_utf16(u, n);
    }
    /* the batched kernel's per-piece arithmetic: every piece of random
     * 32-unit (and 32-byte) chunks, with both neighbour cases */
    for (int t = 0; t < 200; t++) {
        uint32_t m80 = 0, m3 = 0, hi = 0, lo = 0, lb = 0, fb = 0;
        for (int g = 0; g < 8; g++) {
            uint32_t w[2];
            for (int i = 0; i < 2; i++) {
                const uint64_t r = next_rand();
                const uint32_t u0 = r % 3 == 0 ? (0xD800u | ((r >> 8) & 0x7FF)) : (uint32_t)((r >> 20) & 0xFFFF);
                const uint32_t u1 = (r >> 40) % 3 == 0 ? (0xD800u | ((r >> 44) & 0x7FF)) : (uint32_t)((r >> 48) & 0xFFFF);
                w[i] = u0 | (u1 << 16);
            }
            uint32_t a, b4, h, l, l4, f4;
            gputf_u16_unit_bits4(w[0], w[1], &a, &b4, &h, &l);
            m80 |= a << (4 * g);
            m3 |= b4 << (4 * g);
            hi |= h << (4 * g);
            lo |= l << (4 * g);
            gputf_u8_lead_bits((uint32_t)next_rand(), &l4, &f4);
            lb |= l4 << (4 * g);
            fb |= f4 << (4 * g);
        }
        for (int j = 0; j < 32; j++)
            for (int pe = j + 1; pe <= 32; pe++) {
                uint32_t bad;
                (void)gputf_u16_piece(m80, m3, hi, lo, j, pe, (pe + t) & 1, (j + t) & 1, &bad);
                (void)gputf_u8_piece_units(lb, fb, j, pe);
            }
        calls += 2;
    }
    /* the loops over many strings */
    {
        static uint8_t fixed[64 * 7];
        static uint16_t fixed16[64 * 5];
        int32_t err[64];
        uint64_t pos[64], off[65];
        for (size_t k = 0; k < sizeof fixed; k++) fixed[k] = (uint8_t)next_rand();
        for (size_t k = 0; k < sizeof fixed16 / 2; k++) fixed16[k] = (uint16_t)next_rand();
        oracle_validate_utf8_fixed(fixed, 64, 7, err, pos);
        oracle_validate_utf16_fixed(fixed16, 64, 5, err, pos);
        off[0] = 0;
        for (int k = 0; k < 64; k++) off[k + 1] = off[k] + next_rand() % 8;
        oracle_validate_utf8_csr(fixed, off, 64, err, pos);
        calls += 3;
    }
    printf("%llu calls\n", (unsigned long long)calls);
    return 0;
}
