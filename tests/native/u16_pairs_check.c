/*
 * Test harness: the oracle's UTF-16 validator and UTF-16 -> UTF-8 transcoder
 * on every sequence of two 16-bit units (all 2^32 of them), against what
 * Section 3 of the paper fixes for them.  Test infrastructure only.
 *
 * Expected values come from outside the oracle:
 *   - validity and the error position from the closed form of Section 3's
 *     UTF-16 paragraph: a unit D800-DBFF (high) must be followed by a unit
 *     DC00-DFFF (low), and a low unit must follow a high one.  So (a, b) is
 *     valid iff neither unit is a surrogate, or a is high and b is low; the
 *     first invalid unit is a (position 0) when a is a surrogate that does
 *     not start a pair, else b (position 1);
 *   - the UTF-8 bytes from tables the caller builds with CPython's own
 *     codec: the encoding of every BMP scalar value and of every
 *     supplementary one.  A valid pair (a, b) of surrogates must give the
 *     bytes of the code point ((a - 0xD800) << 10 | (b - 0xDC00)) + 0x10000
 *     (Section 3, Fig. 4), two other valid units the bytes of a then of b.
 *     On an error at position 1 the valid prefix is a alone.
 * Returns the number of sequences where the oracle disagrees; the first one
 * goes to *first.
 */
#include <pthread.h>
#include <stdint.h>
#include <string.h>

#include "oracle.c"

static int is_hi(uint32_t u) { return u >= 0xD800 && u <= 0xDBFF; }
static int is_lo(uint32_t u) { return u >= 0xDC00 && u <= 0xDFFF; }

typedef struct {
    const uint8_t *bmp;    /* 65536 x 4: CPython's UTF-8 bytes of each BMP value */
    const uint8_t *blen;   /* 65536: their lengths (0 for surrogates)          */
    const uint8_t *supp;   /* 2^20 x 4: CPython's UTF-8 of U+10000 + i          */
    uint32_t a0, a1;       /* this thread's first units [a0, a1)               */
    uint64_t mismatches;
    uint64_t first;
} job;

static void *run(void *arg)
{
    job *j = (job *)arg;
    for (uint32_t a = j->a0; a < j->a1; a++) {
        for (uint32_t b = 0; b < 65536; b++) {
            const uint16_t in[2] = {(uint16_t)a, (uint16_t)b};
            const int sa = is_hi(a) || is_lo(a), sb = is_hi(b) || is_lo(b);
            const int pair = is_hi(a) && is_lo(b);
            const int valid = (!sa && !sb) || pair;
            const uint64_t epos = valid ? 2 : ((sa && !pair) ? 0 : 1);
            uint8_t want[8];
            uint64_t wlen = 0;
            if (pair) {
                const uint32_t i = ((a - 0xD800) << 10) | (b - 0xDC00);
                memcpy(want, j->supp + 4 * (uint64_t)i, 4);
                wlen = 4;
            } else if (valid || epos == 1) {
                memcpy(want, j->bmp + 4 * a, 4);
                wlen = j->blen[a];
                if (valid) {
                    memcpy(want + wlen, j->bmp + 4 * b, 4);
                    wlen += j->blen[b];
                }
            }
            oracle_result v, t;
            uint8_t out[8];
            memset(out, 0xEE, sizeof out);
            oracle_validate_utf16(in, 2, &v);
            oracle_utf16_to_utf8(in, 2, out, sizeof out, &t);
            int ok = v.position == epos && v.written == 0 &&
                     v.error == (valid ? ORC_OK : ORC_SURROGATE) &&
                     t.position == epos && t.error == v.error && t.written == wlen &&
                     memcmp(out, want, wlen) == 0;
            if (!ok) {
                if (j->mismatches == 0) j->first = ((uint64_t)a << 16) | b;
                j->mismatches++;
            }
        }
    }
    return 0;
}

uint64_t u16_pairs_check(const uint8_t *bmp, const uint8_t *blen, const uint8_t *supp,
                         uint32_t a_begin, uint32_t a_end, int threads, uint64_t *first)
{
    enum { MAXT = 64 };
    job jobs[MAXT];
    pthread_t tid[MAXT];
    if (threads < 1) threads = 1;
    if (threads > MAXT) threads = MAXT;
    const uint32_t span = a_end - a_begin;
    for (int k = 0; k < threads; k++) {
        jobs[k] = (job){bmp, blen, supp, a_begin + (uint32_t)((uint64_t)span * k / threads),
                        a_begin + (uint32_t)((uint64_t)span * (k + 1) / threads), 0, 0};
        pthread_create(&tid[k], 0, run, &jobs[k]);
    }
    uint64_t total = 0;
    *first = ~0ull;
    for (int k = 0; k < threads; k++) {
        pthread_join(tid[k], 0);
        if (jobs[k].mismatches && *first == ~0ull) *first = jobs[k].first;
        total += jobs[k].mismatches;
    }
    return total;
}
