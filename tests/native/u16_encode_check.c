/*
 * Test harness: runs the UTF-16 -> UTF-8 kernel's encoding of a thread's run
 * of units on the host and checks the bytes it leaves against the CPU
 * oracle.  Test infrastructure only.
 *
 * The byte values come from the CUDA path's own header (utf16_scheme.h:
 * gputf_u16_utf8_bytes and gputf_u16_utf8_bytes_back, compiled here for the
 * host), the per-unit counts from the same header's classification.  The
 * store pattern is the kernel's:
 *   - front to back: the lead at the unit's first byte, then b1, b2, b3 at
 *     its last, second-to-last and third-to-last byte as far as its length
 *     goes;
 *   - back to front, units n-1 down to 3 (the "every unit inside the input"
 *     path): b3, b2, b1 at the three bytes before the unit's end whatever its
 *     length, then the lead at its first byte unless it has none; units 2,
 *     1, 0 after them front to back.
 *
 * For a run u[0..n) with neighbours pu and nu, written at base G of a
 * buffer, both patterns must satisfy:
 *   1. every store lands in [G, G + total), total the sum of the counts: no
 *      stray reaches the bytes of the run before (another thread's);
 *   2. the bytes [G, G + w) equal the oracle's UTF-8 of the units from the
 *      first one that does not end a pair begun by pu, with nu appended when
 *      u[n-1] and nu form a pair (that pair's 4 bytes are this run's), where
 *      w is the oracle's output length up to its first error (all of it for
 *      valid text);
 *   3. the counts of the units before that error add up to w (total, for
 *      valid text);
 *   4. the two patterns leave the same bytes in [G, G + total).
 */
#include <pthread.h>
#include <stdint.h>
#include <string.h>

#include "oracle.c"
#include "utf16_scheme.h"

#define MAXN 64
#define G 8                         /* guard bytes before the run */
#define BUF (G + 3 * MAXN + 1 + 8)  /* the run's worst case, and guard bytes after it */

static int hi16(uint32_t u) { return (u & 0xFC00) == 0xD800; }
static int lo16(uint32_t u) { return (u & 0xFC00) == 0xDC00; }

/* the kernel's per-unit counts (as in phase A) */
static void counts(const uint16_t *u, int n, uint32_t pu, uint32_t nu, uint8_t *c)
{
    uint32_t bad = 0, hprev = gputf_is_high(pu) ? 0x80000000u : 0u;
    uint32_t p_c3 = 0, p_hi = 0, p_lo = 0, p_N = 0, p_A = 0;
    for (int g = 0; g <= n / 4; g++) {
        uint32_t c3 = 0, hi = 0, lo = gputf_is_low(nu) ? 0x80u : 0u, N = 0, A = 0;
        if (g < n / 4) {
            const uint32_t w0 = u[4 * g] | ((uint32_t)u[4 * g + 1] << 16);
            const uint32_t w1 = u[4 * g + 2] | ((uint32_t)u[4 * g + 3] << 16);
            gputf_u16_classify(w0, w1, &hprev, &bad, &c3, &hi, &lo, &N, &A);
        }
        if (g > 0) {
            const uint32_t L = gputf_u16_counts(p_c3, p_hi, p_lo, p_N, p_A, lo);
            for (int k = 0; k < 4; k++) c[4 * (g - 1) + k] = (uint8_t)(L >> (8 * k));
        }
        p_c3 = c3;
        p_hi = hi;
        p_lo = lo;
        p_N = N;
        p_A = A;
    }
}

/* One byte store of the encoding; returns 0 when it falls outside [lo, hi). */
static int put(uint8_t *buf, long a, uint32_t v, long lo, long hi)
{
    if (a < lo || a >= hi) return 0;
    buf[a] = (uint8_t)v;
    return 1;
}

/* Encodes the run ending at buffer position end; returns 0 if a store left
 * [lo, hi). */
static int encode(const uint16_t *u, int n, uint32_t nu, const uint8_t *c, uint8_t *buf, long end, long lo,
                  long hi, int back)
{
    long e = end;
    int ok = 1;
    for (int k = n - 1; k >= 0; k--) {
        const uint32_t next = k + 1 < n ? u[k + 1] : nu, l = c[k];
        uint32_t lead, b1, b2, b3;
        if (back && k >= 3) {
            gputf_u16_utf8_bytes_back(u[k], next, l, &lead, &b1, &b2, &b3);
            ok &= put(buf, e - 3, b3, lo, hi);
            ok &= put(buf, e - 2, b2, lo, hi);
            ok &= put(buf, e - 1, b1, lo, hi);
            e -= l;
            if (l) ok &= put(buf, e, lead, lo, hi);
        } else {
            gputf_u16_utf8_bytes(u[k], next, l, &lead, &b1, &b2, &b3);
            e -= l;
            const long se = e + l;
            if (l >= 1) ok &= put(buf, e, lead, lo, hi);
            if (l >= 2) ok &= put(buf, se - 1, b1, lo, hi);
            if (l >= 3) ok &= put(buf, se - 2, b2, lo, hi);
            if (l == 4) ok &= put(buf, se - 3, b3, lo, hi);
        }
    }
    return ok;
}

/* 0 when the run passes all four checks, else the number of the check. */
static int check_run(const uint16_t *u, int n, uint32_t pu, uint32_t nu)
{
    uint8_t c[MAXN];
    counts(u, n, pu, nu, c);
    long total = 0;
    for (int k = 0; k < n; k++) total += c[k];

    uint8_t fwd[BUF], bwd[BUF];
    memset(fwd, 0xA5, sizeof fwd);
    memset(bwd, 0x5A, sizeof bwd);
    if (!encode(u, n, nu, c, fwd, G + total, G, G + total, 0)) return 1;
    if (!encode(u, n, nu, c, bwd, G + total, G, G + total, 1)) return 1;

    /* the oracle's bytes for the text this run writes */
    uint16_t s[MAXN + 1];
    const int j0 = lo16(u[0]) && hi16(pu);
    int m = 0;
    for (int k = j0; k < n; k++) s[m++] = u[k];
    if (hi16(u[n - 1]) && lo16(nu)) s[m++] = (uint16_t)nu;
    uint8_t want[4 * (MAXN + 1)];
    oracle_result r;
    oracle_utf16_to_utf8(s, (uint64_t)m, want, sizeof want, &r);
    const long w = (long)r.written;
    if (memcmp(fwd + G, want, (size_t)w) != 0 || memcmp(bwd + G, want, (size_t)w) != 0) return 2;

    long before = 0;
    const long stop = r.error == 0 ? n : j0 + (long)r.position;
    for (long k = 0; k < stop; k++) before += c[k];
    if (before != w) return 3;
    if (memcmp(fwd + G, bwd + G, (size_t)total) != 0) return 4;
    return 0;
}

typedef struct {
    const uint16_t *data;
    uint64_t begin, end;
    int n;
    uint64_t mismatches, first_bad;
    int first_check;
} job_t;

static void *run(void *arg)
{
    job_t *j = (job_t *)arg;
    for (uint64_t k = j->begin; k < j->end; k++) {
        const uint16_t *row = j->data + k * (uint64_t)(j->n + 2);
        const int r = check_run(row, j->n, row[j->n], row[j->n + 1]);
        if (r) {
            if (!j->mismatches) {
                j->first_bad = k;
                j->first_check = r;
            }
            j->mismatches++;
        }
    }
    return 0;
}

/* Runs of width n (units, then pu, then nu: n + 2 values each).  Returns the
 * number of failing runs; *first_bad / *first_check describe the first. */
uint64_t u16_encode_check(const uint16_t *data, uint64_t count, int n, int threads, uint64_t *first_bad,
                          int *first_check)
{
    if (n < 4 || n > MAXN || n % 4) return ~0ull;
    if (threads < 1) threads = 1;
    if (threads > 64) threads = 64;
    pthread_t th[64];
    job_t jobs[64];
    const uint64_t per = (count + threads - 1) / threads;
    for (int t = 0; t < threads; t++) {
        jobs[t].data = data;
        jobs[t].n = n;
        jobs[t].begin = per * t < count ? per * t : count;
        jobs[t].end = per * (t + 1) < count ? per * (t + 1) : count;
        jobs[t].mismatches = 0;
        jobs[t].first_bad = 0;
        jobs[t].first_check = 0;
        pthread_create(&th[t], 0, run, &jobs[t]);
    }
    uint64_t total = 0;
    *first_bad = ~0ull;
    *first_check = 0;
    for (int t = 0; t < threads; t++) {
        pthread_join(th[t], 0);
        total += jobs[t].mismatches;
        if (jobs[t].mismatches && jobs[t].first_bad < *first_bad) {
            *first_bad = jobs[t].first_bad;
            *first_check = jobs[t].first_check;
        }
    }
    return total;
}
