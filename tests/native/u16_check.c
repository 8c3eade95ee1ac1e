/*
 * Test harness: runs the CUDA path's four-units-per-step UTF-16
 * classification (utf16_scheme.h, compiled for the host from the same header
 * the UTF-16 -> UTF-8 kernel uses) beside the CPU oracle on chunks of units
 * with a unit before and a unit after, and counts chunks where they
 * disagree.  Test infrastructure only.
 *
 * For a chunk u[0..n) with neighbours pu and nu, the scheme's per-unit byte
 * counts c[] and pairing flag must satisfy:
 *   1. for every split k that does not fall between the two halves of a
 *      pair, c[0] + ... + c[k-1] equals the oracle's UTF-8 length of
 *      u[0..k), less 2 when u[0] is the low half of a pair begun by pu, plus
 *      2 when k = n and u[n-1] is the high half of a pair ended by nu (the
 *      pair's 4 bytes sit on its high unit);
 *   2. every c[j] is at most 3, except 4 exactly at the high half of a pair,
 *      and 0 exactly at the low half of a pair, so a chunk's bytes never
 *      exceed 3 n + 1 (the staging bound of the kernel);
 *   3. the pairing flag is set exactly when two adjacent units of
 *      pu, u[0..n), nu break the rule of Section 3; when pu is no low
 *      surrogate and nu no high one, exactly when the oracle finds the
 *      sequence pu, u, nu invalid;
 *   4. the validate-only pass's check (gputf_u16_mismatch4 over the groups,
 *      then gputf_u16_end_mismatch) gives the same flag;
 *   5. the length-only pass's count (n plus the bytes of
 *      gputf_u16_utf8_extra4 over the groups) equals the oracle's UTF-8
 *      length of u[0..n).
 */
#include <pthread.h>
#include <stdint.h>
#include <string.h>

#include "oracle.c"
#include "utf16_scheme.h"

#define MAXN 64

static int hi16(uint32_t u) { return (u & 0xFC00) == 0xD800; }
static int lo16(uint32_t u) { return (u & 0xFC00) == 0xDC00; }

/* 0 when the chunk passes all three checks, else the number of the check. */
static int check_chunk(const uint16_t *u, int n, uint32_t pu, uint32_t nu)
{
    /* the kernel's loop: classify group g, then finish group g-1 with its
     * successor's "is low" flags (the unit after the run for the last) */
    uint8_t c[MAXN];
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
    bad |= gputf_u16_end_mismatch(hprev, nu);

    /* 1: sums against the oracle's lengths */
    const int cut_start = lo16(u[0]) && hi16(pu);
    uint64_t sum = 0;
    for (int k = 0; k <= n; k++) {
        if (k > 0) sum += c[k - 1];
        if (k > 0 && k < n && hi16(u[k - 1]) && lo16(u[k])) continue;
        uint64_t want = oracle_utf8_length_from_utf16(u, (uint64_t)k);
        if (k > 0 && cut_start) want -= 2;
        if (k == n && hi16(u[n - 1]) && lo16(nu)) want += 2;
        if (sum != want) return 1;
    }
    /* 2: per-unit bounds */
    for (int j = 0; j < n; j++) {
        const uint32_t prev = j ? u[j - 1] : pu, next = j + 1 < n ? u[j + 1] : nu;
        const int pair_hi = hi16(u[j]) && lo16(next), pair_lo = lo16(u[j]) && hi16(prev);
        if (c[j] > 4 || (c[j] == 4) != pair_hi || (c[j] == 0) != pair_lo) return 2;
    }
    if (sum > 3 * (uint64_t)n + 1) return 2;
    /* 3: the pairing flag */
    uint16_t ext[MAXN + 2];
    ext[0] = (uint16_t)pu;
    memcpy(ext + 1, u, 2 * (size_t)n);
    ext[n + 1] = (uint16_t)nu;
    int broken = 0;
    for (int j = 0; j + 1 < n + 2; j++) broken |= hi16(ext[j]) != lo16(ext[j + 1]);
    if ((bad != 0) != broken) return 3;
    if (!lo16(pu) && !hi16(nu)) {
        oracle_result r;
        oracle_validate_utf16(ext, (uint64_t)n + 2, &r);
        if ((r.error != 0) != broken) return 3;
    }
    /* 4, 5: the validate-only and length-only passes */
    uint32_t vbad = 0, vprev = gputf_is_high(pu) ? 0x80000000u : 0u;
    uint64_t len = (uint64_t)n;
    for (int g = 0; g < n / 4; g++) {
        const uint32_t w0 = u[4 * g] | ((uint32_t)u[4 * g + 1] << 16);
        const uint32_t w1 = u[4 * g + 2] | ((uint32_t)u[4 * g + 3] << 16);
        vbad |= gputf_u16_mismatch4(w0, w1, &vprev);
        const uint32_t e = gputf_u16_utf8_extra4(w0, w1);
        len += (e & 0xFF) + ((e >> 8) & 0xFF) + ((e >> 16) & 0xFF) + (e >> 24);
    }
    vbad |= gputf_u16_end_mismatch(vprev, nu);
    if ((vbad != 0) != broken) return 4;
    if (len != oracle_utf8_length_from_utf16(u, (uint64_t)n)) return 5;
    return 0;
}

/* Chunks: count chunks of width n (units, then pu, then nu: n + 2 values each). */
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
        const int r = check_chunk(row, j->n, row[j->n], row[j->n + 1]);
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

/* Returns the number of failing chunks; *first_bad / *first_check describe
 * the first one. */
uint64_t u16_check(const uint16_t *data, uint64_t count, int n, int threads, uint64_t *first_bad,
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
