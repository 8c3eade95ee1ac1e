/*
 * Test harness: runs the CUDA path's UTF-8 nibble scheme and fix-up decoder
 * (compiled for the host from the same header the kernels use) and the CPU
 * oracle side by side, and counts strings where (error class, position)
 * differ.  Test infrastructure only.
 */
#include <pthread.h>
#include <stdint.h>
#include <string.h>

#include "oracle.c"
#include "utf8_scheme.h"

typedef struct {
    const uint8_t *data;
    const uint64_t *offsets;   /* NULL: fixed width */
    uint32_t width;
    uint64_t begin, end;
    uint64_t mismatches;
    uint64_t first_bad;
} job_t;

static int scheme_result(const uint8_t *in, uint64_t n, int *cls, uint64_t *pos)
{
    uint64_t f = gputf_utf8_first_flag(in, n);
    if (f == UINT64_MAX) {
        *cls = GPUTF_E_OK;
        *pos = n;
        return 0;
    }
    return gputf_utf8_fixup(in, n, f, cls, pos);
}

static void *run(void *arg)
{
    job_t *j = (job_t *)arg;
    for (uint64_t k = j->begin; k < j->end; k++) {
        const uint8_t *s;
        uint64_t n;
        if (j->offsets) {
            s = j->data + j->offsets[k];
            n = j->offsets[k + 1] - j->offsets[k];
        } else {
            s = j->data + k * j->width;
            n = j->width;
        }
        oracle_result r;
        oracle_validate_utf8(s, n, &r);
        int cls = -2;
        uint64_t pos = 0;
        int rc = scheme_result(s, n, &cls, &pos);
        if (rc != 0 || cls != r.error || pos != r.position) {
            if (j->mismatches == 0) j->first_bad = k;
            j->mismatches++;
        }
    }
    return 0;
}

/* Returns the number of mismatching strings; *first_bad = index of the first. */
uint64_t scheme_check(const uint8_t *data, const uint64_t *offsets, uint64_t count,
                      uint32_t width, int threads, uint64_t *first_bad)
{
    if (threads < 1) threads = 1;
    if (threads > 64) threads = 64;
    pthread_t tid[64];
    job_t jobs[64];
    for (int t = 0; t < threads; t++) {
        jobs[t].data = data;
        jobs[t].offsets = offsets;
        jobs[t].width = width;
        jobs[t].begin = count * (uint64_t)t / (uint64_t)threads;
        jobs[t].end = count * (uint64_t)(t + 1) / (uint64_t)threads;
        jobs[t].mismatches = 0;
        jobs[t].first_bad = UINT64_MAX;
        pthread_create(&tid[t], 0, run, &jobs[t]);
    }
    uint64_t total = 0;
    *first_bad = UINT64_MAX;
    for (int t = 0; t < threads; t++) {
        pthread_join(tid[t], 0);
        total += jobs[t].mismatches;
        if (jobs[t].first_bad < *first_bad) *first_bad = jobs[t].first_bad;
    }
    return total;
}

/* The scheme's result alone, for reporting. */
void scheme_one(const uint8_t *in, uint64_t n, int *cls, uint64_t *pos, uint64_t *flag)
{
    *flag = gputf_utf8_first_flag(in, n);
    scheme_result(in, n, cls, pos);
}
