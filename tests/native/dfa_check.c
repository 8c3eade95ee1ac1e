/*
 * Test harness: the UTF-8 automaton of the validate-only pass
 * (utf8_dfa.h, compiled here for the host) against the CPU oracle.
 * Test infrastructure only.
 *
 * For a string x[0..n): running the automaton from ACCEPT over x and then a
 * zero byte must reject iff the oracle rejects x, and the first rejected
 * position f (n for the zero byte) must satisfy s <= f <= s + 3, where s is
 * the oracle's error position; valid strings end in ACCEPT.  The chunked
 * form must agree: a thread starting at any position c replays the three
 * bytes before c from SYNC0, then runs from c; if the input before c is
 * valid, its state at c equals the state of a run from the start.
 *
 * dfa_check_all(len): every string of `len` bytes (len <= 3: all 2^(8 len)).
 * dfa_check_list(buf, count, len): the given strings.
 * Returns the number of failures; the first failing string goes to *first.
 */
#include <stdint.h>
#include <string.h>

#include "oracle.c"
#include "utf8_dfa.h"

static uint32_t run(const uint8_t *x, int n, uint32_t s, int *first_reject)
{
    *first_reject = -1;
    for (int i = 0; i <= n; i++) {
        s = gputf_dfa_next(s, gputf_dfa_class(i < n ? x[i] : 0u));
        if (s == GPUTF_DFA_REJECT) {
            *first_reject = i;
            return s;
        }
        if (i == n) break;
    }
    return s;
}

static int check_one(const uint8_t *x, int n)
{
    oracle_result r;
    oracle_validate_utf8(x, (uint64_t)n, &r);
    int f;
    run(x, n, GPUTF_DFA_ACCEPT, &f);
    if (r.error == 0) {
        if (f >= 0) return 1;
    } else {
        if (f < 0) return 2;
        if ((uint64_t)f < r.position || (uint64_t)f > r.position + 3) return 3;
    }
    /* chunked: the state at every start c after a valid prefix */
    uint32_t s = GPUTF_DFA_ACCEPT;
    for (int c = 0; c <= n; c++) {
        if (r.error != 0 && (uint64_t)c > r.position) break;   /* prefix before c no longer valid */
        uint32_t t = GPUTF_DFA_SYNC0;
        for (int k = 3; k >= 1; k--) t = gputf_dfa_next(t, gputf_dfa_class(c - k >= 0 ? x[c - k] : 0u));
        if (t != s) return 4;
        if (c < n) s = gputf_dfa_next(s, gputf_dfa_class(x[c]));
    }
    return 0;
}

uint64_t dfa_check_all(int len, uint64_t *first)
{
    uint64_t fails = 0;
    uint8_t x[4];
    const uint64_t total = 1ull << (8 * len);
    for (uint64_t v = 0; v < total; v++) {
        for (int k = 0; k < len; k++) x[k] = (uint8_t)(v >> (8 * k));
        if (check_one(x, len)) {
            if (!fails) *first = v;
            fails++;
        }
    }
    return fails;
}

uint64_t dfa_check_list(const uint8_t *buf, uint64_t count, int len, uint64_t *first)
{
    uint64_t fails = 0;
    for (uint64_t i = 0; i < count; i++) {
        if (check_one(buf + i * (uint64_t)len, len)) {
            if (!fails) *first = i;
            fails++;
        }
    }
    return fails;
}
