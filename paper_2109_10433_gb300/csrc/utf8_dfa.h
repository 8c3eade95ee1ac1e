/*
 * UTF-8 validation as a byte-at-a-time automaton, for the validate-only
 * pass.
 *
 * The states say what the next byte must be (Section 3's rules 1-6, RFC 3629
 * Table 3): any character start (ACCEPT), one, two or three more
 * continuation bytes, or the restricted second byte after E0 (A0-BF), ED
 * (80-9F), F0 (90-BF) or F4 (80-8F); REJECT is absorbing.  Bytes fall into
 * twelve classes by how these states treat them.  Three more states let a
 * thread start anywhere: it replays the three bytes before its chunk from
 * SYNC0, where continuation bytes are skipped (at most three; a fourth
 * would be an error, which the thread before reports) and any other byte
 * acts as from ACCEPT.  So the state at the chunk's first byte is exact
 * whenever the input before it is valid.
 *
 * The same source compiles for the GPU (nvcc) and for the host (gcc); the
 * host suite checks the automaton against the oracle.
 */
#ifndef GPUTF_UTF8_DFA_H
#define GPUTF_UTF8_DFA_H

#include <stdint.h>
#include "utf8_scheme.h"   /* GPUTF_HD */

enum {
    GPUTF_DFA_ACCEPT = 0,
    GPUTF_DFA_NEED1 = 1,
    GPUTF_DFA_NEED2 = 2,
    GPUTF_DFA_NEED3 = 3,
    GPUTF_DFA_AFTER_E0 = 4,
    GPUTF_DFA_AFTER_ED = 5,
    GPUTF_DFA_AFTER_F0 = 6,
    GPUTF_DFA_AFTER_F4 = 7,
    GPUTF_DFA_REJECT = 8,
    GPUTF_DFA_SYNC0 = 9,
    GPUTF_DFA_SYNC1 = 10,
    GPUTF_DFA_SYNC2 = 11,
    GPUTF_DFA_STATES = 12,
    GPUTF_DFA_CLASSES = 12
};

/* Class of a byte: 0 ASCII; 1, 2, 3 continuation bytes 80-8F, 90-9F,
 * A0-BF; 4 never valid (C0, C1, F5-FF); 5 lead C2-DF; 6 E0; 7 E1-EC and
 * EE-EF; 8 ED; 9 F0; 10 F1-F3; 11 F4. */
GPUTF_HD uint32_t gputf_dfa_class(uint32_t b)
{
    if (b < 0x80) return 0;
    if (b < 0x90) return 1;
    if (b < 0xA0) return 2;
    if (b < 0xC0) return 3;
    if (b < 0xC2) return 4;
    if (b < 0xE0) return 5;
    if (b == 0xE0) return 6;
    if (b == 0xED) return 8;
    if (b < 0xF0) return 7;
    if (b == 0xF0) return 9;
    if (b < 0xF4) return 10;
    if (b == 0xF4) return 11;
    return 4;
}

/* Next state from state s on a byte of class c. */
GPUTF_HD uint32_t gputf_dfa_next(uint32_t s, uint32_t c)
{
    const int cont = c >= 1 && c <= 3;
    switch (s) {
    case GPUTF_DFA_SYNC0:
    case GPUTF_DFA_SYNC1:
    case GPUTF_DFA_SYNC2:
        if (cont) return s == GPUTF_DFA_SYNC2 ? GPUTF_DFA_ACCEPT : s + 1;
        /* fall through: a byte that is not a continuation starts over */
    case GPUTF_DFA_ACCEPT:
        switch (c) {
        case 0: return GPUTF_DFA_ACCEPT;
        case 5: return GPUTF_DFA_NEED1;
        case 6: return GPUTF_DFA_AFTER_E0;
        case 7: return GPUTF_DFA_NEED2;
        case 8: return GPUTF_DFA_AFTER_ED;
        case 9: return GPUTF_DFA_AFTER_F0;
        case 10: return GPUTF_DFA_NEED3;
        case 11: return GPUTF_DFA_AFTER_F4;
        default: return GPUTF_DFA_REJECT;   /* a continuation or a never-valid byte */
        }
    case GPUTF_DFA_NEED1: return cont ? GPUTF_DFA_ACCEPT : GPUTF_DFA_REJECT;
    case GPUTF_DFA_NEED2: return cont ? GPUTF_DFA_NEED1 : GPUTF_DFA_REJECT;
    case GPUTF_DFA_NEED3: return cont ? GPUTF_DFA_NEED2 : GPUTF_DFA_REJECT;
    case GPUTF_DFA_AFTER_E0: return c == 3 ? GPUTF_DFA_NEED1 : GPUTF_DFA_REJECT;                /* A0-BF */
    case GPUTF_DFA_AFTER_ED: return (c == 1 || c == 2) ? GPUTF_DFA_NEED1 : GPUTF_DFA_REJECT;   /* 80-9F */
    case GPUTF_DFA_AFTER_F0: return (c == 2 || c == 3) ? GPUTF_DFA_NEED2 : GPUTF_DFA_REJECT;   /* 90-BF */
    case GPUTF_DFA_AFTER_F4: return c == 1 ? GPUTF_DFA_NEED2 : GPUTF_DFA_REJECT;                /* 80-8F */
    default: return GPUTF_DFA_REJECT;
    }
}

/* A state inside a character (a thread runs on past its chunk's end until
 * the character it is in completes). */
GPUTF_HD int gputf_dfa_inside(uint32_t s)
{
    return s != GPUTF_DFA_ACCEPT && s != GPUTF_DFA_REJECT && s < GPUTF_DFA_SYNC0;
}

#endif
