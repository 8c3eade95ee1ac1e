/*
 * Test harness: runs the batched kernel's per-piece arithmetic
 * (batch_piece.h, compiled for the host from the same header batch.cu uses)
 * beside the CPU oracle, and counts the cases where they disagree.  Test
 * infrastructure only.
 *
 * UTF-16 -> UTF-8: a string u[0..L) is cut into pieces at the given points
 * (as chunk edges cut it); each piece is placed in a 32-unit chunk at an
 * offset that varies with the case, the rest of the chunk filled with other
 * strings' units, and worked by gputf_u16_unit_bits4 and gputf_u16_piece,
 * told whether the unit before / after the piece in its string is a high /
 * low surrogate.  Then:
 *   1. the pieces' bytes add up to the per-unit convention's total (a pair's
 *      4 bytes on its high half, 2 for a lone surrogate, Table 2 else);
 *   2. a valid string (oracle_validate_utf16) has no unit flagged, and its
 *      bytes equal the oracle's UTF-8 length;
 *   3. in an invalid string the first unit flagged, over the pieces in
 *      order, is the oracle's error position.
 * UTF-8 -> UTF-16: gputf_u8_lead_bits flags every byte value at every byte
 * position of a word as Table 2 says (a lead: not 10xxxxxx; a 4-byte lead:
 * 0xF0 and above), whatever the other bytes; and gputf_u8_piece_units of a
 * piece equals the oracle's UTF-16 length of its bytes.
 */
#include <pthread.h>
#include <stdint.h>
#include <string.h>

#include "oracle.c"
#include "batch_piece.h"

static int hi16(uint32_t u) { return (u & 0xFC00) == 0xD800; }
static int lo16(uint32_t u) { return (u & 0xFC00) == 0xDC00; }

/* 0 when the string passes, else the number of the failed check.  cuts: bit
 * b set when a chunk edge falls before unit b (1 <= b < L). */
static int check16(const uint16_t *u, int L, uint64_t cuts, const uint16_t *filler, int salt)
{
    uint64_t total = 0;
    long first_bad = -1;
    int a = 0;
    while (a < L) {
        int b = a + 1;
        while (b < L && !((cuts >> b) & 1)) b++;
        const int n = b - a;
        if (n > 32) return 9;
        const int j0 = (a * 5 + L + salt) % (33 - n);
        uint16_t ch[32];
        for (int k = 0; k < 32; k++) ch[k] = filler[(k + salt) % 8];
        memcpy(ch + j0, u + a, 2 * (size_t)n);
        uint32_t m80 = 0, m3 = 0, hi = 0, lo = 0;
        for (int g = 0; g < 8; g++) {
            const uint32_t w0 = ch[4 * g] | ((uint32_t)ch[4 * g + 1] << 16);
            const uint32_t w1 = ch[4 * g + 2] | ((uint32_t)ch[4 * g + 3] << 16);
            uint32_t x80, x3, xh, xl;
            gputf_u16_unit_bits4(w0, w1, &x80, &x3, &xh, &xl);
            m80 |= x80 << (4 * g);
            m3 |= x3 << (4 * g);
            hi |= xh << (4 * g);
            lo |= xl << (4 * g);
        }
        const int ph = a > 0 && hi16(u[a - 1]), nl = b < L && lo16(u[b]);
        uint32_t bad;
        total += gputf_u16_piece(m80, m3, hi, lo, j0, j0 + n, ph, nl, &bad);
        if (bad && first_bad < 0) first_bad = a + (__builtin_ctz(bad) - j0);
        a = b;
    }
    uint64_t conv = 0;
    for (int k = 0; k < L; k++) {
        const uint32_t prev = k ? u[k - 1] : 0, next = k + 1 < L ? u[k + 1] : 0, x = u[k];
        if (lo16(x) && hi16(prev)) continue;
        if (hi16(x) && lo16(next)) conv += 4;
        else conv += x < 0x80 ? 1 : ((x < 0x800 || hi16(x) || lo16(x)) ? 2 : 3);
    }
    if (total != conv) return 1;
    oracle_result r;
    oracle_validate_utf16(u, (uint64_t)L, &r);
    if (r.error == 0) {
        if (first_bad >= 0) return 2;
        if (oracle_utf8_length_from_utf16(u, (uint64_t)L) != total) return 2;
    } else if (first_bad != (long)r.position) {
        return 3;
    }
    return 0;
}

/* UTF-16 cases: count strings of width L (L units, then the cut mask as four
 * 16-bit words, then 8 filler units, then the salt). */
typedef struct {
    const uint16_t *data;
    uint64_t begin, end;
    int L;
    uint64_t mismatches, first_bad;
    int first_check;
} job16_t;

static void *run16(void *arg)
{
    job16_t *j = (job16_t *)arg;
    const int w = j->L + 4 + 8 + 1;
    for (uint64_t k = j->begin; k < j->end; k++) {
        const uint16_t *row = j->data + k * (uint64_t)w;
        const uint64_t cuts = (uint64_t)row[j->L] | ((uint64_t)row[j->L + 1] << 16) |
                              ((uint64_t)row[j->L + 2] << 32) | ((uint64_t)row[j->L + 3] << 48);
        const int r = check16(row, j->L, cuts, row + j->L + 4, row[j->L + 12]);
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

uint64_t piece16_check(const uint16_t *data, uint64_t count, int L, int threads, uint64_t *first_bad,
                       int *first_check)
{
    pthread_t t[64];
    job16_t jobs[64];
    if (threads < 1) threads = 1;
    if (threads > 64) threads = 64;
    for (int i = 0; i < threads; i++) {
        jobs[i] = (job16_t){data, count * (uint64_t)i / threads, count * (uint64_t)(i + 1) / threads, L, 0, 0, 0};
        pthread_create(&t[i], 0, run16, &jobs[i]);
    }
    uint64_t total = 0;
    *first_bad = 0;
    *first_check = 0;
    for (int i = 0; i < threads; i++) {
        pthread_join(t[i], 0);
        if (jobs[i].mismatches && !total) {
            *first_bad = jobs[i].first_bad;
            *first_check = jobs[i].first_check;
        }
        total += jobs[i].mismatches;
    }
    return total;
}

/* UTF-8: the lead bits of every byte value at every position of a word, the
 * other three bytes from `others` (count values); returns the number of
 * words flagged wrongly. */
uint64_t lead_bits_check(const uint8_t *others, int count)
{
    uint64_t bad = 0;
    for (int p = 0; p < 4; p++)
        for (int b = 0; b < 256; b++)
            for (int o = 0; o < count; o++) {
                uint32_t x = 0;
                for (int q = 0; q < 4; q++) x |= (uint32_t)(q == p ? b : others[(o + q) % count]) << (8 * q);
                uint32_t lead, lead4;
                gputf_u8_lead_bits(x, &lead, &lead4);
                for (int q = 0; q < 4; q++) {
                    const uint32_t v = (x >> (8 * q)) & 0xFF;
                    if (((lead >> q) & 1) != ((v & 0xC0) != 0x80) || ((lead4 >> q) & 1) != (v >= 0xF0)) {
                        bad++;
                        break;
                    }
                }
            }
    return bad;
}

/* UTF-8 pieces: each row holds 32 bytes, then the piece's start and end;
 * returns the number of rows whose piece units differ from the oracle's. */
uint64_t piece8_check(const uint8_t *rows, uint64_t count)
{
    uint64_t bad = 0;
    for (uint64_t k = 0; k < count; k++) {
        const uint8_t *row = rows + 34 * k;
        uint32_t lb = 0, fb = 0;
        for (int w = 0; w < 8; w++) {
            uint32_t x = 0, l4, f4;
            for (int q = 0; q < 4; q++) x |= (uint32_t)row[4 * w + q] << (8 * q);
            gputf_u8_lead_bits(x, &l4, &f4);
            lb |= l4 << (4 * w);
            fb |= f4 << (4 * w);
        }
        const int j = row[32], pe = row[33];
        if (gputf_u8_piece_units(lb, fb, j, pe) != oracle_utf16_length_from_utf8(row + j, (uint64_t)(pe - j))) bad++;
    }
    return bad;
}
