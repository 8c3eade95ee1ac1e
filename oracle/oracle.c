/*
 * Scalar CPU oracle for validating UTF-8 <-> UTF-16LE transcoding.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * definition that the CUDA path is checked against.  Only the test suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load it; the
 * library's own code path never does.  It shares no code, header, table or
 * constant with the CUDA path.
 *
 * Everything here follows the format definitions of Section 3 ("The UTF-8 and
 * UTF-16 Formats") of Lemire & Mula, "Transcoding Billions of Unicode
 * Characters per Second with SIMD Instructions" (arXiv 2109.10433), which
 * restates RFC 3629 (UTF-8) and RFC 2781 (UTF-16):
 *   - Table 2 gives the byte length of each character range;
 *   - the UTF-8 paragraph gives the lead-byte prefixes 0 / 110 / 1110 / 11110,
 *     the continuation prefix 10, the big-endian placement of payload bits and
 *     the six validation rules;
 *   - the UTF-16 paragraph gives the surrogate-pair construction and its
 *     validation (a high unit D800-DBFF must be followed by a low unit
 *     DC00-DFFF, and a low unit must follow a high one).
 * The surrogate split used when encoding (subtract 0x10000, low ten bits under
 * 110111, high ten bits under 110110) is the one stated in the caption of
 * Fig. 4.
 *
 * Where the paper is silent the readings are:
 *   - the reported error offset is the start of the first character that cannot
 *     be decoded (its lead byte, or the stray continuation byte itself), in code
 *     units of the input encoding;
 *   - when several rules fail on one character, the class is taken in decoding
 *     order: a stray continuation (TOO_LONG) or a byte >= 0xF8 (HEADER_BITS) at
 *     the lead, then a missing continuation (TOO_SHORT), then OVERLONG,
 *     TOO_LARGE, SURROGATE;
 *   - UTF-16 has a single error class, SURROGATE, at the offending unit;
 *   - on error, `written` counts the output units of the valid prefix;
 *   - the two length functions are closed forms that do not validate;
 *   - no byte-order mark is detected or stripped; U+0000 is an ordinary
 *     character.
 */
#include <stdint.h>
#include <stddef.h>
#include <string.h>

/* Error classes (numbering fixed by the library's public interface). */
enum {
    ORC_OK = 0,
    ORC_HEADER_BITS = 1,      /* rule 1: byte 0xF8..0xFF                        */
    ORC_TOO_SHORT = 2,        /* rule 2: lead without enough continuation bytes */
    ORC_TOO_LONG = 3,         /* rule 3: continuation byte without a lead       */
    ORC_OVERLONG = 4,         /* rule 4: value fits in a shorter sequence       */
    ORC_TOO_LARGE = 5,        /* rule 5: value above U+10FFFF                   */
    ORC_SURROGATE = 6,        /* rule 6 (UTF-8) / unpaired surrogate (UTF-16)   */
    ORC_OUTPUT_TOO_SMALL = 7  /* next character does not fit in the output      */
};

typedef struct {
    int32_t error;
    int32_t reserved;
    uint64_t position;
    uint64_t written;
} oracle_result;

static int is_continuation(uint8_t b) { return b >= 0x80 && b <= 0xBF; }

/* ---------------------------------------------------------------------------
 * One UTF-8 decoding step at in[p] (Section 3, rules 1-6).
 * Returns the error class; on success stores the code point and the sequence
 * length in *cp and *len.
 * ------------------------------------------------------------------------- */
static int utf8_decode_one(const uint8_t *in, uint64_t n, uint64_t p,
                           uint32_t *cp, int *len)
{
    uint8_t b = in[p];
    int L;
    uint32_t v;

    if (b < 0x80) {                 /* leading bit 0: one-byte (ASCII) sequence */
        *cp = b;
        *len = 1;
        return ORC_OK;
    }
    if (b <= 0xBF)                  /* 10xxxxxx with no lead before it: rule 3 */
        return ORC_TOO_LONG;
    if (b >= 0xF8)                  /* five leading ones: rule 1 */
        return ORC_HEADER_BITS;

    if (b >= 0xF0) {                /* 11110xxx: 21 payload bits */
        L = 4;
        v = b & 0x07;
    } else if (b >= 0xE0) {         /* 1110xxxx: 16 payload bits */
        L = 3;
        v = b & 0x0F;
    } else {                        /* 110xxxxx: 11 payload bits */
        L = 2;
        v = b & 0x1F;
    }

    /* rule 2: the lead must be followed by L-1 continuation bytes */
    for (int k = 1; k < L; k++) {
        if (p + (uint64_t)k >= n || !is_continuation(in[p + k]))
            return ORC_TOO_SHORT;
    }
    /* big-endian payload: 6 bits from each continuation byte */
    for (int k = 1; k < L; k++)
        v = (v << 6) | (uint32_t)(in[p + k] & 0x3F);

    /* rule 4: shortest form only */
    if ((L == 2 && v <= 0x7F) || (L == 3 && v <= 0x7FF) || (L == 4 && v <= 0xFFFF))
        return ORC_OVERLONG;
    /* rule 5: below U+110000 */
    if (v > 0x10FFFF)
        return ORC_TOO_LARGE;
    /* rule 6: not a surrogate code point */
    if (v >= 0xD800 && v <= 0xDFFF)
        return ORC_SURROGATE;

    *cp = v;
    *len = L;
    return ORC_OK;
}

/* Number of UTF-16 units for a scalar value (Table 2: 2 bytes below U+10000,
 * 4 bytes, i.e. a surrogate pair, above). */
static int utf16_units_of(uint32_t cp) { return cp >= 0x10000 ? 2 : 1; }

/* Number of UTF-8 bytes for a scalar value (Table 2). */
static int utf8_bytes_of(uint32_t cp)
{
    if (cp <= 0x7F) return 1;
    if (cp <= 0x7FF) return 2;
    if (cp <= 0xFFFF) return 3;
    return 4;
}

/* Write cp as UTF-16 units (Section 3; surrogate split of the Fig. 4 caption). */
static void utf16_put(uint32_t cp, uint16_t *out)
{
    if (cp < 0x10000) {
        out[0] = (uint16_t)cp;
    } else {
        uint32_t x = cp - 0x10000;                 /* a 20-bit value */
        out[0] = (uint16_t)(0xD800 | (x >> 10));   /* 110110 + high ten bits */
        out[1] = (uint16_t)(0xDC00 | (x & 0x3FF)); /* 110111 + low ten bits */
    }
}

/* Write cp as UTF-8 bytes (Section 3: lead prefix, then 10xxxxxx bytes, most
 * significant payload bits first). */
static void utf8_put(uint32_t cp, uint8_t *out)
{
    int L = utf8_bytes_of(cp);
    if (L == 1) {
        out[0] = (uint8_t)cp;
        return;
    }
    static const uint8_t lead_prefix[5] = {0, 0, 0xC0, 0xE0, 0xF0};
    static const uint8_t lead_payload_mask[5] = {0, 0, 0x1F, 0x0F, 0x07};
    for (int k = L - 1; k >= 1; k--) {
        out[k] = (uint8_t)(0x80 | (cp & 0x3F));
        cp >>= 6;
    }
    out[0] = (uint8_t)(lead_prefix[L] | (cp & lead_payload_mask[L]));
}

/* ---------------------------------------------------------------------------
 * Public oracle entry points.
 * ------------------------------------------------------------------------- */

/* Encode one scalar value; returns its length, or 0 if cp is not a scalar
 * value (a surrogate, or above U+10FFFF). */
int oracle_encode_utf8(uint32_t cp, uint8_t *out)
{
    if (cp > 0x10FFFF || (cp >= 0xD800 && cp <= 0xDFFF)) return 0;
    utf8_put(cp, out);
    return utf8_bytes_of(cp);
}

int oracle_encode_utf16(uint32_t cp, uint16_t *out)
{
    if (cp > 0x10FFFF || (cp >= 0xD800 && cp <= 0xDFFF)) return 0;
    utf16_put(cp, out);
    return utf16_units_of(cp);
}

/* Validating UTF-8 -> UTF-16LE.  `out` may be NULL when cap == 0.  The output
 * of the valid prefix is written; on failure `position` is the start of the
 * first character that is invalid or does not fit. */
void oracle_utf8_to_utf16(const uint8_t *in, uint64_t n, uint16_t *out,
                          uint64_t cap, oracle_result *r)
{
    uint64_t p = 0, q = 0;
    while (p < n) {
        uint32_t cp = 0;
        int len = 0;
        int e = utf8_decode_one(in, n, p, &cp, &len);
        if (e != ORC_OK) {
            r->error = e;
            r->position = p;
            r->written = q;
            return;
        }
        int units = utf16_units_of(cp);
        if (q + (uint64_t)units > cap) {
            r->error = ORC_OUTPUT_TOO_SMALL;
            r->position = p;
            r->written = q;
            return;
        }
        utf16_put(cp, out + q);
        q += (uint64_t)units;
        p += (uint64_t)len;
    }
    r->error = ORC_OK;
    r->position = n;
    r->written = q;
}

/* One UTF-16 step at in[i]: returns the error class, the code point and the
 * number of units consumed (Section 3, surrogate pairs). */
static int utf16_decode_one(const uint16_t *in, uint64_t n, uint64_t i,
                            uint32_t *cp, int *len)
{
    uint16_t u = in[i];
    if (u < 0xD800 || u > 0xDFFF) {
        *cp = u;
        *len = 1;
        return ORC_OK;
    }
    if (u <= 0xDBFF && i + 1 < n && in[i + 1] >= 0xDC00 && in[i + 1] <= 0xDFFF) {
        /* ten bits from the high unit above ten bits from the low unit,
         * then add 0x10000 */
        uint32_t hi10 = u & 0x3FF;
        uint32_t lo10 = in[i + 1] & 0x3FF;
        *cp = ((hi10 << 10) | lo10) + 0x10000;
        *len = 2;
        return ORC_OK;
    }
    return ORC_SURROGATE;   /* lone low, or high not followed by low */
}

/* Validating UTF-16LE -> UTF-8. */
void oracle_utf16_to_utf8(const uint16_t *in, uint64_t n, uint8_t *out,
                          uint64_t cap, oracle_result *r)
{
    uint64_t i = 0, q = 0;
    while (i < n) {
        uint32_t cp = 0;
        int len = 0;
        int e = utf16_decode_one(in, n, i, &cp, &len);
        if (e != ORC_OK) {
            r->error = e;
            r->position = i;
            r->written = q;
            return;
        }
        int bytes = utf8_bytes_of(cp);
        if (q + (uint64_t)bytes > cap) {
            r->error = ORC_OUTPUT_TOO_SMALL;
            r->position = i;
            r->written = q;
            return;
        }
        utf8_put(cp, out + q);
        q += (uint64_t)bytes;
        i += (uint64_t)len;
    }
    r->error = ORC_OK;
    r->position = n;
    r->written = q;
}

void oracle_validate_utf8(const uint8_t *in, uint64_t n, oracle_result *r)
{
    uint64_t p = 0;
    r->written = 0;
    while (p < n) {
        uint32_t cp = 0;
        int len = 0;
        int e = utf8_decode_one(in, n, p, &cp, &len);
        if (e != ORC_OK) {
            r->error = e;
            r->position = p;
            return;
        }
        p += (uint64_t)len;
    }
    r->error = ORC_OK;
    r->position = n;
}

void oracle_validate_utf16(const uint16_t *in, uint64_t n, oracle_result *r)
{
    uint64_t i = 0;
    r->written = 0;
    while (i < n) {
        uint32_t cp = 0;
        int len = 0;
        int e = utf16_decode_one(in, n, i, &cp, &len);
        if (e != ORC_OK) {
            r->error = e;
            r->position = i;
            return;
        }
        i += (uint64_t)len;
    }
    r->error = ORC_OK;
    r->position = n;
}

/* UTF-16 length of UTF-8 input, without validation: every byte that is not a
 * continuation byte starts a character worth one unit, and a four-byte lead
 * (0xF0 and above) starts a character worth two (Table 2). */
uint64_t oracle_utf16_length_from_utf8(const uint8_t *in, uint64_t n)
{
    uint64_t total = 0;
    for (uint64_t p = 0; p < n; p++) {
        uint8_t b = in[p];
        if (!is_continuation(b)) total += 1;
        if (b >= 0xF0) total += 1;
    }
    return total;
}

/* UTF-8 length of UTF-16 input, without validation: 1, 2 or 3 bytes per unit
 * by value (Table 2), and 2 bytes for each surrogate unit, so that a pair
 * counts the 4 bytes of its character. */
uint64_t oracle_utf8_length_from_utf16(const uint16_t *in, uint64_t n)
{
    uint64_t total = 0;
    for (uint64_t i = 0; i < n; i++) {
        uint16_t u = in[i];
        if (u <= 0x7F) total += 1;
        else if (u <= 0x7FF) total += 2;
        else if (u >= 0xD800 && u <= 0xDFFF) total += 2;
        else total += 3;
    }
    return total;
}

/* ---------------------------------------------------------------------------
 * Loops over many strings, for the test suite (each string handled by the
 * single-string entry points above).
 * ------------------------------------------------------------------------- */

/* `count` strings of `width` bytes each, stored back to back. */
void oracle_validate_utf8_fixed(const uint8_t *in, uint64_t count, uint32_t width,
                                int32_t *err, uint64_t *pos)
{
    for (uint64_t k = 0; k < count; k++) {
        oracle_result r;
        oracle_validate_utf8(in + k * width, width, &r);
        err[k] = r.error;
        pos[k] = r.position;
    }
}

void oracle_validate_utf16_fixed(const uint16_t *in, uint64_t count, uint32_t width,
                                 int32_t *err, uint64_t *pos)
{
    for (uint64_t k = 0; k < count; k++) {
        oracle_result r;
        oracle_validate_utf16(in + k * width, width, &r);
        err[k] = r.error;
        pos[k] = r.position;
    }
}

/* Strings given by CSR offsets (in code units of their own encoding). */
void oracle_validate_utf8_csr(const uint8_t *in, const uint64_t *offsets, uint64_t count,
                              int32_t *err, uint64_t *pos)
{
    for (uint64_t k = 0; k < count; k++) {
        oracle_result r;
        oracle_validate_utf8(in + offsets[k], offsets[k + 1] - offsets[k], &r);
        err[k] = r.error;
        pos[k] = r.position;
    }
}
