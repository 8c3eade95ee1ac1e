"""Derive the three 16-entry UTF-8 error tables from the validation rules.

The UTF-8 validation rules 1-6 of Section 3 of the paper are re-expressed as
"pair terms": conditions on a byte pair (p, c), with p the byte before c, of
the form  p>>4 in H1  and  p&15 in L1  and  c>>4 in H3.  A term of that product
form can be evaluated with one lookup per factor, ANDed: table T1 indexed by
p>>4, T2 by p&15, T3 by c>>4, each term owning one bit of the table bytes.

Two terms share a bit only when every cross combination of their factor sets
is itself an error; the two merged bits below are checked for that.

TWO_CONTS (bit 7) is not an error by itself: byte c must be a continuation
byte exactly when a three- or four-byte lead sits two or three bytes back, so
the kernel compares that bit with the lead test on the bytes before p.

Run as a script to (re)write utf8_tables.h next to this file.
"""
import os

ALL = set(range(16))
LEAD = {0xC, 0xD, 0xE, 0xF}
ASCII = set(range(8))
CONT = {0x8, 0x9, 0xA, 0xB}

# (bit, name, H1 = p>>4, L1 = p&15, H3 = c>>4, reason)
TERMS = [
    (0x01, "TOO_SHORT", LEAD, ALL, ASCII | LEAD,
     "rule 2: a lead byte must be followed by a continuation byte"),
    (0x02, "TOO_LONG", ASCII, ALL, CONT,
     "rule 3: a continuation byte may not follow an ASCII byte"),
    (0x04, "OVERLONG_2", {0xC}, {0x0, 0x1}, CONT,
     "rule 4: C0 and C1 leads only encode values below U+0080"),
    (0x08, "OVERLONG_3", {0xE}, {0x0}, {0x8, 0x9},
     "rule 4: E0 followed by 80..9F encodes a value below U+0800"),
    (0x10, "SURROGATE", {0xE}, {0xD}, {0xA, 0xB},
     "rule 6: ED followed by A0..BF encodes U+D800..DFFF"),
    (0x20, "OVERLONG_4_TOO_LARGE", {0xF}, {0x0} | set(range(5, 16)), {0x8},
     "rule 4: F0 followed by 80..8F is below U+10000; rules 1 and 5: F5..FF never start a character"),
    (0x40, "TOO_LARGE", {0xF}, set(range(4, 16)), {0x9, 0xA, 0xB},
     "rule 5: F4 followed by 90..BF is above U+10FFFF; rules 1 and 5: F5..FF never start a character"),
    (0x80, "TWO_CONTS", CONT, ALL, CONT,
     "rules 2 and 3: a continuation after a continuation, checked against the leads further back"),
]


def pair_is_error(p: int, c: int) -> bool:
    """Is the pair (p, c) wrong whatever comes before p?  Used to check that
    each term (all cross combinations included) only flags real errors."""
    if p < 0x80:                       # ASCII: only a continuation is wrong
        return 0x80 <= c <= 0xBF
    if p <= 0xBF:                      # continuation: depends on bytes further back
        return False
    if p in (0xC0, 0xC1) or p >= 0xF5:
        return True                    # never part of a valid sequence
    lo, hi = 0x80, 0xBF                # allowed range of the byte after a lead
    if p == 0xE0:
        lo = 0xA0
    elif p == 0xED:
        hi = 0x9F
    elif p == 0xF0:
        lo = 0x90
    elif p == 0xF4:
        hi = 0x8F
    return not (lo <= c <= hi)


def tables():
    t1, t2, t3 = [0] * 16, [0] * 16, [0] * 16
    for bit, _name, h1, l1, h3, _why in TERMS:
        for i in h1:
            t1[i] |= bit
        for i in l1:
            t2[i] |= bit
        for i in h3:
            t3[i] |= bit
    return t1, t2, t3


def check_terms():
    """Every (p, c) flagged by an error term is a wrong pair, and every wrong
    pair with a lead or ASCII first byte is flagged by some error term."""
    t1, t2, t3 = tables()
    for p in range(256):
        for c in range(256):
            e = t1[p >> 4] & t2[p & 15] & t3[c >> 4] & 0x7F
            if e:
                assert pair_is_error(p, c), (hex(p), hex(c), hex(e))
            elif not (0x80 <= p <= 0xBF):
                assert not pair_is_error(p, c), (hex(p), hex(c))


def pack(t):
    """Four little-endian words: entries 0-3, 4-7, 8-11, 12-15."""
    return [sum(t[4 * w + k] << (8 * k) for k in range(4)) for w in range(4)]


def header_text() -> str:
    t1, t2, t3 = tables()
    lines = [
        "/* Generated by gen_utf8_tables.py from the UTF-8 validation rules of",
        " * Section 3 of the paper; do not edit by hand.",
        " *",
        " * Error-class bits of the three 16-entry tables (one per bit):",
    ]
    for bit, name, _h1, _l1, _h3, why in TERMS:
        lines.append(f" *   0x{bit:02X} {name:<22} {why}")
    lines += [
        " *",
        " * T1 is indexed by the high nibble of the previous byte, T2 by its low",
        " * nibble and T3 by the high nibble of the current byte; each table is",
        " * stored as four words holding entries 0-3, 4-7, 8-11, 12-15.",
        " */",
        "#ifndef GPUTF_UTF8_TABLES_H",
        "#define GPUTF_UTF8_TABLES_H",
    ]
    for name, t in (("T1", t1), ("T2", t2), ("T3", t3)):
        for w, v in enumerate(pack(t)):
            lines.append(f"#define GPUTF_{name}_W{w} 0x{v:08X}u")
    lines.append("#define GPUTF_TWO_CONTS 0x80u")
    lines.append("#endif")
    return "\n".join(lines) + "\n"


if __name__ == "__main__":
    check_terms()
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "utf8_tables.h")
    with open(path, "w") as f:
        f.write(header_text())
    print("wrote", path)
