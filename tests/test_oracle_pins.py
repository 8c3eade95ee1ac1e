"""Pins for the CPU oracle, against things other than the oracle itself.

- the worked example and Table 2 ranges printed in the paper (tests/golden/);
- CPython's strict UTF-8 / UTF-16LE codecs, an independent library routine,
  on every Unicode scalar value and on corrupted text (error offsets);
- brute-force validity of every 1-, 2- and 3-byte string and of every 4-byte
  string with a lead byte 0xF0-0xF7, where the valid set is built from
  CPython's encodings of individual characters;
- the closed-form validity of UTF-16 unit pairs (Section 3: a high unit must be
  followed by a low one and conversely);
- the error classes labelled on generated error tokens.
"""
import os

import numpy as np
import pytest

import oracle as O
import workloads as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append([c.strip() for c in line.split("|")])
    return rows


ALL_SCALARS = np.concatenate([np.arange(0, 0xD800), np.arange(0xE000, 0x110000)]).astype(np.uint32)


def cps_to_str(cps):
    return np.asarray(cps, dtype="<u4").tobytes().decode("utf-32-le")


# ---------------------------------------------------------------------------
# Values printed in the paper
# ---------------------------------------------------------------------------
def test_worked_example_u93e1():
    rows = read_golden("paper_examples.txt")
    assert rows
    for cp_hex, u8_hex, u16_hex, _cite in rows:
        cp = int(cp_hex, 16)
        u8 = bytes.fromhex(u8_hex)
        u16 = [int(x, 16) for x in u16_hex.split()]
        assert O.encode_utf8(cp) == u8
        assert O.encode_utf16(cp) == u16
        r, out = O.utf8_to_utf16(u8)
        assert r == (O.OK, len(u8), len(u16)) and out.tolist() == u16
        r, out = O.utf16_to_utf8(np.array(u16, dtype=np.uint16))
        assert r == (O.OK, len(u16), len(u8)) and out.tobytes() == u8
    # the bit groups printed for U+93E1: 1110|1001, 10|001111, 10|100001
    assert [format(b, "08b") for b in O.encode_utf8(0x93E1)] == ["11101001", "10001111", "10100001"]


def test_table2_lengths_every_scalar():
    rows = read_golden("table2_ranges.txt")
    covered = 0
    for lo_hex, hi_hex, n8, n16, _cite in rows:
        lo, hi, n8, n16 = int(lo_hex, 16), int(hi_hex, 16), int(n8), int(n16)
        cps = np.arange(lo, hi + 1, dtype=np.uint32)
        covered += cps.size
        u16 = W.to_utf16(cps)
        # every character of the range costs n16 bytes in UTF-16 ...
        assert u16.size * 2 == cps.size * n16
        # ... and the oracle writes exactly n8 UTF-8 bytes for each of them
        r, out = O.utf16_to_utf8(u16)
        assert r == (O.OK, u16.size, cps.size * n8)
        for cp in [lo, hi, (lo + hi) // 2]:
            assert len(O.encode_utf8(cp)) == n8
            assert len(O.encode_utf16(cp)) * 2 == n16
    assert covered == ALL_SCALARS.size == 1112064
    # Section 3: U+D800-DFFF are forbidden, and nothing lies above U+10FFFF
    for cp in [0xD800, 0xDBFF, 0xDC00, 0xDFFF, 0x110000, 0x1FFFFF]:
        assert O.encode_utf8(cp) == b"" and O.encode_utf16(cp) == []


def test_surrogate_pair_construction():
    g = {k: v for k, v, _c in read_golden("surrogates.txt")}
    hi_units = np.arange(int(g["high_first"], 16), int(g["high_last"], 16) + 1, dtype=np.uint16)
    lo_units = np.arange(int(g["low_first"], 16), int(g["low_last"], 16) + 1, dtype=np.uint16)
    pairs = np.stack(np.meshgrid(hi_units, lo_units, indexing="ij"), axis=-1).reshape(-1)
    r, u8 = O.utf16_to_utf8(pairs)
    assert r.error == O.OK and r.written == 4 * hi_units.size * lo_units.size
    values = np.frombuffer(u8.tobytes().decode("utf-8").encode("utf-32-le"), dtype="<u4")
    # every (high, low) pair in lexicographic order gives the next value of
    # U+10000..U+10FFFF: the low unit holds the 10 low bits, the high unit the
    # next 10, and 0x10000 is added
    assert values[0] == int(g["supplementary_first"], 16) == int(g["offset"], 16)
    assert values[-1] == int(g["supplementary_last"], 16)
    assert np.array_equal(values, np.arange(0x10000, 0x110000, dtype=np.uint32))
    # Fig. 4: low unit = 110111 + low ten bits, high unit = 110110 + high ten bits
    for cp in [0x10000, 0x1F600, 0x10FFFF]:
        hi, lo = O.encode_utf16(cp)
        x = cp - 0x10000
        assert format(hi >> 10, "06b") == g["high_prefix_bits"] and (hi & 0x3FF) == x >> 10
        assert format(lo >> 10, "06b") == g["low_prefix_bits"] and (lo & 0x3FF) == x & 0x3FF


# ---------------------------------------------------------------------------
# CPython's codecs as an independent routine
# ---------------------------------------------------------------------------
def test_round_trip_every_scalar_value_matches_cpython():
    s = cps_to_str(ALL_SCALARS)
    u8 = np.frombuffer(s.encode("utf-8"), dtype=np.uint8)
    u16 = np.frombuffer(s.encode("utf-16-le"), dtype="<u2")
    r, out16 = O.utf8_to_utf16(u8)
    assert r == (O.OK, u8.size, u16.size)
    assert np.array_equal(out16, u16)
    r, out8 = O.utf16_to_utf8(u16)
    assert r == (O.OK, u16.size, u8.size)
    assert np.array_equal(out8, u8)
    assert O.utf16_length_from_utf8(u8) == u16.size
    assert O.utf8_length_from_utf16(u16) == u8.size
    # one character at a time, on a sample spread over the whole range
    for cp in ALL_SCALARS[::997].tolist() + [0, 0x7F, 0x80, 0x7FF, 0x800, 0xD7FF, 0xE000,
                                             0xFFFF, 0x10000, 0x10FFFF]:
        assert O.encode_utf8(cp) == chr(cp).encode("utf-8")
        assert O.encode_utf16(cp) == list(np.frombuffer(chr(cp).encode("utf-16-le"), "<u2"))


def cpython_utf8_start(b: bytes):
    try:
        b.decode("utf-8")
        return None
    except UnicodeDecodeError as e:
        return e.start


def cpython_utf16_start(units: np.ndarray):
    try:
        units.astype("<u2").tobytes().decode("utf-16-le")
        return None
    except UnicodeDecodeError as e:
        return e.start // 2


def _valid_mask_short(length):
    """Valid UTF-8 strings of `length` bytes, as a bool mask over all 256**length
    strings (big-endian index), built from CPython's encodings of characters."""
    by_len = {1: [], 2: [], 3: []}
    for cp in ALL_SCALARS[ALL_SCALARS < 0x10000].tolist():
        e = chr(cp).encode("utf-8")
        by_len[len(e)].append(int.from_bytes(e, "big"))
    by_len = {k: np.array(v, dtype=np.int64) for k, v in by_len.items()}

    def seqs(total):   # all concatenations of characters with `total` bytes
        if total == 0:
            return np.zeros(1, dtype=np.int64)
        out = []
        for first in (1, 2, 3):
            if first <= total:
                rest = seqs(total - first)
                out.append((by_len[first][:, None] << (8 * (total - first)) | rest[None, :]).ravel())
        return np.concatenate(out)

    mask = np.zeros(256 ** length, dtype=bool)
    mask[seqs(length)] = True
    return mask


@pytest.mark.parametrize("length", [1, 2, 3])
def test_every_short_utf8_string(length):
    idx = np.arange(256 ** length, dtype=np.int64)
    strings = np.stack([(idx >> (8 * (length - 1 - k))) & 0xFF for k in range(length)],
                       axis=1).astype(np.uint8)
    err, pos = O.validate_utf8_fixed(strings)
    valid = _valid_mask_short(length)
    assert np.array_equal(err == O.OK, valid)
    assert np.all(pos[valid] == length)
    # error offsets against CPython: all invalid strings up to 2 bytes, a
    # sample of the 3-byte ones
    bad = np.nonzero(~valid)[0]
    if bad.size > 60000:
        bad = np.random.default_rng(7).choice(bad, 60000, replace=False)
    for i in bad.tolist():
        assert int(pos[i]) == cpython_utf8_start(strings[i].tobytes())


def test_every_four_byte_string_with_a_four_byte_lead():
    four = ALL_SCALARS[ALL_SCALARS >= 0x10000]
    enc = np.frombuffer(cps_to_str(four).encode("utf-8"), dtype=np.uint8).reshape(-1, 4)
    enc_idx = (enc[:, 0].astype(np.int64) << 24 | enc[:, 1].astype(np.int64) << 16
               | enc[:, 2].astype(np.int64) << 8 | enc[:, 3])
    tails = np.arange(1 << 24, dtype=np.int64)
    rng = np.random.default_rng(11)
    for lead in range(0xF0, 0xF8):
        strings = np.empty((1 << 24, 4), dtype=np.uint8)
        strings[:, 0] = lead
        strings[:, 1] = tails >> 16
        strings[:, 2] = (tails >> 8) & 0xFF
        strings[:, 3] = tails & 0xFF
        err, pos = O.validate_utf8_fixed(strings)
        valid = np.zeros(1 << 24, dtype=bool)
        mine = enc_idx[(enc_idx >> 24) == lead] & 0xFFFFFF
        valid[mine] = True
        assert np.array_equal(err == O.OK, valid), hex(lead)
        assert np.all(pos[~valid] == 0)   # the first character starts at the lead
        for i in rng.choice(np.nonzero(~valid)[0], 2000, replace=False).tolist():
            assert cpython_utf8_start(strings[i].tobytes()) == 0


def test_utf16_units_and_pairs_closed_form():
    allu = np.arange(1 << 16, dtype=np.uint16)
    reps = np.array([0, 0x41, 0x7F, 0x80, 0x7FF, 0x800, 0xD7FF, 0xD800, 0xDA12, 0xDBFF,
                     0xDC00, 0xDE34, 0xDFFF, 0xE000, 0xFFFD, 0xFFFF], dtype=np.uint16)

    def hi(x):
        return (x >= 0xD800) & (x <= 0xDBFF)

    def lo(x):
        return (x >= 0xDC00) & (x <= 0xDFFF)

    # single units: valid iff not in D800-DFFF (Section 3)
    err, pos = O.validate_utf16_fixed(allu[:, None])
    assert np.array_equal(err == O.OK, ~(hi(allu) | lo(allu)))
    a = np.concatenate([np.repeat(allu, reps.size), np.tile(reps, allu.size)])
    b = np.concatenate([np.tile(reps, allu.size), np.repeat(allu, reps.size)])
    err, pos = O.validate_utf16_fixed(np.stack([a, b], axis=1))
    sa, sb = hi(a) | lo(a), hi(b) | lo(b)
    pair = hi(a) & lo(b)
    valid = (~sa & ~sb) | pair
    assert np.array_equal(err == O.OK, valid)
    expect_pos = np.where(valid, 2, np.where(sa & ~pair, 0, 1))
    assert np.array_equal(pos.astype(np.int64), expect_pos)
    assert np.all(err[~valid] == O.SURROGATE)
    for i in np.random.default_rng(5).choice(np.nonzero(~valid)[0], 3000, replace=False).tolist():
        assert cpython_utf16_start(np.array([a[i], b[i]])) == int(pos[i])


def _corrupt(rng, data, nflips):
    d = data.copy()
    for _ in range(nflips):
        i = int(rng.integers(0, d.size))
        d[i] = int(rng.integers(0, 256 if d.dtype == np.uint8 else 65536))
    return d


@pytest.mark.parametrize("mix", [W.MIX_LATIN_CYRILLIC, W.MIX_FOUR_BYTE_HEAVY, W.SCRIPT_CJK,
                                 W.SCRIPT_MIXED])
def test_error_offsets_match_cpython_on_corrupted_text(mix):
    rng = np.random.default_rng(3)
    for trial in range(300):
        text = W.utf8_text(1000 + trial, int(rng.integers(1, 400)), mix)
        bad = _corrupt(rng, text, int(rng.integers(0, 3)))
        r = O.validate_utf8(bad)
        start = cpython_utf8_start(bad.tobytes())
        assert r.position == (bad.size if start is None else start)
        assert (r.error == O.OK) == (start is None)
        r2, out = O.utf8_to_utf16(bad)
        assert (r2.error, r2.position) == (r.error, r.position)
        prefix16 = np.frombuffer(bad[:r.position].tobytes().decode("utf-8").encode("utf-16-le"), "<u2")
        assert r2.written == prefix16.size and np.array_equal(out, prefix16)

        t16 = W.utf16_text(2000 + trial, int(rng.integers(1, 200)), mix)
        bad16 = t16.copy()
        for _ in range(int(rng.integers(0, 3))):
            bad16[int(rng.integers(0, bad16.size))] = int(rng.integers(0xD700, 0xE100))
        r = O.validate_utf16(bad16)
        start = cpython_utf16_start(bad16)
        assert r.position == (bad16.size if start is None else start)
        r2, out = O.utf16_to_utf8(bad16)
        assert (r2.error, r2.position) == (r.error, r.position)
        prefix8 = bad16[:r.position].astype("<u2").tobytes().decode("utf-16-le").encode("utf-8")
        assert out.tobytes() == prefix8


# ---------------------------------------------------------------------------
# Error classes: generated tokens carry their class as a label
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_injected_error_tokens_first_error_and_class(seed):
    et = W.utf8_error_text(seed, 256 * 1024, W.MIX_FOUR_BYTE_HEAVY, mean_gap=4096,
                           kinds=W.UTF8_TOKEN_KINDS + ("header",))
    assert len(et.tokens) > 20
    r = O.validate_utf8(et.data)
    assert (r.error, r.position) == (et.tokens[0][2], et.tokens[0][0])
    for k, (off, _ln, cls) in enumerate(et.tokens):
        d = et.repaired_before(k)
        r = O.validate_utf8(d)
        assert (r.error, r.position) == (cls, off), k
        assert cpython_utf8_start(d.tobytes()) == off
    repaired = et.repaired_before(len(et.tokens))
    assert O.validate_utf8(repaired) == (O.OK, repaired.size, 0)


# The readings for several failing rules on one character (decoding order).
PRECEDENCE = [
    ("C0 41", O.TOO_SHORT, 0), ("C0 80", O.OVERLONG, 0), ("C1 BF", O.OVERLONG, 0),
    ("E0 80 41", O.TOO_SHORT, 0), ("E0 9F BF", O.OVERLONG, 0), ("F0 8F BF BF", O.OVERLONG, 0),
    ("F5 41", O.TOO_SHORT, 0), ("F5 80 80 80", O.TOO_LARGE, 0), ("F4 90 80 80", O.TOO_LARGE, 0),
    ("F7 BF BF BF", O.TOO_LARGE, 0), ("ED A0 80", O.SURROGATE, 0), ("ED BF BF", O.SURROGATE, 0),
    ("F8", O.HEADER_BITS, 0), ("FF 80", O.HEADER_BITS, 0), ("80", O.TOO_LONG, 0),
    ("41 80", O.TOO_LONG, 1), ("41 E9 8F", O.TOO_SHORT, 1), ("E9 8F A1 BF", O.TOO_LONG, 3),
    ("F0 90 80", O.TOO_SHORT, 0), ("C2", O.TOO_SHORT, 0), ("", O.OK, 0),
    ("ED 9F BF", O.OK, 3), ("EE 80 80", O.OK, 3), ("F4 8F BF BF", O.OK, 4), ("00", O.OK, 1),
]


@pytest.mark.parametrize("hexstr,cls,pos", PRECEDENCE)
def test_precedence_readings(hexstr, cls, pos):
    r = O.validate_utf8(bytes.fromhex(hexstr))
    assert (r.error, r.position) == (cls, pos)
    if cls != O.OK:
        assert cpython_utf8_start(bytes.fromhex(hexstr)) == pos


# ---------------------------------------------------------------------------
# Length functions and output capacity
# ---------------------------------------------------------------------------
def test_length_functions_match_encoded_lengths_and_add_up():
    rng = np.random.default_rng(9)
    for mix in [W.MIX_LATIN_CYRILLIC, W.MIX_CJK_EMOJI, W.MIX_FOUR_BYTE_HEAVY, W.SCRIPT_MIXED]:
        cps = W.draw_chars(rng, mix, 5000, "utf8")
        s = cps_to_str(cps)
        u8 = np.frombuffer(s.encode("utf-8"), np.uint8)
        u16 = np.frombuffer(s.encode("utf-16-le"), "<u2")
        assert O.utf16_length_from_utf8(u8) == u16.size
        assert O.utf8_length_from_utf16(u16) == u8.size
    # on arbitrary input they are sums over code units: splitting anywhere adds up
    for _ in range(50):
        b = rng.integers(0, 256, int(rng.integers(0, 300))).astype(np.uint8)
        k = int(rng.integers(0, b.size + 1))
        assert O.utf16_length_from_utf8(b) == O.utf16_length_from_utf8(b[:k]) + O.utf16_length_from_utf8(b[k:])
        u = rng.integers(0, 65536, int(rng.integers(0, 300))).astype(np.uint16)
        k = int(rng.integers(0, u.size + 1))
        assert O.utf8_length_from_utf16(u) == O.utf8_length_from_utf16(u[:k]) + O.utf8_length_from_utf16(u[k:])


def test_output_capacity_stops_at_first_character_that_does_not_fit():
    rng = np.random.default_rng(13)
    cps = W.draw_chars(rng, W.SCRIPT_MIXED, 120, "utf8")
    s = cps_to_str(cps)
    u8 = np.frombuffer(s.encode("utf-8"), np.uint8)
    u16 = np.frombuffer(s.encode("utf-16-le"), "<u2")
    n8 = [len(c.encode("utf-8")) for c in s]
    n16 = [len(c.encode("utf-16-le")) // 2 for c in s]
    c8 = np.concatenate([[0], np.cumsum(n8)])
    c16 = np.concatenate([[0], np.cumsum(n16)])
    for cap in range(0, u16.size + 2):
        r, out = O.utf8_to_utf16(u8, cap=cap)
        if cap >= u16.size:
            assert r == (O.OK, u8.size, u16.size)
        else:
            k = int(np.searchsorted(c16, cap, side="right")) - 1   # characters that fit
            assert r == (O.OUTPUT_TOO_SMALL, int(c8[k]), int(c16[k]))
            assert np.array_equal(out, u16[:c16[k]])
    for cap in range(0, u8.size + 2):
        r, out = O.utf16_to_utf8(u16, cap=cap)
        if cap >= u8.size:
            assert r == (O.OK, u16.size, u8.size)
        else:
            k = int(np.searchsorted(c8, cap, side="right")) - 1
            assert r == (O.OUTPUT_TOO_SMALL, int(c16[k]), int(c8[k]))
            assert out.tobytes() == u8[:c8[k]].tobytes()


# ---------------------------------------------------------------------------
# UTF-16BE: CPython's utf-16-be codec as the independent routine
# ---------------------------------------------------------------------------
def test_utf16be_every_scalar_value_matches_cpython():
    s = cps_to_str(ALL_SCALARS)
    u8 = np.frombuffer(s.encode("utf-8"), dtype=np.uint8)
    be = np.frombuffer(s.encode("utf-16-be"), dtype=">u2").astype(np.uint16)   # units as stored in memory
    be_mem = np.frombuffer(s.encode("utf-16-be"), dtype=np.uint16)
    assert not np.array_equal(be, be_mem)
    r, out16 = O.utf8_to_utf16be(u8)
    assert r == (O.OK, u8.size, be_mem.size)
    assert out16.tobytes() == s.encode("utf-16-be")
    r, out8 = O.utf16be_to_utf8(be_mem)
    assert r == (O.OK, be_mem.size, u8.size) and out8.tobytes() == u8.tobytes()
    assert O.validate_utf16be(be_mem) == (O.OK, be_mem.size, 0)
    assert O.utf8_length_from_utf16be(be_mem) == u8.size


def test_utf16be_error_offsets_match_cpython():
    rng = np.random.default_rng(17)
    for trial in range(300):
        t16 = W.utf16_text(3000 + trial, int(rng.integers(1, 200)), W.SCRIPT_MIXED)
        bad = t16.copy()
        for _ in range(int(rng.integers(0, 3))):
            bad[int(rng.integers(0, bad.size))] = int(rng.integers(0xD700, 0xE100))
        mem = np.frombuffer(bad.astype(">u2").tobytes(), dtype=np.uint16)   # big-endian storage
        try:
            mem.tobytes().decode("utf-16-be")
            start = None
        except UnicodeDecodeError as e:
            start = e.start // 2
        r = O.validate_utf16be(mem)
        assert r.position == (bad.size if start is None else start)
        assert (r.error == O.OK) == (start is None)
        r2, out = O.utf16be_to_utf8(mem)
        assert (r2.error, r2.position) == (r.error, r.position)
        assert out.tobytes() == mem[:r.position].tobytes().decode("utf-16-be").encode("utf-8")
