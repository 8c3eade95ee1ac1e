"""Proof, on the host, of the batched kernel's per-piece arithmetic.

The batched kernel works a thread's chunk one string piece at a time from
bit masks over the chunk (csrc/batch_piece.h).  tests/native/batch_piece_check.c
compiles that header for the CPU and checks it beside the oracle:
  - UTF-16 -> UTF-8: every string of up to 4 units over a set holding every
    class boundary, cut into pieces at every combination of points, every
    string of 5 units with four cut patterns, and random strings of up to 40
    units with random cuts, each piece placed in a 32-unit chunk among other
    strings' units (ASCII, high or low surrogates).  The pieces' bytes add up
    to the kernel's per-unit convention and, for a valid string, to the
    oracle's UTF-8 length; the first unit flagged is the oracle's error
    position, and a valid string has none;
  - UTF-8 -> UTF-16: the lead and 4-byte-lead bits of every byte value at
    every position of a word, and random pieces' units against the oracle's
    UTF-16 length.
Planted mistakes in copies of the header each fail the proof.
"""
import ctypes
import itertools
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2109_10433_gb300", "csrc")

SYMS = np.array([0x0041, 0x007F, 0x0080, 0x07FF, 0x0800, 0xD7FF, 0xE000, 0xFFFF,
                 0xD800, 0xDBFF, 0xDC00, 0xDFFF], dtype=np.uint16)
FILLERS = [[0x0041] * 8, [0xD800] * 8, [0xDC00] * 8, [0xD800, 0xDC00, 0xDC00, 0xD800, 0x0041, 0xDBFF, 0xDFFF, 0x4E00]]
BYTES = np.array([0x00, 0x41, 0x7F, 0x80, 0xBF, 0xC0, 0xC2, 0xDF, 0xE0, 0xED, 0xEF, 0xF0, 0xF4, 0xF5, 0xFF],
                 dtype=np.uint8)


def build_checker(out_dir, csrc=CSRC):
    out = os.path.join(str(out_dir), "batch_piece_check.so")
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared",
                           "-I" + os.path.join(ROOT, "oracle"), "-I" + csrc, "-o", out,
                           os.path.join(ROOT, "tests", "native", "batch_piece_check.c"), "-lpthread"])
    lib = ctypes.CDLL(out)
    lib.piece16_check.restype = ctypes.c_uint64
    lib.piece16_check.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                  ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_int)]
    lib.lead_bits_check.restype = ctypes.c_uint64
    lib.lead_bits_check.argtypes = [ctypes.c_void_p, ctypes.c_int]
    lib.piece8_check.restype = ctypes.c_uint64
    lib.piece8_check.argtypes = [ctypes.c_void_p, ctypes.c_uint64]
    return lib


def rows16(strings, cuts, salt):
    """Rows of the UTF-16 checker: units, the cut mask as four words, the
    filler, the salt; one row per (string, cut mask, filler)."""
    n, L = strings.shape
    out = []
    for f, filler in enumerate(FILLERS):
        r = np.empty((n * len(cuts), L + 13), dtype=np.uint16)
        r[:, :L] = np.repeat(strings, len(cuts), axis=0)
        c = np.tile(np.asarray(cuts, dtype=np.uint64), n)
        for q in range(4):
            r[:, L + q] = (c >> np.uint64(16 * q)) & np.uint64(0xFFFF)
        r[:, L + 4:L + 12] = filler
        r[:, L + 12] = (salt + f) % 8
        out.append(r)
    return np.concatenate(out)


def run16(lib, rows, L):
    fb, fc = ctypes.c_uint64(), ctypes.c_int()
    rows = np.ascontiguousarray(rows)
    m = lib.piece16_check(rows.ctypes.data, rows.shape[0], L, max(1, min(8, os.cpu_count() or 1)),
                          ctypes.byref(fb), ctypes.byref(fc))
    return m, (rows[fb.value].tolist() if m else None), fc.value


def utf16_cases():
    rng = np.random.default_rng(41)
    for L in range(1, 5):
        strings = np.array(list(itertools.product(SYMS, repeat=L)), dtype=np.uint16)
        yield L, rows16(strings, [c << 1 for c in range(1 << (L - 1))], L)
    strings = np.array(list(itertools.product(SYMS, repeat=5)), dtype=np.uint16)
    yield 5, rows16(strings, [0, 0b11110, 0b00100, 0b01010], 5)
    for L in (7, 16, 33, 40):
        s = rng.choice(SYMS, size=(4000, L)).astype(np.uint16)
        cuts = [int(c) << 1 for c in rng.integers(0, 1 << min(L - 1, 62), size=6, dtype=np.uint64)]
        yield L, rows16(s, cuts, L)


def utf8_rows():
    rng = np.random.default_rng(43)
    count = 100_000
    rows = np.empty((count, 34), dtype=np.uint8)
    rows[:, :32] = rng.choice(np.concatenate([BYTES, rng.integers(0, 256, 64).astype(np.uint8)]), size=(count, 32))
    j = rng.integers(0, 32, count)
    pe = j + 1 + (rng.random(count) * (32 - j)).astype(np.int64)
    rows[:, 32] = j
    rows[:, 33] = np.minimum(pe, 32)
    return rows


def failures(lib):
    """The first failing case, or None."""
    for L, rows in utf16_cases():
        m, bad, check = run16(lib, rows, L)
        if m:
            return ("utf16", L, check, bad)
    if lib.lead_bits_check(BYTES.ctypes.data, BYTES.size):
        return ("lead bits",)
    rows = utf8_rows()
    if lib.piece8_check(rows.ctypes.data, rows.shape[0]):
        return ("utf8 pieces",)
    return None


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    return build_checker(tmp_path_factory.mktemp("batchpiece"))


def test_batch_piece_arithmetic_matches_oracle(checker):
    assert failures(checker) is None


MUTANTS = [
    ("no correction where a pair's low half opens the piece", "if ((lo & fb) && ph) bytes -= 2;", ""),
    ("the unit after the piece ignored", "| (nl ? lb : 0u);", ";"),
    ("surrogates counted as 3-byte units", "*m3 = gputf_bit7_nibble(ge08 & ~sur);", "*m3 = gputf_bit7_nibble(ge08);"),
    ("E0-EF leads taken for 4-byte leads", "x & (x << 1) & (x << 2) & (x << 3) & 0x80808080u",
     "x & (x << 1) & (x << 2) & 0x80808080u"),
    ("piece one unit short", "const uint32_t pm = gputf_bit_range(j, pe), fb",
     "const uint32_t pm = gputf_bit_range(j, pe - 1 > j ? pe - 1 : pe), fb"),
]


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistakes_fail_the_proof(tmp_path, name, old, new):
    csrc = tmp_path / "csrc"
    shutil.copytree(CSRC, csrc, ignore=shutil.ignore_patterns("__pycache__", "*.o", "*.so"))
    p = csrc / "batch_piece.h"
    s = p.read_text()
    assert s.count(old) == 1, name
    p.write_text(s.replace(old, new))
    assert failures(build_checker(tmp_path, str(csrc))) is not None, name
