"""Pin of the oracle on every sequence of two UTF-16 units (all 2^32).

tests/native/u16_pairs_check.c calls the oracle's UTF-16 validator and its
UTF-16 -> UTF-8 transcoder on each pair (a, b) and compares them with values
fixed outside the oracle: validity and the first invalid position from the
closed form of Section 3's UTF-16 paragraph (valid iff neither unit is a
surrogate, or a is D800-DBFF and b is DC00-DFFF; the error is at a when a is
a surrogate that starts no pair, else at b), and the UTF-8 bytes from
CPython's codec (every BMP scalar value, every supplementary one).  The run
is split over the host's cores; on 8 cores it takes well under a minute.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def build_checker(out_dir, oracle_dir=os.path.join(ROOT, "oracle")):
    """Builds the checker against the oracle source in `oracle_dir`."""
    out = os.path.join(str(out_dir), "u16_pairs_check.so")
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-I" + oracle_dir,
                           "-o", out, os.path.join(ROOT, "tests", "native", "u16_pairs_check.c"),
                           "-lpthread"])
    lib = ctypes.CDLL(out)
    lib.u16_pairs_check.restype = ctypes.c_uint64
    lib.u16_pairs_check.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int,
                                    ctypes.POINTER(ctypes.c_uint64)]
    return lib


def cpython_tables():
    """CPython's UTF-8 bytes of every BMP value (surrogates left empty) and
    of every supplementary value, 4 bytes a value, zero-padded."""
    bmp = np.zeros((1 << 16, 4), dtype=np.uint8)
    blen = np.zeros(1 << 16, dtype=np.uint8)
    for u in range(1 << 16):
        if 0xD800 <= u <= 0xDFFF:
            continue
        b = chr(u).encode("utf-8")
        bmp[u, :len(b)] = np.frombuffer(b, dtype=np.uint8)
        blen[u] = len(b)
    supp = np.frombuffer("".join(map(chr, range(0x10000, 0x110000))).encode("utf-8"),
                         dtype=np.uint8).reshape(-1, 4).copy()
    assert supp.shape == (1 << 20, 4)
    return bmp, blen, supp


@pytest.fixture(scope="module")
def tables():
    return cpython_tables()


def run_pairs(lib, tables, a_begin=0, a_end=1 << 16):
    bmp, blen, supp = tables
    first = ctypes.c_uint64()
    threads = max(1, min(64, os.cpu_count() or 1))
    m = lib.u16_pairs_check(bmp.ctypes.data, blen.ctypes.data, supp.ctypes.data, a_begin, a_end,
                            threads, ctypes.byref(first))
    return m, first.value


def test_every_utf16_unit_pair(tmp_path, tables):
    lib = build_checker(tmp_path)
    m, first = run_pairs(lib, tables)
    assert m == 0, f"{m} pairs disagree; first (a, b) = ({first >> 16:#06x}, {first & 0xFFFF:#06x})"


# Planted mistakes in copies of the oracle that this pin must catch, each on
# the unit ranges where the mistake shows (first units near every class
# boundary, every second unit): (what, text in oracle.c, replacement).
MISTAKES = [
    ("two/three-byte bound", "if (cp <= 0x7FF) return 2;", "if (cp < 0x7FF) return 2;"),
    ("three/four-byte bound", "if (cp <= 0xFFFF) return 3;", "if (cp < 0xFFFF) return 3;"),
    ("continuation mask", "out[k] = (uint8_t)(0x80 | (cp & 0x3F));", "out[k] = (uint8_t)(0x80 | (cp & 0x7F));"),
    ("lead prefixes transposed", "{0, 0, 0xC0, 0xE0, 0xF0}", "{0, 0, 0xC0, 0xF0, 0xE0}"),
    ("payload shift", "cp >>= 6;", "cp >>= 5;"),
    ("low unit's upper bound dropped", "in[i + 1] >= 0xDC00 && in[i + 1] <= 0xDFFF)", "in[i + 1] >= 0xDC00)"),
    ("0x10000 not added", "*cp = ((hi10 << 10) | lo10) + 0x10000;", "*cp = ((hi10 << 10) | lo10);"),
    ("0xDFFF outside the surrogates", "if (u < 0xD800 || u > 0xDFFF) {", "if (u < 0xD800 || u >= 0xDFFF) {"),
    ("a low unit opens a pair", "if (u <= 0xDBFF && i + 1 < n", "if (u <= 0xDFFF && i + 1 < n"),
    ("transcoder error offset one past the unit",
     "r->error = e;\n            r->position = i;\n            r->written = q;",
     "r->error = e;\n            r->position = i + 1;\n            r->written = q;"),
    ("validator error offset one past the unit",
     "r->error = e;\n            r->position = i;\n            return;",
     "r->error = e;\n            r->position = i + 1;\n            return;"),
]

# first units: both sides of every class boundary of Section 3 and Table 2
A_RANGES = [(0x0000, 0x0100), (0x07F0, 0x0810), (0xD7F0, 0xE010), (0xFFF0, 0x10000)]


def _mismatches_on_ranges(lib, tables):
    return sum(run_pairs(lib, tables, a, b)[0] for a, b in A_RANGES)


def test_unmodified_oracle_copy_passes_on_the_ranges(tmp_path, tables):
    d = tmp_path / "same"
    d.mkdir()
    (d / "oracle.c").write_text(open(os.path.join(ROOT, "oracle", "oracle.c")).read())
    assert _mismatches_on_ranges(build_checker(d, str(d)), tables) == 0


@pytest.mark.parametrize("what,old,new", MISTAKES, ids=[m[0] for m in MISTAKES])
def test_planted_mistake_fails_the_pair_pin(tmp_path, tables, what, old, new):
    text = open(os.path.join(ROOT, "oracle", "oracle.c")).read()
    assert text.count(old) == 1, old
    d = tmp_path / "mut"
    d.mkdir()
    (d / "oracle.c").write_text(text.replace(old, new))
    assert _mismatches_on_ranges(build_checker(d, str(d)), tables) > 0, what
