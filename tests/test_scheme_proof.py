"""Proof, on the host, of the UTF-8 validation scheme the kernels use.

tests/native/scheme_check.c compiles the CUDA path's own header
(utf8_scheme.h: nibble tables, four-bytes-at-a-time flags, and the scalar
fix-up) for the CPU and runs it beside the oracle.  For every string in each
domain below, the pair (error class, position) must be identical:
  - every string of 0 to 3 bytes;
  - every 4-byte string with one byte position running over all 256 values
    and the others over a representative set that holds every boundary of
    the UTF-8 byte classes;
  - every 5-byte string over the representative set;
  - every 6-byte string over a smaller representative set;
  - corrupted synthetic text of all the benchmark mixes.
The flags depend only on the four bytes ending at each position, so these
domains meet every window class in every context the oracle distinguishes.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

REPS = np.array([0x00, 0x41, 0x7F, 0x80, 0x85, 0x8F, 0x90, 0x95, 0x9F, 0xA0, 0xA5, 0xAF, 0xB0,
                 0xB5, 0xBF, 0xC0, 0xC1, 0xC2, 0xCF, 0xD0, 0xD5, 0xDF, 0xE0, 0xE1, 0xE5, 0xEC,
                 0xED, 0xEE, 0xEF, 0xF0, 0xF1, 0xF3, 0xF4, 0xF5, 0xF7, 0xF8, 0xFB, 0xFF], dtype=np.uint8)
REPS6 = np.array([0x41, 0x80, 0x90, 0xA0, 0xBF, 0xC1, 0xC2, 0xE0, 0xED, 0xEF, 0xF0, 0xF4, 0xF5,
                  0xF8], dtype=np.uint8)


CSRC = os.path.join(ROOT, "paper_2109_10433_gb300", "csrc")


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    return build_checker(tmp_path_factory.mktemp("scheme"))


def build_checker(out_dir, csrc=CSRC):
    """Builds the checker against the kernel headers in `csrc`."""
    out = os.path.join(str(out_dir), "scheme_check.so")
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared",
                           "-I" + os.path.join(ROOT, "oracle"), "-I" + csrc,
                           "-o", out, os.path.join(ROOT, "tests", "native", "scheme_check.c"),
                           "-lpthread"])
    lib = ctypes.CDLL(out)
    lib.scheme_check.restype = ctypes.c_uint64
    lib.scheme_check.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64,
                                 ctypes.c_uint32, ctypes.c_int, ctypes.POINTER(ctypes.c_uint64)]

    def run(strings=None, data=None, offsets=None):
        fb = ctypes.c_uint64()
        threads = max(1, min(8, os.cpu_count() or 1))
        if strings is not None:
            s = np.ascontiguousarray(strings, dtype=np.uint8)
            m = lib.scheme_check(s.ctypes.data, None, s.shape[0], s.shape[1], threads, ctypes.byref(fb))
            return m, (s[fb.value].tobytes().hex() if m else None)
        d = np.ascontiguousarray(data, dtype=np.uint8)
        o = np.ascontiguousarray(offsets, dtype=np.uint64)
        m = lib.scheme_check(d.ctypes.data, o.ctypes.data, o.size - 1, 0, threads, ctypes.byref(fb))
        return m, (d[o[fb.value]:o[fb.value + 1]].tobytes().hex() if m else None)
    return run


def grid(*axes):
    return np.stack(np.meshgrid(*axes, indexing="ij"), -1).reshape(-1, len(axes)).astype(np.uint8)


@pytest.mark.parametrize("length", [1, 2, 3])
def test_every_short_string(checker, length):
    idx = np.arange(256 ** length, dtype=np.int64)
    s = np.stack([(idx >> (8 * (length - 1 - k))) & 0xFF for k in range(length)], axis=1)
    assert checker(strings=s) == (0, None)


def test_empty_string(checker):
    assert checker(data=np.zeros(1, np.uint8), offsets=np.array([0, 0])) == (0, None)


@pytest.mark.parametrize("free", [0, 1, 2, 3])
def test_four_byte_strings(checker, free):
    axes = [REPS] * 4
    axes[free] = np.arange(256)
    assert checker(strings=grid(*axes)) == (0, None)


def test_five_byte_strings(checker):
    assert checker(strings=grid(*([REPS] * 5))) == (0, None)


def test_six_byte_strings(checker):
    assert checker(strings=grid(*([REPS6] * 6))) == (0, None)


def test_corrupted_synthetic_text(checker):
    rng = np.random.default_rng(21)
    parts, offs = [], [0]
    for mix in [W.MIX_LATIN_CYRILLIC, W.MIX_CJK_EMOJI, W.MIX_FOUR_BYTE_HEAVY, W.SCRIPT_MIXED,
                W.SCRIPT_TWO_BYTE]:
        for i in range(3000):
            t = W.utf8_text(int(rng.integers(1 << 30)), int(rng.integers(1, 120)), mix).copy()
            for _ in range(int(rng.integers(0, 3))):
                t[int(rng.integers(0, t.size))] = int(rng.integers(0, 256))
            parts.append(t)
            offs.append(offs[-1] + t.size)
    assert checker(data=np.concatenate(parts), offsets=np.array(offs)) == (0, None)
