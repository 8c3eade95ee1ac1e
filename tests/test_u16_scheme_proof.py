"""Proof, on the host, of the UTF-16 classification the UTF-16 -> UTF-8 kernel
uses for its per-unit byte counts and its pairing check.

tests/native/u16_check.c compiles the CUDA path's own header
(utf16_scheme.h: four units per step on their gathered high bytes) for the
CPU and checks it beside the oracle on chunks of units with a unit before
and a unit after (the kernel's thread chunk and its neighbours): prefix sums
of the counts against the oracle's UTF-8 lengths at every split that does
not cut a surrogate pair, the per-unit bounds that make the kernel's staging
buffer big enough, and the pairing flag against the rule of Section 3 and
the oracle's validator; and the same header's arithmetic of the validate-only
and length-only UTF-16 passes (pairing flag, and UTF-8 length against the
oracle's).  Domains:
  - every 16-bit value at every position of a 24-unit chunk, the other units
    drawn from a set holding every class boundary;
  - every combination of boundary values over the five units around a group
    boundary, with the neighbours;
  - random chunks rich in surrogates, of the kernel's width and of 4 units.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# one value on each side of every class boundary the scheme distinguishes
REPS = np.array([0x0000, 0x0041, 0x007F, 0x0080, 0x00FF, 0x0100, 0x07FF, 0x0800, 0x4E00, 0xD7FF,
                 0xD800, 0xDB7F, 0xDBFF, 0xDC00, 0xDEAD, 0xDFFF, 0xE000, 0xFEFF, 0xFFFF], dtype=np.uint16)


CSRC = os.path.join(ROOT, "paper_2109_10433_gb300", "csrc")


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    return build_checker(tmp_path_factory.mktemp("u16scheme"))


def build_checker(out_dir, csrc=CSRC):
    """Builds the checker against the kernel headers in `csrc`."""
    out = os.path.join(str(out_dir), "u16_check.so")
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared",
                           "-I" + os.path.join(ROOT, "oracle"), "-I" + csrc,
                           "-o", out, os.path.join(ROOT, "tests", "native", "u16_check.c"),
                           "-lpthread"])
    lib = ctypes.CDLL(out)
    lib.u16_check.restype = ctypes.c_uint64
    lib.u16_check.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                              ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_int)]

    def run(chunks):
        """chunks: uint16 array (count, n + 2): n units, then pu, then nu."""
        c = np.ascontiguousarray(chunks, dtype=np.uint16)
        fb, fc = ctypes.c_uint64(), ctypes.c_int()
        threads = max(1, min(8, os.cpu_count() or 1))
        m = lib.u16_check(c.ctypes.data, c.shape[0], c.shape[1] - 2, threads, ctypes.byref(fb), ctypes.byref(fc))
        return m, (c[fb.value].tolist() if m else None), fc.value
    return run


def test_every_value_at_every_position(checker):
    rng = np.random.default_rng(41)
    n = 24
    vals = np.arange(1 << 16, dtype=np.uint16)
    for pos in range(n + 2):          # positions n and n + 1 are pu and nu
        chunks = REPS[rng.integers(0, REPS.size, size=(vals.size, n + 2))]
        chunks[:, pos] = vals
        assert checker(chunks) == (0, None, 0), pos


def test_every_boundary_combination_around_a_group_boundary(checker):
    # units 2..6 of an 8-unit chunk take every combination of REPS; the rest,
    # pu and nu, random boundary values
    rng = np.random.default_rng(42)
    axes = np.meshgrid(*([np.arange(REPS.size)] * 5), indexing="ij")
    combo = np.stack([a.ravel() for a in axes], axis=1)
    chunks = REPS[rng.integers(0, REPS.size, size=(combo.shape[0], 10))]
    chunks[:, 2:7] = REPS[combo]
    assert checker(chunks) == (0, None, 0)


@pytest.mark.parametrize("n", [4, 24])
def test_random_surrogate_rich_chunks(checker, n):
    rng = np.random.default_rng(43 + n)
    count = 400_000
    kind = rng.integers(0, 4, size=(count, n + 2))
    chunks = np.where(kind == 0, rng.integers(0xD800, 0xE000, size=(count, n + 2)),
                      np.where(kind == 1, rng.integers(0, 0x800, size=(count, n + 2)),
                               rng.integers(0, 0x10000, size=(count, n + 2)))).astype(np.uint16)
    assert checker(chunks) == (0, None, 0)
