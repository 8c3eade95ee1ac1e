"""Proof, on the host, of the UTF-16 -> UTF-8 kernel's encoding: the bytes
each unit writes and the order the kernel stores them in.

tests/native/u16_encode_check.c compiles the CUDA path's own header
(utf16_scheme.h: the per-unit counts and gputf_u16_utf8_bytes /
gputf_u16_utf8_bytes_back, the byte values of the kernel's two store
orders) for the CPU.  It replays the kernel's stores for a thread's run of
units and checks the bytes left against the oracle's UTF-8 (Section 3 pair
construction, Section 5 byte layout, Table 2 lengths).  It also checks that
no store of the back-to-front order reaches the bytes before the run, which
belong to another thread.  Domains:
  - every 16-bit value at every position of a 24-unit run (and as the unit
    before or after it), the other units drawn from a set holding every
    class boundary;
  - every combination of boundary values over the unit before and the first
    four units (where the stray stores of the back-to-front order could
    leave the run), and over the last four units and the unit after;
  - every surrogate pair (2^20 of them) at the start of a run, across the
    change from back-to-front to front-to-back stores, and across the run's
    end;
  - random runs rich in surrogates, of the kernel's width and of 4 units.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# one value on each side of every class boundary the encoding distinguishes
REPS = np.array([0x0000, 0x0041, 0x007F, 0x0080, 0x00FF, 0x0100, 0x07FF, 0x0800, 0x0FFF, 0x1000,
                 0x4E00, 0xD7FF, 0xD800, 0xDB7F, 0xDBFF, 0xDC00, 0xDEAD, 0xDFFF, 0xE000, 0xFEFF,
                 0xFFFF], dtype=np.uint16)


CSRC = os.path.join(ROOT, "paper_2109_10433_gb300", "csrc")


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    return build_checker(tmp_path_factory.mktemp("u16encode"))


def build_checker(out_dir, csrc=CSRC):
    """Builds the checker against the kernel headers in `csrc`."""
    out = os.path.join(str(out_dir), "u16_encode_check.so")
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared",
                           "-I" + os.path.join(ROOT, "oracle"), "-I" + csrc,
                           "-o", out, os.path.join(ROOT, "tests", "native", "u16_encode_check.c"),
                           "-lpthread"])
    lib = ctypes.CDLL(out)
    lib.u16_encode_check.restype = ctypes.c_uint64
    lib.u16_encode_check.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                     ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_int)]

    def run(runs):
        """runs: uint16 array (count, n + 2): n units, then pu, then nu."""
        c = np.ascontiguousarray(runs, dtype=np.uint16)
        fb, fc = ctypes.c_uint64(), ctypes.c_int()
        threads = max(1, min(8, os.cpu_count() or 1))
        m = lib.u16_encode_check(c.ctypes.data, c.shape[0], c.shape[1] - 2, threads, ctypes.byref(fb),
                                 ctypes.byref(fc))
        return m, (c[fb.value].tolist() if m else None), fc.value
    return run


def test_every_value_at_every_position(checker):
    rng = np.random.default_rng(51)
    n = 24
    vals = np.arange(1 << 16, dtype=np.uint16)
    for pos in range(n + 2):          # positions n and n + 1 are pu and nu
        runs = REPS[rng.integers(0, REPS.size, size=(vals.size, n + 2))]
        runs[:, pos] = vals
        assert checker(runs) == (0, None, 0), pos


@pytest.mark.parametrize("cols", [(8, 0, 1, 2, 3), (4, 5, 6, 7, 9)])
def test_every_boundary_combination_at_the_ends(checker, cols):
    # an 8-unit run (pu at column 8, nu at column 9): the unit before and
    # units 0-3, or units 4-7 and the unit after, take every combination
    rng = np.random.default_rng(52 + cols[0])
    axes = np.meshgrid(*([np.arange(REPS.size)] * 5), indexing="ij")
    combo = np.stack([a.ravel() for a in axes], axis=1)
    runs = REPS[rng.integers(0, REPS.size, size=(combo.shape[0], 10))]
    runs[:, list(cols)] = REPS[combo]
    assert checker(runs) == (0, None, 0)


@pytest.mark.parametrize("at", [0, 2, 3, 7])
def test_every_surrogate_pair(checker, at):
    # an 8-unit run of 'A' with the pair's high half at unit `at` and its
    # low half after it (the unit after the run when at = 7)
    hi = np.repeat(np.arange(0xD800, 0xDC00, dtype=np.uint16), 1024)
    lo = np.tile(np.arange(0xDC00, 0xE000, dtype=np.uint16), 1024)
    runs = np.full((hi.size, 10), 0x41, dtype=np.uint16)
    runs[:, at] = hi
    runs[:, at + 1 if at < 7 else 9] = lo
    assert checker(runs) == (0, None, 0)


@pytest.mark.parametrize("n", [4, 24])
def test_random_surrogate_rich_runs(checker, n):
    rng = np.random.default_rng(53 + n)
    count = 400_000
    kind = rng.integers(0, 4, size=(count, n + 2))
    runs = np.where(kind == 0, rng.integers(0xD800, 0xE000, size=(count, n + 2)),
                    np.where(kind == 1, rng.integers(0, 0x800, size=(count, n + 2)),
                             rng.integers(0, 0x10000, size=(count, n + 2)))).astype(np.uint16)
    assert checker(runs) == (0, None, 0)
