"""Proof, on the host, of the UTF-8 character decoder the UTF-8 -> UTF-16
kernel uses (gputf_utf8_decode in utf8_scheme.h: byte reversal, the length
from the lead's leading ones, the prefixes cleared by shifts and a mask, the
6-bit groups packed in two steps).

tests/native/decode_check.c compiles the kernel's header for the CPU:
  - every scalar value, encoded by the oracle and followed by filler bytes of
    every kind (zero, ASCII, continuation, lead, 0xFF), decodes to the
    oracle's UTF-16 units;
  - every lead byte with every second byte (and fillers after) gives the unit
    count the length pass assigns it, 1 + [lead >= 0xF0], so invalid input
    never moves the output of the characters after it.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FILL = np.array([0x00000000, 0xFFFFFFFF, 0x80808080, 0xBFBFBFBF, 0x41414141, 0xC2C2C2C2, 0xE0E0E0E0,
                 0xF0F0F0F0, 0x7F80BFC0, 0x12345678, 0xDEADBEEF, 0xF4908080], dtype=np.uint32)


CSRC = os.path.join(ROOT, "paper_2109_10433_gb300", "csrc")


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    return build_checker(tmp_path_factory.mktemp("decode"))


def build_checker(out_dir, csrc=CSRC):
    """Builds the checker against the kernel headers in `csrc`."""
    out = os.path.join(str(out_dir), "decode_check.so")
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared",
                           "-I" + os.path.join(ROOT, "oracle"), "-I" + csrc,
                           "-o", out, os.path.join(ROOT, "tests", "native", "decode_check.c")])
    L = ctypes.CDLL(out)
    for f in (L.decode_check_scalars, L.decode_check_counts):
        f.restype = ctypes.c_uint64
        f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_uint32)]
    return L


def test_every_scalar_value_with_every_filler(lib):
    fb = ctypes.c_uint32()
    n = lib.decode_check_scalars(FILL.ctypes.data, FILL.size, ctypes.byref(fb))
    assert n == 0, hex(fb.value)


def test_unit_count_of_every_lead_and_second_byte(lib):
    fb = ctypes.c_uint32()
    n = lib.decode_check_counts(FILL.ctypes.data, FILL.size, ctypes.byref(fb))
    assert n == 0, hex(fb.value)
