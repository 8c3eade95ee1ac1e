"""Scalar CPU oracle for validating UTF-8 <-> UTF-16 transcoding (UTF-16LE;
UTF-16BE through a byte swap of each unit).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg load this module; the library's code path never does.

The arithmetic lives in ``oracle.c`` (plain C, one character at a time,
following Section 3 of Lemire & Mula, arXiv 2109.10433: Table 2 lengths, the
UTF-8 lead/continuation structure and validation rules 1-6, and the UTF-16
surrogate-pair construction).  This module compiles it with gcc into
``liboracle.so`` next to the source and wraps it with ctypes and numpy.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import NamedTuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

# Error classes, as numbered in oracle.c.
OK = 0
HEADER_BITS = 1
TOO_SHORT = 2
TOO_LONG = 3
OVERLONG = 4
TOO_LARGE = 5
SURROGATE = 6
OUTPUT_TOO_SMALL = 7

ERROR_NAMES = {
    OK: "OK", HEADER_BITS: "HEADER_BITS", TOO_SHORT: "TOO_SHORT",
    TOO_LONG: "TOO_LONG", OVERLONG: "OVERLONG", TOO_LARGE: "TOO_LARGE",
    SURROGATE: "SURROGATE", OUTPUT_TOO_SMALL: "OUTPUT_TOO_SMALL",
}


class Result(NamedTuple):
    error: int
    position: int
    written: int


class _CResult(ctypes.Structure):
    _fields_ = [("error", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("position", ctypes.c_uint64), ("written", ctypes.c_uint64)]


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, -O2, no target-specific flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        U64 = ctypes.c_uint64
        R = ctypes.POINTER(_CResult)
        for name, args, res in [
            ("oracle_utf8_to_utf16", [P, U64, P, U64, R], None),
            ("oracle_utf16_to_utf8", [P, U64, P, U64, R], None),
            ("oracle_validate_utf8", [P, U64, R], None),
            ("oracle_validate_utf16", [P, U64, R], None),
            ("oracle_utf16_length_from_utf8", [P, U64], U64),
            ("oracle_utf8_length_from_utf16", [P, U64], U64),
            ("oracle_encode_utf8", [ctypes.c_uint32, P], ctypes.c_int),
            ("oracle_encode_utf16", [ctypes.c_uint32, P], ctypes.c_int),
            ("oracle_validate_utf8_fixed", [P, U64, ctypes.c_uint32, P, P], None),
            ("oracle_validate_utf16_fixed", [P, U64, ctypes.c_uint32, P, P], None),
            ("oracle_validate_utf8_csr", [P, P, U64, P, P], None),
        ]:
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
    return _lib


def _u8(data) -> np.ndarray:
    if isinstance(data, (bytes, bytearray, memoryview)):
        return np.frombuffer(bytes(data), dtype=np.uint8)
    a = np.ascontiguousarray(data)
    if a.dtype != np.uint8:
        raise TypeError("expected uint8 data")
    return a


def _u16(data) -> np.ndarray:
    if isinstance(data, (bytes, bytearray, memoryview)):
        return np.frombuffer(bytes(data), dtype="<u2")
    a = np.ascontiguousarray(data)
    if a.dtype != np.uint16:
        raise TypeError("expected uint16 data")
    return a


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data) if a.size else ctypes.c_void_p(0)


def _res(r: _CResult) -> Result:
    return Result(int(r.error), int(r.position), int(r.written))


def utf8_to_utf16(data, cap: int | None = None):
    """Returns (Result, uint16 array of the `written` output units)."""
    a = _u8(data)
    n = a.size
    cap = n if cap is None else int(cap)
    out = np.zeros(max(cap, 1), dtype=np.uint16)
    r = _CResult()
    _load().oracle_utf8_to_utf16(_ptr(a), n, _ptr(out), cap, ctypes.byref(r))
    res = _res(r)
    return res, out[:res.written].copy()


def utf16_to_utf8(units, cap: int | None = None):
    """Returns (Result, uint8 array of the `written` output bytes)."""
    a = _u16(units)
    n = a.size
    cap = 3 * n if cap is None else int(cap)
    out = np.zeros(max(cap, 1), dtype=np.uint8)
    r = _CResult()
    _load().oracle_utf16_to_utf8(_ptr(a), n, _ptr(out), cap, ctypes.byref(r))
    res = _res(r)
    return res, out[:res.written].copy()


def validate_utf8(data) -> Result:
    a = _u8(data)
    r = _CResult()
    _load().oracle_validate_utf8(_ptr(a), a.size, ctypes.byref(r))
    return _res(r)


def validate_utf16(units) -> Result:
    a = _u16(units)
    r = _CResult()
    _load().oracle_validate_utf16(_ptr(a), a.size, ctypes.byref(r))
    return _res(r)


def utf16_length_from_utf8(data) -> int:
    a = _u8(data)
    return int(_load().oracle_utf16_length_from_utf8(_ptr(a), a.size))


def utf8_length_from_utf16(units) -> int:
    a = _u16(units)
    return int(_load().oracle_utf8_length_from_utf16(_ptr(a), a.size))


# UTF-16BE.  The paper's UTF-16 is little-endian (Section 3); big-endian
# UTF-16 stores the same 16-bit units with their two bytes exchanged.  The
# oracle therefore swaps the bytes of each unit and applies the UTF-16LE
# definitions above (and swaps the units it writes).

def _swap16(a: np.ndarray) -> np.ndarray:
    return a.byteswap()


def utf16be_to_utf8(units, cap: int | None = None):
    return utf16_to_utf8(_swap16(_u16(units)), cap)


def utf8_to_utf16be(data, cap: int | None = None):
    res, out = utf8_to_utf16(data, cap)
    return res, _swap16(out)


def validate_utf16be(units) -> Result:
    return validate_utf16(_swap16(_u16(units)))


def utf8_length_from_utf16be(units) -> int:
    return utf8_length_from_utf16(_swap16(_u16(units)))


def encode_utf8(cp: int) -> bytes:
    buf = (ctypes.c_uint8 * 4)()
    k = _load().oracle_encode_utf8(cp, buf)
    return bytes(buf[:k])


def encode_utf16(cp: int) -> list[int]:
    buf = (ctypes.c_uint16 * 2)()
    k = _load().oracle_encode_utf16(cp, buf)
    return list(buf[:k])


def validate_utf8_fixed(strings: np.ndarray):
    """strings: uint8 array of shape (count, width).  Returns (err, pos)."""
    s = np.ascontiguousarray(strings, dtype=np.uint8)
    count, width = s.shape
    err = np.empty(count, dtype=np.int32)
    pos = np.empty(count, dtype=np.uint64)
    _load().oracle_validate_utf8_fixed(_ptr(s), count, width, _ptr(err), _ptr(pos))
    return err, pos


def validate_utf16_fixed(strings: np.ndarray):
    s = np.ascontiguousarray(strings, dtype=np.uint16)
    count, width = s.shape
    err = np.empty(count, dtype=np.int32)
    pos = np.empty(count, dtype=np.uint64)
    _load().oracle_validate_utf16_fixed(_ptr(s), count, width, _ptr(err), _ptr(pos))
    return err, pos


def validate_utf8_csr(data: np.ndarray, offsets: np.ndarray):
    d = _u8(data)
    off = np.ascontiguousarray(offsets, dtype=np.uint64)
    count = off.size - 1
    err = np.empty(count, dtype=np.int32)
    pos = np.empty(count, dtype=np.uint64)
    _load().oracle_validate_utf8_csr(_ptr(d), _ptr(off), count, _ptr(err), _ptr(pos))
    return err, pos
