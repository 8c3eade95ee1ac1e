"""Python binding of libgputf: validating UTF-8 <-> UTF-16LE transcoding on
NVIDIA GB300 (sm_103a).

This module only marshals arguments: every step of the work runs in the CUDA
kernels of libgputf.so, reached through its C ABI (include/gputf.h).  PyTorch
provides device memory and streams.  There is no CPU fallback: if the library
is not built, or the device is not an sm_103 part, calls raise.

Two levels:
  - `lib()` gives the raw ctypes functions, named as in the C header;
  - the functions below (utf8_to_utf16, utf16_to_utf8, validate_utf8,
    validate_utf16, utf16_length_from_utf8, utf8_length_from_utf16) take CUDA
    tensors and a Workspace, enqueue the call on the current (or given)
    stream and, unless sync=False, return the result read back from the GPU.
"""
from __future__ import annotations

import ctypes
import os
from typing import NamedTuple

from . import _build

__all__ = [
    "build", "lib", "Result", "Workspace", "GputfError",
    "utf8_to_utf16", "utf16_to_utf8", "validate_utf8", "validate_utf16",
    "utf16_length_from_utf8", "utf8_length_from_utf16",
    "utf8_to_utf16_host", "utf16_to_utf8_host",
    "ERROR_NAMES", "OK", "HEADER_BITS", "TOO_SHORT", "TOO_LONG", "OVERLONG", "TOO_LARGE",
    "SURROGATE", "OUTPUT_TOO_SMALL", "TIMEOUT", "INTERNAL",
]

OK, HEADER_BITS, TOO_SHORT, TOO_LONG, OVERLONG, TOO_LARGE, SURROGATE = 0, 1, 2, 3, 4, 5, 6
OUTPUT_TOO_SMALL, TIMEOUT, INTERNAL = 7, 8, 9
ERROR_NAMES = ["OK", "HEADER_BITS", "TOO_SHORT", "TOO_LONG", "OVERLONG", "TOO_LARGE",
               "SURROGATE", "OUTPUT_TOO_SMALL", "TIMEOUT", "INTERNAL"]
STATUS_NAMES = ["OK", "INVALID_ARGUMENT", "WORKSPACE_TOO_SMALL", "INPUT_TOO_LARGE",
                "CUDA_ERROR", "UNSUPPORTED_DEVICE"]

LIB_PATH = _build.LIB

# name -> (argtypes, restype); every entry point declared in include/gputf.h
_P, _S, _I = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int
SIGNATURES = {
    "gputf_workspace_bytes": ([_S], _S),
    "gputf_workspace_init": ([_P, _S, _P], _I),
    "gputf_utf8_to_utf16": ([_P, _S, _P, _S, _P, _S, _P, _P], _I),
    "gputf_utf16_to_utf8": ([_P, _S, _P, _S, _P, _S, _P, _P], _I),
    "gputf_utf8_to_utf16_unchecked": ([_P, _S, _P, _S, _P, _S, _P, _P], _I),
    "gputf_utf16_to_utf8_unchecked": ([_P, _S, _P, _S, _P, _S, _P, _P], _I),
    "gputf_validate_utf8": ([_P, _S, _P, _S, _P, _P], _I),
    "gputf_validate_utf16": ([_P, _S, _P, _S, _P, _P], _I),
    "gputf_utf16_length_from_utf8": ([_P, _S, _P, _S, _P, _P], _I),
    "gputf_utf8_length_from_utf16": ([_P, _S, _P, _S, _P, _P], _I),
    "gputf_utf16be_to_utf8": ([_P, _S, _P, _S, _P, _S, _P, _P], _I),
    "gputf_utf8_to_utf16be": ([_P, _S, _P, _S, _P, _S, _P, _P], _I),
    "gputf_validate_utf16be": ([_P, _S, _P, _S, _P, _P], _I),
    "gputf_utf8_length_from_utf16be": ([_P, _S, _P, _S, _P, _P], _I),
    "gputf_utf8_to_utf16_host": ([_P, _S, _P, _S, _P, _P, _P, _S, _P, _P, _P], _I),
    "gputf_utf16_to_utf8_host": ([_P, _S, _P, _S, _P, _P, _P, _S, _P, _P, _P], _I),
    "gputf_utf8_to_utf16_host_chunked": ([_P, _S, _P, _S, _P, _P, _P, _S, _P, _P, _P, _S], _I),
    "gputf_utf16_to_utf8_host_chunked": ([_P, _S, _P, _S, _P, _P, _P, _S, _P, _P, _P, _S], _I),
    "gputf_utf8_chunk_end": ([_P, _S, _S], _S),
    "gputf_utf16_chunk_end": ([_P, _S, _S], _S),
    "gputf_utf16_to_utf8_static": ([_P, _S, _P, _S, _P, _P], _I),
    "gputf_test_wait_timeout": ([_P, _S, _I, ctypes.c_uint32, _P, _P], _I),
    "gputf_batch_workspace_bytes": ([ctypes.c_uint64] * 4, _S),
    "gputf_batch_config_count": ([], _I),
    "gputf_batch_transcode": ([_P, _P, _I, _P, _S, _P], _I),
    "gputf_batch_graph_create": ([_P, _P, _I, _P, _S, _P, _P], _I),
    "gputf_graph_launch": ([_P, _P], _I),
    "gputf_graph_destroy": ([_P], None),
    "gputf_gather": ([_P, ctypes.c_uint64, _P, _P], _I),
    "gputf_serve_meta_bytes": ([ctypes.c_uint64, ctypes.c_uint64], _S),
    "gputf_serve_plan": ([_P, ctypes.c_uint64, ctypes.c_uint64, _P, _P, _P], _I),
    "gputf_serve_launch": ([_P, _P, ctypes.c_uint64, ctypes.c_uint64, _I, _P, _P], _I),
    "gputf_error_name": ([ctypes.c_int32], ctypes.c_char_p),
    "gputf_status_name": ([_I], ctypes.c_char_p),
    "gputf_last_cuda_error": ([], _I),
    "gputf_version": ([], _I),
}


class GputfError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile libgputf.so for sm_103a (nvcc) next to this file."""
    return _build.build(force=force)


_lib = None


def lib():
    """The loaded library, with ctypes signatures set.  Raises if missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise GputfError(f"{LIB_PATH} is not built: run paper_2109_10433_gb300.build() "
                             "(nvcc for sm_103a); there is no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in SIGNATURES.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


class Result(NamedTuple):
    error: int
    position: int
    written: int

    @property
    def ok(self) -> bool:
        return self.error == OK

    @property
    def name(self) -> str:
        return ERROR_NAMES[self.error] if 0 <= self.error < len(ERROR_NAMES) else "UNKNOWN"


class _CResult(ctypes.Structure):
    _fields_ = [("error", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("position", ctypes.c_uint64), ("written", ctypes.c_uint64)]


def _check(status: int, what: str):
    if status != 0:
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        extra = f" (CUDA error {lib().gputf_last_cuda_error()})" if name == "CUDA_ERROR" else ""
        raise GputfError(f"{what}: {name}{extra}")


def _torch():
    import torch
    return torch


def _stream(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr() if t.numel() else 0)


def _nbytes(t) -> int:
    return t.numel() * t.element_size()


def _on_device(t, what: str, min_bytes: int = 0):
    """Checks a tensor whose address goes to a kernel.  The kernels read and
    write t.data_ptr() as device memory, contiguously, for as many bytes as
    the call's sizes say; a CPU tensor, a strided view or a short result
    buffer would hand them the wrong memory, so those are refused here,
    before anything is enqueued."""
    if not getattr(t, "is_cuda", False):
        raise ValueError(f"{what}: expected a CUDA tensor, got one on {getattr(t, 'device', type(t))}")
    if not t.is_contiguous():
        raise ValueError(f"{what}: expected a contiguous tensor")
    if _nbytes(t) < min_bytes:
        raise ValueError(f"{what}: {_nbytes(t)} bytes, at least {min_bytes} needed")
    return t


def _on_host(t, what: str):
    """Checks a host buffer of the host-buffer forms (read or written by
    cudaMemcpyAsync at t.data_ptr(), contiguously)."""
    if getattr(t, "is_cuda", True):
        raise ValueError(f"{what}: expected a CPU tensor (pinned for speed)")
    if not t.is_contiguous():
        raise ValueError(f"{what}: expected a contiguous tensor")
    return t


def _utf16_units(t, what: str) -> int:
    nb = _nbytes(t)
    if nb % 2:
        raise ValueError(f"{what}: UTF-16 input of {nb} bytes (an odd count)")
    return nb // 2


class Workspace:
    """Device scratch for the calls: a header and one status word per input
    tile.  Owned by PyTorch's allocator; prepared once here."""

    def __init__(self, max_units: int, device=None, stream=None):
        torch = _torch()
        self.max_units = int(max_units)
        self.nbytes = int(lib().gputf_workspace_bytes(self.max_units))
        self.buf = torch.empty(self.nbytes, dtype=torch.uint8,
                               device=device if device is not None else "cuda")
        _check(lib().gputf_workspace_init(_ptr(self.buf), self.nbytes, _stream(stream)),
               "gputf_workspace_init")

    @classmethod
    def of_bytes(cls, nbytes: int, device=None, stream=None):
        """A workspace of exactly `nbytes` (for example gputf_batch_workspace_bytes)."""
        torch = _torch()
        ws = cls.__new__(cls)
        ws.max_units = 0
        ws.nbytes = int(nbytes)
        ws.buf = torch.empty(ws.nbytes, dtype=torch.uint8, device=device if device is not None else "cuda")
        _check(lib().gputf_workspace_init(_ptr(ws.buf), ws.nbytes, _stream(stream)), "gputf_workspace_init")
        return ws

    @property
    def ptr(self):
        return _ptr(self.buf)

    def reset(self, stream=None):
        _check(lib().gputf_workspace_init(self.ptr, self.nbytes, _stream(stream)),
               "gputf_workspace_init")


def _res_tensor(res, device):
    """The caller's result tensor (24 bytes on the device), or a new one."""
    torch = _torch()
    if res is not None:
        return _on_device(res, "res", 24)
    return torch.empty(3, dtype=torch.int64, device=device)


def read_result(res) -> Result:
    """Reads a 24-byte result tensor (synchronises with the GPU)."""
    v = res.cpu().tolist()
    return Result(int(v[0]) & 0xFFFFFFFF, int(v[1]), int(v[2]))


def _ws_for(ws, n, device):
    if ws is None:
        ws = Workspace(max(int(n), 1), device=device)
    return ws


def _utf16_name(base, validate, big_endian):
    if big_endian and not validate:
        raise ValueError("the non-validating transcoders take UTF-16LE only")
    if big_endian:
        return base.replace("utf16", "utf16be")
    return base if validate else base + "_unchecked"


def utf8_to_utf16(inp, out=None, ws: Workspace | None = None, res=None, stream=None, sync=True,
                  validate: bool = True, big_endian: bool = False):
    """UTF-8 bytes (CUDA uint8 tensor) -> UTF-16LE units (UTF-16BE when
    big_endian).  Returns (Result, out) when sync, else (res tensor, out);
    `out` defaults to n units (torch.int16 storage).  validate=False calls the
    non-validating form."""
    _on_device(inp, "inp")
    torch = _torch()
    n = _nbytes(inp)
    if out is None:
        out = torch.empty(max(n, 1), dtype=torch.int16, device=inp.device)
    cap = _nbytes(_on_device(out, "out")) // 2
    name = _utf16_name("gputf_utf8_to_utf16", validate, big_endian)
    ws, res = _ws_for(ws, n, inp.device), _res_tensor(res, inp.device)
    _check(getattr(lib(), name)(_ptr(inp), n, _ptr(out), cap, ws.ptr, ws.nbytes, _ptr(res), _stream(stream)), name)
    return (read_result(res) if sync else res), out


def utf16_to_utf8(inp, out=None, ws: Workspace | None = None, res=None, stream=None, sync=True,
                  validate: bool = True, big_endian: bool = False):
    """UTF-16LE units (UTF-16BE when big_endian; CUDA tensor of 2-byte
    elements) -> UTF-8 bytes.  `out` defaults to 3 bytes per unit
    (torch.uint8).  validate=False calls the non-validating form."""
    n = _utf16_units(_on_device(inp, "inp"), "inp")
    torch = _torch()
    if out is None:
        out = torch.empty(max(3 * n, 1), dtype=torch.uint8, device=inp.device)
    cap = _nbytes(_on_device(out, "out"))
    name = _utf16_name("gputf_utf16_to_utf8", validate, big_endian)
    ws, res = _ws_for(ws, n, inp.device), _res_tensor(res, inp.device)
    _check(getattr(lib(), name)(_ptr(inp), n, _ptr(out), cap, ws.ptr, ws.nbytes, _ptr(res), _stream(stream)), name)
    return (read_result(res) if sync else res), out


def validate_utf8(inp, ws: Workspace | None = None, res=None, stream=None, sync=True):
    n = _nbytes(_on_device(inp, "inp"))
    ws, res = _ws_for(ws, n, inp.device), _res_tensor(res, inp.device)
    _check(lib().gputf_validate_utf8(_ptr(inp), n, ws.ptr, ws.nbytes, _ptr(res), _stream(stream)),
           "gputf_validate_utf8")
    return read_result(res) if sync else res


def validate_utf16(inp, ws: Workspace | None = None, res=None, stream=None, sync=True, big_endian: bool = False):
    n = _utf16_units(_on_device(inp, "inp"), "inp")
    ws, res = _ws_for(ws, n, inp.device), _res_tensor(res, inp.device)
    name = "gputf_validate_utf16be" if big_endian else "gputf_validate_utf16"
    _check(getattr(lib(), name)(_ptr(inp), n, ws.ptr, ws.nbytes, _ptr(res), _stream(stream)), name)
    return read_result(res) if sync else res


def _len_tensor(out, device):
    """The caller's length tensor (8 bytes on the device), or a new one."""
    torch = _torch()
    if out is not None:
        return _on_device(out, "out", 8)
    return torch.empty(1, dtype=torch.int64, device=device)


def utf16_length_from_utf8(inp, ws: Workspace | None = None, out=None, stream=None, sync=True):
    n = _nbytes(_on_device(inp, "inp"))
    ws, out = _ws_for(ws, n, inp.device), _len_tensor(out, inp.device)
    _check(lib().gputf_utf16_length_from_utf8(_ptr(inp), n, ws.ptr, ws.nbytes, _ptr(out),
                                              _stream(stream)), "gputf_utf16_length_from_utf8")
    return int(out.item()) if sync else out


def utf8_length_from_utf16(inp, ws: Workspace | None = None, out=None, stream=None, sync=True,
                           big_endian: bool = False):
    n = _utf16_units(_on_device(inp, "inp"), "inp")
    ws, out = _ws_for(ws, n, inp.device), _len_tensor(out, inp.device)
    name = "gputf_utf8_length_from_utf16be" if big_endian else "gputf_utf8_length_from_utf16"
    _check(getattr(lib(), name)(_ptr(inp), n, ws.ptr, ws.nbytes, _ptr(out), _stream(stream)), name)
    return int(out.item()) if sync else out


def _host_form_buffers(h_in, h_out, d_in, d_out, d_res):
    """The host forms copy all of h_in into d_in and read up to all of h_out's
    capacity from d_out, so the device buffers must be at least as large."""
    _on_host(h_in, "h_in")
    _on_host(h_out, "h_out")
    _on_device(d_in, "d_in", _nbytes(h_in))
    _on_device(d_out, "d_out", _nbytes(h_out))
    _on_device(d_res, "d_res", 24)


def utf8_to_utf16_host(h_in, h_out, d_in, d_out, ws: Workspace, d_res, stream=None, chunk=None) -> Result:
    """Host-buffer form: h_in / h_out are CPU tensors (pinned for speed),
    d_in / d_out / d_res device tensors of matching sizes.  `chunk` (input
    bytes) overrides the size of the pieces whose copies and transcoding
    overlap."""
    _host_form_buffers(h_in, h_out, d_in, d_out, d_res)
    r = _CResult()
    n = _nbytes(h_in)
    cap = _nbytes(h_out) // 2
    args = (_ptr(h_in), n, _ptr(h_out), cap, _ptr(d_in), _ptr(d_out), ws.ptr, ws.nbytes, _ptr(d_res),
            ctypes.byref(r), _stream(stream))
    name = "gputf_utf8_to_utf16_host" if chunk is None else "gputf_utf8_to_utf16_host_chunked"
    _check(getattr(lib(), name)(*args) if chunk is None else getattr(lib(), name)(*args, int(chunk)), name)
    return Result(r.error, r.position, r.written)


def utf16_to_utf8_host(h_in, h_out, d_in, d_out, ws: Workspace, d_res, stream=None, chunk=None) -> Result:
    """As utf8_to_utf16_host, UTF-16LE in (`chunk` in input units)."""
    _host_form_buffers(h_in, h_out, d_in, d_out, d_res)
    r = _CResult()
    n = _utf16_units(h_in, "h_in")
    cap = _nbytes(h_out)
    args = (_ptr(h_in), n, _ptr(h_out), cap, _ptr(d_in), _ptr(d_out), ws.ptr, ws.nbytes, _ptr(d_res),
            ctypes.byref(r), _stream(stream))
    name = "gputf_utf16_to_utf8_host" if chunk is None else "gputf_utf16_to_utf8_host_chunked"
    _check(getattr(lib(), name)(*args) if chunk is None else getattr(lib(), name)(*args, int(chunk)), name)
    return Result(r.error, r.position, r.written)
