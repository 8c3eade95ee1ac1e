"""Batched transcoding through the C ABI (gputf_batch_transcode).

A DeviceBatch holds one direction's strings on the device in CSR form: the
strings back to back, their offsets, an output arena with one capacity per
string, and a result per string.  batch_transcode() runs both directions in
one launch.  Everything here is argument marshalling; the work is the batched
kernel of libgputf.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import GputfError, Result, Workspace, _check, _ptr, _stream, lib

UTF8_TO_UTF16 = 0
UTF16_TO_UTF8 = 1


class CBatch(ctypes.Structure):
    _fields_ = [("count", ctypes.c_uint64), ("units", ctypes.c_uint64),
                ("in_", ctypes.c_void_p), ("in_offsets", ctypes.c_void_p),
                ("out", ctypes.c_void_p), ("out_offsets", ctypes.c_void_p),
                ("results", ctypes.c_void_p)]


def default_capacity(direction: int, n_units: np.ndarray) -> np.ndarray:
    """Output units that always suffice: n units for UTF-8 -> UTF-16, 3n
    bytes for UTF-16 -> UTF-8."""
    return n_units.copy() if direction == UTF8_TO_UTF16 else 3 * n_units


class DeviceBatch:
    """One direction of a batch, resident on the device."""

    def __init__(self, strings, direction: int, capacities=None, device="cuda", validate_only: bool = False):
        import torch
        self.direction = direction
        self.validate_only = validate_only
        dtype = np.uint8 if direction == UTF8_TO_UTF16 else np.uint16
        sizes = np.array([len(s) for s in strings], dtype=np.int64)
        self.count = len(strings)
        self.in_offsets_host = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        self.units = int(self.in_offsets_host[-1])
        caps = default_capacity(direction, sizes) if capacities is None else np.asarray(capacities, np.int64)
        self.out_offsets_host = np.concatenate([[0], np.cumsum(caps)]).astype(np.int64)
        data = np.concatenate([np.asarray(s, dtype=dtype) for s in strings]) if self.count else np.zeros(0, dtype)
        if direction == UTF8_TO_UTF16:
            self.inp = torch.from_numpy(data.copy()).to(device)
            self.out = torch.empty(max(int(self.out_offsets_host[-1]), 1), dtype=torch.int16, device=device)
        else:
            self.inp = torch.from_numpy(data.view(np.int16).copy()).to(device)
            self.out = torch.empty(max(int(self.out_offsets_host[-1]), 1), dtype=torch.uint8, device=device)
        self.in_offsets = torch.from_numpy(self.in_offsets_host).to(device)
        self.out_offsets = torch.from_numpy(self.out_offsets_host).to(device)
        self.results = torch.zeros((max(self.count, 1), 3), dtype=torch.int64, device=device)

    def cstruct(self) -> CBatch:
        """The C descriptor; validate-only batches pass no output (out = NULL)."""
        out = None if self.validate_only else _ptr(self.out).value
        out_off = None if self.validate_only else _ptr(self.out_offsets).value
        return CBatch(self.count, self.units, _ptr(self.inp).value, _ptr(self.in_offsets).value,
                      out, out_off, _ptr(self.results).value)

    def read_results(self) -> list:
        v = self.results.cpu().numpy()[:self.count]
        return [Result(int(r[0]) & 0xFFFFFFFF, int(r[1]), int(r[2])) for r in v]

    def output(self, s: int, written: int) -> np.ndarray:
        a = int(self.out_offsets_host[s])
        o = self.out[a:a + written].cpu().numpy()
        return o.view(np.uint16) if self.direction == UTF8_TO_UTF16 else o


def workspace_for(b8: DeviceBatch | None, b16: DeviceBatch | None, device="cuda") -> Workspace:
    n = lib().gputf_batch_workspace_bytes(b8.units if b8 else 0, b8.count if b8 else 0,
                                          b16.units if b16 else 0, b16.count if b16 else 0)
    return Workspace.of_bytes(int(n), device=device)


def config_count() -> int:
    return int(lib().gputf_batch_config_count())


def batch_transcode(b8: DeviceBatch | None, b16: DeviceBatch | None, ws: Workspace, config: int = 0,
                    stream=None):
    """Enqueue both directions in one launch (results stay on the device)."""
    c8 = ctypes.byref(b8.cstruct()) if b8 is not None else None
    c16 = ctypes.byref(b16.cstruct()) if b16 is not None else None
    _check(lib().gputf_batch_transcode(c8, c16, int(config), ws.ptr, ws.nbytes, _stream(stream)),
           "gputf_batch_transcode")


class BatchGraph:
    """A batched launch captured into a CUDA graph (gputf_batch_graph_create)
    on a stream of its own; replay() enqueues it on that stream."""

    def __init__(self, b8: DeviceBatch | None, b16: DeviceBatch | None, ws: Workspace, config: int = 0):
        import torch
        self.stream = torch.cuda.Stream()
        self._keep = (b8, b16, ws)
        self._c8 = b8.cstruct() if b8 is not None else None
        self._c16 = b16.cstruct() if b16 is not None else None
        self.handle = ctypes.c_void_p()
        torch.cuda.synchronize()
        _check(lib().gputf_batch_graph_create(
            ctypes.byref(self._c8) if self._c8 is not None else None,
            ctypes.byref(self._c16) if self._c16 is not None else None,
            int(config), ws.ptr, ws.nbytes, _stream(self.stream), ctypes.byref(self.handle)),
            "gputf_batch_graph_create")

    def replay(self):
        _check(lib().gputf_graph_launch(self.handle, _stream(self.stream)), "gputf_graph_launch")

    def close(self):
        if self.handle:
            lib().gputf_graph_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


__all__ = ["BatchGraph", "DeviceBatch", "batch_transcode", "workspace_for", "config_count", "UTF8_TO_UTF16",
           "UTF16_TO_UTF8", "GputfError"]
