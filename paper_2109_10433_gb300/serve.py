"""Continuous-batching request server over the library's batched calls.

Requests are transcode or validate requests in either direction whose inputs
already sit in device memory.  The server owns a fixed device-memory budget,
split evenly into batch slots.  A slot is one stream with its own arena (the
back-to-back inputs and the outputs of a batch), a workspace for the batched
calls, a workspace for single-buffer calls, a metadata block (gather spans
and CSR offsets) and result rows.

The loop (step):
  - completes every slot whose last launch has finished (a CUDA event),
    handing each of its requests its result and the arena view of its
    output, stamped with the completion time;
  - drops, unrun, the waiting requests whose deadline (optional, host clock)
    has passed; a waiting request can also be withdrawn with cancel();
  - fills every free slot with waiting requests in arrival order while they
    fit: a request takes its input bytes plus its output capacity from the
    slot's arena (admission by memory budget), and the first request that
    does not fit stops the filling, so requests are served in order;
  - launches each slot it filled with one native call, gputf_serve_launch,
    which plans the batch and enqueues on the slot's stream one copy of the
    metadata, one gather of the small requests' inputs into the arena
    (gputf_gather), one batched launch for the small transcode requests of
    both directions and one for the small validate requests
    (gputf_batch_transcode), one single-buffer call per large request run in
    place on its own input, then one copy of the results back to host.

So requests that arrive while other slots are on the GPU go out in the next
free slot, and the slots' launches overlap on the device.  Every request gets
the output and result that the single-string call gives it: batching only
changes where the bytes sit.  Host work here is bookkeeping; every byte of
every request is copied and transcoded by the library's kernels.
"""
from __future__ import annotations

import ctypes
import time
from dataclasses import dataclass

import numpy as np

from . import Result, Workspace, _check, _stream, lib
from . import batch as B

TRANSCODE, VALIDATE = 0, 1
_ALIGN = 256


def _up(x: int, a: int = _ALIGN) -> int:
    return (x + a - 1) // a * a


@dataclass
class Request:
    """One request: `units` input code units at device address `ptr`."""
    rid: int
    direction: int               # batch.UTF8_TO_UTF16 or batch.UTF16_TO_UTF8
    op: int                      # TRANSCODE or VALIDATE
    ptr: int                     # device address of the input
    units: int
    arrival: float = 0.0         # host clock (time.perf_counter) of arrival
    result: Result | None = None
    done: float | None = None
    output: object | None = None  # kept output (a device tensor) when the server keeps outputs
    batch: int = -1              # index of the launch that served it
    deadline: float | None = None  # host clock after which a request still waiting is dropped unrun
    bypassed: int = 0            # times a later request was admitted while this one waited

    @property
    def unit_bytes(self) -> int:
        return 1 if self.direction == B.UTF8_TO_UTF16 else 2

    @property
    def in_bytes(self) -> int:
        return self.units * self.unit_bytes

    @property
    def out_units(self) -> int:
        """Output capacity in output code units: always enough (n UTF-16 units
        for n UTF-8 bytes, 3 bytes per UTF-16 unit)."""
        if self.op == VALIDATE:
            return 0
        return self.units if self.direction == B.UTF8_TO_UTF16 else 3 * self.units

    @property
    def out_bytes(self) -> int:
        return self.out_units * (2 if self.direction == B.UTF8_TO_UTF16 else 1)


REQUEST_DTYPE = np.dtype([("in", "<u8"), ("units", "<u8"), ("direction", "<u4"), ("op", "<u4")])
PLACEMENT_DTYPE = np.dtype([("row", "<u8"), ("in_offset", "<u8"), ("out_offset", "<u8")])
NOWHERE = (1 << 64) - 1


class CSlot(ctypes.Structure):
    _fields_ = [("arena", ctypes.c_void_p), ("arena_bytes", ctypes.c_uint64), ("meta", ctypes.c_void_p),
                ("meta_host", ctypes.c_void_p), ("meta_bytes", ctypes.c_uint64), ("results", ctypes.c_void_p),
                ("results_host", ctypes.c_void_p), ("max_requests", ctypes.c_uint64), ("ws", ctypes.c_void_p),
                ("ws_bytes", ctypes.c_uint64), ("ws1", ctypes.c_void_p), ("ws1_bytes", ctypes.c_uint64)]


def request_array(reqs: list) -> np.ndarray:
    a = np.zeros(len(reqs), dtype=REQUEST_DTYPE)
    a["in"] = [r.ptr for r in reqs]
    a["units"] = [r.units for r in reqs]
    a["direction"] = [r.direction for r in reqs]
    a["op"] = [r.op for r in reqs]
    return a


def plan(reqs: list, big_units: int):
    """gputf_serve_plan: (placements, arena bytes, metadata bytes) of a batch."""
    a = request_array(reqs)
    place = np.zeros(len(reqs), dtype=PLACEMENT_DTYPE)
    arena, meta = ctypes.c_uint64(), ctypes.c_uint64()
    _check(lib().gputf_serve_plan(a.ctypes.data, len(reqs), big_units, place.ctypes.data, ctypes.byref(arena),
                                  ctypes.byref(meta)), "gputf_serve_plan")
    return place, arena.value, meta.value


class _Slot:
    def __init__(self, index: int, arena_bytes: int, max_requests: int, ws_batch: int, ws_single: int,
                 meta_bytes: int, device: str):
        import torch
        self.index = index
        self.stream = torch.cuda.Stream(device=device)
        self.event = torch.cuda.Event()
        self.arena = torch.empty(arena_bytes, dtype=torch.uint8, device=device)
        self.arena_bytes = arena_bytes
        self.ws = Workspace.of_bytes(ws_batch, device=device)
        self.ws1 = Workspace.of_bytes(ws_single, device=device)
        self.meta_bytes = meta_bytes
        self.meta = torch.empty(meta_bytes // 8, dtype=torch.int64, device=device)
        self.meta_host = torch.empty(meta_bytes // 8, dtype=torch.int64).pin_memory()
        self.res = torch.zeros((max_requests, 3), dtype=torch.int64, device=device)
        self.res_host = torch.zeros((max_requests, 3), dtype=torch.int64).pin_memory()
        self.req_buf = np.zeros(max_requests, dtype=REQUEST_DTYPE)
        self.place = np.zeros(max_requests, dtype=PLACEMENT_DTYPE)
        self.cslot = CSlot(self.arena.data_ptr(), arena_bytes, self.meta.data_ptr(), self.meta_host.data_ptr(),
                           meta_bytes, self.res.data_ptr(), self.res_host.data_ptr(), max_requests,
                           self.ws.buf.data_ptr(), self.ws.nbytes, self.ws1.buf.data_ptr(), self.ws1.nbytes)
        self.requests: list[Request] = []
        self.used = 0
        self.in_flight = False

    def device_bytes(self) -> int:
        return self.arena_bytes + self.ws.nbytes + self.ws1.nbytes + self.meta_bytes + self.res.numel() * 8


class Server:
    """Continuous batching over `slots` batch slots within `budget_bytes` of
    device memory.  Requests of at least `big_units` input units run as
    single-buffer calls on their own input; smaller ones are gathered into
    the slot's arena and transcoded by one batched launch per kind."""

    def __init__(self, budget_bytes: int = 8 << 30, slots: int = 4, max_requests: int = 4096,
                 big_units: int = 1 << 20, config: int = 0, keep_outputs: bool = False, trace: bool = False,
                 device: str = "cuda"):
        import torch
        self.torch = torch
        self.trace = trace
        self.trace_events: list = []   # (slot, start event, end event, requests) per launch when tracing
        self.max_requests = max_requests
        self.big_units = big_units
        self.config = config
        self.keep_outputs = keep_outputs
        L = lib()
        per_slot = budget_bytes // slots
        # fixed per-slot costs, sized for an arena as large as the slot
        ws_batch = int(L.gputf_batch_workspace_bytes(per_slot, max_requests, per_slot // 2, max_requests))
        ws_single = int(L.gputf_workspace_bytes(per_slot))
        meta_bytes = int(L.gputf_serve_meta_bytes(max_requests, per_slot))
        fixed = ws_batch + ws_single + meta_bytes + 24 * max_requests
        arena = (per_slot - fixed) // _ALIGN * _ALIGN
        if arena <= 0:
            raise ValueError("budget too small for the slot count")
        self.slots = [_Slot(i, arena, max_requests, ws_batch, ws_single, meta_bytes, device) for i in range(slots)]
        self.budget_bytes = budget_bytes
        self.device_bytes = sum(s.device_bytes() for s in self.slots)
        self.waiting: list[Request] = []
        self.completed: list[Request] = []
        self.cancelled: list[Request] = []   # withdrawn by cancel() while waiting
        self.expired: list[Request] = []     # still waiting at their deadline, never run
        self._deadlines = 0                  # waiting requests that carry a deadline
        self.batches = 0
        self.launches = 0           # library kernels enqueued

    # ---- admission ------------------------------------------------------
    def footprint(self, r: Request) -> int:
        """Arena bytes a request takes: its input (gathered, or counted
        against the budget where it runs in place), its output capacity and
        alignment slack."""
        return r.in_bytes + r.out_bytes + _ALIGN

    def submit(self, r: Request):
        if self.footprint(r) + 4 * _ALIGN > self.slots[0].arena_bytes:
            raise ValueError(f"request {r.rid} ({r.in_bytes} bytes) does not fit a batch slot")
        self.waiting.append(r)
        if r.deadline is not None:
            self._deadlines += 1

    def cancel(self, rid: int) -> bool:
        """Withdraws the waiting request `rid` (True), or does nothing (False)
        when it is not waiting: a request already in a slot runs to the end."""
        for k, r in enumerate(self.waiting):
            if r.rid == rid:
                del self.waiting[k]
                if r.deadline is not None:
                    self._deadlines -= 1
                self.cancelled.append(r)
                return True
        return False

    def _expire(self, now: float):
        """Drops, unrun, the waiting requests whose deadline has passed."""
        keep = []
        for r in self.waiting:
            if r.deadline is not None and now > r.deadline:
                r.done = now
                self.expired.append(r)
                self._deadlines -= 1
            else:
                keep.append(r)
        self.waiting = keep

    # A waiting request that does not fit what is left of a slot lets later
    # requests that do fit go ahead of it, in at most MAX_BYPASS fills; after
    # that it holds back every request behind it until a slot has room for
    # it, so no request waits for ever.  Only LOOKAHEAD requests past the
    # first one left behind are looked at per fill.
    MAX_BYPASS = 8
    LOOKAHEAD = 256

    def _fill(self, slot: _Slot):
        cap = slot.arena_bytes - 4 * _ALIGN   # the three group paddings of the layout
        left: list[tuple[int, Request]] = []  # passed over: (position, request), in arrival order
        last_taken = -1
        k = 0
        n = len(self.waiting)
        while k < n and len(slot.requests) < self.max_requests:
            if left and k - left[0][0] > self.LOOKAHEAD:
                break
            r = self.waiting[k]
            f = self.footprint(r)
            if slot.used + f <= cap:
                slot.requests.append(r)
                slot.used += f
                last_taken = k
                if r.deadline is not None:
                    self._deadlines -= 1
            else:
                left.append((k, r))
                if r.bypassed >= self.MAX_BYPASS:
                    k += 1
                    break
            k += 1
        for pos, r in left:
            if pos < last_taken:   # a later request went ahead of it in this fill
                r.bypassed += 1
        self.waiting = [r for _, r in left] + self.waiting[k:]

    # ---- launch ---------------------------------------------------------
    def _launch(self, slot: _Slot):
        torch = self.torch
        reqs = slot.requests
        n = len(reqs)
        a = slot.req_buf[:n]
        a["in"] = [r.ptr for r in reqs]
        a["units"] = [r.units for r in reqs]
        a["direction"] = [r.direction for r in reqs]
        a["op"] = [r.op for r in reqs]
        with torch.cuda.stream(slot.stream):
            if self.trace:
                started = torch.cuda.Event(enable_timing=True)
                started.record(slot.stream)
        _check(lib().gputf_serve_launch(ctypes.byref(slot.cslot), a.ctypes.data, n, self.big_units, self.config,
                                        slot.place.ctypes.data, _stream(slot.stream)), "gputf_serve_launch")
        # kernels enqueued: the gather, the batched transcode and validate
        # launches, one per large request
        place = slot.place[:n]
        small = place["in_offset"] != NOWHERE
        ops = a["op"][small]
        self.launches += (int(bool(np.any(a["units"][small] > 0))) + int(bool(np.any(ops == TRANSCODE)))
                          + int(bool(np.any(ops == VALIDATE))) + int(n - int(small.sum())))
        for r in reqs:
            r.batch = self.batches
        with torch.cuda.stream(slot.stream):
            if self.keep_outputs:
                for r, off in zip(reqs, place["out_offset"].tolist()):
                    if off != NOWHERE:
                        r.output = slot.arena[off:off + r.out_bytes].clone()
            slot.event.record(slot.stream)
            if self.trace:
                ended = torch.cuda.Event(enable_timing=True)
                ended.record(slot.stream)
                self.trace_events.append((slot.index, started, ended, n))
        slot.in_flight = True
        self.batches += 1

    # ---- completion -----------------------------------------------------
    def _complete(self, slot: _Slot, now: float):
        n = len(slot.requests)
        res = slot.res_host.numpy()[slot.place["row"][:n].astype(np.int64)].tolist()
        for r, (e, p, w) in zip(slot.requests, res):
            r.result = Result(e & 0xFFFFFFFF, p, w)
            r.done = now
        self.completed.extend(slot.requests)
        slot.requests = []
        slot.used = 0
        slot.in_flight = False

    def step(self) -> bool:
        """One pass of the loop; True while requests are waiting or in flight."""
        for slot in self.slots:
            if slot.in_flight and slot.event.query():
                self._complete(slot, time.perf_counter())
        if self._deadlines:
            self._expire(time.perf_counter())
        for slot in self.slots:
            if not slot.in_flight and self.waiting:
                self._fill(slot)
                if slot.requests:
                    self._launch(slot)
        return bool(self.waiting) or any(s.in_flight for s in self.slots)

    def drain(self):
        while self.step():
            pass


class DevicePool:
    """Client-side input store: host arrays copied once into one device
    buffer, each starting on a 256-byte boundary, so that requests can point
    at inputs that are resident on the device before they arrive."""

    def __init__(self, arrays, device: str = "cuda"):
        import torch
        offs, pos = [], 0
        for a in arrays:
            offs.append(pos)
            pos = _up(pos + a.nbytes)
        self.offsets = offs
        self.buf = torch.empty(max(pos, 1), dtype=torch.uint8, device=device)
        for a, o in zip(arrays, offs):
            if a.nbytes:
                host = np.array(a, copy=True).view(np.uint8)     # writable, contiguous
                self.buf[o:o + a.nbytes].copy_(torch.from_numpy(host))

    def ptr(self, k: int, byte_offset: int = 0) -> int:
        return self.buf.data_ptr() + self.offsets[k] + byte_offset

    def view(self, k: int, byte_offset: int, nbytes: int):
        a = self.offsets[k] + byte_offset
        return self.buf[a:a + nbytes]


def latency_ms(reqs: list[Request]) -> dict:
    lat = np.array([r.done - r.arrival for r in reqs]) * 1e3
    return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "max_ms": float(lat.max())}


def run_arrivals(server: Server, requests: list[Request], times: np.ndarray) -> float:
    """Feeds `requests` to the server at host times t0 + times[i] (seconds)
    and runs the loop until every request is complete.  A request's arrival
    time is its scheduled time.  Returns t0."""
    order = np.argsort(times, kind="stable")
    n = len(requests)
    i = 0
    t0 = time.perf_counter()
    while True:
        now = time.perf_counter() - t0
        while i < n and times[order[i]] <= now:
            r = requests[order[i]]
            r.arrival = t0 + float(times[order[i]])
            server.submit(r)
            i += 1
        busy = server.step()
        if i >= n and not busy:
            return t0
        if not busy:
            wait = float(times[order[i]]) - (time.perf_counter() - t0)
            if wait > 2e-4:
                time.sleep(wait - 1e-4)
