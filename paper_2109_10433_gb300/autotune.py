"""Autotuner for the batched kernel's tile configuration.

For a batch, every configuration gputf_batch_transcode accepts is timed on the
device (CUDA events, median of a few launches) and the fastest is kept.
Choices are cached in a JSON file keyed by the GPU (name, SM count, driver)
and by the batch's input mix: the share of UTF-16 input, the size of the
batch and the mean string length, each bucketed on a log or linear scale.
"""
from __future__ import annotations

import json
import math
import os
import threading

from . import batch as B
from . import lib

CACHE_PATH = os.environ.get("GPUTF_AUTOTUNE_CACHE",
                            os.path.join(os.path.dirname(os.path.abspath(__file__)), "_autotune_cache.json"))
_lock = threading.Lock()


def driver_version() -> int:
    """The installed CUDA driver's version (cuDriverGetVersion), 0 if the
    driver library cannot be asked."""
    import ctypes
    try:
        v = ctypes.c_int(0)
        if ctypes.CDLL("libcuda.so.1").cuDriverGetVersion(ctypes.byref(v)) == 0:
            return int(v.value)
    except OSError:
        pass
    return 0


def _device_key() -> str:
    import torch
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return f"{p.name}|{p.multi_processor_count}|driver={driver_version()}"


def mix_key(b8: B.DeviceBatch | None, b16: B.DeviceBatch | None) -> str:
    u8 = b8.units if b8 else 0
    u16 = 2 * b16.units if b16 else 0
    strings = (b8.count if b8 else 0) + (b16.count if b16 else 0)
    total = u8 + u16
    share16 = round(4 * u16 / total) if total else 0            # quarters of UTF-16 input bytes
    size = int(math.log2(total)) if total else 0                 # batch bytes, power of two
    mean = int(math.log2(max(total // max(strings, 1), 1)))      # mean string bytes, power of two
    return f"share16={share16}|size=2^{size}|mean=2^{mean}"


def _load() -> dict:
    try:
        with open(CACHE_PATH) as f:
            return json.load(f)
    except Exception:
        return {}


def _store(cache: dict):
    tmp = CACHE_PATH + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, CACHE_PATH)


def time_config(b8, b16, ws, config: int, reps: int = 5) -> float:
    """Median device time (ms) of one batched launch with `config`."""
    import torch
    B.batch_transcode(b8, b16, ws, config=config)
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        B.batch_transcode(b8, b16, ws, config=config)
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    ts.sort()
    return ts[len(ts) // 2]


def tune(b8, b16, ws, reps: int = 5) -> tuple[int, dict]:
    times = {c: time_config(b8, b16, ws, c, reps) for c in range(int(lib().gputf_batch_config_count()))}
    best = min(times, key=times.get)
    return best, times


def best_config(b8, b16, ws, reps: int = 5, retune: bool = False) -> int:
    """The cached choice for this GPU and mix, tuning it on first use."""
    key = _device_key() + "|" + mix_key(b8, b16)
    with _lock:
        cache = _load()
        if not retune and key in cache:
            return int(cache[key]["config"])
    best, times = tune(b8, b16, ws, reps)
    with _lock:
        cache = _load()
        cache[key] = {"config": best, "ms": {str(k): v for k, v in times.items()}}
        _store(cache)
    return best
