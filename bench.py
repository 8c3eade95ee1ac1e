"""Benchmark of validating UTF-16LE -> UTF-8 transcoding on GB300.

Workload (one step = one call over the whole buffer): 256 MiB of UTF-16LE,
20% U+0020-007E, 70% U+4E00-9FFF, 10% U+1F300-1FAFF as surrogate pairs
(seeded synthetic text standing in for the paper's CJK/emoji files), fully
validated and transcoded to UTF-8 by one kernel launch.  The input is larger
than L2, so no flush is needed between steps.

Prints one JSON line: input GB/s (device-timed, inputs resident in HBM), the
same metric end to end through the host-buffer C-ABI call (copies included)
beside the host link's own copy ceiling, the roofline of the kernel against
the measured HBM copy bandwidth, SM clocks sampled during the timed region,
and the CPU oracle's throughput on a sample.  On one GPU the line also holds,
under "configs", the other workloads, each timed on its own with its own
clock record: the 1 MiB UTF-8 buffer, the 64 MiB error-injected UTF-8 buffer
(and its mix at 256 MiB), every validate / length pass at 256 MiB, the
100,000-string batch against per-string launches, the served request stream
with p50 / p99 latency, and the input-size sweep; results are checked against
the oracle (whole buffers, or the stated samples).  --headline-only skips
them.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun each rank transcodes its own buffer (independent replicas; the
path needs no exchange), and the reported value is all ranks' input bytes over
the slowest rank's time.
"""
from __future__ import annotations

import argparse
import gc
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "validated UTF-8<->UTF-16 input GB/s, % of HBM roofline; serving p99 latency"
WORKLOAD = "utf16le_to_utf8_validating_256MiB_cjk70_ascii20_emoji10"
KERNEL = "utf16_to_utf8_kernel"
KERNEL_SOURCES = ["paper_2109_10433_gb300/csrc/utf16_to_utf8.cu",
                  "paper_2109_10433_gb300/csrc/common.cuh",
                  "paper_2109_10433_gb300/csrc/utf16_scheme.h",
                  "paper_2109_10433_gb300/csrc/utf8_scheme.h"]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "utf16_to_utf8_256MiB_traffic.json")
L2_BYTES = 129 * 10 ** 6   # GB300's L2 cache
BATCH_SEED, SERVE_SEED = 3, 4


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def ncu_traffic():
    """DRAM bytes per launch from the committed ncu capture, if it was taken
    on the current kernel source."""
    try:
        with open(TRAFFIC_FILE) as f:
            t = json.load(f)
        if t.get("source_hash") == kernel_source_hash():
            return float(t["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi samples of the GPU's SM clock and throttle reasons."""

    FIELDS = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.uuid = uuid
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        try:
            with open(self.path) as f:
                for line in f:
                    c = [x.strip() for x in line.split(",")]
                    if len(c) < 9:
                        continue
                    if self.uuid and c[0] != self.uuid:
                        continue
                    rows.append(c)
            os.unlink(self.path)
        except Exception:
            return None
        if not rows:
            return None

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def slowest(value: float, device) -> float:
    """The largest of every rank's value (the slowest rank's time); the value
    itself when no process group is running."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_gbs(world: int, bytes_per_rank_step: int, steps: int, seconds: float) -> float:
    """Whole-job throughput of independent replicas: every rank's bytes over
    the slowest rank's time."""
    return world * steps * bytes_per_rank_step / seconds / 1e9


def rank_seed(rank: int) -> int:
    """Each replica transcodes its own buffer of the same mix."""
    return 1 + rank


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def pair_safe_chunks(data: np.ndarray, parts: int) -> list:
    """Cuts UTF-16 units into about equal chunks, never between the two
    halves of a surrogate pair (the transcoding of the whole is then the
    concatenation of the chunks' transcodings)."""
    cuts = [0]
    for k in range(1, parts):
        c = k * data.size // parts
        if c > 0 and 0xD800 <= int(data[c - 1]) <= 0xDBFF:
            c -= 1
        cuts.append(max(c, cuts[-1]))
    cuts.append(data.size)
    return [data[a:b] for a, b in zip(cuts[:-1], cuts[1:]) if b > a]


def cpu_oracle_parallel(data: np.ndarray, min_seconds: float, threads: int):
    """The oracle, as it stands, on all host cores: the buffer cut into one
    chunk per thread (at pair-safe points), each chunk transcoded by one
    oracle call in its own thread (the oracle's C code runs outside the
    interpreter lock)."""
    from concurrent.futures import ThreadPoolExecutor

    import oracle
    oracle.build()
    chunks = pair_safe_chunks(data, threads)
    runs, t0 = 0, time.perf_counter()
    with ThreadPoolExecutor(threads) as ex:
        while True:
            results = list(ex.map(lambda c: oracle.utf16_to_utf8(c)[0], chunks))
            runs += 1
            el = time.perf_counter() - t0
            if el >= min_seconds:
                break
    assert all(r.error == 0 for r in results)
    return runs * data.nbytes / el / 1e9, runs, el


def cpu_oracle_baseline(data: np.ndarray, min_seconds: float):
    """The oracle, as it stands, on the host cores: one thread."""
    import oracle
    oracle.build()
    sample = data
    runs, t0 = 0, time.perf_counter()
    res = None
    while True:
        res = oracle.utf16_to_utf8(sample)[0]
        runs += 1
        el = time.perf_counter() - t0
        if el >= min_seconds:
            break
    assert res.error == 0
    gbs = runs * sample.nbytes / el / 1e9
    return gbs, runs, el


def workload_config(data: np.ndarray, out_bytes: int, world: int, mib: int) -> dict:
    """The `config` object of the bench line, the same for both arms."""
    return {"workload": WORKLOAD if mib == 256 else WORKLOAD.replace("256MiB", f"{mib}MiB"),
            "input_bytes": int(data.nbytes),
            "output_bytes": int(out_bytes), "chars": count_chars(data),
            "l2": (f"input ({mib} MiB) larger than L2, no flush" if data.nbytes > L2_BYTES
                   else f"input ({mib} MiB) fits in L2, no flush: L2-resident timing"),
            "parallelism": f"replicas{world}", "seeds": [rank_seed(r) for r in range(world)]}


def count_chars(data: np.ndarray) -> int:
    """Characters of UTF-16 text: every unit but the low half of a pair
    (a low surrogate right after a high one)."""
    top = data & np.uint16(0xFC00)
    low = top == 0xDC00
    low[1:] &= top[:-1] == 0xD800
    low[:1] = False
    return int(data.size - np.count_nonzero(low))


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    data = W.cjk_emoji_utf16_256mib(seed=rank_seed(0), nbytes=args.mib << 20)
    # each step: the oracle over a bounded 32 MiB slice of the workload
    k = min((32 << 20) // 2, data.size)
    if k < data.size and 0xD800 <= int(data[k - 1]) <= 0xDBFF:   # do not split a surrogate pair
        k -= 1
    sample = data[:k]
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    oracle.build()
    cores = os.cpu_count() or 1
    chunks = pair_safe_chunks(sample, cores)
    times = []
    with ThreadPoolExecutor(cores) as ex:
        for _ in range(args.warmup):
            list(ex.map(lambda c: oracle.utf16_to_utf8(c)[0], chunks))
        for _ in range(args.steps):
            t0 = time.perf_counter()
            rs = list(ex.map(lambda c: oracle.utf16_to_utf8(c)[0], chunks))
            times.append(time.perf_counter() - t0)
            assert all(r.error == 0 for r in rs)
    total = sum(times)
    value = args.steps * sample.nbytes / total / 1e9
    out_bytes = oracle.utf8_length_from_utf16(data)   # the transcoded length (the text is valid)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u16", "data": "synthetic",
        "config": workload_config(data, out_bytes, world, args.mib),
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": cores, "kind": "oracle",
                         "sample": f"first {sample.nbytes >> 20} MiB of the {args.mib} MiB workload per step, "
                                   f"in {cores} pair-safe chunks, one oracle call per chunk on its own thread"},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_gpu(args):
    import torch

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    import paper_2109_10433_gb300 as g
    g.build()

    data = W.cjk_emoji_utf16_256mib(seed=rank_seed(rank), nbytes=args.mib << 20)
    n = data.size
    inp = torch.from_numpy(data.view(np.int16)).to(dev)
    out = torch.empty(3 * n, dtype=torch.uint8, device=dev)
    ws = g.Workspace(n, device=dev)
    res = torch.zeros(3, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream(dev)
    L = g.lib()
    args_c = (g._ptr(inp), n, g._ptr(out), out.numel(), ws.ptr, ws.nbytes, g._ptr(res),
              g._stream(stream))

    def step():
        st = L.gputf_utf16_to_utf8(*args_c)
        if st != 0:
            raise RuntimeError(f"gputf_utf16_to_utf8 status {st}")

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    r = g.read_result(res)
    assert r.error == 0 and r.position == n, r
    out_bytes = r.written

    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    clocks = ClockSampler(uuid) if rank == 0 else None
    if clocks:
        clocks.start()
        time.sleep(0.3)

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    region0 = torch.cuda.Event(enable_timing=True)
    region1 = torch.cuda.Event(enable_timing=True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    region0.record(stream)
    for i in range(args.steps):
        starts[i].record(stream)
        step()
        ends[i].record(stream)
    region1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clock_info = clocks.stop() if clocks else None
    r = g.read_result(res)
    assert r.error == 0 and r.written == out_bytes, r

    region_ms = region0.elapsed_time(region1)
    launch_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    region_ms = slowest(region_ms, dev)
    ms_per_step = region_ms / args.steps
    value = replica_gbs(world, data.nbytes, args.steps, region_ms * 1e-3)

    # end to end through the host-buffer C-ABI call: pinned host input in,
    # UTF-8 out to pinned host memory, result read back every step
    h_in = torch.from_numpy(data.view(np.int16)).pin_memory()
    h_out = torch.empty(3 * n, dtype=torch.uint8).pin_memory()
    e2e_times = []
    for i in range(args.e2e_warmup + args.e2e_steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rr = g.utf16_to_utf8_host(h_in, h_out, inp, out, ws, res)
        el = time.perf_counter() - t0
        assert rr.error == 0 and rr.written == out_bytes
        if i >= args.e2e_warmup:
            e2e_times.append(el)
    e2e_total = slowest(max(sum(e2e_times), 1e-12), dev)
    e2e_val = replica_gbs(world, data.nbytes, len(e2e_times), e2e_total) if e2e_times else None
    ceiling = e2e_ceiling(h_in, h_out[:out_bytes], inp, out[:out_bytes]) if rank == 0 else None
    del h_in, h_out

    if rank != 0:
        torch.distributed.destroy_process_group()
        return 0

    peak, peak_kind = measured_peak()
    avg_launch_s = statistics.mean(launch_ms) * 1e-3
    algo_bytes = data.nbytes + out_bytes
    achieved = algo_bytes / avg_launch_s / 1e9
    traffic = ncu_traffic() if args.mib == 256 else None   # the capture is of the 256 MiB launch
    chars = count_chars(data)

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        gbs1, runs1, el1 = cpu_oracle_baseline(data, args.cpu_seconds / 2)
        cores = os.cpu_count() or 1
        gbs, runs, el = cpu_oracle_parallel(data, args.cpu_seconds / 2, cores)
        cpu = {"value": gbs, "unit": "GB/s", "cores": cores, "kind": "oracle",
               "sample": f"the whole 256 MiB buffer in {cores} pair-safe chunks, one oracle call per chunk "
                         f"on its own thread, {runs} run(s) in {el:.1f} s; single thread: {gbs1:.3f} GB/s "
                         f"({runs1} run(s) in {el1:.1f} s)",
               "single_thread_value": gbs1}

    line = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world,
        "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u16",
        "data": "synthetic",
        "config": workload_config(data, out_bytes, world, args.mib),
        "gchar_s": world * args.steps * chars / (region_ms * 1e-3) / 1e9,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "traffic_note": ("steady-state DRAM bytes per launch: one ncu launch of the 128 MiB case "
                                      "with --cache-control none, times 2") if traffic else None,
                     "algorithmic_bytes": int(algo_bytes), "kernel": KERNEL,
                     "avg_launch_us": avg_launch_s * 1e6, "peak_source": peak_kind},
        "e2e": {"value": e2e_val, "unit": "GB/s", "h2d_bytes_per_step": int(data.nbytes),
                "d2h_bytes_per_step": int(out_bytes + 24), "steps": len(e2e_times),
                "copy_ceiling": ceiling,
                "frac_of_copy_ceiling": (e2e_val / ceiling["input_gbs_ceiling"]) if (ceiling and e2e_val) else None},
        "gpu_launches": args.steps,
        "clocks": clock_info,
        "cpu_baseline": cpu,
    }
    if world == 1 and not args.headline_only:
        # the other configurations, each timed on its own with its own clock
        # record (outside the headline's timed region)
        del inp, out, ws, res
        torch.cuda.empty_cache()
        sections = {}
        for name, fn in (("config1_utf8_1MiB", config1_section), ("config3_utf8_64MiB_errors", config3_section),
                         ("passes_256MiB", passes_section), ("config4_batch", batch_section),
                         ("config5_serve", serve_section), ("sweep", sweep_section)):
            t0 = time.perf_counter()
            sections[name] = fn(args)
            sections[name]["section_s"] = time.perf_counter() - t0
            torch.cuda.synchronize()
            torch.cuda.empty_cache()
        line["configs"] = sections
        sv = sections["config5_serve"]
        line["serving_p99_ms"] = sv["p99_ms"]
        line["serving_p50_ms"] = sv["p50_ms"]
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def event_times(fn, stream, reps, before=None):
    """Device time (ms) of each of `reps` calls of fn, CUDA events on the
    launching stream; `before` (not timed) runs ahead of each call."""
    import torch
    ms = []
    for _ in range(reps):
        if before is not None:
            before()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = fn()
        e1.record(stream)
        if st not in (None, 0):
            raise RuntimeError(f"call status {st}")
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    return ms


def device_uuid():
    import torch
    try:
        return "GPU-" + str(torch.cuda.get_device_properties(torch.cuda.current_device()).uuid)
    except Exception:
        return None


def config1_section(args):
    """Configuration 1: one 1 MiB UTF-8 buffer (90% U+0020-007E, 10%
    U+0400-04FF, seed 0) to UTF-16LE with validation.  It fits in L2 and a
    launch costs more than its bytes: reported in microseconds per call
    (no flush, L2-resident), with the output checked against the oracle."""
    import torch

    import oracle
    import paper_2109_10433_gb300 as g
    data = W.latin_cyrillic_utf8_1mib()
    n = int(data.size)
    d = torch.from_numpy(data.copy()).cuda()
    out = torch.empty(n, dtype=torch.int16, device="cuda")
    ws = g.Workspace(n + 16)
    res = torch.zeros(3, dtype=torch.int64, device="cuda")
    s = torch.cuda.current_stream()
    L = g.lib()
    fn = lambda: L.gputf_utf8_to_utf16(g._ptr(d), n, g._ptr(out), n, ws.ptr, ws.nbytes, g._ptr(res), g._stream(s))
    event_times(fn, s, 5)
    clocks = ClockSampler(device_uuid())
    clocks.start()
    ms = event_times(fn, s, 200)
    clk = clocks.stop()
    r = g.read_result(res)
    ref, ref_out = oracle.utf8_to_utf16(data)
    exact = tuple(r) == tuple(ref) and np.array_equal(out[:r.written].cpu().numpy().view(np.uint16), ref_out)
    us = statistics.median(ms) * 1e3
    peak, _ = measured_peak()
    algo = n + 2 * int(r.written)
    return {"workload": "utf8_to_utf16le_validating_1MiB_ascii90_cyrillic10", "seed": 0, "input_bytes": n,
            "output_units": int(r.written), "median_us": us, "min_us": min(ms) * 1e3, "calls": len(ms),
            "input_gbs": n / (us * 1e-6) / 1e9, "gchar_s": int(r.written) / (us * 1e-6) / 1e9,
            "achieved_gbs": algo / (us * 1e-6) / 1e9, "frac": algo / (us * 1e-6) / 1e9 / peak,
            "l2": "1 MiB fits in L2; no flush (L2-resident, launch-bound)", "identical_to_oracle": bool(exact),
            "clocks": clk}


def config3_section(args):
    """Configuration 3: 64 MiB of four-byte-heavy UTF-8 (40% U+10000-10FFFF,
    30% U+0800-FFFF without surrogates, 30% ASCII; seed 2) with error tokens
    about once per MiB.  The full buffer's result (the first error: class,
    offset, output count) and output are checked against the oracle; the
    clean buffer (every token repaired) is timed with L2 flushed before each
    call (a 512 MB write), and the same mix at 256 MiB (larger than L2, no
    flush)."""
    import torch

    import oracle
    import paper_2109_10433_gb300 as g
    L = g.lib()
    s = torch.cuda.current_stream()
    sp = g._stream(s)
    peak, _ = measured_peak()
    et = W.four_byte_heavy_utf8_64mib()
    n = int(et.data.size)
    out = torch.empty(n, dtype=torch.int16, device="cuda")
    ws = g.Workspace(4 * n + 16)
    res = torch.zeros(3, dtype=torch.int64, device="cuda")
    d = torch.from_numpy(et.data.copy()).cuda()
    assert L.gputf_utf8_to_utf16(g._ptr(d), n, g._ptr(out), n, ws.ptr, ws.nbytes, g._ptr(res), sp) == 0
    r = g.read_result(res)
    ref, ref_out = oracle.utf8_to_utf16(et.data)
    first_ok = (tuple(r) == tuple(ref) == (et.tokens[0][2], et.tokens[0][0], ref.written)
                and np.array_equal(out[:r.written].cpu().numpy().view(np.uint16), ref_out))
    clean = et.repaired_before(len(et.tokens))
    d = torch.from_numpy(clean.copy()).cuda()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    fn = lambda: L.gputf_utf8_to_utf16(g._ptr(d), n, g._ptr(out), n, ws.ptr, ws.nbytes, g._ptr(res), sp)
    event_times(fn, s, 3)
    clocks = ClockSampler(device_uuid())
    clocks.start()
    ms = event_times(fn, s, 20, before=lambda: flush.fill_(1))
    clk = clocks.stop()
    rc = g.read_result(res)
    us = statistics.median(ms) * 1e3
    algo = n + 2 * int(rc.written)
    row64 = {"input_bytes": n, "output_units": int(rc.written), "median_us": us, "min_us": min(ms) * 1e3,
             "input_gbs": n / (us * 1e-6) / 1e9, "achieved_gbs": algo / (us * 1e-6) / 1e9,
             "frac": algo / (us * 1e-6) / 1e9 / peak, "l2": "flushed before each call", "clean_ok": rc.error == 0,
             "clocks": clk}
    del d, flush
    big = W.utf8_text(2, 256 << 20, W.MIX_FOUR_BYTE_HEAVY)
    nb = int(big.size)
    db = torch.from_numpy(big).cuda()
    outb = torch.empty(nb, dtype=torch.int16, device="cuda")
    fnb = lambda: L.gputf_utf8_to_utf16(g._ptr(db), nb, g._ptr(outb), nb, ws.ptr, ws.nbytes, g._ptr(res), sp)
    event_times(fnb, s, 3)
    clocks = ClockSampler(device_uuid())
    clocks.start()
    ms = event_times(fnb, s, 10)
    clk = clocks.stop()
    rb = g.read_result(res)
    us = statistics.median(ms) * 1e3
    algo = nb + 2 * int(rb.written)
    row256 = {"input_bytes": nb, "output_units": int(rb.written), "median_us": us, "min_us": min(ms) * 1e3,
              "input_gbs": nb / (us * 1e-6) / 1e9, "achieved_gbs": algo / (us * 1e-6) / 1e9,
              "frac": algo / (us * 1e-6) / 1e9 / peak, "l2": "input larger than L2, no flush",
              "clean_ok": rb.error == 0, "clocks": clk}
    return {"workload": "utf8_to_utf16le_validating_64MiB_four_byte_heavy_errors_1_per_MiB", "seed": 2,
            "error_tokens": len(et.tokens), "first_error": {"class": int(r.error), "position": int(r.position),
                                                            "written": int(r.written)},
            "first_error_identical_to_oracle": bool(first_ok), "clean_64MiB": row64, "clean_256MiB": row256,
            "roofline_kernel": "utf8_to_utf16_kernel", "algorithmic_bytes": "n + 2 U (input bytes, output units)"}


def e2e_ceiling(h_in, h_out, d_in, d_out, reps=5):
    """The host link alone: the pinned input copied to the device while the
    output is copied back, on two streams (as the host-buffer call overlaps
    them), no kernel; and each direction alone."""
    import torch
    a, b = torch.cuda.Stream(), torch.cuda.Stream()
    nin, nout = h_in.numel() * h_in.element_size(), d_out.numel() * d_out.element_size()

    def one(h2d, d2h):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if h2d:
            with torch.cuda.stream(a):
                d_in.copy_(h_in, non_blocking=True)
        if d2h:
            with torch.cuda.stream(b):
                h_out.copy_(d_out, non_blocking=True)
        torch.cuda.synchronize()
        return time.perf_counter() - t0

    res = {}
    for name, h2d, d2h in (("both", True, True), ("h2d", True, False), ("d2h", False, True)):
        one(h2d, d2h)
        res[name] = min(one(h2d, d2h) for _ in range(reps))
    return {"h2d_bytes": nin, "d2h_bytes": nout, "both_s": res["both"], "h2d_s": res["h2d"], "d2h_s": res["d2h"],
            "input_gbs_ceiling": nin / res["both"] / 1e9, "h2d_gbs": nin / res["h2d"] / 1e9,
            "d2h_gbs": nout / res["d2h"] / 1e9}


def batch_section(args):
    """Batched form: 100,000 strings (log-normal lengths, median 1 KiB,
    clipped 16 B - 64 KiB, per-string script, half in each direction, 1%
    invalid) in one graph-replayed launch with the autotuned tile shape,
    against per-string plain launches through the same C ABI."""
    import ctypes

    import torch

    import paper_2109_10433_gb300 as g
    from paper_2109_10433_gb300 import autotune
    from paper_2109_10433_gb300 import batch as B

    g.build()
    torch.cuda.set_device(0)
    bt = W.string_batch(BATCH_SEED, args.strings)
    s8 = [s for s, d in zip(bt.strings, bt.directions) if d == 0]
    s16 = [s for s, d in zip(bt.strings, bt.directions) if d == 1]
    b8 = B.DeviceBatch(s8, B.UTF8_TO_UTF16)
    b16 = B.DeviceBatch(s16, B.UTF16_TO_UTF8)
    ws = B.workspace_for(b8, b16)
    cfg = autotune.best_config(b8, b16, ws)
    graph = B.BatchGraph(b8, b16, ws, cfg)
    for _ in range(max(args.warmup, 3)):
        graph.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(graph.stream)
    for _ in range(args.steps):
        graph.replay()
    e1.record(graph.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    n_strings = len(bt.strings)
    in_bytes = b8.units + 2 * b16.units
    res8, res16 = b8.read_results(), b16.read_results()

    # per-string plain launches on a sample, into the same output regions
    rng = np.random.default_rng(0)
    sample = rng.choice(n_strings, size=min(args.sample, n_strings), replace=False)
    pos8 = {int(i): k for k, i in enumerate(np.nonzero(bt.directions == 0)[0])}
    pos16 = {int(i): k for k, i in enumerate(np.nonzero(bt.directions == 1)[0])}
    ws1 = g.Workspace(64 * 1024 + 16)
    r1 = torch.zeros((len(sample), 3), dtype=torch.int64, device="cuda")
    L = g.lib()
    stream = torch.cuda.current_stream()
    calls = []
    for j, i in enumerate(sample.tolist()):
        if bt.directions[i] == 0:
            k = pos8[i]
            a, e = int(b8.in_offsets_host[k]), int(b8.in_offsets_host[k + 1])
            oa, oe = int(b8.out_offsets_host[k]), int(b8.out_offsets_host[k + 1])
            calls.append((L.gputf_utf8_to_utf16, b8.inp.data_ptr() + a, e - a, b8.out.data_ptr() + 2 * oa, oe - oa,
                          r1.data_ptr() + 24 * j, res8[k]))
        else:
            k = pos16[i]
            a, e = int(b16.in_offsets_host[k]), int(b16.in_offsets_host[k + 1])
            oa, oe = int(b16.out_offsets_host[k]), int(b16.out_offsets_host[k + 1])
            calls.append((L.gputf_utf16_to_utf8, b16.inp.data_ptr() + 2 * a, e - a, b16.out.data_ptr() + oa, oe - oa,
                          r1.data_ptr() + 24 * j, res16[k]))
    sp = ctypes.c_void_p(stream.cuda_stream)

    def per_string():
        for fn, ip, n, op, cap, rp, _ in calls:
            st = fn(ctypes.c_void_p(ip), n, ctypes.c_void_p(op), cap, ws1.ptr, ws1.nbytes, ctypes.c_void_p(rp), sp)
            if st != 0:
                raise RuntimeError(f"status {st}")
    per_string()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    per_string()
    torch.cuda.synchronize()
    per_s = time.perf_counter() - t0
    got = r1.cpu().numpy()
    same = all((int(got[j][0]) & 0xFFFFFFFF, int(got[j][1]), int(got[j][2])) == tuple(c[6])
               for j, c in enumerate(calls))
    bad = sum(1 for r in res8 + res16 if r.error != 0)
    # the batched results and outputs of the same sample (and of every
    # invalid string) against the oracle
    import oracle
    out8 = b8.out.cpu().numpy().view(np.uint16)
    out16 = b16.out.cpu().numpy()
    check = set(sample.tolist()) | {i for i in range(n_strings) if bt.invalid[i]}
    oracle_ok = True
    for i in sorted(check):
        if bt.directions[i] == 0:
            k = pos8[i]
            ref, ref_out = oracle.utf8_to_utf16(bt.strings[i])
            a = int(b8.out_offsets_host[k])
            ok = tuple(res8[k]) == tuple(ref) and np.array_equal(out8[a:a + ref.written], ref_out)
        else:
            k = pos16[i]
            ref, ref_out = oracle.utf16_to_utf8(bt.strings[i])
            a = int(b16.out_offsets_host[k])
            ok = tuple(res16[k]) == tuple(ref) and np.array_equal(out16[a:a + ref.written], ref_out)
        oracle_ok = oracle_ok and ok
    line = {
        "metric": "batched transcoding strings/s (one graph-replayed launch) vs per-string launches",
        "value": n_strings / (ms * 1e-3), "unit": "strings/s", "n_gpus": 1, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True, "dtype": "u8/u16",
        "data": "synthetic",
        "config": {"workload": f"batch_{n_strings}_strings_lognormal_median1KiB_half_each_direction",
                   "input_bytes": int(in_bytes), "tile_config": cfg, "graph": True, "seed": BATCH_SEED},
        "input_gbs": in_bytes / (ms * 1e-3) / 1e9,
        "invalid_strings": bad,
        "per_string_launches": {"strings": len(calls), "seconds": per_s,
                                "strings_per_s": len(calls) / per_s, "results_identical": same},
        "speedup_vs_per_string": (n_strings / (ms * 1e-3)) / (len(calls) / per_s),
        "oracle_check": {"strings": len(check), "identical": bool(oracle_ok),
                         "sample": "the per-string sample and every invalid string"},
        "gpu_launches": args.steps,
    }
    return line


def run_batch(args):
    print(json.dumps(batch_section(args)), flush=True)
    return 0


def serve_section(args):
    """Served form: requests with Poisson arrivals, sizes log-uniform
    64 B - 16 MiB of input, scripts and directions as in the batched form,
    a fifth of them validate-only and 1% invalid, inputs resident on the
    device before they arrive, an 8 GB admission budget over four batch
    slots.  Reports the saturated throughput (every request waiting at
    start) and p50/p99 latency at 50/80/95% of it, with every request's
    result checked against its standalone call."""
    import ctypes

    import torch

    import paper_2109_10433_gb300 as g
    from paper_2109_10433_gb300 import serve as S

    g.build()
    torch.cuda.set_device(0)
    t_gen = time.perf_counter()
    w = W.serve_workload(SERVE_SEED, args.requests)
    gen_s = time.perf_counter() - t_gen
    pool = S.DevicePool(list(w.texts) + list(w.payloads))
    nt = len(w.texts)

    def requests():
        out = []
        for i in range(w.units.size):
            s = int(w.source[i])
            k = s if s >= 0 else nt + (-1 - s)
            ub = 1 + int(w.direction[i])
            out.append(S.Request(i, int(w.direction[i]), S.VALIDATE if w.validate_only[i] else S.TRANSCODE,
                                 pool.ptr(k, int(w.offset[i]) * ub), int(w.units[i])))
        return out

    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(0).uuid)
    except Exception:
        pass
    srv = S.Server(budget_bytes=args.budget_gb << 30, slots=args.slots, max_requests=args.max_requests,
                   big_units=args.big_units)
    in_bytes = int(w.input_bytes().sum())
    mean_bytes = in_bytes / w.units.size

    def run(times, reqs):
        srv.completed = []
        l0 = srv.launches
        b0 = srv.batches
        clocks = ClockSampler(uuid)
        clocks.start()
        # the host loop runs in Python: its garbage collector is run before
        # and held off during the run, so that a collection pause is not
        # counted as serving latency
        gc.collect()
        gc.disable()
        try:
            t0 = S.run_arrivals(srv, reqs, times)
        finally:
            gc.enable()
        clk = clocks.stop()
        t_end = max(r.done for r in reqs)
        lat = S.latency_ms(reqs)
        return {"requests": len(reqs), "seconds": t_end - t0, "achieved_gbs": in_bytes / (t_end - t0) / 1e9,
                "batches": srv.batches - b0, "gpu_launches": srv.launches - l0, **lat, "clocks": clk}

    # warm-up: a few hundred requests, all at once
    warm = requests()[:min(400, w.units.size)]
    S.run_arrivals(srv, warm, np.zeros(len(warm)))
    torch.cuda.synchronize()

    sat_reqs = requests()
    sat = run(np.zeros(len(sat_reqs)), sat_reqs)
    cap_gbs = sat["achieved_gbs"]
    levels = []
    for frac in (0.5, 0.8, 0.95):
        offered = frac * cap_gbs
        times = np.cumsum(w.gaps) * (mean_bytes / (offered * 1e9))
        lv = run(times, requests())
        lv["offered_frac"] = frac
        lv["offered_gbs"] = offered
        levels.append(lv)

    # every result of the saturated run against the standalone call on the same input
    L = g.lib()
    ws1 = g.Workspace(16 << 20)
    r1 = torch.zeros((len(sat_reqs), 3), dtype=torch.int64, device="cuda")
    scratch = torch.empty(3 * (16 << 20) + 256, dtype=torch.uint8, device="cuda")
    sp = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for j, r in enumerate(sat_reqs):
        rp, ip = ctypes.c_void_p(r1.data_ptr() + 24 * j), ctypes.c_void_p(r.ptr)
        if r.op == S.TRANSCODE:
            fn = L.gputf_utf8_to_utf16 if r.direction == 0 else L.gputf_utf16_to_utf8
            st = fn(ip, r.units, ctypes.c_void_p(scratch.data_ptr()), r.out_units, ws1.ptr, ws1.nbytes, rp, sp)
        else:
            fn = L.gputf_validate_utf8 if r.direction == 0 else L.gputf_validate_utf16
            st = fn(ip, r.units, ws1.ptr, ws1.nbytes, rp, sp)
        if st != 0:
            raise RuntimeError(f"standalone call status {st}")
    got = r1.cpu().numpy()
    same = all((int(got[j][0]) & 0xFFFFFFFF, int(got[j][1]), int(got[j][2])) == tuple(r.result)
               for j, r in enumerate(sat_reqs))
    invalid = sum(1 for r in sat_reqs if r.result.error != 0)
    # served results and output bytes against the oracle: a seeded sample of
    # the requests, every invalid one, and the largest ones
    import oracle

    def host_input(i):
        src = int(w.source[i])
        if src >= 0:
            return w.texts[src][int(w.offset[i]):int(w.offset[i]) + int(w.units[i])]
        return w.payloads[-1 - src]
    pick = set(np.random.default_rng(1).choice(len(sat_reqs), size=min(args.oracle_sample, len(sat_reqs)),
                                               replace=False).tolist())
    pick |= {j for j, r in enumerate(sat_reqs) if r.result.error != 0}
    pick |= set(np.argsort(w.units)[-10:].tolist())
    # the picked requests served again, all at once, by a server of the same
    # configuration that keeps their outputs: each result must be the timed
    # run's, and result and bytes the oracle's
    vsrv = S.Server(budget_bytes=args.budget_gb << 30, slots=args.slots, max_requests=args.max_requests,
                    big_units=args.big_units, keep_outputs=True)
    all_reqs = requests()
    vreqs = [all_reqs[j] for j in sorted(pick)]
    S.run_arrivals(vsrv, vreqs, np.zeros(len(vreqs)))
    torch.cuda.synchronize()
    oracle_ok = True
    for r in vreqs:
        if tuple(r.result) != tuple(sat_reqs[r.rid].result):
            oracle_ok = False
        h = host_input(r.rid)
        if r.op == S.VALIDATE:
            ref = (oracle.validate_utf8 if r.direction == 0 else oracle.validate_utf16)(h)
            ok = tuple(r.result) == tuple(ref)
        else:
            ref, ref_out = (oracle.utf8_to_utf16 if r.direction == 0 else oracle.utf16_to_utf8)(h)
            ub = 2 if r.direction == 0 else 1
            got_b = r.output[:r.result.written * ub].cpu().numpy()
            ok = tuple(r.result) == tuple(ref) and np.array_equal(got_b, ref_out.view(np.uint8))
        oracle_ok = oracle_ok and ok
    line = {
        "metric": "served transcoding: sustained input GB/s with p50/p99 latency",
        "value": cap_gbs, "unit": "GB/s", "n_gpus": 1, "steps": 1, "warmup": 1,
        "ms_per_step": sat["seconds"] * 1e3, "higher_is_better": True, "dtype": "u8/u16", "data": "synthetic",
        "config": {"workload": f"serve_{w.units.size}_requests_loguniform_64B_16MiB_poisson",
                   "input_bytes": in_bytes, "budget_bytes": srv.budget_bytes, "device_bytes": srv.device_bytes,
                   "slots": len(srv.slots), "max_requests_per_slot": srv.max_requests, "big_units": srv.big_units,
                   "validate_only_requests": int(w.validate_only.sum()), "generation_s": gen_s, "seed": SERVE_SEED},
        "saturated": sat, "levels": levels,
        "p50_ms": levels[1]["p50_ms"], "p99_ms": levels[1]["p99_ms"],
        "invalid_requests": invalid, "results_identical_to_standalone": same,
        "identical_to_oracle": bool(oracle_ok),
        "oracle_check": {"requests": len(pick), "sample": f"{min(args.oracle_sample, len(sat_reqs))} seeded "
                         "requests, every invalid one and the 10 largest, results and output bytes"},
        "gpu_launches": sat["gpu_launches"],
    }
    return line


def run_serve(args):
    print(json.dumps(serve_section(args)), flush=True)
    return 0


def passes_section(args):
    """Every kernel of the path on its own: the two transcoders and the four
    validate / length passes, each timed per launch with CUDA events, with
    achieved algorithmic bytes per second against the measured HBM peak.
    UTF-16 input: the 256 MiB headline buffer (larger than L2).  UTF-8 input:
    --u8-mib MiB (256 by default) of the 4-byte-heavy mix (40% U+10000-10FFFF,
    30% U+0800-FFFF, 30% ASCII), valid; L2 is flushed (a 512 MB write) before
    every timed launch; and the 1 MiB Latin/Cyrillic buffer (90% U+0020-007E, 10%
    U+0400-04FF), which stays in L2 (not flushed): a launch-bound case."""
    import torch

    import paper_2109_10433_gb300 as g

    g.build()
    torch.cuda.set_device(0)
    peak, peak_kind = measured_peak()
    L = g.lib()
    s = torch.cuda.current_stream()
    sp = g._stream(s)
    u16 = W.cjk_emoji_utf16_256mib(nbytes=args.mib << 20)
    u8 = W.utf8_text(2, args.u8_mib << 20, W.MIX_FOUR_BYTE_HEAVY)
    d16 = torch.from_numpy(u16.view(np.int16).copy()).cuda()
    d8 = torch.from_numpy(u8.copy()).cuda()
    n16, n8 = int(u16.size), int(u8.size)
    u8s = W.latin_cyrillic_utf8_1mib()
    d8s = torch.from_numpy(u8s.copy()).cuda()
    n8s = int(u8s.size)
    # script-uniform UTF-16 text of the same size: all U+4E00-9FFF, all ASCII
    cjk = torch.from_numpy(W.utf16_text(5, n16, W.SCRIPT_CJK).view(np.int16).copy()).cuda()
    asc = torch.from_numpy(W.utf16_text(6, n16, W.SCRIPT_ASCII).view(np.int16).copy()).cuda()
    out8 = torch.empty(3 * n16, dtype=torch.uint8, device="cuda")
    out16 = torch.empty(n8, dtype=torch.int16, device="cuda")
    ws = g.Workspace(max(n16, n8) + 16)
    res = torch.zeros(3, dtype=torch.int64, device="cuda")
    ln = torch.zeros(1, dtype=torch.int64, device="cuda")
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    len8 = g.utf8_length_from_utf16(d16, ws=ws)
    len16 = g.utf16_length_from_utf8(d8, ws=ws)
    len16s = g.utf16_length_from_utf8(d8s, ws=ws)
    inputs = {"utf16": ("utf16 %d MiB cjk/emoji" % args.mib, 2 * n16),
              "utf8": ("utf8 %d MiB four-byte-heavy" % args.u8_mib, n8),
              "utf8_l2": ("utf8 1 MiB latin/cyrillic, L2-resident", n8s)}
    cases = [
        ("utf16_to_utf8", "utf16", lambda: L.gputf_utf16_to_utf8(g._ptr(d16), n16, g._ptr(out8), 3 * n16, ws.ptr,
                                                                 ws.nbytes, g._ptr(res), sp), 2 * n16 + len8),
        ("utf16_to_utf8_unchecked", "utf16", lambda: L.gputf_utf16_to_utf8_unchecked(
            g._ptr(d16), n16, g._ptr(out8), 3 * n16, ws.ptr, ws.nbytes, g._ptr(res), sp), 2 * n16 + len8),
        ("utf16_to_utf8 cjk-only", "utf16", lambda: L.gputf_utf16_to_utf8(
            g._ptr(cjk), n16, g._ptr(out8), 3 * n16, ws.ptr, ws.nbytes, g._ptr(res), sp), 2 * n16 + 3 * n16),
        ("utf16_to_utf8 ascii-only", "utf16", lambda: L.gputf_utf16_to_utf8(
            g._ptr(asc), n16, g._ptr(out8), 3 * n16, ws.ptr, ws.nbytes, g._ptr(res), sp), 2 * n16 + n16),
        ("validate_utf16", "utf16", lambda: L.gputf_validate_utf16(g._ptr(d16), n16, ws.ptr, ws.nbytes, g._ptr(res),
                                                                   sp), 2 * n16),
        ("utf8_length_from_utf16", "utf16", lambda: L.gputf_utf8_length_from_utf16(g._ptr(d16), n16, ws.ptr,
                                                                                   ws.nbytes, g._ptr(ln), sp), 2 * n16),
        ("utf8_to_utf16", "utf8", lambda: L.gputf_utf8_to_utf16(g._ptr(d8), n8, g._ptr(out16), n8, ws.ptr, ws.nbytes,
                                                                g._ptr(res), sp), n8 + 2 * len16),
        ("utf8_to_utf16_unchecked", "utf8", lambda: L.gputf_utf8_to_utf16_unchecked(
            g._ptr(d8), n8, g._ptr(out16), n8, ws.ptr, ws.nbytes, g._ptr(res), sp), n8 + 2 * len16),
        ("validate_utf8", "utf8", lambda: L.gputf_validate_utf8(g._ptr(d8), n8, ws.ptr, ws.nbytes, g._ptr(res), sp),
         n8),
        ("utf16_length_from_utf8", "utf8", lambda: L.gputf_utf16_length_from_utf8(g._ptr(d8), n8, ws.ptr, ws.nbytes,
                                                                                   g._ptr(ln), sp), n8),
        ("utf8_to_utf16 1 MiB", "utf8_l2", lambda: L.gputf_utf8_to_utf16(g._ptr(d8s), n8s, g._ptr(out16), n8s, ws.ptr,
                                                                         ws.nbytes, g._ptr(res), sp), n8s + 2 * len16s),
    ]
    rows = []
    clocks = ClockSampler(None)
    clocks.start()
    for name, src, fn, algo in cases:
        for _ in range(max(args.warmup, 3)):
            if fn() != 0:
                raise RuntimeError(name)
        torch.cuda.synchronize()
        ms = []
        for _ in range(args.steps):
            if src == "utf8":
                flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            fn()
            e1.record(s)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        us = statistics.median(ms) * 1e3
        gbs = algo / (us * 1e-6) / 1e9
        desc, in_bytes = inputs[src]
        rows.append({"kernel": name, "input": desc, "input_bytes": in_bytes,
                     "algorithmic_bytes": int(algo), "median_us": us, "min_us": min(ms) * 1e3,
                     "input_gbs": in_bytes / (us * 1e-6) / 1e9,
                     "achieved_gbs": gbs, "frac": gbs / peak})
    clk = clocks.stop()
    return {"metric": "per-kernel algorithmic GB/s vs HBM roofline", "unit": "GB/s",
            "peak": peak, "peak_source": peak_kind, "steps": args.steps, "kernels": rows, "clocks": clk}


def run_passes(args):
    print(json.dumps(passes_section(args)), flush=True)
    return 0


def sweep_section(args):
    """Throughput against input size: single calls of both transcoders on
    sizes from 16 units to the whole buffer, and the batched call on many
    strings of one size (up to 64 Ki units), each timed over back-to-back
    launches with CUDA events.  UTF-16 input: the headline mix; UTF-8 input:
    the 4-byte-heavy mix; cuts never split a character."""
    import ctypes

    import torch

    import paper_2109_10433_gb300 as g
    from paper_2109_10433_gb300 import batch as B

    g.build()
    torch.cuda.set_device(0)
    L = g.lib()
    s = torch.cuda.current_stream()
    sp = g._stream(s)
    u16 = W.cjk_emoji_utf16_256mib(nbytes=args.mib << 20)
    u8 = W.utf8_text(2, 64 << 20, W.MIX_FOUR_BYTE_HEAVY)
    d16 = torch.from_numpy(u16.view(np.int16).copy()).cuda()
    d8 = torch.from_numpy(u8.copy()).cuda()
    out8 = torch.empty(3 * u16.size, dtype=torch.uint8, device="cuda")
    out16 = torch.empty(u8.size, dtype=torch.int16, device="cuda")
    ws = g.Workspace(max(u16.size, u8.size) + 16)
    res = torch.zeros(3, dtype=torch.int64, device="cuda")
    is_high = (u16 & 0xFC00) == 0xD800
    is_cont8 = (u8 & 0xC0) == 0x80

    def timed(fn, reps):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(reps):
            fn()
        e1.record(s)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) * 1e3 / reps

    rows = []
    clocks = ClockSampler(device_uuid())
    clocks.start()
    sizes = [16 << (2 * k) for k in range(12)] + [u16.size]
    for n in sizes:
        n16 = min(n, u16.size)
        if is_high[n16 - 1]:
            n16 -= 1
        reps = 200 if n16 < (1 << 20) else 20
        us16 = timed(lambda: L.gputf_utf16_to_utf8(g._ptr(d16), n16, g._ptr(out8), 3 * n16, ws.ptr, ws.nbytes,
                                                   g._ptr(res), sp), reps)
        row = {"units": n16, "utf16_to_utf8_us": us16, "utf16_to_utf8_input_gbs": 2 * n16 / us16 / 1e3}
        n8 = min(n, u8.size)
        while n8 < u8.size and is_cont8[n8]:
            n8 -= 1
        us8 = timed(lambda: L.gputf_utf8_to_utf16(g._ptr(d8), n8, g._ptr(out16), n8, ws.ptr, ws.nbytes,
                                                  g._ptr(res), sp), reps)
        row.update({"utf8_bytes": n8, "utf8_to_utf16_us": us8, "utf8_to_utf16_input_gbs": n8 / us8 / 1e3})
        if n <= (64 << 10):
            count = min(100000, (u16.size - 1) // n)
            cuts = np.arange(count + 1, dtype=np.int64) * n
            cuts[1:] -= is_high[cuts[1:] - 1]          # never split a pair
            off = torch.from_numpy(cuts).cuda()
            caps = torch.from_numpy(cuts * 3).cuda()
            results = torch.zeros((count, 3), dtype=torch.int64, device="cuda")
            cb = B.CBatch(count, int(cuts[-1]), d16.data_ptr(), off.data_ptr(), out8.data_ptr(), caps.data_ptr(),
                          results.data_ptr())
            bws = g.Workspace.of_bytes(int(L.gputf_batch_workspace_bytes(0, 0, int(cuts[-1]), count)))
            usb = timed(lambda: L.gputf_batch_transcode(None, ctypes.byref(cb), 0, bws.ptr, bws.nbytes, sp), 20)
            row.update({"batch_strings": count, "batch_us": usb, "batch_strings_per_s": count / (usb * 1e-6),
                        "batch_input_gbs": 2 * int(cuts[-1]) / usb / 1e3})
        rows.append(row)
    clk = clocks.stop()
    return {"metric": "throughput vs input size (single calls and batched)", "sweep": rows, "clocks": clk}


def run_sweep(args):
    print(json.dumps(sweep_section(args)), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--e2e-warmup", type=int, default=2)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mib", type=int, default=256,
                    help="input MiB of the UTF-16 workload (256 is the measured configuration; "
                         "smaller sizes are for profiler captures)")
    ap.add_argument("--u8-mib", type=int, default=256,
                    help="input MiB of the four-byte-heavy UTF-8 workload in --workload passes")
    ap.add_argument("--workload", default="utf16_256mib", choices=["utf16_256mib", "batch", "serve", "passes", "sweep"])
    ap.add_argument("--requests", type=int, default=20000)
    ap.add_argument("--budget-gb", type=int, default=8)
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--max-requests", type=int, default=4096)
    ap.add_argument("--big-units", type=int, default=1 << 20)
    ap.add_argument("--strings", type=int, default=100000)
    ap.add_argument("--sample", type=int, default=2000)
    ap.add_argument("--oracle-sample", type=int, default=400)
    ap.add_argument("--headline-only", action="store_true",
                    help="time only the 256 MiB UTF-16 -> UTF-8 configuration (profiler captures)")
    args = ap.parse_args()
    if args.workload == "batch" and args.impl != "reference":
        return run_batch(args)
    if args.workload == "serve" and args.impl != "reference":
        return run_serve(args)
    if args.workload == "passes" and args.impl != "reference":
        return run_passes(args)
    if args.workload == "sweep" and args.impl != "reference":
        return run_sweep(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
