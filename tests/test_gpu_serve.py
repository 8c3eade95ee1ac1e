"""GPU tests of the continuous-batching server: every request's result and
output are those it gets alone (the single-string call on the same input)
and those of the oracle; requests are admitted in arrival order within each
slot's memory budget; slots' work overlaps on the device."""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MiB = 1 << 20


@pytest.fixture(scope="module")
def g():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2109_10433_gb300 as g
    g.build()
    return g


@pytest.fixture(scope="module")
def work():
    return W.serve_workload(5, 400, min_bytes=64, max_bytes=2 * MiB, text_bytes=4 * MiB)


def host_input(w, i):
    s = int(w.source[i])
    if s >= 0:
        return w.texts[s][int(w.offset[i]):int(w.offset[i]) + int(w.units[i])]
    return w.payloads[-1 - s]


def build_requests(w, extra_empty=True):
    from paper_2109_10433_gb300 import serve as S
    pool = S.DevicePool(list(w.texts) + list(w.payloads))
    reqs = []
    for i in range(w.units.size):
        s = int(w.source[i])
        k = s if s >= 0 else len(w.texts) + (-1 - s)
        ub = 1 + int(w.direction[i])
        reqs.append(S.Request(i, int(w.direction[i]), S.VALIDATE if w.validate_only[i] else S.TRANSCODE,
                              pool.ptr(k, int(w.offset[i]) * ub), int(w.units[i])))
    if extra_empty:   # empty requests of every kind
        for d in (0, 1):
            for op in (S.TRANSCODE, S.VALIDATE):
                reqs.append(S.Request(len(reqs), d, op, pool.ptr(0), 0))
    return pool, reqs


def standalone(g, pool, r):
    """The single-string call on the request's own input."""
    from paper_2109_10433_gb300 import serve as S
    k_off = r.ptr - pool.buf.data_ptr()
    inp = pool.buf[k_off:k_off + r.in_bytes]
    if r.direction == 1:
        inp = inp.view(torch.int16)
    if r.op == S.VALIDATE:
        return (g.validate_utf8(inp) if r.direction == 0 else g.validate_utf16(inp)), None
    return g.utf8_to_utf16(inp) if r.direction == 0 else g.utf16_to_utf8(inp)


def check_all(g, w, pool, reqs):
    from paper_2109_10433_gb300 import serve as S
    torch.cuda.synchronize()
    n_invalid = 0
    for r in reqs:
        assert r.result is not None, r.rid
        alone, out = standalone(g, pool, r)
        assert tuple(r.result) == tuple(alone), (r.rid, r.result, alone)
        host = host_input(w, r.rid) if r.rid < w.units.size else np.zeros(0, np.uint8 if r.direction == 0 else np.uint16)
        if r.op == S.VALIDATE:
            ref = (oracle.validate_utf8 if r.direction == 0 else oracle.validate_utf16)(host)
        else:
            ref, ref_out = (oracle.utf8_to_utf16 if r.direction == 0 else oracle.utf16_to_utf8)(host)
        assert tuple(r.result) == tuple(ref), (r.rid, r.result, ref)
        n_invalid += r.result.error != 0
        if r.op == S.TRANSCODE:
            ub = 2 if r.direction == 0 else 1
            got = r.output[:r.result.written * ub].cpu().numpy()
            alone_b = out.reshape(-1).view(torch.uint8)[:r.result.written * ub].cpu().numpy()
            assert np.array_equal(got, alone_b), r.rid
            assert np.array_equal(got, ref_out.view(np.uint8)), r.rid
    return n_invalid


def test_served_results_equal_standalone_and_oracle(g, work):
    """Poisson arrivals over several slots; small requests batched, large
    ones in place: each result and output is the single call's and the
    oracle's, bit for bit."""
    from paper_2109_10433_gb300 import serve as S
    pool, reqs = build_requests(work)
    srv = S.Server(budget_bytes=256 * MiB, slots=3, max_requests=256, big_units=128 << 10, keep_outputs=True)
    rng = np.random.default_rng(0)
    times = np.cumsum(rng.exponential(2e-4, len(reqs)))
    S.run_arrivals(srv, reqs, times)
    assert len(srv.completed) == len(reqs)
    assert srv.batches > 3
    n_invalid = check_all(g, work, pool, reqs)
    assert n_invalid >= int(work.invalid.sum()) > 0


def test_served_form_at_full_request_sizes(g):
    """The served form's own sizes: requests log-uniform from 64 B to 16 MiB
    of input (a tenth of them 4 MiB or more), an 8 GiB admission budget over
    four slots, the benchmark's split between batched and in-place requests,
    Poisson arrivals that keep several slots busy.  Every result and every
    output byte equals the oracle's and the single call's."""
    from paper_2109_10433_gb300 import serve as S
    w = W.serve_workload(9, 240)
    sizes = w.input_bytes()
    assert int((sizes >= 4 * MiB).sum()) >= 10 and int(sizes.max()) > 12 * MiB and int(sizes.min()) < 256
    pool, reqs = build_requests(w)
    srv = S.Server(budget_bytes=8 << 30, slots=4, max_requests=4096, big_units=1 << 20, keep_outputs=True)
    rng = np.random.default_rng(1)
    times = np.cumsum(rng.exponential(1e-4, len(reqs)))
    S.run_arrivals(srv, reqs, times)
    assert len(srv.completed) == len(reqs)
    assert srv.batches >= 4
    n_invalid = check_all(g, w, pool, reqs)
    assert n_invalid >= int(w.invalid.sum())


def test_one_request_at_a_time_equals_mix(g, work):
    """The same requests served one per batch give the same results as in
    the mix (a request's result does not depend on its batch)."""
    from paper_2109_10433_gb300 import serve as S
    pool, reqs = build_requests(work, extra_empty=False)
    reqs = reqs[:120]
    mix = S.Server(budget_bytes=128 * MiB, slots=2, max_requests=512, big_units=1 << 30, keep_outputs=True)
    for r in reqs:
        mix.submit(r)
    mix.drain()
    torch.cuda.synchronize()
    got = {r.rid: (tuple(r.result), r.output.cpu().numpy() if r.output is not None else None) for r in reqs}
    _, alone_reqs = build_requests(work, extra_empty=False)
    alone_reqs = alone_reqs[:120]
    one = S.Server(budget_bytes=128 * MiB, slots=1, max_requests=1, big_units=1 << 30, keep_outputs=True)
    for r in alone_reqs:
        one.submit(r)
        one.drain()
    torch.cuda.synchronize()
    assert one.batches == len(alone_reqs)
    for r in alone_reqs:
        res, out = got[r.rid]
        assert tuple(r.result) == res, r.rid
        if out is not None:
            ub = 2 if r.direction == 0 else 1
            assert np.array_equal(out[:res[2] * ub], r.output.cpu().numpy()[:res[2] * ub]), r.rid


def test_admission_order_budget_and_overlap(g, work):
    """A small budget forces many batches: requests leave in arrival order
    except where a later one that fits went ahead of one that did not (a
    bounded number of times), no batch holds more than its arena, and the
    slots' launches overlap in device time."""
    from paper_2109_10433_gb300 import serve as S
    pool, reqs = build_requests(work, extra_empty=False)
    # every request through the batched kernel, so that a batch's device time
    # exceeds the host time of the next launch
    srv = S.Server(budget_bytes=192 * MiB, slots=4, max_requests=32, big_units=1 << 30, trace=True)
    too_big = S.Request(-1, 1, S.TRANSCODE, pool.ptr(0), srv.slots[0].arena_bytes)
    with pytest.raises(ValueError):
        srv.submit(too_big)
    S.run_arrivals(srv, reqs, np.zeros(len(reqs)))
    torch.cuda.synchronize()
    # a request is served after a later one only when that one went ahead
    # of it while it did not fit, and that happens in a bounded number of fills
    by_rid = sorted(reqs, key=lambda r: r.rid)
    for i, r in enumerate(by_rid):
        overtaken = any(q.batch < r.batch for q in by_rid[i + 1:])
        assert not overtaken or r.bypassed >= 1, r.rid
        assert r.bypassed <= S.Server.MAX_BYPASS, r.rid
    per_batch = {}
    for r in reqs:
        per_batch[r.batch] = per_batch.get(r.batch, 0) + srv.footprint(r)
    assert max(per_batch.values()) <= srv.slots[0].arena_bytes
    assert srv.batches >= 8
    ref = srv.trace_events[0][1]
    spans = [(sl, ref.elapsed_time(a), ref.elapsed_time(b)) for sl, a, b, _ in srv.trace_events]
    overlaps = sum(1 for i, (si, a0, a1) in enumerate(spans) for sj, b0, b1 in spans[i + 1:]
                   if si != sj and a0 < b1 and b0 < a1)
    assert overlaps > 0, spans
    check_ok = [r for r in reqs if r.result is None]
    assert not check_ok
