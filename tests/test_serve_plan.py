"""Host logic of the served batches, without a GPU: gputf_serve_plan (the
planning pass of gputf_serve_launch) gives every request a result row and
arena ranges that do not overlap, aligned where the kernels need it, grouped
as the header states, and never needs more arena than the admission
footprints the server charges."""
import numpy as np
import pytest

from paper_2109_10433_gb300 import serve as S

NOWHERE = S.NOWHERE


def make(rng, n, big_units):
    reqs = []
    ptr = 1 << 40
    for i in range(n):
        d = int(rng.integers(0, 2))
        op = int(rng.integers(0, 2))
        units = int(rng.choice([0, 1, 3, 1000, 70000, big_units - 1, big_units, 3 * big_units]))
        reqs.append(S.Request(i, d, op, ptr + (i % 7) * (1 + d), units))
        ptr += 1 << 30
    return reqs


def footprint(r):
    return r.in_bytes + r.out_bytes + 256


@pytest.mark.parametrize("trial", range(20))
def test_plan_rows_ranges_and_budget(trial):
    rng = np.random.default_rng(trial)
    big_units = 200000
    reqs = make(rng, int(rng.integers(1, 80)), big_units)
    place, arena, meta = S.plan(reqs, big_units)
    n = len(reqs)
    rows = place["row"].astype(np.int64)
    assert sorted(rows.tolist()) == list(range(n))
    # rows: groups (direction, op) in order, then large requests; order kept within each
    def key(r):
        return (4, 0) if r.units >= big_units else (2 * r.direction + r.op, 0)
    expect = sorted(range(n), key=lambda i: (key(reqs[i]), i))
    assert [int(np.nonzero(rows == k)[0][0]) for k in range(n)] == expect
    ranges = []
    for r, p in zip(reqs, place):
        big = r.units >= big_units
        assert (int(p["in_offset"]) == NOWHERE) == big
        if not big and r.units:
            a = int(p["in_offset"])
            if r.direction == 1:
                assert a % 2 == 0
            ranges.append((a, a + r.in_bytes))
        if r.op == S.VALIDATE:
            assert int(p["out_offset"]) == NOWHERE
        elif r.units:
            a = int(p["out_offset"])
            if r.direction == 0:
                assert a % 2 == 0
            if big:
                assert a % 256 == 0
            ranges.append((a, a + r.out_bytes))
    ranges.sort()
    for (a0, a1), (b0, b1) in zip(ranges, ranges[1:]):
        assert a1 <= b0
    assert not ranges or ranges[-1][1] <= arena
    # the server admits a batch when its footprints fit arena - 4 * 256
    assert arena <= sum(footprint(r) for r in reqs) + 4 * 256
    # metadata within what a slot allocates for this many requests and bytes
    from paper_2109_10433_gb300 import lib
    assert meta <= lib().gputf_serve_meta_bytes(n, arena)


def test_plan_rejects_bad_requests():
    from paper_2109_10433_gb300 import GputfError
    with pytest.raises(GputfError):
        S.plan([S.Request(0, 2, S.TRANSCODE, 1 << 40, 5)], 100)       # bad direction
    with pytest.raises(GputfError):
        S.plan([S.Request(0, 1, S.TRANSCODE, (1 << 40) + 1, 5)], 100)  # misaligned UTF-16
    with pytest.raises(GputfError):
        S.plan([S.Request(0, 0, S.TRANSCODE, 0, 5)], 100)              # NULL input


def test_capacities_always_suffice():
    r8 = S.Request(0, 0, S.TRANSCODE, 0, 10)
    r16 = S.Request(1, 1, S.TRANSCODE, 0, 10)
    v = S.Request(2, 1, S.VALIDATE, 0, 10)
    assert (r8.out_units, r8.out_bytes) == (10, 20)      # n units for n bytes
    assert (r16.out_units, r16.out_bytes) == (30, 30)    # 3 bytes per unit
    assert (v.out_units, v.out_bytes) == (0, 0)
