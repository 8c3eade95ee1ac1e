"""Host logic of the serving loop, without a GPU: admission and completion.

The server's slots are replaced by stand-ins (no stream, no device memory) and
its launch by a recorder, so the test sees what the loop itself decides:
  - a free slot takes waiting requests in arrival order while their
    footprints (input bytes, output capacity, alignment slack) fit its arena,
    and at most max_requests of them; a request that does not fit lets later
    ones that do go ahead, in at most MAX_BYPASS fills, and then holds back
    every request behind it until it is admitted;
  - a request larger than any slot is refused when submitted;
  - a slot is launched once per fill and not refilled while in flight;
  - on completion every request of the slot gets the result row its
    placement names, and the slot is free again;
  - requests that arrive while a slot is in flight go to another free slot;
  - a waiting request can be withdrawn, one in a slot cannot; a request
    still waiting at its deadline is dropped unrun, and requests without a
    deadline never are.
"""
from types import SimpleNamespace

import numpy as np
import pytest

from paper_2109_10433_gb300 import serve as S

A = S._ALIGN


class FakeEvent:
    def __init__(self):
        self.done = False

    def query(self):
        return self.done


class FakeHost:
    def __init__(self, rows):
        self.rows = rows

    def numpy(self):
        return self.rows


def fake_slot(index, arena_bytes, max_requests=8):
    return SimpleNamespace(index=index, arena_bytes=arena_bytes, requests=[], used=0, in_flight=False,
                           event=FakeEvent(), place=np.zeros(max_requests, dtype=S.PLACEMENT_DTYPE),
                           res_host=FakeHost(np.zeros((max_requests, 3), dtype=np.int64)))


def fake_server(slots, max_requests=8):
    srv = object.__new__(S.Server)
    srv.slots = slots
    srv.max_requests = max_requests
    srv.waiting, srv.completed, srv.cancelled, srv.expired = [], [], [], []
    srv._deadlines = 0
    srv.batches = 0
    srv.launched = []

    def launch(slot):
        srv.launched.append((slot.index, [r.rid for r in slot.requests]))
        # placement rows in reverse order, so that results must follow the rows
        n = len(slot.requests)
        slot.place["row"][:n] = np.arange(n)[::-1]
        slot.in_flight = True
        srv.batches += 1
    srv._launch = launch
    return srv


def req(rid, units, direction=0, op=S.TRANSCODE):
    return S.Request(rid, direction, op, 1 << 20, units)


def test_footprint():
    srv = fake_server([fake_slot(0, 1 << 20)])
    assert srv.footprint(req(0, 100)) == 100 + 200 + A                      # UTF-8 in, n UTF-16 units out
    assert srv.footprint(req(1, 100, direction=1)) == 200 + 300 + A         # UTF-16 in, 3n bytes out
    assert srv.footprint(req(2, 100, direction=1, op=S.VALIDATE)) == 200 + A


def test_fill_in_arrival_order_within_the_arena():
    cap = 10 * 1024
    slot = fake_slot(0, cap + 4 * A)
    srv = fake_server([slot])
    big = req(2, 3000)                          # 3000 + 6000 + 256 bytes
    srv.waiting = [req(0, 1000), req(1, 200), big, req(3, 10), req(4, 10)]
    srv._fill(slot)
    # 3256 + 856 fit; the big one would pass the cap and waits, the two small
    # ones after it go ahead of it
    assert [r.rid for r in slot.requests] == [0, 1, 3, 4]
    assert [r.rid for r in srv.waiting] == [2]
    assert big.bypassed == 1
    assert slot.used == sum(srv.footprint(r) for r in slot.requests)
    assert slot.used <= cap


def test_a_request_left_behind_is_overtaken_a_bounded_number_of_times():
    cap = 10 * 1024
    srv = fake_server([fake_slot(0, cap + 4 * A)])
    big = req(1, 3000)                          # 9256 bytes: fits only an empty slot
    srv.waiting = [req(0, 300), big] + [req(2 + i, 300) for i in range(40)]
    slot = fake_slot(0, cap + 4 * A)
    srv._fill(slot)
    assert slot.requests[0].rid == 0 and big in srv.waiting and big.bypassed == 1
    slot = fake_slot(0, cap + 4 * A)            # the next free slot takes it first
    srv._fill(slot)
    assert slot.requests[0] is big
    # once overtaken MAX_BYPASS times, nothing behind it goes ahead any more
    srv = fake_server([fake_slot(0, cap + 4 * A)])
    big = req(1, 3000)
    big.bypassed = S.Server.MAX_BYPASS
    srv.waiting = [req(0, 300), big] + [req(2 + i, 300) for i in range(10)]
    slot = fake_slot(0, cap + 4 * A)
    srv._fill(slot)
    assert [r.rid for r in slot.requests] == [0]
    assert [r.rid for r in srv.waiting] == list(range(1, 12))


def test_lookahead_is_bounded():
    cap = 10 * 1024
    srv = fake_server([fake_slot(0, cap + 4 * A)], max_requests=10000)
    srv.waiting = [req(0, 3000), req(1, 3000)] + [req(2 + i, 1) for i in range(1000)]
    slot = fake_slot(0, cap + 4 * A, max_requests=10000)
    srv._fill(slot)
    assert len(slot.requests) <= S.Server.LOOKAHEAD + 2


def test_fill_stops_at_max_requests():
    slot = fake_slot(0, 1 << 20, max_requests=3)
    srv = fake_server([slot], max_requests=3)
    srv.waiting = [req(i, 10) for i in range(7)]
    srv._fill(slot)
    assert [r.rid for r in slot.requests] == [0, 1, 2]
    assert len(srv.waiting) == 4


def test_submit_refuses_a_request_larger_than_a_slot():
    srv = fake_server([fake_slot(0, 4096 + 4 * A)])
    srv.submit(req(0, 1000))
    with pytest.raises(ValueError):
        srv.submit(req(1, 2000))                # 2000 + 4000 + 256 > 4096
    assert [r.rid for r in srv.waiting] == [0]


def test_step_launches_completes_and_refills():
    s0, s1 = fake_slot(0, 1 << 16), fake_slot(1, 1 << 16)
    srv = fake_server([s0, s1])
    for i in range(3):
        srv.submit(req(i, 10))
    assert srv.step() is True                  # all three go to slot 0 (they fit), slot 1 stays idle
    assert srv.launched == [(0, [0, 1, 2])] and s0.in_flight and not s1.in_flight
    # requests arriving while slot 0 is in flight go to slot 1
    srv.submit(req(3, 10))
    srv.submit(req(4, 10))
    assert srv.step() is True
    assert srv.launched[-1] == (1, [3, 4])
    # nothing new while both are in flight
    assert srv.step() is True and len(srv.launched) == 2
    # slot 0 completes: results by placement row (rows were assigned in reverse)
    s0.res_host.rows[:3] = [[0, 10, 20], [5, 7, 0], [6, 3, 1]]
    s0.event.done = True
    assert srv.step() is True                  # slot 1 still in flight
    got = {r.rid: tuple(r.result) for r in srv.completed}
    assert got == {0: (6, 3, 1), 1: (5, 7, 0), 2: (0, 10, 20)}
    assert all(r.done is not None for r in srv.completed)
    assert not s0.in_flight and s0.requests == [] and s0.used == 0
    s1.event.done = True
    assert srv.step() is False                 # nothing waiting, nothing in flight
    assert sorted(r.rid for r in srv.completed) == [0, 1, 2, 3, 4]


def test_result_error_word_keeps_the_low_32_bits():
    """The result row's first word holds the error class in its low 32 bits
    (the C struct's int32 error and int32 reserved)."""
    slot = fake_slot(0, 1 << 16)
    srv = fake_server([slot])
    srv.submit(req(0, 10))
    srv.step()
    slot.res_host.rows[0] = [(0x1234 << 32) | 6, 4, 2]
    slot.event.done = True
    srv.step()
    assert tuple(srv.completed[0].result) == (6, 4, 2)


def test_cancel_withdraws_only_waiting_requests():
    slot = fake_slot(0, 1 << 16, max_requests=2)
    srv = fake_server([slot], max_requests=2)
    for i in range(4):
        srv.submit(req(i, 10))
    srv.step()                                   # 0 and 1 go out, 2 and 3 wait
    assert srv.cancel(0) is False                # in flight: runs to the end
    assert srv.cancel(3) is True and srv.cancel(3) is False
    assert [r.rid for r in srv.cancelled] == [3] and [r.rid for r in srv.waiting] == [2]
    slot.event.done = True
    srv.step()                                   # 0 and 1 complete, 2 goes out
    slot.event.done = False
    assert srv.launched[-1] == (0, [2])
    slot.event.done = True
    assert srv.step() is False
    assert sorted(r.rid for r in srv.completed) == [0, 1, 2]


def test_deadlines_drop_requests_still_waiting():
    slot = fake_slot(0, 1 << 16, max_requests=1)
    srv = fake_server([slot], max_requests=1)
    now = S.time.perf_counter()
    r0 = req(0, 10)
    r0.deadline = now - 1.0                      # already past when the loop first runs
    srv.submit(r0)
    r1, r2, r3 = req(1, 10), req(2, 10), req(3, 10)
    r1.deadline = now - 1.0                      # past: dropped while waiting
    r2.deadline = now + 3600.0                   # far ahead: runs
    for r in (r1, r2, r3):                       # r3 has no deadline
        srv.submit(r)
    assert srv._deadlines == 3
    srv.step()
    # expiry comes before filling: r0 and r1 are dropped unrun, r2 goes out
    assert sorted(r.rid for r in srv.expired) == [0, 1]
    assert all(r.result is None and r.done is not None for r in srv.expired)
    assert srv.launched == [(0, [2])] and srv._deadlines == 0
    slot.event.done = True
    srv.step()
    slot.event.done = False
    assert srv.launched[-1] == (0, [3])
    slot.event.done = True
    assert srv.step() is False
    assert sorted(r.rid for r in srv.completed) == [2, 3]


def test_budget_too_small_for_the_slots_is_refused():
    with pytest.raises(ValueError):
        S.Server(budget_bytes=1 << 20, slots=4, max_requests=4096)


def test_server_splits_the_budget_into_slots(monkeypatch):
    """The constructor's arithmetic with stand-in slots: every slot's arena,
    workspaces, metadata and result rows fit its share of the budget."""
    made = []

    class StandInSlot:
        def __init__(self, index, arena_bytes, max_requests, ws_batch, ws_single, meta_bytes, device):
            self.index, self.arena_bytes = index, arena_bytes
            self.parts = (arena_bytes, ws_batch, ws_single, meta_bytes, 24 * max_requests)
            made.append(self)

        def device_bytes(self):
            return sum(self.parts)

    monkeypatch.setattr(S, "_Slot", StandInSlot)
    srv = S.Server(budget_bytes=8 << 30, slots=4, max_requests=4096)
    assert len(made) == 4 and all(s.arena_bytes % A == 0 for s in made)
    assert all(s.device_bytes() <= (8 << 30) // 4 for s in made)
    assert srv.device_bytes <= 8 << 30
    assert made[0].arena_bytes > (8 << 30) // 4 * 0.9          # the arena takes most of the share
    assert srv.waiting == [] and srv.expired == [] and srv.cancelled == [] and srv._deadlines == 0
