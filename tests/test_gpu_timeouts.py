"""GPU tests of failure detection: the kernels' bounded waits end.

gputf_test_wait_timeout runs one of the waits the kernels use between
thread blocks, the decoupled look-back of the output offsets and the wait on
a tile copy's shared-memory barrier, against a partner that never arrives,
with a small poll limit.  Each must come back as GPUTF_TIMEOUT, quickly, with
the GPU still usable; the workspace it ran on must then serve a normal call
bit-exactly, without being prepared again (every call's last block resets
it) and after being prepared again."""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TIMEOUT = 8


@pytest.fixture(scope="module")
def g():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2109_10433_gb300 as g
    g.build()
    return g


def _timed_out_call(g, ws, which, polls):
    res = torch.zeros(3, dtype=torch.int64, device="cuda")
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    st = g.lib().gputf_test_wait_timeout(ws.ptr, ws.nbytes, which, polls, g._ptr(res), g._stream(s))
    e1.record(s)
    torch.cuda.synchronize()
    assert st == 0
    return g.read_result(res), e0.elapsed_time(e1)


def _exact_call(g, ws, units):
    r, out = g.utf16_to_utf8(torch.from_numpy(units.view(np.int16).copy()).cuda(), ws=ws)
    ref, ref_out = oracle.utf16_to_utf8(units)
    assert tuple(r) == tuple(ref)
    assert np.array_equal(out[:r.written].cpu().numpy(), ref_out)


@pytest.mark.parametrize("which,polls,limit_ms", [(0, 256, 1.0), (1, 256, 50.0)],
                         ids=["look-back", "copy-barrier"])
def test_bounded_wait_times_out_and_the_workspace_serves_again(g, which, polls, limit_ms):
    units = W.utf16_text(77, 300_001, W.MIX_CJK_EMOJI)
    ws = g.Workspace(units.size)
    _exact_call(g, ws, units)                     # the workspace in use before
    r, ms = _timed_out_call(g, ws, which, polls)
    assert r.error == TIMEOUT and r.position == 0 and r.written == 0
    assert ms < limit_ms, ms
    _exact_call(g, ws, units)                     # no re-initialisation needed
    _exact_call(g, ws, W.utf16_text(78, 123_457, W.SCRIPT_MIXED))
    r, _ = _timed_out_call(g, ws, which, polls)
    assert r.error == TIMEOUT
    ws.reset()                                    # and re-initialising is harmless
    _exact_call(g, ws, units)
