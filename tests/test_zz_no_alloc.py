"""GPU test of gputf_utf16_to_utf8_static, the UTF-16 -> UTF-8 entry point
that allocates nothing and keeps its scratch in a fixed array inside the
library (for callers that cannot allocate device memory while they run).

Its results and output must equal those of gputf_utf16_to_utf8 (which takes a
workspace from the caller) and the oracle's, exactly, on two calls in a row: the second call
reuses the array as the first left it.  The file is collected last so that a
run stopping at the first failure has run every other test before it."""
import ctypes

import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2109_10433_gb300 as g
    g.build()
    return g


def _static_call(g, inp, out, res):
    n = inp.numel()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return g.lib().gputf_utf16_to_utf8_static(g._ptr(inp), n, g._ptr(out), out.numel(), g._ptr(res), stream)


def _compare(g, units):
    inp = torch.from_numpy(np.ascontiguousarray(units).view(np.int16)).cuda()
    cap = 3 * units.size + 1
    out_ref = torch.full((cap,), 0x5A, dtype=torch.uint8, device="cuda")
    out_new = torch.full((cap,), 0xA5, dtype=torch.uint8, device="cuda")
    ref, _ = g.utf16_to_utf8(inp, out=out_ref)
    res = torch.zeros(3, dtype=torch.int64, device="cuda")
    assert _static_call(g, inp, out_new, res) == 0
    got = g.read_result(res)
    assert tuple(got) == tuple(ref)
    assert torch.equal(out_new[:got.written], out_ref[:ref.written])
    # and against the oracle itself, result and bytes
    o_res, o_out = oracle.utf16_to_utf8(units)
    assert tuple(got) == tuple(o_res)
    assert np.array_equal(out_new[:got.written].cpu().numpy(), o_out)
    return got


def test_static_scratch_matches_workspace_entry_point_on_two_calls(g):
    # first call: a valid multi-tile buffer, sized at the stated maximum
    big = W.utf16_text(41, 1 << 25, W.MIX_CJK_EMOJI)
    r1 = _compare(g, big)
    assert r1.error == 0 and r1.position == big.size
    # second call, straight after: other text with a lone surrogate
    small = W.utf16_text(42, 3_000_001, W.SCRIPT_MIXED).copy()
    small[2_500_000] = 0xDC00
    r2 = _compare(g, small)
    assert r2.error == 6


def test_static_scratch_refuses_inputs_past_the_maximum(g):
    n = (1 << 25) + 1
    status = g.lib().gputf_utf16_to_utf8_static(ctypes.c_void_p(16), n, ctypes.c_void_p(16), 3 * n,
                                                ctypes.c_void_p(16), ctypes.c_void_p(0))
    assert status == 3   # GPUTF_STATUS_INPUT_TOO_LARGE, checked before any GPU work
