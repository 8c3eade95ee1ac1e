"""Call-level failures of the C ABI, on the CPU.

Every entry point checks its arguments before it touches a GPU: NULL or
misaligned pointers give GPUTF_STATUS_INVALID_ARGUMENT, inputs above the
stated maximum GPUTF_STATUS_INPUT_TOO_LARGE, and a workspace (or serving slot)
too small for the call GPUTF_STATUS_WORKSPACE_TOO_SMALL.  These tests call
each entry point with one bad argument at a time and stand-in addresses that
nothing dereferences (every case fails a check that comes before the first
CUDA call), so they run without a GPU and give the same statuses with one.
The Python binding's own checks (CUDA, contiguous and large-enough tensors)
are covered at the end, also before any GPU work.
"""
import ctypes

import numpy as np
import pytest

OK, INVALID, WS_SMALL, TOO_LARGE = 0, 1, 2, 3
MAX_UNITS = 1 << 38
STATIC_MAX_UNITS = 1 << 25
A = 1 << 20            # a stand-in device address, 256-byte aligned
NULL = None


@pytest.fixture(scope="module")
def g():
    import paper_2109_10433_gb300 as g
    g.build()
    return g


@pytest.fixture(scope="module")
def L(g):
    return g.lib()


def P(x):
    return ctypes.c_void_p(x)


TRANSCODERS = [
    # name, input is UTF-16, output is UTF-16
    ("gputf_utf8_to_utf16", False, True),
    ("gputf_utf8_to_utf16_unchecked", False, True),
    ("gputf_utf8_to_utf16be", False, True),
    ("gputf_utf16_to_utf8", True, False),
    ("gputf_utf16_to_utf8_unchecked", True, False),
    ("gputf_utf16be_to_utf8", True, False),
]

PASSES = [
    # name, input is UTF-16
    ("gputf_validate_utf8", False),
    ("gputf_validate_utf16", True),
    ("gputf_validate_utf16be", True),
    ("gputf_utf16_length_from_utf8", False),
    ("gputf_utf8_length_from_utf16", True),
    ("gputf_utf8_length_from_utf16be", True),
]


@pytest.mark.parametrize("name,in16,out16", TRANSCODERS)
def test_transcoder_argument_checks(L, name, in16, out16):
    f = getattr(L, name)
    n = 1000
    ws_bytes = L.gputf_workspace_bytes(n)

    def call(inp=A, n=n, out=A, cap=3 * n, ws=A, wsb=ws_bytes, res=A):
        return f(P(inp), n, P(out), cap, P(ws), wsb, P(res), P(0))

    assert call(inp=NULL) == INVALID                  # NULL input with n > 0
    assert call(ws=NULL) == INVALID
    assert call(res=NULL) == INVALID
    assert call(out=NULL) == INVALID                  # NULL output with a capacity
    assert call(res=A + 4) == INVALID                 # result not 8-byte aligned
    assert call(ws=A + 8) == INVALID                  # workspace not 16-byte aligned
    if in16:
        assert call(inp=A + 1) == INVALID             # UTF-16 input not 2-byte aligned
    if out16:
        assert call(out=A + 1) == INVALID             # UTF-16 output not 2-byte aligned
    assert call(n=MAX_UNITS + 1) == TOO_LARGE
    assert call(wsb=100) == WS_SMALL                  # not even the header
    assert call(n=1 << 24, wsb=L.gputf_workspace_bytes(1024)) == WS_SMALL   # too few tile words


@pytest.mark.parametrize("name,in16", PASSES)
def test_pass_argument_checks(L, name, in16):
    f = getattr(L, name)
    n = 1000
    ws_bytes = L.gputf_workspace_bytes(n)

    def call(inp=A, n=n, ws=A, wsb=ws_bytes, res=A):
        return f(P(inp), n, P(ws), wsb, P(res), P(0))

    assert call(inp=NULL) == INVALID
    assert call(ws=NULL) == INVALID
    assert call(res=NULL) == INVALID
    assert call(res=A + 4) == INVALID
    assert call(ws=A + 8) == INVALID
    if in16:
        assert call(inp=A + 1) == INVALID
    assert call(n=MAX_UNITS + 1) == TOO_LARGE
    assert call(wsb=100) == WS_SMALL


def test_workspace_init_argument_checks(L):
    assert L.gputf_workspace_init(P(NULL), 4096, P(0)) == INVALID
    assert L.gputf_workspace_init(P(A + 8), 4096, P(0)) == INVALID
    assert L.gputf_workspace_init(P(A), 255, P(0)) == INVALID   # smaller than the 256-byte header


def test_workspace_sizes_cover_every_tile(L):
    """The workspace has a status word for every tile of the smallest tile
    size (1024 units) at any alignment of the input, plus the header."""
    for n in (0, 1, 1023, 1024, 1025, 6144, 10 ** 6, 1 << 30, MAX_UNITS):
        b = L.gputf_workspace_bytes(n)
        assert b >= 256 + 8 * ((n + 15) // 1024 + 1)
        assert b % 8 == 0


@pytest.mark.parametrize("name", ["gputf_utf8_to_utf16_host", "gputf_utf16_to_utf8_host"])
def test_host_form_argument_checks(L, name):
    f = getattr(L, name)
    n = 1000
    h = np.zeros(4 * n, dtype=np.uint8)
    hp = h.ctypes.data
    r = ctypes.create_string_buffer(24)

    def call(h_in=hp, h_out=hp, d_in=A, d_out=A, d_res=A, h_res=ctypes.addressof(r), cap=n):
        return f(P(h_in), n, P(h_out), cap, P(d_in), P(d_out), P(A), L.gputf_workspace_bytes(n), P(d_res),
                 P(h_res), P(0))

    assert call(h_in=NULL) == INVALID
    assert call(d_in=NULL) == INVALID
    assert call(h_res=NULL) == INVALID
    assert call(d_res=NULL) == INVALID
    assert call(h_out=NULL) == INVALID
    assert call(d_out=NULL) == INVALID


def test_static_entry_point_argument_checks(L):
    f = L.gputf_utf16_to_utf8_static
    n = STATIC_MAX_UNITS + 1
    assert f(P(A), n, P(A), 3 * n, P(A), P(0)) == TOO_LARGE           # above its fixed scratch
    assert f(P(NULL), 10, P(A), 30, P(A), P(0)) == INVALID
    assert f(P(A), 10, P(A), 30, P(NULL), P(0)) == INVALID
    assert f(P(A), 10, P(NULL), 30, P(A), P(0)) == INVALID
    assert f(P(A + 1), 10, P(A), 30, P(A), P(0)) == INVALID           # UTF-16 input not 2-byte aligned
    assert f(P(A), 10, P(A), 30, P(A + 4), P(0)) == INVALID           # result not 8-byte aligned


def test_wait_timeout_entry_argument_checks(L):
    f = L.gputf_test_wait_timeout
    assert f(P(NULL), 4096, 0, 100, P(A), P(0)) == INVALID
    assert f(P(A + 8), 4096, 0, 100, P(A), P(0)) == INVALID           # workspace not 16-byte aligned
    assert f(P(A), 256, 0, 100, P(A), P(0)) == INVALID                # no room for a tile's status word
    assert f(P(A), 4096, 2, 100, P(A), P(0)) == INVALID               # no such wait
    assert f(P(A), 4096, 1, 0, P(A), P(0)) == INVALID                 # no polls
    assert f(P(A), 4096, 1, (1 << 20) + 1, P(A), P(0)) == INVALID     # above the limit
    assert f(P(A), 4096, 0, 100, P(NULL), P(0)) == INVALID
    assert f(P(A), 4096, 0, 100, P(A + 4), P(0)) == INVALID           # result not 8-byte aligned


def test_batch_argument_checks(g, L):
    from paper_2109_10433_gb300.batch import CBatch

    def batch(**kw):
        b = CBatch(count=2, units=100, in_=A, in_offsets=A, out=A, out_offsets=A, results=A)
        for k, v in kw.items():
            setattr(b, k, v)
        return b

    wsb = L.gputf_batch_workspace_bytes(100, 2, 100, 2)

    def call(b8=None, b16=None, config=0, ws=A, ws_bytes=wsb):
        return L.gputf_batch_transcode(ctypes.byref(b8) if b8 is not None else None,
                                       ctypes.byref(b16) if b16 is not None else None,
                                       config, P(ws), ws_bytes, P(0))

    for d in ("b8", "b16"):
        assert call(**{d: batch(in_offsets=NULL)}) == INVALID
        assert call(**{d: batch(results=NULL)}) == INVALID
        assert call(**{d: batch(results=A + 4)}) == INVALID
        assert call(**{d: batch(in_offsets=A + 4)}) == INVALID
        assert call(**{d: batch(in_=NULL)}) == INVALID                 # NULL input with units > 0
        assert call(**{d: batch(out_offsets=NULL)}) == INVALID         # output without capacities
        assert call(**{d: batch(units=MAX_UNITS + 1)}) == TOO_LARGE
        assert call(**{d: batch()}, config=L.gputf_batch_config_count()) == INVALID
        assert call(**{d: batch()}, ws=NULL) == INVALID
        assert call(**{d: batch()}, ws=A + 8) == INVALID
        assert call(**{d: batch()}, ws_bytes=wsb // 2) == WS_SMALL
    assert call(b16=batch(in_=A + 1)) == INVALID        # UTF-16 input not 2-byte aligned
    assert call(b8=batch(out=A + 1)) == INVALID         # UTF-16 output not 2-byte aligned


def test_graph_and_gather_argument_checks(L):
    out = ctypes.c_void_p()
    assert L.gputf_batch_graph_create(None, None, 0, P(A), 4096, P(A), None) == INVALID   # no handle
    assert L.gputf_batch_graph_create(None, None, 0, P(A), 4096, P(0), ctypes.byref(out)) == INVALID  # legacy stream
    assert L.gputf_graph_launch(None, P(0)) == INVALID
    L.gputf_graph_destroy(None)                                       # a no-op
    assert L.gputf_gather(P(A), 0, P(A), P(0)) == OK                  # nothing to copy: no GPU work
    assert L.gputf_gather(P(NULL), 3, P(A), P(0)) == INVALID
    assert L.gputf_gather(P(A), 3, P(NULL), P(0)) == INVALID
    assert L.gputf_gather(P(A + 4), 3, P(A), P(0)) == INVALID


def test_serve_launch_argument_checks(g, L):
    from paper_2109_10433_gb300 import serve as S

    meta_host = np.zeros(1 << 12, dtype=np.uint64)

    def slot(**kw):
        s = S.CSlot(arena=A, arena_bytes=1 << 20, meta=A, meta_host=meta_host.ctypes.data,
                    meta_bytes=meta_host.nbytes, results=A, results_host=0, max_requests=8, ws=A,
                    ws_bytes=1 << 16, ws1=A, ws1_bytes=1 << 16)
        for k, v in kw.items():
            setattr(s, k, v)
        return s

    def reqs(*items):
        return S.request_array([S.Request(i, d, op, ptr, units) for i, (d, op, ptr, units) in enumerate(items)])

    place = np.zeros(16 * 3, dtype=np.uint64)

    def call(s, r, big_units=1 << 20):
        return L.gputf_serve_launch(ctypes.byref(s), r.ctypes.data, r.size, big_units, 0, place.ctypes.data,
                                    P(0))

    good = reqs((0, 0, A, 100), (1, 0, A, 50))
    assert L.gputf_serve_launch(None, good.ctypes.data, good.size, 1 << 20, 0, place.ctypes.data, P(0)) == INVALID
    assert call(slot(arena=NULL), good) == INVALID
    assert call(slot(arena=A + 16), good) == INVALID                 # arena not 256-byte aligned
    assert call(slot(meta=A + 4), good) == INVALID
    assert call(slot(results=A + 4), good) == INVALID
    assert call(slot(ws=NULL), good) == INVALID
    assert call(slot(), reqs((2, 0, A, 100))) == INVALID              # no such direction
    assert call(slot(), reqs((0, 2, A, 100))) == INVALID              # no such operation
    assert call(slot(), reqs((1, 0, A + 1, 100))) == INVALID          # UTF-16 input not 2-byte aligned
    assert call(slot(), reqs((0, 0, 0, 100))) == INVALID              # NULL input
    assert call(slot(), reqs((0, 0, A, MAX_UNITS + 1))) == TOO_LARGE
    assert call(slot(), S.request_array([])) == OK                    # an empty batch: nothing enqueued
    assert call(slot(max_requests=1), good) == WS_SMALL               # more requests than result rows
    assert call(slot(arena_bytes=256), good) == WS_SMALL              # gathered inputs do not fit
    assert call(slot(meta_bytes=8), good) == WS_SMALL
    assert call(slot(ws_bytes=256), good) == WS_SMALL                 # batched workspace too small
    assert call(slot(ws1=NULL), good, big_units=10) == WS_SMALL       # in-place requests need ws1
    assert call(slot(ws1_bytes=256), good, big_units=10) == WS_SMALL


def test_status_names_and_binding_errors(g, L):
    names = [L.gputf_status_name(k).decode() for k in range(6)]
    assert names == g.STATUS_NAMES
    assert L.gputf_status_name(99) == b"UNKNOWN"
    assert [L.gputf_error_name(k).decode() for k in range(10)] == g.ERROR_NAMES
    assert L.gputf_error_name(-1) == b"UNKNOWN"
    g._check(0, "x")
    with pytest.raises(g.GputfError, match="x: WORKSPACE_TOO_SMALL"):
        g._check(WS_SMALL, "x")
    with pytest.raises(g.GputfError, match="INPUT_TOO_LARGE"):
        g._check(TOO_LARGE, "y")


def test_binding_refuses_tensors_the_kernels_cannot_use(g):
    """CPU tensors, strided views, odd UTF-16 byte counts and short result
    buffers are refused by the binding before any GPU work (the kernels would
    otherwise be given host addresses or too little memory)."""
    torch = pytest.importorskip("torch")
    u8 = torch.zeros(64, dtype=torch.uint8)
    u16 = torch.zeros(64, dtype=torch.int16)
    for call in (lambda: g.utf8_to_utf16(u8), lambda: g.validate_utf8(u8), lambda: g.utf16_length_from_utf8(u8),
                 lambda: g.utf16_to_utf8(u16), lambda: g.validate_utf16(u16),
                 lambda: g.utf8_length_from_utf16(u16), lambda: g.utf16_to_utf8(u16, big_endian=True)):
        with pytest.raises(ValueError, match="CUDA tensor"):
            call()
    with pytest.raises(ValueError, match="contiguous"):
        g._on_device(_FakeCuda(contiguous=False), "x")
    with pytest.raises(ValueError, match="at least 24"):
        g._on_device(_FakeCuda(nbytes=16), "res", 24)
    assert g._on_device(_FakeCuda(nbytes=24), "res", 24) is not None
    with pytest.raises(ValueError, match="odd"):
        g._utf16_units(torch.zeros(7, dtype=torch.uint8), "inp")
    assert g._utf16_units(torch.zeros(8, dtype=torch.uint8), "inp") == 4
    # host forms: host buffers on the CPU, device buffers on the GPU and large enough
    with pytest.raises(ValueError, match="CPU tensor"):
        g._on_host(_FakeCuda(), "h_in")
    with pytest.raises(ValueError, match="contiguous"):
        g._on_host(torch.zeros((4, 4), dtype=torch.uint8).t(), "h_in")
    with pytest.raises(ValueError, match="CUDA tensor"):
        g.utf8_to_utf16_host(u8, u16, u8, u16, None, torch.zeros(3, dtype=torch.int64))
    with pytest.raises(ValueError, match="d_in: .* at least 64"):
        g._host_form_buffers(u8, u16, _FakeCuda(nbytes=32), _FakeCuda(nbytes=128), _FakeCuda(nbytes=24))
    with pytest.raises(ValueError, match="d_out: .* at least 128"):
        g._host_form_buffers(u8, u16, _FakeCuda(nbytes=64), _FakeCuda(nbytes=127), _FakeCuda(nbytes=24))
    g._host_form_buffers(u8, u16, _FakeCuda(nbytes=64), _FakeCuda(nbytes=128), _FakeCuda(nbytes=24))


class _FakeCuda:
    """Stands in for a CUDA tensor in the binding's checks (no device here)."""

    is_cuda = True

    def __init__(self, nbytes=64, contiguous=True):
        self._n = nbytes
        self._c = contiguous

    def numel(self):
        return self._n

    def element_size(self):
        return 1

    def is_contiguous(self):
        return self._c
