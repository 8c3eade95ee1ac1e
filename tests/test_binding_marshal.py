"""The Python binding's argument marshalling, on the CPU.

The binding turns tensors into the C ABI's pointers and sizes.  Here the
library is replaced by a recorder and the tensors by stand-ins with known
addresses and sizes, so the test sees exactly what each binding function
would pass to the C entry point: which entry point (validating, unchecked,
UTF-16BE, host form), the input size in code units of the input encoding
(bytes for UTF-8, 16-bit units for UTF-16), the output capacity in code units
of the output encoding, the workspace and result addresses, and the stream.
"""
import ctypes

import pytest


class FakeTensor:
    """Stands in for a contiguous tensor at address `ptr` (no device here)."""

    def __init__(self, ptr, numel, element_size, cuda=True, values=(0, 0, 0)):
        self.ptr, self.n, self.es, self.is_cuda = ptr, numel, element_size, cuda
        self.values = list(values)
        self.device = "cuda:0" if cuda else "cpu"

    def data_ptr(self):
        return self.ptr

    def numel(self):
        return self.n

    def element_size(self):
        return self.es

    def is_contiguous(self):
        return True

    def cpu(self):
        return self

    def tolist(self):
        return self.values

    def item(self):
        return self.values[0]


class FakeStream:
    cuda_stream = 0x5000


class Recorder:
    """Every attribute is a C function that records its arguments and returns 0."""

    def __init__(self):
        self.calls = []

    def __getattr__(self, name):
        def f(*args):
            self.calls.append((name, [a.value if isinstance(a, ctypes.c_void_p) else a for a in args]))
            return 0
        return f


@pytest.fixture
def g(monkeypatch):
    import paper_2109_10433_gb300 as g
    rec = Recorder()
    monkeypatch.setattr(g, "_lib", rec)
    return g, rec


def workspace(g, ptr=0x9000, nbytes=4096):
    ws = object.__new__(g.Workspace)
    ws.max_units, ws.nbytes, ws.buf = 0, nbytes, FakeTensor(ptr, nbytes, 1)
    return ws


RES = dict(values=(7, 12, 34))   # error (low 32 bits of word 0), position, written


def test_utf8_to_utf16_marshalling(g):
    g, rec = g
    inp = FakeTensor(0x1001, 1001, 1)              # 1001 UTF-8 bytes at an odd address
    out = FakeTensor(0x2000, 300, 2)               # 300 UTF-16 units
    res = FakeTensor(0x3000, 3, 8, **RES)
    r, o = g.utf8_to_utf16(inp, out=out, ws=workspace(g), res=res, stream=FakeStream())
    assert o is out and tuple(r) == (7, 12, 34)
    assert rec.calls == [("gputf_utf8_to_utf16", [0x1001, 1001, 0x2000, 300, 0x9000, 4096, 0x3000, 0x5000])]
    for kw, name in ((dict(validate=False), "gputf_utf8_to_utf16_unchecked"),
                     (dict(big_endian=True), "gputf_utf8_to_utf16be")):
        rec.calls.clear()
        g.utf8_to_utf16(inp, out=out, ws=workspace(g), res=res, stream=FakeStream(), **kw)
        assert rec.calls[0][0] == name and rec.calls[0][1][1] == 1001 and rec.calls[0][1][3] == 300


def test_utf16_to_utf8_marshalling(g):
    g, rec = g
    inp = FakeTensor(0x1002, 500, 2)               # 500 UTF-16 units
    out = FakeTensor(0x2001, 1499, 1)              # 1499 bytes
    res = FakeTensor(0x3000, 3, 8, **RES)
    g.utf16_to_utf8(inp, out=out, ws=workspace(g), res=res, stream=FakeStream())
    assert rec.calls == [("gputf_utf16_to_utf8", [0x1002, 500, 0x2001, 1499, 0x9000, 4096, 0x3000, 0x5000])]
    # UTF-16 given as bytes: the unit count is half the bytes
    rec.calls.clear()
    g.utf16_to_utf8(FakeTensor(0x1002, 1000, 1), out=out, ws=workspace(g), res=res, stream=FakeStream(),
                    big_endian=True)
    assert rec.calls[0][0] == "gputf_utf16be_to_utf8" and rec.calls[0][1][1] == 500
    rec.calls.clear()
    g.utf16_to_utf8(inp, out=out, ws=workspace(g), res=res, stream=FakeStream(), validate=False)
    assert rec.calls[0][0] == "gputf_utf16_to_utf8_unchecked"
    with pytest.raises(ValueError):
        g.utf16_to_utf8(inp, out=out, ws=workspace(g), res=res, stream=FakeStream(), validate=False,
                        big_endian=True)


def test_validate_and_length_marshalling(g):
    g, rec = g
    u8 = FakeTensor(0x1003, 77, 1)
    u16 = FakeTensor(0x1004, 40, 2)
    res = FakeTensor(0x3000, 3, 8, **RES)
    ln = FakeTensor(0x3100, 1, 8, values=(123,))
    s = FakeStream()
    g.validate_utf8(u8, ws=workspace(g), res=res, stream=s)
    g.validate_utf16(u16, ws=workspace(g), res=res, stream=s)
    g.validate_utf16(u16, ws=workspace(g), res=res, stream=s, big_endian=True)
    assert g.utf16_length_from_utf8(u8, ws=workspace(g), out=ln, stream=s) == 123
    assert g.utf8_length_from_utf16(u16, ws=workspace(g), out=ln, stream=s) == 123
    g.utf8_length_from_utf16(u16, ws=workspace(g), out=ln, stream=s, big_endian=True)
    assert rec.calls == [
        ("gputf_validate_utf8", [0x1003, 77, 0x9000, 4096, 0x3000, 0x5000]),
        ("gputf_validate_utf16", [0x1004, 40, 0x9000, 4096, 0x3000, 0x5000]),
        ("gputf_validate_utf16be", [0x1004, 40, 0x9000, 4096, 0x3000, 0x5000]),
        ("gputf_utf16_length_from_utf8", [0x1003, 77, 0x9000, 4096, 0x3100, 0x5000]),
        ("gputf_utf8_length_from_utf16", [0x1004, 40, 0x9000, 4096, 0x3100, 0x5000]),
        ("gputf_utf8_length_from_utf16be", [0x1004, 40, 0x9000, 4096, 0x3100, 0x5000]),
    ]


def test_empty_input_passes_null(g):
    g, rec = g
    res = FakeTensor(0x3000, 3, 8, **RES)
    g.validate_utf8(FakeTensor(0x1000, 0, 1), ws=workspace(g), res=res, stream=FakeStream())
    assert rec.calls[0][1][:2] == [None, 0]      # no data: a NULL pointer and size 0


def test_host_form_marshalling(g):
    g, rec = g
    h_in = FakeTensor(0x7000, 600, 2, cuda=False)      # 600 UTF-16 units on the host
    h_out = FakeTensor(0x8000, 1800, 1, cuda=False)
    d_in = FakeTensor(0x1000, 600, 2)
    d_out = FakeTensor(0x2000, 1800, 1)
    d_res = FakeTensor(0x3000, 3, 8)
    r = g.utf16_to_utf8_host(h_in, h_out, d_in, d_out, workspace(g), d_res, stream=FakeStream())
    name, args = rec.calls[0]
    assert name == "gputf_utf16_to_utf8_host"
    assert args[:9] == [0x7000, 600, 0x8000, 1800, 0x1000, 0x2000, 0x9000, 4096, 0x3000]
    assert args[10] == 0x5000 and tuple(r) == (0, 0, 0)
    rec.calls.clear()
    h8 = FakeTensor(0x7000, 999, 1, cuda=False)
    h16 = FakeTensor(0x8000, 999, 2, cuda=False)
    g.utf8_to_utf16_host(h8, h16, FakeTensor(0x1000, 999, 1), FakeTensor(0x2000, 999, 2), workspace(g), d_res,
                         stream=FakeStream(), chunk=4096)
    name, args = rec.calls[0]
    assert name == "gputf_utf8_to_utf16_host_chunked"
    assert args[1] == 999 and args[3] == 999 and args[11] == 4096
