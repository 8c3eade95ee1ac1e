"""Host side of the batched call, without a GPU: the CSR layout DeviceBatch
builds (strings back to back, input offsets, output offsets from the
capacities) and the C descriptor it hands to gputf_batch_transcode.  The
tensors live on the CPU here; only their layout and addresses are checked."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2109_10433_gb300 import batch as B  # noqa: E402


def test_utf8_batch_layout_and_descriptor():
    strings = [np.frombuffer("héllo".encode(), np.uint8), np.zeros(0, np.uint8),
               np.frombuffer("🌍!".encode(), np.uint8)]
    b = B.DeviceBatch(strings, B.UTF8_TO_UTF16, device="cpu")
    assert b.count == 3 and b.units == 6 + 0 + 5
    assert b.in_offsets_host.tolist() == [0, 6, 6, 11]
    # default capacities: n UTF-16 units for n UTF-8 bytes, always enough
    assert b.out_offsets_host.tolist() == [0, 6, 6, 11]
    assert bytes(b.inp.numpy().tobytes()) == "héllo🌍!".encode()
    c = b.cstruct()
    assert (c.count, c.units) == (3, 11)
    assert c.in_ == b.inp.data_ptr() and c.in_offsets == b.in_offsets.data_ptr()
    assert c.out == b.out.data_ptr() and c.out_offsets == b.out_offsets.data_ptr()
    assert c.results == b.results.data_ptr()
    assert b.out.dtype == torch.int16 and b.out.numel() == 11


def test_utf16_batch_capacities_and_validate_only():
    s = [np.array([0x41, 0xD83D, 0xDE00], np.uint16), np.array([0x4E2D], np.uint16)]
    b = B.DeviceBatch(s, B.UTF16_TO_UTF8, capacities=[5, 0], device="cpu")
    assert b.units == 4 and b.in_offsets_host.tolist() == [0, 3, 4]
    assert b.out_offsets_host.tolist() == [0, 5, 5]          # the capacities given, back to back
    assert b.inp.dtype == torch.int16 and b.inp.numpy().view(np.uint16).tolist() == [0x41, 0xD83D, 0xDE00, 0x4E2D]
    d = B.DeviceBatch(s, B.UTF16_TO_UTF8, device="cpu")
    assert d.out_offsets_host.tolist() == [0, 9, 12]         # 3 bytes per unit by default
    v = B.DeviceBatch(s, B.UTF16_TO_UTF8, device="cpu", validate_only=True).cstruct()
    assert v.out is None and v.out_offsets is None           # NULL: validate only


def test_results_and_outputs_are_read_per_string():
    s = [np.frombuffer(b"ab", np.uint8), np.frombuffer(b"cde", np.uint8)]
    b = B.DeviceBatch(s, B.UTF8_TO_UTF16, device="cpu")
    b.results[:] = torch.tensor([[(7 << 32) | 0, 2, 2], [3, 1, 1]])
    assert [tuple(r) for r in b.read_results()] == [(0, 2, 2), (3, 1, 1)]
    b.out[:5] = torch.tensor([0x61, 0x62, 0x63, 0x64, 0x65], dtype=torch.int16)
    assert b.output(1, 2).tolist() == [0x63, 0x64]            # string 1's output starts at its offset
    assert b.output(0, 2).dtype == np.uint16


def test_empty_batch():
    b = B.DeviceBatch([], B.UTF8_TO_UTF16, device="cpu")
    assert b.count == 0 and b.units == 0 and b.in_offsets_host.tolist() == [0]
    assert b.cstruct().count == 0
