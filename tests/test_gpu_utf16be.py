"""GPU parity for big-endian UTF-16: the four UTF-16BE calls through the C ABI
against the CPU oracle, bit for bit (output, error class, position, units
written, lengths), with guard bands around every output buffer.

Covers ragged sizes of every character mix, sizes around the tile
boundaries of each kernel, unaligned pointers, every UTF-16 error form near
tile boundaries, random units, output capacities that cut the output short,
and a buffer larger than L2.
"""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TILE8 = 8192      # input bytes per tile, UTF-8 -> UTF-16
TILE16 = 6144     # input units per tile, UTF-16 -> UTF-8
PASS16 = 4096     # input units per tile of the UTF-16 validate / length passes
GUARD = 0x5A

MIXES = [W.MIX_LATIN_CYRILLIC, W.MIX_CJK_EMOJI, W.MIX_FOUR_BYTE_HEAVY, W.SCRIPT_MIXED,
         W.SCRIPT_ASCII, W.SCRIPT_TWO_BYTE, W.SCRIPT_CJK]


@pytest.fixture(scope="module")
def g():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2109_10433_gb300 as g
    g.build()
    return g


@pytest.fixture(scope="module")
def ws(g):
    return g.Workspace(80 << 20)


def be(units):
    """UTF-16 code-unit values -> the uint16 words of their big-endian storage."""
    return np.asarray(units, dtype=np.uint16).byteswap()


def dev(a, dtype, off=0):
    pad = 32 if dtype == torch.uint8 else 16
    buf = torch.zeros(a.size + off + pad, dtype=dtype, device="cuda")
    if a.size:
        host = np.ascontiguousarray(a)
        buf[off:off + a.size] = torch.from_numpy(host if dtype == torch.uint8 else host.view(np.int16)).cuda()
    return buf[off:off + a.size]


def check_be_to_8(g, ws, mem, cap=None, in_off=0, out_off=0):
    mem = np.asarray(mem, dtype=np.uint16)
    cap = 3 * mem.size if cap is None else cap
    outbuf = torch.full((cap + out_off + 32,), GUARD, dtype=torch.uint8, device="cuda")
    out = outbuf[out_off:out_off + cap]
    res, _ = g.utf16_to_utf8(dev(mem, torch.int16, in_off), out=out, ws=ws, big_endian=True)
    ref, ref_out = oracle.utf16be_to_utf8(mem, cap=cap)
    assert tuple(res) == tuple(ref), (res, ref, mem.size, cap, in_off, out_off)
    host = outbuf.cpu().numpy()
    assert np.array_equal(host[out_off:out_off + res.written], ref_out)
    assert np.all(host[:out_off] == GUARD) and np.all(host[out_off + cap:] == GUARD)
    return res


def check_8_to_be(g, ws, data, cap=None, in_off=0, out_off=0):
    data = np.asarray(data, dtype=np.uint8)
    cap = data.size if cap is None else cap
    outbuf = torch.full((cap + out_off + 16,), GUARD * 257, dtype=torch.int16, device="cuda")
    out = outbuf[out_off:out_off + cap]
    res, _ = g.utf8_to_utf16(dev(data, torch.uint8, in_off), out=out, ws=ws, big_endian=True)
    ref, ref_out = oracle.utf8_to_utf16be(data, cap=cap)
    assert tuple(res) == tuple(ref), (res, ref, data.size, cap, in_off, out_off)
    host = outbuf.cpu().numpy().view(np.uint16)
    assert np.array_equal(host[out_off:out_off + res.written], ref_out)
    assert np.all(host[:out_off] == GUARD * 257) and np.all(host[out_off + cap:] == GUARD * 257)
    return res


def check_passes_be(g, ws, mem, in_off=0):
    mem = np.asarray(mem, dtype=np.uint16)
    d = dev(mem, torch.int16, in_off)
    assert tuple(g.validate_utf16(d, ws=ws, big_endian=True)) == tuple(oracle.validate_utf16be(mem))
    assert g.utf8_length_from_utf16(d, ws=ws, big_endian=True) == oracle.utf8_length_from_utf16be(mem)


# ---------------------------------------------------------------------------
def test_empty(g, ws):
    for off in (0, 3):
        check_be_to_8(g, ws, np.zeros(0, np.uint16), in_off=off)
        check_8_to_be(g, ws, np.zeros(0, np.uint8), in_off=off)
        check_passes_be(g, ws, np.zeros(0, np.uint16), in_off=off)


def test_small_sizes_all_mixes(g, ws):
    rng = np.random.default_rng(31)
    for n in list(range(1, 70)) + [127, 128, 129, 255, 256, 257, 513, 1000]:
        mix = MIXES[n % len(MIXES)]
        mem = be(W.utf16_text(n, n, mix))
        off = int(rng.integers(0, 8))
        check_be_to_8(g, ws, mem, in_off=off, out_off=int(rng.integers(0, 16)))
        check_passes_be(g, ws, mem, in_off=off)
        check_8_to_be(g, ws, W.utf8_text(n, n, mix), in_off=int(rng.integers(0, 16)),
                      out_off=int(rng.integers(0, 8)))


def test_sizes_around_tile_boundaries(g, ws):
    rng = np.random.default_rng(32)
    for k in (1, 2, 5):
        for delta in (-3, -1, 0, 1, 2):
            for T16 in (TILE16, PASS16):
                mem = be(W.utf16_text(k + 40, k * T16 + delta, MIXES[(k + delta) % len(MIXES)]))
                off = int(rng.integers(0, 8))
                check_be_to_8(g, ws, mem, in_off=off, out_off=int(rng.integers(0, 16)))
                check_passes_be(g, ws, mem, in_off=off)
            d8 = W.utf8_text(k + 50, k * TILE8 + delta, MIXES[(k - delta) % len(MIXES)])
            check_8_to_be(g, ws, d8, in_off=int(rng.integers(0, 16)), out_off=int(rng.integers(0, 8)))


def test_every_utf16_error_form_around_tile_boundaries(g, ws):
    rng = W.rng_for(33)
    base = W.utf16_text(7, 3 * TILE16 + 50, W.MIX_CJK_EMOJI)
    near = [b + d for b in (TILE16, 2 * TILE16, PASS16, 24 * 5, 16 * 9) for d in range(-4, 4)]
    for pos in near + [0, 1, base.size - 1]:
        tok, _ = W.utf16_error_token(rng)
        mem = be(np.concatenate([base[:pos], np.array(tok, np.uint16), base[pos:]]))
        check_be_to_8(g, ws, mem, in_off=pos % 8)
        check_passes_be(g, ws, mem)
    check_be_to_8(g, ws, be(np.concatenate([base[:TILE16 - 1], [0xD83D]])))
    check_be_to_8(g, ws, be(np.concatenate([[0xDE00], base[:100]])))


def test_utf8_errors_with_big_endian_output(g, ws):
    rng = W.rng_for(34)
    base = W.utf8_text(8, 2 * TILE8 + 100, W.MIX_FOUR_BYTE_HEAVY)
    starts = np.cumsum([0] + [len(c.encode()) for c in base.tobytes().decode()])[:-1]
    near = [s for s in starts if abs(int(s) - TILE8) <= 6]
    for s, kind in zip(near, W.UTF8_TOKEN_KINDS * 4):
        tok, cls = W.utf8_error_token(rng, kind)
        d = np.concatenate([base[:s], np.frombuffer(tok, np.uint8), base[s:]])
        r = check_8_to_be(g, ws, d, in_off=int(s) % 16)
        assert (r.error, r.position) == (cls, int(s))


def test_random_units(g, ws):
    rng = np.random.default_rng(35)
    for trial in range(30):
        n = int(rng.integers(1, 20000))
        u = rng.integers(0, 65536, n).astype(np.uint16)
        u[: n - n // 8] = np.where((u[: n - n // 8] & 0xF800) == 0xD800, 0x41, u[: n - n // 8])
        check_be_to_8(g, ws, u)        # the raw words as stored: any values
        check_passes_be(g, ws, u)
        check_be_to_8(g, ws, be(u))


def test_output_capacity(g, ws):
    mem = be(W.utf16_text(9, 3000, W.SCRIPT_MIXED))
    full = oracle.utf8_length_from_utf16be(mem)
    for cap in (0, 1, 2, 3, 4, 5, 100, full // 2, full - 3, full - 1, full):
        check_be_to_8(g, ws, mem, cap=cap, out_off=cap % 7)
    d8 = W.utf8_text(10, 3000, W.SCRIPT_MIXED)
    full16 = oracle.utf16_length_from_utf8(d8)
    for cap in (0, 1, 2, 3, 100, full16 // 2, full16 - 1, full16):
        check_8_to_be(g, ws, d8, cap=cap, out_off=cap % 5)


def test_big_endian_is_the_byte_swapped_little_endian_call(g, ws):
    """Above L2 (64 MiB of UTF-16): the BE calls on byte-swapped storage give
    exactly the LE calls' results, and the UTF-8 -> UTF-16BE output is the
    byte-swapped UTF-16LE output."""
    units = W.utf16_text(11, 32 << 20, W.MIX_CJK_EMOJI)
    le = torch.from_numpy(units.view(np.int16)).cuda()
    bed = torch.from_numpy(be(units).view(np.int16)).cuda()
    big_ws = g.Workspace(units.size * 2)
    r_le, out_le = g.utf16_to_utf8(le, ws=big_ws)
    r_be, out_be = g.utf16_to_utf8(bed, ws=big_ws, big_endian=True)
    assert tuple(r_le) == tuple(r_be) == (0, units.size, r_le.written)
    assert torch.equal(out_le[:r_le.written], out_be[:r_be.written])
    assert tuple(g.validate_utf16(bed, ws=big_ws, big_endian=True)) == tuple(g.validate_utf16(le, ws=big_ws))
    assert g.utf8_length_from_utf16(bed, ws=big_ws, big_endian=True) == r_le.written
    # sampled windows against the oracle
    host8 = out_be[:r_be.written].cpu().numpy()
    ref8 = oracle.utf16_to_utf8(units[: 1 << 20])[1]
    assert np.array_equal(host8[:ref8.size], ref8)
    d8 = out_le[:r_le.written].contiguous()
    r16le, o16le = g.utf8_to_utf16(d8, ws=big_ws)
    r16be, o16be = g.utf8_to_utf16(d8, ws=big_ws, big_endian=True)
    assert tuple(r16le) == tuple(r16be) == (0, r_le.written, units.size)
    a = o16le[:units.size].cpu().numpy().view(np.uint16)
    b = o16be[:units.size].cpu().numpy().view(np.uint16)
    assert np.array_equal(a, units) and np.array_equal(b, be(units))
