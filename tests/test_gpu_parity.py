"""GPU parity: every call through the C ABI against the CPU oracle, bit for bit
(output units, error class, error position, units written, lengths).

Covers empty and ragged sizes, sizes around tile boundaries, unaligned input
and output pointers, every error class at offsets around tile boundaries,
output capacities that cut the output short, workspace reuse, the host-buffer
forms, and the benchmark workloads at full size.  Guard bands around every
output buffer check that nothing is written outside the caller's capacity.
"""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TILE8 = 8192      # input bytes per tile, UTF-8 -> UTF-16 and the UTF-8 passes (32 per thread)
TILE16 = 6144     # input units per tile, UTF-16 -> UTF-8 (24 units per thread)
PASS16 = 4096     # input units per tile of the UTF-16 validate / length passes (16 per thread)
GUARD = 0x5A


@pytest.fixture(scope="module")
def g():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2109_10433_gb300 as g
    g.build()
    return g


@pytest.fixture(scope="module")
def ws(g):
    return g.Workspace(300 << 20)


def dev_u8(a, off=0):
    buf = torch.zeros(a.size + off + 32, dtype=torch.uint8, device="cuda")
    if a.size:
        buf[off:off + a.size] = torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return buf[off:off + a.size]


def dev_u16(a, off=0):
    buf = torch.zeros(a.size + off + 16, dtype=torch.int16, device="cuda")
    if a.size:
        buf[off:off + a.size] = torch.from_numpy(np.ascontiguousarray(a).view(np.int16)).cuda()
    return buf[off:off + a.size]


def check_8to16(g, ws, data, cap=None, in_off=0, out_off=0):
    data = np.asarray(data, dtype=np.uint8)
    cap = data.size if cap is None else cap
    outbuf = torch.full((cap + out_off + 16,), GUARD * 257, dtype=torch.int16, device="cuda")
    out = outbuf[out_off:out_off + cap]
    res, _ = g.utf8_to_utf16(dev_u8(data, in_off), out=out, ws=ws)
    ref, ref_out = oracle.utf8_to_utf16(data, cap=cap)
    assert tuple(res) == tuple(ref), (res, ref, data.size, cap, in_off, out_off)
    host = outbuf.cpu().numpy().view(np.uint16)
    assert np.array_equal(host[out_off:out_off + res.written], ref_out)
    assert np.all(host[:out_off] == GUARD * 257) and np.all(host[out_off + cap:] == GUARD * 257)
    return res


def check_16to8(g, ws, units, cap=None, in_off=0, out_off=0):
    units = np.asarray(units, dtype=np.uint16)
    cap = 3 * units.size if cap is None else cap
    outbuf = torch.full((cap + out_off + 32,), GUARD, dtype=torch.uint8, device="cuda")
    out = outbuf[out_off:out_off + cap]
    res, _ = g.utf16_to_utf8(dev_u16(units, in_off), out=out, ws=ws)
    ref, ref_out = oracle.utf16_to_utf8(units, cap=cap)
    assert tuple(res) == tuple(ref), (res, ref, units.size, cap, in_off, out_off)
    host = outbuf.cpu().numpy()
    assert np.array_equal(host[out_off:out_off + res.written], ref_out)
    assert np.all(host[:out_off] == GUARD) and np.all(host[out_off + cap:] == GUARD)
    return res


def check_passes8(g, ws, data, in_off=0):
    d = dev_u8(np.asarray(data, np.uint8), in_off)
    assert tuple(g.validate_utf8(d, ws=ws)) == tuple(oracle.validate_utf8(data))
    assert g.utf16_length_from_utf8(d, ws=ws) == oracle.utf16_length_from_utf8(data)


def check_passes16(g, ws, units, in_off=0):
    d = dev_u16(np.asarray(units, np.uint16), in_off)
    assert tuple(g.validate_utf16(d, ws=ws)) == tuple(oracle.validate_utf16(units))
    assert g.utf8_length_from_utf16(d, ws=ws) == oracle.utf8_length_from_utf16(units)


MIXES = [W.MIX_LATIN_CYRILLIC, W.MIX_CJK_EMOJI, W.MIX_FOUR_BYTE_HEAVY, W.SCRIPT_MIXED,
         W.SCRIPT_ASCII, W.SCRIPT_TWO_BYTE, W.SCRIPT_CJK]


# ---------------------------------------------------------------------------
def test_empty(g, ws):
    for off in (0, 3):
        check_8to16(g, ws, np.zeros(0, np.uint8), in_off=off)
        check_16to8(g, ws, np.zeros(0, np.uint16), in_off=off)
        check_passes8(g, ws, np.zeros(0, np.uint8), in_off=off)
        check_passes16(g, ws, np.zeros(0, np.uint16), in_off=off)


def test_small_sizes_all_mixes(g, ws):
    rng = np.random.default_rng(1)
    for n in list(range(1, 80)) + [127, 128, 129, 255, 256, 257, 511, 512, 513, 1000]:
        mix = MIXES[n % len(MIXES)]
        d8 = W.utf8_text(n, n, mix)
        off = int(rng.integers(0, 16))
        check_8to16(g, ws, d8, in_off=off, out_off=int(rng.integers(0, 8)))
        check_passes8(g, ws, d8, in_off=off)
        d16 = W.utf16_text(n, n, mix)
        off = int(rng.integers(0, 8))
        check_16to8(g, ws, d16, in_off=off, out_off=int(rng.integers(0, 16)))
        check_passes16(g, ws, d16, in_off=off)


def test_sizes_around_tile_boundaries(g, ws):
    rng = np.random.default_rng(2)
    for k in (1, 2, 3, 7):
        for delta in range(-4, 5):
            n = k * TILE8 + delta
            for off in (0, 1, 7, 15):
                d8 = W.utf8_text(n + off, n, MIXES[(k + delta) % len(MIXES)])
                check_8to16(g, ws, d8, in_off=off, out_off=int(rng.integers(0, 8)))
            for T16 in (TILE16, PASS16):
                d16 = W.utf16_text(n, k * T16 + delta, MIXES[(k - delta) % len(MIXES)])
                for off in (0, 1, 5, 7):
                    check_16to8(g, ws, d16, in_off=off, out_off=int(rng.integers(0, 16)))
                check_passes16(g, ws, d16)
            check_passes8(g, ws, d8)


def test_random_bytes_and_units(g, ws):
    rng = np.random.default_rng(3)
    for trial in range(60):
        n = int(rng.integers(1, 20000))
        b = rng.integers(0, 256, n).astype(np.uint8)
        if trial % 2:
            b[: n // 2] &= 0x7F        # a valid ASCII prefix, garbage after
        check_8to16(g, ws, b)
        check_passes8(g, ws, b)
        u = rng.integers(0, 65536, n).astype(np.uint16)
        u[: n - n // 8] = np.where((u[: n - n // 8] & 0xF800) == 0xD800, 0x41, u[: n - n // 8])
        check_16to8(g, ws, u)
        check_passes16(g, ws, u)


@pytest.mark.parametrize("kind", W.UTF8_TOKEN_KINDS + ("header",))
def test_every_utf8_error_class_around_tile_boundaries(g, ws, kind):
    rng = W.rng_for(17)
    base = W.utf8_text(5, 3 * TILE8 + 100, W.MIX_FOUR_BYTE_HEAVY)
    # character starts of the clean text, from CPython's decoding
    starts = np.cumsum([0] + [len(c.encode()) for c in base.tobytes().decode()])[:-1]
    near = [s for s in starts if any(abs(int(s) - b) <= 8 for b in (TILE8, 2 * TILE8))]
    for s in near:
        tok, cls = W.utf8_error_token(rng, kind)
        d = np.concatenate([base[:s], np.frombuffer(tok, np.uint8), base[s:]])
        r = check_8to16(g, ws, d, in_off=int(s) % 16)
        assert (r.error, r.position) == (cls, int(s))
        check_passes8(g, ws, d)


def test_every_utf16_error_form_around_tile_boundaries(g, ws):
    rng = W.rng_for(19)
    base = W.utf16_text(6, 3 * TILE16 + 50, W.MIX_CJK_EMOJI)
    near = [b + d for b in (TILE16, 2 * TILE16, PASS16, 24 * 5, 24 * 32, 16 * 9) for d in range(-6, 6)]
    for pos in near + [0, 1, base.size - 1]:
        tok, _ = W.utf16_error_token(rng)
        d = np.concatenate([base[:pos], np.array(tok, np.uint16), base[pos:]])
        check_16to8(g, ws, d, in_off=pos % 8)
        check_passes16(g, ws, d)
    # a high surrogate as the very last unit, and a low one as the first
    check_16to8(g, ws, np.concatenate([base[:TILE16 - 1], [0xD83D]]).astype(np.uint16))
    check_16to8(g, ws, np.concatenate([[0xDE00], base[:100]]).astype(np.uint16))


def test_truncated_tail_at_every_alignment(g, ws):
    for seq in (b"\xc3", b"\xe9\x8f", b"\xf0\x9f\x98", b"\xe9", b"\xf0", b"\xf0\x9f"):
        for n in (TILE8 - 3, TILE8 - 2, TILE8 - 1, TILE8, 2 * TILE8 + 1):
            d = np.concatenate([np.full(n, 0x41, np.uint8), np.frombuffer(seq, np.uint8)])
            r = check_8to16(g, ws, d)
            assert r.error == oracle.TOO_SHORT
            check_passes8(g, ws, d)


def test_output_capacity(g, ws):
    rng = np.random.default_rng(4)
    for mix in (W.SCRIPT_MIXED, W.MIX_FOUR_BYTE_HEAVY, W.MIX_CJK_EMOJI):
        d8 = W.utf8_text(7, 5 * TILE8 + 13, mix)
        d16 = W.utf16_text(8, 5 * TILE16 + 13, mix)
        need16 = oracle.utf16_length_from_utf8(d8)
        need8 = oracle.utf8_length_from_utf16(d16)
        for cap in [0, 1, 2, 3, need16 - 1, need16, need16 + 1] + list(rng.integers(0, need16, 12)):
            check_8to16(g, ws, d8, cap=int(cap), out_off=int(rng.integers(0, 8)))
        for cap in [0, 1, 2, 3, 4, need8 - 1, need8, need8 + 1] + list(rng.integers(0, need8, 12)):
            check_16to8(g, ws, d16, cap=int(cap), out_off=int(rng.integers(0, 16)))
    # invalid input that would need more than n units: all four-byte leads
    check_8to16(g, ws, np.full(3 * TILE8 + 5, 0xF0, np.uint8))


def test_workspace_reuse_many_calls(g):
    ws = g.Workspace(1 << 20)
    rng = np.random.default_rng(5)
    for i in range(200):
        n = int(rng.integers(0, 70000))
        if i % 2:
            check_8to16(g, ws, W.utf8_text(i, n, MIXES[i % len(MIXES)]))
        else:
            check_16to8(g, ws, W.utf16_text(i, n // 2, MIXES[i % len(MIXES)]))


def test_host_buffer_forms(g, ws):
    d8 = W.utf8_text(9, 100000, W.SCRIPT_MIXED)
    h_in = torch.from_numpy(d8).pin_memory()
    h_out = torch.empty(d8.size, dtype=torch.int16).pin_memory()
    d_in = torch.empty(d8.size, dtype=torch.uint8, device="cuda")
    d_out = torch.empty(d8.size, dtype=torch.int16, device="cuda")
    d_res = torch.empty(3, dtype=torch.int64, device="cuda")
    r = g.utf8_to_utf16_host(h_in, h_out, d_in, d_out, ws, d_res)
    ref, ref_out = oracle.utf8_to_utf16(d8)
    assert tuple(r) == tuple(ref)
    assert np.array_equal(h_out.numpy().view(np.uint16)[:r.written], ref_out)

    d16 = W.utf16_text(10, 100000, W.MIX_CJK_EMOJI)
    h_in = torch.from_numpy(d16.view(np.int16)).pin_memory()
    h_out = torch.empty(3 * d16.size, dtype=torch.uint8).pin_memory()
    d_in = torch.empty(d16.size, dtype=torch.int16, device="cuda")
    d_out = torch.empty(3 * d16.size, dtype=torch.uint8, device="cuda")
    r = g.utf16_to_utf8_host(h_in, h_out, d_in, d_out, ws, d_res)
    ref, ref_out = oracle.utf16_to_utf8(d16)
    assert tuple(r) == tuple(ref)
    assert np.array_equal(h_out.numpy()[:r.written], ref_out)


def chunk_ends(chunk, n):
    """Where the host forms cut an input of n units with chunk size `chunk`,
    before each cut moves back to a character start: an eighth, a quarter
    and half of `chunk` first (at least 64 units), then `chunk`."""
    chunk = max(chunk, 64)
    if n // chunk >= 60:   # at most 64 chunks
        chunk = n // 59
    ends, step, at = [], max(chunk // 8, 64), 0
    while at < n:
        at += step
        ends.append(at)
        step = min(2 * step, chunk)
    return ends


def test_host_forms_in_chunks(g, ws):
    """The host forms cut into many chunks: every result, the host output,
    the device output and the device result equal the single call's, with
    errors and capacity ends placed near the cuts."""
    rng = np.random.default_rng(12)
    d_res = torch.empty(3, dtype=torch.int64, device="cuda")
    clean8 = W.utf8_text(13, 200_000, W.MIX_FOUR_BYTE_HEAVY)
    clean16 = W.utf16_text(14, 150_000, W.MIX_CJK_EMOJI)
    for chunk in (64, 1000, 4099, 50_000):
        for variant in range(4):
            a = clean8.copy()
            if variant:   # a corrupted byte next to where a chunk ends
                a[min(a.size - 1, int(rng.choice(chunk_ends(chunk, a.size)[:8])) + int(rng.integers(-3, 4)))] = 0xFF
            for cap in (a.size, int(rng.integers(1, a.size))):
                h_in = torch.from_numpy(a).pin_memory()
                h_out = torch.full((cap,), GUARD * 257, dtype=torch.int16).pin_memory()
                d_in = torch.empty(a.size, dtype=torch.uint8, device="cuda")
                d_out = torch.empty(cap, dtype=torch.int16, device="cuda")
                r = g.utf8_to_utf16_host(h_in, h_out, d_in, d_out, ws, d_res, chunk=chunk)
                ref, ref_out = oracle.utf8_to_utf16(a, cap=cap)
                assert tuple(r) == tuple(ref), (chunk, variant, cap, r, ref)
                assert tuple(g.read_result(d_res)) == tuple(ref)
                assert np.array_equal(h_out.numpy().view(np.uint16)[:r.written], ref_out)
                assert np.array_equal(d_out.cpu().numpy().view(np.uint16)[:r.written], ref_out)
        for variant in range(4):
            u = clean16.copy()
            if variant:   # a lone surrogate next to where a chunk ends
                u[min(u.size - 1, int(rng.choice(chunk_ends(chunk, u.size)[:8])) + int(rng.integers(-2, 3)))] = \
                    0xD800 + variant
            for cap in (3 * u.size, int(rng.integers(1, 3 * u.size))):
                h_in = torch.from_numpy(u.view(np.int16)).pin_memory()
                h_out = torch.full((cap,), GUARD, dtype=torch.uint8).pin_memory()
                d_in = torch.empty(u.size, dtype=torch.int16, device="cuda")
                d_out = torch.empty(cap, dtype=torch.uint8, device="cuda")
                r = g.utf16_to_utf8_host(h_in, h_out, d_in, d_out, ws, d_res, chunk=chunk)
                ref, ref_out = oracle.utf16_to_utf8(u, cap=cap)
                assert tuple(r) == tuple(ref), (chunk, variant, cap, r, ref)
                assert tuple(g.read_result(d_res)) == tuple(ref)
                assert np.array_equal(h_out.numpy()[:r.written], ref_out)
                assert np.array_equal(d_out.cpu().numpy()[:r.written], ref_out)


# ---------------------------------------------------------------------------
# The benchmark workloads at full size
# ---------------------------------------------------------------------------
def test_latin_cyrillic_utf8_1mib(g, ws):
    d = W.latin_cyrillic_utf8_1mib()
    r = check_8to16(g, ws, d)
    assert r.error == oracle.OK and r.position == d.size
    check_passes8(g, ws, d)


def test_cjk_emoji_utf16_256mib(g, ws):
    d = W.cjk_emoji_utf16_256mib()
    inp = dev_u16(d)
    out = torch.empty(3 * d.size, dtype=torch.uint8, device="cuda")
    res, _ = g.utf16_to_utf8(inp, out=out, ws=ws)
    ref, ref_out = oracle.utf16_to_utf8(d)
    assert tuple(res) == tuple(ref) and res.error == oracle.OK
    assert torch.equal(out[:res.written].cpu(), torch.from_numpy(ref_out))
    assert tuple(g.validate_utf16(inp, ws=ws)) == tuple(oracle.validate_utf16(d))
    assert g.utf8_length_from_utf16(inp, ws=ws) == ref.written


def test_four_byte_heavy_utf8_64mib_every_error(g, ws):
    et = W.four_byte_heavy_utf8_64mib()
    assert len(et.tokens) > 30
    out = torch.empty(et.data.size, dtype=torch.int16, device="cuda")
    # (i) the buffer with all its errors: the first one is reported
    res, _ = g.utf8_to_utf16(dev_u8(et.data), out=out, ws=ws)
    ref, ref_out = oracle.utf8_to_utf16(et.data)
    assert tuple(res) == tuple(ref) == (et.tokens[0][2], et.tokens[0][0], ref.written)
    assert np.array_equal(out[:res.written].cpu().numpy().view(np.uint16), ref_out)
    # (ii) with errors before k repaired, error k is the first
    for k, (off, _ln, cls) in enumerate(et.tokens):
        d = et.repaired_before(k)
        res, _ = g.utf8_to_utf16(dev_u8(d), out=out, ws=ws)
        v = g.validate_utf8(dev_u8(d), ws=ws)
        assert (res.error, res.position) == (cls, off) == (v.error, v.position), k
        ref = oracle.utf8_to_utf16(d)[0]
        assert tuple(res) == tuple(ref)
    # (iii) the clean buffer
    clean = et.repaired_before(len(et.tokens))
    res, _ = g.utf8_to_utf16(dev_u8(clean), out=out, ws=ws)
    ref, ref_out = oracle.utf8_to_utf16(clean)
    assert tuple(res) == tuple(ref) and res.error == oracle.OK
    assert np.array_equal(out[:res.written].cpu().numpy().view(np.uint16), ref_out)
    assert g.utf16_length_from_utf8(dev_u8(clean), ws=ws) == ref.written


def test_validate_utf16_one_error_anywhere_in_a_long_buffer(g, ws):
    """The validate-only pass checks surrogate pairs two units at a time and
    streams several tiles per CTA: one lone or broken surrogate placed at
    thread (16 units), warp (512), tile (4096) boundaries and in tiles a CTA
    reaches only after prefetching is found at its exact position."""
    base = W.utf16_text(31, 6 << 20, W.MIX_CJK_EMOJI)
    n = base.size
    positions = []
    for b in (16 * 7, 512 * 3, 4096 * 5, 4096 * 1500, n - 4096 * 3, n - 2):
        positions += [b - 1, b, b + 1]
    positions += [0, n - 1, 15, 31, 32]
    for form in range(3):
        for p in positions:
            d = base.copy()
            if form == 0:      # a lone high surrogate
                d[p] = 0xD83D
                if p + 1 < n:
                    d[p + 1] = 0x4E00
            elif form == 1:    # a lone low surrogate
                d[p] = 0xDE00
                if p > 0:
                    d[p - 1] = 0x4E00
            else:              # a high followed by a low in the wrong order
                d[p] = 0xDE00
                if p + 1 < n:
                    d[p + 1] = 0xD83D
                if p > 0:
                    d[p - 1] = 0x4E00
                if p + 2 < n:
                    d[p + 2] = 0x4E00
            inp = dev_u16(d, p % 8)
            assert tuple(g.validate_utf16(inp, ws=ws)) == tuple(oracle.validate_utf16(d)), (form, p)
            assert g.utf8_length_from_utf16(inp, ws=ws) == oracle.utf8_length_from_utf16(d), (form, p)


def test_unchecked_equals_checked_on_valid_input(g, ws):
    """The non-validating calls give the validating calls' result and output
    on valid input: every mix, sizes across tiles and alignments, and the
    256 MiB benchmark buffer."""
    for i, mix in enumerate(MIXES):
        for n in (1, 37, TILE8 - 1, 3 * TILE8 + 17):
            d8 = W.utf8_text(50 + i, n, mix)
            a, oa = g.utf8_to_utf16(dev_u8(d8, i % 16), ws=ws)
            b, ob = g.utf8_to_utf16(dev_u8(d8, i % 16), ws=ws, validate=False)
            assert tuple(a) == tuple(b) and a.error == 0
            assert torch.equal(oa[:a.written], ob[:b.written])
        for n in (1, 37, TILE16 - 1, 3 * TILE16 + 17):
            d16 = W.utf16_text(60 + i, n, mix)
            a, oa = g.utf16_to_utf8(dev_u16(d16, i % 8), ws=ws)
            b, ob = g.utf16_to_utf8(dev_u16(d16, i % 8), ws=ws, validate=False)
            assert tuple(a) == tuple(b) and a.error == 0
            assert torch.equal(oa[:a.written], ob[:b.written])
    d = W.cjk_emoji_utf16_256mib()
    inp = dev_u16(d)
    a, oa = g.utf16_to_utf8(inp, ws=ws)
    b, ob = g.utf16_to_utf8(inp, ws=ws, validate=False)
    assert tuple(a) == tuple(b) and torch.equal(oa[:a.written], ob[:b.written])


def test_unchecked_on_invalid_input_stays_in_bounds(g, ws):
    """Without validation, invalid input gives OK or OUTPUT_TOO_SMALL and an
    unspecified output, but nothing outside the output buffer is touched,
    also with capacities that cut the output short."""
    rng = np.random.default_rng(23)
    for trial in range(40):
        n = int(rng.integers(1, 3 * TILE8))
        b = rng.integers(0, 256, n).astype(np.uint8)
        cap = int(rng.integers(0, 2 * n + 4)) if trial % 3 == 0 else n
        outbuf = torch.full((cap + 32,), GUARD * 257, dtype=torch.int16, device="cuda")
        r, _ = g.utf8_to_utf16(dev_u8(b, trial % 16), out=outbuf[8:8 + cap], ws=ws, validate=False)
        assert r.error in (oracle.OK, oracle.OUTPUT_TOO_SMALL) and r.written <= cap
        host = outbuf.cpu().numpy().view(np.uint16)
        assert np.all(host[:8] == GUARD * 257) and np.all(host[8 + cap:] == GUARD * 257)
        u = rng.integers(0, 65536, n).astype(np.uint16)
        u[rng.random(n) < 0.3] = rng.integers(0xD800, 0xE000, int((rng.random(n) < 0.3).sum()) or 1)[0]
        cap = int(rng.integers(0, 3 * n + 4)) if trial % 3 == 0 else 3 * n
        outbuf = torch.full((cap + 64,), GUARD, dtype=torch.uint8, device="cuda")
        r, _ = g.utf16_to_utf8(dev_u16(u, trial % 8), out=outbuf[16:16 + cap], ws=ws, validate=False)
        assert r.error in (oracle.OK, oracle.OUTPUT_TOO_SMALL) and r.written <= cap
        host = outbuf.cpu().numpy()
        assert np.all(host[:16] == GUARD) and np.all(host[16 + cap:] == GUARD)


def test_dense_lone_surrogates_fit_the_staging_buffer(g, ws):
    """Input made of lone or mis-ordered surrogates over several tiles: a
    lone surrogate counts 2 bytes, so no tile's output outgrows the staging
    buffer.  The validating call reports the oracle's first error; the
    non-validating call stays inside the output buffer."""
    rng = np.random.default_rng(29)
    n = 3 * TILE16 + 5
    cases = [np.full(n, 0xD800, np.uint16), np.full(n, 0xDFFF, np.uint16),
             np.tile(np.array([0xDC00, 0xD800], np.uint16), n // 2),
             rng.integers(0xD800, 0xE000, n).astype(np.uint16),
             np.where(rng.random(n) < 0.5, 0xDBFF, 0x9FFF).astype(np.uint16)]
    for u in cases:
        check_16to8(g, ws, u)
        check_passes16(g, ws, u)
        for cap in (3 * u.size, u.size):
            outbuf = torch.full((cap + 64,), GUARD, dtype=torch.uint8, device="cuda")
            r, _ = g.utf16_to_utf8(dev_u16(u), out=outbuf[16:16 + cap], ws=ws, validate=False)
            assert r.error in (oracle.OK, oracle.OUTPUT_TOO_SMALL) and r.written <= cap
            host = outbuf.cpu().numpy()
            assert np.all(host[:16] == GUARD) and np.all(host[16 + cap:] == GUARD)


def test_uniform_and_mixed_warps_in_one_tile(g, ws):
    """Runs of one script (all 3-byte, all ASCII, all 2-byte, 2-byte with lone
    surrogates) next to mixed text, with run lengths that are not multiples
    of a warp's 768 units: warps on the uniform-class fast paths and warps on
    the general path share tiles and write adjacent bytes."""
    rng = np.random.default_rng(31)
    scripts = [W.SCRIPT_CJK, W.SCRIPT_ASCII, W.SCRIPT_TWO_BYTE, W.MIX_CJK_EMOJI]
    for trial in range(12):
        parts = []
        for p in range(int(rng.integers(3, 9))):
            n = int(rng.integers(1, 4000)) if p % 2 else int(rng.integers(700, 6000))
            parts.append(W.utf16_text(1000 + 10 * trial + p, n, scripts[int(rng.integers(0, 4))]))
        d = np.concatenate(parts).astype(np.uint16)
        check_16to8(g, ws, d, in_off=trial % 8, out_off=trial % 16)
    # a 2-byte run with lone surrogates in it: the error is reported, the prefix exact
    d = W.utf16_text(77, 5000, W.SCRIPT_TWO_BYTE).copy()
    d[3001] = 0xD800
    check_16to8(g, ws, d)
    check_16to8(g, ws, d, cap=2500)


def test_uniform_two_and_three_byte_warps_utf8(g, ws):
    """UTF-8 -> UTF-16 warps whose chunks hold only 2-byte or only 3-byte
    characters take the uniform-pattern paths (leads every other or every
    third byte); covered at every start phase of the characters against the
    chunks, with one character of another length planted in one thread's
    chunk (the warp falls back), and with errors inside uniform runs (an
    overlong 2-byte lead, an encoded surrogate, a 3-byte character cut short
    at a chunk's end, a stray continuation)."""
    rng = np.random.default_rng(7)
    two = np.array([0xC0 | (c >> 6) for c in range(0x400, 0x500)], np.uint8)
    for script, length in ((W.SCRIPT_TWO_BYTE, 2), (W.SCRIPT_CJK, 3)):
        base = W.utf8_text(11 * length, 5 * TILE8 + 777, script)
        for lead_bytes in range(0, 6):           # 0-5 ASCII bytes shift the character phase
            data = np.concatenate([np.full(lead_bytes, 0x41, np.uint8), base])
            check_8to16(g, ws, data)
            check_8to16(g, ws, data, in_off=lead_bytes % 3, out_off=lead_bytes % 2)
            # one character of another length in the middle of a chunk
            d2 = data.copy()
            p = 2 * TILE8 + 96 * 32 + 7
            p -= (p - lead_bytes) % length
            d2 = np.concatenate([d2[:p], np.array([0x41], np.uint8), d2[p:]])
            check_8to16(g, ws, d2)
        # errors inside a uniform run, near chunk (32-byte) and tile ends
        for at in (TILE8 - 3, TILE8 - 1, 3 * TILE8 + 32 * 17 + 1, 4 * TILE8 + 31):
            q = at - at % length                      # a character start (no ASCII prefix)
            for kind in range(4):
                bad = base.copy()
                if kind == 0:
                    bad[q] = 0xC1 if length == 2 else 0xE0   # overlong lead (E0 then 80-9F only if the next byte is low)
                    if length == 3:
                        bad[q + 1] = 0x80 | (bad[q + 1] & 0x1F)
                elif kind == 1:
                    if length == 3:
                        bad[q], bad[q + 1] = 0xED, 0xA0 | (bad[q + 1] & 0x1F)   # U+D800-DFFF
                    else:
                        bad[q + 1] = 0x41                                     # 2-byte lead cut short
                elif kind == 2:
                    bad = bad[:q + length - 1]                                # cut short at the end
                else:
                    bad[q] = 0x80 | (bad[q] & 0x3F)                           # stray continuation
                check_8to16(g, ws, bad)
    # random 2-byte text with random planted ASCII bytes, many sizes
    for n in rng.integers(1, 3 * TILE8, 12):
        t = W.utf8_text(int(n), int(n), W.SCRIPT_TWO_BYTE).copy()
        t[rng.integers(0, t.size, 2)] = 0x20
        check_8to16(g, ws, t)
