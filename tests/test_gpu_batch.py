"""GPU parity of the batched C-ABI call: every string's result and output in a
batch are those of the oracle on that string alone, for every tile
configuration, with strings of all lengths (empty, one unit, spanning many
tiles), errors at string edges, capacities that cut outputs short, and tiles
holding more strings than the kernel caches."""
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


def check(g, strings8, strings16, caps8=None, caps16=None, config=0):
    from paper_2109_10433_gb300 import batch as B
    b8 = B.DeviceBatch(strings8, B.UTF8_TO_UTF16, caps8) if strings8 is not None else None
    b16 = B.DeviceBatch(strings16, B.UTF16_TO_UTF8, caps16) if strings16 is not None else None
    ws = B.workspace_for(b8, b16)
    B.batch_transcode(b8, b16, ws, config=config)
    torch.cuda.synchronize()
    for b, strings, fn in ((b8, strings8, oracle.utf8_to_utf16), (b16, strings16, oracle.utf16_to_utf8)):
        if b is None:
            continue
        res = b.read_results()
        caps = np.diff(b.out_offsets_host)
        for s, data in enumerate(strings):
            ref, ref_out = fn(data, cap=int(caps[s]))
            assert tuple(res[s]) == tuple(ref), (s, len(data), res[s], ref, config)
            assert np.array_equal(b.output(s, ref.written), ref_out), s
    return b8, b16


def test_workload_batch_every_config(g):
    from paper_2109_10433_gb300 import batch as B
    bt = W.string_batch(3, 1500)
    s8 = [s for s, d in zip(bt.strings, bt.directions) if d == 0]
    s16 = [s for s, d in zip(bt.strings, bt.directions) if d == 1]
    assert bt.invalid.sum() > 5
    for cfg in range(B.config_count()):
        check(g, s8, s16, config=cfg)


def test_empty_tiny_and_long_strings(g):
    rng = np.random.default_rng(1)
    s8, s16 = [], []
    for i in range(400):
        k = int(rng.integers(0, 6))
        n = [0, 1, 2, 3, 5000, 70000][k]
        s8.append(W.utf8_text(i, n, W.SCRIPT_MIXED))
        s16.append(W.utf16_text(i, n, W.MIX_CJK_EMOJI))
    check(g, s8, s16)
    check(g, [np.zeros(0, np.uint8)] * 50, [np.zeros(0, np.uint16)] * 7)
    check(g, [W.utf8_text(9, 300000, W.MIX_FOUR_BYTE_HEAVY)], None)


def test_more_strings_in_a_tile_than_the_cache(g):
    rng = np.random.default_rng(2)
    s8 = [W.utf8_text(i, int(rng.integers(0, 4)), W.SCRIPT_MIXED) for i in range(6000)]
    s16 = [W.utf16_text(i, int(rng.integers(0, 3)), W.MIX_CJK_EMOJI) for i in range(6000)]
    for cfg in (0, 3):
        check(g, s8, s16, config=cfg)


def test_errors_at_string_edges(g):
    rng = W.rng_for(5)
    s8, s16 = [], []
    for i in range(600):
        base = W.utf8_text(i, int(rng.integers(1, 200)), W.MIX_FOUR_BYTE_HEAVY)
        tok, _ = W.utf8_error_token(rng, W.UTF8_TOKEN_KINDS[i % 5])
        tok = np.frombuffer(tok, np.uint8)
        s8.append(np.concatenate([tok, base]) if i % 3 == 0 else
                  np.concatenate([base, tok]) if i % 3 == 1 else base[:-1] if base.size > 1 else base)
        b16 = W.utf16_text(i, int(rng.integers(1, 100)), W.MIX_CJK_EMOJI)
        t16, _ = W.utf16_error_token(rng)
        t16 = np.array(t16, np.uint16)
        s16.append(np.concatenate([t16, b16]) if i % 3 == 0 else
                   np.concatenate([b16, t16]) if i % 3 == 1 else b16)
    # strings that end with a high surrogate and strings that start with a low one, back to back
    s16 += [np.array([0x41, 0xD83D], np.uint16), np.array([0xDE00, 0x42], np.uint16)]
    check(g, s8, s16)


def test_capacities_cut_outputs(g):
    rng = np.random.default_rng(4)
    s8 = [W.utf8_text(i, int(rng.integers(1, 3000)), W.SCRIPT_MIXED) for i in range(300)]
    s16 = [W.utf16_text(i, int(rng.integers(1, 3000)), W.MIX_CJK_EMOJI) for i in range(300)]
    c8 = [int(rng.integers(0, oracle.utf16_length_from_utf8(s) + 2)) for s in s8]
    c16 = [int(rng.integers(0, oracle.utf8_length_from_utf16(s) + 2)) for s in s16]
    check(g, s8, s16, c8, c16)


def test_errors_and_capacity_deep_in_long_strings(g):
    """Strings spanning many tiles with the first error, or the first unit
    that does not fit, in any of their tiles (the result's `written` is then
    found from the tiles' status words plus one tile), for every
    configuration, transcoding and validating."""
    from paper_2109_10433_gb300 import batch as B
    rng = np.random.default_rng(9)
    s8, s16, c8, c16 = [], [], [], []
    for i in range(40):
        n = int(rng.integers(20000, 90000))
        t8 = W.utf8_error_text(100 + i, n, W.SCRIPT_MIXED, mean_gap=int(rng.integers(3000, 60000)))
        t16 = W.utf16_text(200 + i, n // 2, W.MIX_CJK_EMOJI).copy()
        k = int(rng.integers(0, t16.size))
        if i % 3:
            t16[k] = 0xD800 if i % 2 else 0xDC00      # a lone surrogate somewhere inside
        s8.append(t8.data)
        s16.append(t16)
        l8 = oracle.utf16_length_from_utf8(t8.data)
        l16 = oracle.utf8_length_from_utf16(t16)
        # capacities: ample, or cut anywhere in the string
        c8.append(int(rng.integers(0, l8 + 1)) if i % 4 == 0 else len(t8.data))
        c16.append(int(rng.integers(0, l16 + 1)) if i % 4 == 1 else 3 * t16.size)
    for cfg in range(B.config_count()):
        check(g, s8, s16, c8, c16, config=cfg)
    for cfg in (0, B.config_count() - 1):
        b8 = B.DeviceBatch(s8, B.UTF8_TO_UTF16, validate_only=True)
        b16 = B.DeviceBatch(s16, B.UTF16_TO_UTF8, validate_only=True)
        ws = B.workspace_for(b8, b16)
        B.batch_transcode(b8, b16, ws, config=cfg)
        torch.cuda.synchronize()
        for b, strings, val in ((b8, s8, oracle.validate_utf8), (b16, s16, oracle.validate_utf16)):
            res = b.read_results()
            for j, data in enumerate(strings):
                assert tuple(res[j]) == tuple(val(data)), (cfg, j)


def test_batch_equals_single_string_calls(g):
    strings = [W.utf16_text(i, 10000 + 37 * i, W.MIX_CJK_EMOJI) for i in range(5)]
    _, b16 = check(g, None, strings)
    res = b16.read_results()
    for s, data in enumerate(strings):
        r, out = g.utf16_to_utf8(torch.from_numpy(data.view(np.int16)).cuda())
        assert tuple(r) == tuple(res[s])
        assert np.array_equal(out[:r.written].cpu().numpy(), b16.output(s, r.written))


@pytest.mark.parametrize("graph", [False, True])
def test_full_size_workload_batch(g, graph):
    """The 100,000-string workload at full size, in the launch the benchmark
    times (autotuned configuration; graph replay), against the oracle."""
    from paper_2109_10433_gb300 import autotune
    from paper_2109_10433_gb300 import batch as B
    bt = W.string_batch(3, 100000)
    s8 = [s for s, d in zip(bt.strings, bt.directions) if d == 0]
    s16 = [s for s, d in zip(bt.strings, bt.directions) if d == 1]
    b8 = B.DeviceBatch(s8, B.UTF8_TO_UTF16)
    b16 = B.DeviceBatch(s16, B.UTF16_TO_UTF8)
    ws = B.workspace_for(b8, b16)
    cfg = autotune.best_config(b8, b16, ws)   # the benchmark's choice
    if graph:
        gr = B.BatchGraph(b8, b16, ws, cfg)
        for _ in range(3):
            gr.replay()
    else:
        B.batch_transcode(b8, b16, ws, config=cfg)
    torch.cuda.synchronize()
    bad = []
    for b, strings, fn in ((b8, s8, oracle.utf8_to_utf16), (b16, s16, oracle.utf16_to_utf8)):
        res = b.read_results()
        out = b.out.cpu().numpy()
        if b.direction == B.UTF8_TO_UTF16:
            out = out.view(np.uint16)
        for s, data in enumerate(strings):
            ref, ref_out = fn(data)
            a = int(b.out_offsets_host[s])
            if tuple(res[s]) != tuple(ref) or not np.array_equal(out[a:a + ref.written], ref_out):
                bad.append((b.direction, s, len(data), tuple(res[s]), tuple(ref)))
    assert not bad, (len(bad), bad[:5])


def test_one_workspace_across_configurations_and_single_calls(g):
    """One workspace used in turn by every tile configuration (which lay it out
    differently) and by single-string calls: no call may read another's words."""
    from paper_2109_10433_gb300 import batch as B
    rng = W.rng_for(8)
    s8, s16 = [], []
    for i in range(800):
        t = W.utf8_text(i, int(rng.integers(1, 400)), W.SCRIPT_MIXED)
        if i % 7 == 0:
            tok, _ = W.utf8_error_token(rng, W.UTF8_TOKEN_KINDS[i % 5])
            t = np.concatenate([t, np.frombuffer(tok, np.uint8)])
        s8.append(t)
        u = W.utf16_text(i, int(rng.integers(1, 300)), W.MIX_CJK_EMOJI)
        if i % 7 == 3:
            u = np.concatenate([u, np.array([0xD800], np.uint16)])
        s16.append(u)
    b8 = B.DeviceBatch(s8, B.UTF8_TO_UTF16)
    b16 = B.DeviceBatch(s16, B.UTF16_TO_UTF8)
    ws = B.workspace_for(b8, b16)
    expect8 = [oracle.utf8_to_utf16(s)[0] for s in s8]
    expect16 = [oracle.utf16_to_utf8(s)[0] for s in s16]
    for rnd in range(3):
        for cfg in list(range(B.config_count())) + [0, 3, 1]:
            B.batch_transcode(b8, b16, ws, config=cfg)
            torch.cuda.synchronize()
            assert [tuple(r) for r in b8.read_results()] == [tuple(r) for r in expect8], (rnd, cfg)
            assert [tuple(r) for r in b16.read_results()] == [tuple(r) for r in expect16], (rnd, cfg)
        # the same workspace for a single-buffer call in between
        d = torch.from_numpy(s16[0].view(np.int16).copy()).cuda()
        r, _ = g.utf16_to_utf8(d, ws=ws)
        assert tuple(r) == tuple(expect16[0])


def test_validate_only_batch_equals_single_validation(g):
    """out == NULL validates only: each string's result is the oracle's
    validation result (written 0), across tiles and configurations, with one
    direction transcoding and the other validating in the same launch."""
    from paper_2109_10433_gb300 import batch as B
    bt = W.string_batch(11, 600)
    s8 = [s for s, d in zip(bt.strings, bt.directions) if d == 0] + [np.zeros(0, np.uint8), W.utf8_text(5, 90000, W.SCRIPT_MIXED)]
    s16 = [s for s, d in zip(bt.strings, bt.directions) if d == 1] + [np.zeros(0, np.uint16)]
    for cfg in range(B.config_count()):
        for v8, v16 in ((True, True), (True, False), (False, True)):
            b8 = B.DeviceBatch(s8, B.UTF8_TO_UTF16, validate_only=v8)
            b16 = B.DeviceBatch(s16, B.UTF16_TO_UTF8, validate_only=v16)
            ws = B.workspace_for(b8, b16)
            B.batch_transcode(b8, b16, ws, config=cfg)
            torch.cuda.synchronize()
            for b, strings, val, fn in ((b8, s8, oracle.validate_utf8, oracle.utf8_to_utf16),
                                        (b16, s16, oracle.validate_utf16, oracle.utf16_to_utf8)):
                res = b.read_results()
                for s, data in enumerate(strings):
                    if b.validate_only:
                        assert tuple(res[s]) == tuple(val(data)), (cfg, s)
                    else:
                        ref, ref_out = fn(data)
                        assert tuple(res[s]) == tuple(ref), (cfg, s)
                        assert np.array_equal(b.output(s, ref.written), ref_out), (cfg, s)
