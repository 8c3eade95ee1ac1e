"""The chunk boundaries of the host forms, on the CPU against the oracle.

gputf_utf8_chunk_end / gputf_utf16_chunk_end (host code in libgputf) pick the
points where the host-buffer transcoders cut a large input.  The oracle shows
that a cut there changes nothing: the oracle on the two pieces, combined the
way the host forms combine their chunks (the second piece gets the capacity
left and runs only if the first succeeded; its positions are shifted by the
cut), gives the single call's result and output, for every cut position of
short texts with every kind of character and error, and for whole inputs cut
into many chunks with capacities that end the output anywhere.
"""
import ctypes

import numpy as np
import pytest

import oracle
import workloads as W

MAX_CHUNKS = 64


@pytest.fixture(scope="module")
def L():
    import paper_2109_10433_gb300 as g
    g.build()
    return g.lib()


def cut8(L, a):
    return lambda at: int(L.gputf_utf8_chunk_end(a.ctypes.data, a.size, at))


def cut16(L, a):
    return lambda at: int(L.gputf_utf16_chunk_end(a.ctypes.data, a.size, at))


def combined(fn, data, cap, cuts):
    """The host forms' combination of per-chunk calls: chunk k runs on
    data[cuts[k]:cuts[k+1]] with the capacity left, and the first error or
    full output ends the call."""
    out, done = [], 0
    for a, b in zip(cuts[:-1], cuts[1:]):
        r, o = fn(data[a:b], cap=cap - done)
        w = min(r.written, cap - done)
        out.append(np.asarray(o)[:w])
        done += w
        if r.error != oracle.OK:
            return (r.error, a + r.position, done), np.concatenate(out)
    return (oracle.OK, data.size, done), (np.concatenate(out) if out else np.zeros(0))


def host_cuts(cut, n, chunk):
    """The chunk starts the host forms compute (the same clamps)."""
    chunk = max(chunk, 64)
    if chunk and n // chunk >= MAX_CHUNKS:
        chunk = n // (MAX_CHUNKS - 1)
    a = [0]
    while True:
        nxt = n if len(a) == MAX_CHUNKS else cut(a[-1] + chunk)
        a.append(nxt)
        if nxt >= n:
            return a


def soup8(rng, n):
    """Bytes of every class: ASCII, continuation, every lead, 0xF8-0xFF, and
    runs of valid characters of every length."""
    parts = []
    while sum(len(p) for p in parts) < n:
        k = rng.integers(0, 6)
        if k == 0:
            parts.append(bytes(rng.integers(0, 256, size=rng.integers(1, 6)).astype(np.uint8)))
        elif k == 1:
            parts.append(bytes([0x80 | int(rng.integers(0, 64))] * int(rng.integers(1, 6))))
        else:
            cp = int(rng.choice([rng.integers(0, 0x80), rng.integers(0x80, 0x800), rng.integers(0x800, 0xD800),
                                 rng.integers(0xE000, 0x10000), rng.integers(0x10000, 0x110000)]))
            parts.append(chr(cp).encode("utf-8"))
    return np.frombuffer(b"".join(parts)[:n], dtype=np.uint8).copy()


def soup16(rng, n):
    kind = rng.integers(0, 4, size=n)
    return np.where(kind == 0, rng.integers(0xD800, 0xE000, size=n),
                    np.where(kind == 1, rng.integers(0, 0x80, size=n),
                             rng.integers(0, 0x10000, size=n))).astype(np.uint16)


def test_utf8_every_cut_of_short_texts(L):
    rng = np.random.default_rng(61)
    for trial in range(150):
        a = soup8(rng, int(rng.integers(1, 90)))
        whole_r, whole_o = oracle.utf8_to_utf16(a)
        cut = cut8(L, a)
        for at in range(a.size + 2):
            p = cut(at)
            assert p == a.size if at >= a.size else (at - 3 <= p <= at)
            r, o = combined(oracle.utf8_to_utf16, a, a.size, [0, p, a.size] if 0 < p < a.size else [0, a.size])
            assert r == tuple(whole_r), (a.tolist(), at, p)
            assert np.array_equal(o, whole_o)


def test_utf16_every_cut_of_short_texts(L):
    rng = np.random.default_rng(62)
    for trial in range(150):
        a = soup16(rng, int(rng.integers(1, 60)))
        whole_r, whole_o = oracle.utf16_to_utf8(a)
        cut = cut16(L, a)
        for at in range(a.size + 2):
            p = cut(at)
            assert p == a.size if at >= a.size else (at - 1 <= p <= at)
            r, o = combined(oracle.utf16_to_utf8, a, 3 * a.size, [0, p, a.size] if 0 < p < a.size else [0, a.size])
            assert r == tuple(whole_r), (a.tolist(), at, p)
            assert np.array_equal(o, whole_o)


@pytest.mark.parametrize("chunk", [1, 64, 77, 500])
def test_utf8_many_chunks_and_capacities(L, chunk):
    rng = np.random.default_rng(63 + chunk)
    for mix in (W.MIX_FOUR_BYTE_HEAVY, W.SCRIPT_MIXED, W.MIX_LATIN_CYRILLIC):
        clean = W.utf8_text(int(rng.integers(0, 1000)), 6000, mix)
        for variant in range(6):
            a = clean.copy()
            if variant:   # one corrupted byte, anywhere
                a[rng.integers(0, a.size)] = rng.integers(0x80, 0x100)
            for cap in (a.size, int(rng.integers(0, a.size)), 1000):
                whole_r, whole_o = oracle.utf8_to_utf16(a, cap=cap)
                r, o = combined(oracle.utf8_to_utf16, a, cap, host_cuts(cut8(L, a), a.size, chunk))
                assert r == tuple(whole_r), (variant, cap)
                assert np.array_equal(o, whole_o)


@pytest.mark.parametrize("chunk", [1, 64, 77, 500])
def test_utf16_many_chunks_and_capacities(L, chunk):
    rng = np.random.default_rng(73 + chunk)
    for mix in (W.MIX_CJK_EMOJI, W.SCRIPT_MIXED):
        clean = W.utf16_text(int(rng.integers(0, 1000)), 5000, mix)
        for variant in range(6):
            a = clean.copy()
            if variant:   # one lone surrogate, anywhere
                a[rng.integers(0, a.size)] = rng.integers(0xD800, 0xE000)
            for cap in (3 * a.size, int(rng.integers(0, 3 * a.size)), 2000):
                whole_r, whole_o = oracle.utf16_to_utf8(a, cap=cap)
                r, o = combined(oracle.utf16_to_utf8, a, cap, host_cuts(cut16(L, a), a.size, chunk))
                assert r == tuple(whole_r), (variant, cap)
                assert np.array_equal(o, whole_o)


def test_chunk_end_edges(L):
    e = np.zeros(0, dtype=np.uint8)
    assert L.gputf_utf8_chunk_end(None, 0, 0) == 0
    assert L.gputf_utf16_chunk_end(None, 0, 5) == 0
    a = np.frombuffer("€".encode(), dtype=np.uint8).copy()        # E2 82 AC
    assert [cut8(L, a)(at) for at in range(4)] == [0, 0, 0, 3]
    s = np.array([0xD83D, 0xDE00, 0x41], dtype=np.uint16)           # a pair, then 'A'
    assert [cut16(L, s)(at) for at in range(4)] == [0, 0, 2, 3]
    del e


def _cut_breaks_results(fn, texts, cap_of, cut_of):
    """True when some cut that `cut_of(text)` gives changes the combined
    result or output against the single call on the whole text."""
    for a in texts:
        whole_r, whole_o = fn(a, cap=cap_of(a))
        cut = cut_of(a)
        for at in range(a.size + 1):
            p = cut(at)
            r, o = combined(fn, a, cap_of(a), [0, p, a.size] if 0 < p < a.size else [0, a.size])
            if r != tuple(whole_r) or not np.array_equal(o, whole_o):
                return True
    return False


def test_wrong_cut_rules_are_caught(L):
    """The checks above fail for cut rules that are slightly wrong: a UTF-8
    rule that looks back only three bytes (so a cut can fall after the third
    byte of a four-byte character) and a UTF-16 rule that ignores surrogates
    (so a cut can split a pair)."""
    rng = np.random.default_rng(64)
    t8 = [soup8(rng, int(rng.integers(10, 90))) for _ in range(40)]
    t16 = [soup16(rng, int(rng.integers(10, 60))) for _ in range(40)]

    def short8(a):
        def cut(at):
            if at >= a.size:
                return a.size
            for k in range(3):   # one byte short of the four a character can span
                if k <= at and (int(a[at - k]) & 0xC0) != 0x80:
                    return at - k
            return at
        return cut

    def blind16(a):
        return lambda at: min(at, a.size)

    assert _cut_breaks_results(oracle.utf8_to_utf16, t8, lambda a: a.size, short8)
    assert _cut_breaks_results(oracle.utf16_to_utf8, t16, lambda a: 3 * a.size, blind16)
    # the library's rules on the same texts
    assert not _cut_breaks_results(oracle.utf8_to_utf16, t8, lambda a: a.size, lambda a: cut8(L, a))
    assert not _cut_breaks_results(oracle.utf16_to_utf8, t16, lambda a: 3 * a.size, lambda a: cut16(L, a))
