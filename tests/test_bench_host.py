"""Host logic of the benchmark: the CPU baseline cuts the UTF-16 buffer into
chunks for the oracle's threads; the cuts must never fall between the two
halves of a surrogate pair, so that the chunks' transcodings concatenate to
the whole buffer's."""
import numpy as np

import bench
import oracle
import workloads as W


def test_pair_safe_chunks_concatenate_to_the_whole_transcoding():
    d = W.utf16_text(1, 200_000, W.MIX_CJK_EMOJI)
    whole = oracle.utf16_to_utf8(d)[1]
    for parts in (1, 2, 3, 7, 16, 64):
        chunks = bench.pair_safe_chunks(d, parts)
        assert sum(c.size for c in chunks) == d.size
        for c in chunks[:-1]:
            assert not (0xD800 <= int(c[-1]) <= 0xDBFF)
        assert np.array_equal(np.concatenate([oracle.utf16_to_utf8(c)[1] for c in chunks]), whole)


def test_pair_safe_chunks_on_a_buffer_of_pairs():
    d = np.tile(np.array([0xD83D, 0xDE00], np.uint16), 1000)   # every cut point but every other is mid-pair
    chunks = bench.pair_safe_chunks(d, 9)
    assert all(c.size % 2 == 0 for c in chunks)
    assert sum(c.size for c in chunks) == d.size
