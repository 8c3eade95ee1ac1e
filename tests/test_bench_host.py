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


def test_count_chars_counts_a_pair_once():
    d = W.utf16_text(3, 50_000, W.MIX_CJK_EMOJI)
    assert bench.count_chars(d) == len(d.tobytes().decode("utf-16-le"))
    # lone low, a pair, 'A', lone low, lone high at the end: five characters
    assert bench.count_chars(np.array([0xDC00, 0xD800, 0xDC00, 0x41, 0xDC01, 0xD800], np.uint16)) == 5
    assert bench.count_chars(np.zeros(0, np.uint16)) == 0


def test_reference_arm_line(capsys):
    """The reference arm (the oracle on the host cores) prints one JSON line
    with the main arm's metric, unit and config, and the keys of the bench
    contract."""
    import json
    import types
    args = types.SimpleNamespace(mib=2, steps=1, warmup=1, gpus=1)
    assert bench.run_reference(args) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    data = W.cjk_emoji_utf16_256mib(seed=bench.rank_seed(0), nbytes=2 << 20)
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == "GB/s"
    assert line["config"] == bench.workload_config(data, oracle.utf8_length_from_utf16(data), 1, 2)
    assert line["config"]["output_bytes"] == oracle.utf16_to_utf8(data)[0].written
    for key in ("value", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling", "dtype",
                "data", "cpu_baseline", "e2e", "gpu_launches"):
        assert key in line, key
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
