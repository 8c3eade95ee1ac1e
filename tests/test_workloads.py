"""The seeded synthetic inputs follow their stated recipes.

Each benchmark workload is generated (at its full size where that is quick,
else by the same generator at a smaller size) and checked against the recipe:
exact sizes, strict validity under CPython's codecs (or exactly the injected
errors), code points only from the stated ranges, and character-class
fractions, string-length and request-size distributions, direction,
validate-only and invalid fractions within sampling tolerance.
"""
import numpy as np

import workloads as W

MiB = 1 << 20


def cps_of_utf8(b):
    return np.frombuffer(bytes(b).decode("utf-8").encode("utf-32-le"), dtype="<u4")


def cps_of_utf16(u):
    return np.frombuffer(np.asarray(u, np.uint16).tobytes().decode("utf-16-le").encode("utf-32-le"), dtype="<u4")


def frac(cps, lo, hi):
    return float(np.mean((cps >= lo) & (cps <= hi)))


def test_latin_cyrillic_utf8_1mib():
    d = W.latin_cyrillic_utf8_1mib(0)
    assert d.dtype == np.uint8 and d.size == MiB
    cps = cps_of_utf8(d)                                  # strictly valid
    assert np.all(((cps >= 0x20) & (cps <= 0x7E)) | ((cps >= 0x400) & (cps <= 0x4FF)))
    assert abs(frac(cps, 0x400, 0x4FF) - 0.10) < 0.005
    assert np.array_equal(W.latin_cyrillic_utf8_1mib(0), d)   # seeded: the same bytes again


def test_cjk_emoji_utf16_mix():
    u = W.cjk_emoji_utf16_256mib(1, nbytes=8 * MiB)       # the headline generator, at 8 MiB
    assert u.dtype == np.uint16 and u.nbytes == 8 * MiB
    cps = cps_of_utf16(u)
    assert np.all(((cps >= 0x20) & (cps <= 0x7E)) | ((cps >= 0x4E00) & (cps <= 0x9FFF))
                  | ((cps >= 0x1F300) & (cps <= 0x1FAFF)))
    assert abs(frac(cps, 0x20, 0x7E) - 0.20) < 0.005
    assert abs(frac(cps, 0x4E00, 0x9FFF) - 0.70) < 0.005
    assert abs(frac(cps, 0x1F300, 0x1FAFF) - 0.10) < 0.005


def test_four_byte_heavy_utf8_with_errors():
    et = W.four_byte_heavy_utf8_64mib(2, nbytes=16 * MiB, mean_gap=MiB // 4)
    assert et.data.size == 16 * MiB
    n = len(et.tokens)
    assert 40 <= n <= 90                                  # Poisson, mean 64
    offs = [t[0] for t in et.tokens]
    assert offs == sorted(offs) and all(b - a >= t[1] for (a, _, _), b, t in
                                        zip(et.tokens, offs[1:], et.tokens))
    clean = et.repaired_before(n)                         # every token overwritten: valid text
    cps = cps_of_utf8(clean)
    real = cps[cps != 0x41]                               # the repairs write 'A'
    assert abs(frac(real, 0x10000, 0x10FFFF) - 0.40) < 0.01
    assert abs(frac(real, 0x800, 0xFFFF) - 0.30) < 0.01
    assert not np.any((cps >= 0xD800) & (cps <= 0xDFFF))
    kinds = {t[2] for t in et.tokens}
    assert len(kinds) >= 4                                # the error kinds all occur
    for k in range(0, n, 7):                              # token k is the first error once the earlier ones are repaired
        d = bytes(et.repaired_before(k))
        try:
            d.decode("utf-8")
            raise AssertionError("no error")
        except UnicodeDecodeError as e:
            assert e.start == et.tokens[k][0]


def test_string_batch_recipe():
    bt = W.string_batch(3, 6000)
    assert len(bt.strings) == 6000
    nbytes = np.array([s.nbytes for s in bt.strings])
    assert nbytes.min() >= 8 and nbytes.max() <= 64 * 1024 + 8
    assert 900 <= np.median(nbytes) <= 1150               # log-normal, median 1 KiB
    assert abs(np.mean(bt.directions) - 0.5) < 0.03
    assert 30 <= bt.invalid.sum() <= 95                   # 1 % of 6000
    for s, d, bad in zip(bt.strings, bt.directions, bt.invalid):
        try:
            bytes(s).decode("utf-8") if d == 0 else np.asarray(s, np.uint16).tobytes().decode("utf-16-le")
            ok = True
        except UnicodeDecodeError:
            ok = False
        assert ok != bad
    idx, data, off = bt.pack(1)
    assert off[-1] == data.size and len(idx) == len(off) - 1


def test_serve_workload_recipe():
    sw = W.serve_workload(4, 4000, max_bytes=1 * MiB, text_bytes=2 * MiB)
    b = sw.input_bytes()
    assert b.min() >= 32 and b.max() <= MiB
    logs = np.log(np.maximum(b, 1))
    mid = (np.log(64) + np.log(MiB)) / 2
    assert abs(np.median(logs) - mid) < 0.3               # log-uniform sizes
    assert abs(np.mean(sw.direction) - 0.5) < 0.03
    assert abs(np.mean(sw.validate_only) - 0.2) < 0.03
    assert 15 <= sw.invalid.sum() <= 70                   # 1 % of 4000
    assert abs(np.mean(sw.gaps) - 1.0) < 0.06             # exponential gaps of mean 1
    for i in range(0, 4000, 97):
        if sw.source[i] >= 0:
            t = sw.texts[sw.source[i]]
            piece = t[sw.offset[i]:sw.offset[i] + sw.units[i]]
        else:
            piece = sw.payloads[-1 - sw.source[i]]
        try:
            bytes(piece).decode("utf-8") if sw.direction[i] == 0 else piece.tobytes().decode("utf-16-le")
            ok = True
        except UnicodeDecodeError:
            ok = False
        assert ok != bool(sw.invalid[i]), i
