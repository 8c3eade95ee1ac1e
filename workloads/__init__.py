"""Seeded synthetic workloads for the UTF-8 <-> UTF-16LE transcoding path.

This module draws code points and error tokens and nothing else: turning code
points into UTF-8 / UTF-16LE bytes is delegated to CPython's own codecs
(``str.encode``), so the module holds none of the transcoding arithmetic and
serves both the CUDA path and the oracle as plain input.

The paper measures on lipsum and Wikipedia-Mars text files (Section 6, Table
3) that are not available here; the mixes below stand in for them by their
per-class character fractions: ASCII-heavy text, 2-byte scripts (Cyrillic,
Arabic), 3-byte scripts (CJK) and 4-byte emoji.

Random numbers come from NumPy's PCG64 generator seeded with the workload's
seed.  Each character class carries its UTF-8 byte length and UTF-16 unit
count (Table 2 of the paper) as part of its definition, which is what lets a
buffer be cut at a character boundary to an exact size.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

KiB = 1 << 10
MiB = 1 << 20


@dataclass(frozen=True)
class CharClass:
    """Code points drawn uniformly from [lo, hi], skipping D800-DFFF."""
    lo: int
    hi: int
    utf8_len: int
    utf16_len: int

    def size(self) -> int:
        n = self.hi - self.lo + 1
        if self.lo <= 0xD800 and self.hi >= 0xDFFF:
            n -= 0x800
        return n

    def draw(self, rng: np.random.Generator, count: int) -> np.ndarray:
        r = rng.integers(0, self.size(), size=count, dtype=np.int64) + self.lo
        if self.lo <= 0xD800 and self.hi >= 0xDFFF:
            r = np.where(r >= 0xD800, r + 0x800, r)
        return r.astype(np.uint32)


PRINTABLE = CharClass(0x20, 0x7E, 1, 1)
ASCII = CharClass(0x00, 0x7F, 1, 1)
CYRILLIC = CharClass(0x400, 0x4FF, 2, 1)
CYRILLIC_ARABIC = CharClass(0x400, 0x6FF, 2, 1)
CJK = CharClass(0x4E00, 0x9FFF, 3, 1)
BMP3 = CharClass(0x800, 0xFFFF, 3, 1)            # surrogates skipped
EMOJI = CharClass(0x1F300, 0x1FAFF, 4, 2)
SUPPLEMENTARY = CharClass(0x10000, 0x10FFFF, 4, 2)


@dataclass(frozen=True)
class Mix:
    classes: tuple
    probs: tuple

    def cum(self) -> np.ndarray:
        c = np.cumsum(np.asarray(self.probs, dtype=np.float64))
        c[-1] = 1.0
        return c


# The single-buffer mixes of the benchmark configurations.
MIX_LATIN_CYRILLIC = Mix((PRINTABLE, CYRILLIC), (0.9, 0.1))               # 1 MiB UTF-8
MIX_CJK_EMOJI = Mix((PRINTABLE, CJK, EMOJI), (0.2, 0.7, 0.1))             # 256 MiB UTF-16
MIX_FOUR_BYTE_HEAVY = Mix((SUPPLEMENTARY, BMP3, ASCII), (0.4, 0.3, 0.3))  # 64 MiB UTF-8
# The per-string scripts of the batched and served configurations.
SCRIPT_ASCII = Mix((PRINTABLE,), (1.0,))
SCRIPT_TWO_BYTE = Mix((CYRILLIC_ARABIC,), (1.0,))
SCRIPT_CJK = Mix((CJK,), (1.0,))
SCRIPT_MIXED = Mix((PRINTABLE, CYRILLIC_ARABIC, CJK, EMOJI),
                   (0.95 / 3, 0.95 / 3, 0.95 / 3, 0.05))
SCRIPTS = (SCRIPT_ASCII, SCRIPT_TWO_BYTE, SCRIPT_CJK, SCRIPT_MIXED)


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def draw_chars(rng: np.random.Generator, mix: Mix, budget: int, unit: str,
               with_sizes: bool = False):
    """Code points whose encoded size ('utf8' bytes or 'utf16' units) is exactly
    `budget`: characters of the mix while they fit, then printable ASCII.
    With `with_sizes`, also returns each character's size from its class."""
    lens = np.array([c.utf8_len if unit == "utf8" else c.utf16_len for c in mix.classes])
    mean = float(np.dot(lens, mix.probs))
    cum = mix.cum()
    cats = np.zeros(0, dtype=np.int64)
    while True:
        extra = int(budget / mean * 1.02) + 64 - cats.size
        cats = np.concatenate([cats, np.searchsorted(cum, rng.random(max(extra, 64)), side="right")])
        sizes = np.cumsum(lens[cats])
        if sizes[-1] > budget or budget == 0:
            break
    k = int(np.searchsorted(sizes, budget, side="right"))   # characters that fit
    cats = cats[:k]
    used = int(sizes[k - 1]) if k else 0
    cps = np.empty(k, dtype=np.uint32)
    for ci, cls in enumerate(mix.classes):
        sel = np.nonzero(cats == ci)[0]
        cps[sel] = cls.draw(rng, sel.size)
    fill = PRINTABLE.draw(rng, budget - used)
    out = np.concatenate([cps, fill])
    if with_sizes:
        return out, np.concatenate([lens[cats], np.ones(budget - used, dtype=lens.dtype)])
    return out


def to_utf8(cps: np.ndarray) -> np.ndarray:
    s = np.ascontiguousarray(cps, dtype="<u4").tobytes().decode("utf-32-le")
    return np.frombuffer(s.encode("utf-8"), dtype=np.uint8)


def to_utf16(cps: np.ndarray) -> np.ndarray:
    s = np.ascontiguousarray(cps, dtype="<u4").tobytes().decode("utf-32-le")
    return np.frombuffer(s.encode("utf-16-le"), dtype="<u2")


def utf8_text(seed: int, nbytes: int, mix: Mix) -> np.ndarray:
    """Valid UTF-8 of exactly `nbytes` bytes."""
    out = to_utf8(draw_chars(rng_for(seed), mix, nbytes, "utf8"))
    assert out.size == nbytes
    return out


def utf16_text(seed: int, nunits: int, mix: Mix) -> np.ndarray:
    """Valid UTF-16LE of exactly `nunits` 16-bit units."""
    out = to_utf16(draw_chars(rng_for(seed), mix, nunits, "utf16"))
    assert out.size == nunits
    return out


# ---------------------------------------------------------------------------
# Error tokens.  Each token is a byte (or unit) sequence that, placed at a
# character boundary and followed by a character boundary, makes the first
# invalid character start at the token, with the class given by its label.
# Class numbers are those of the library interface.
# ---------------------------------------------------------------------------
HEADER_BITS, TOO_SHORT, TOO_LONG, OVERLONG, TOO_LARGE, SURROGATE = 1, 2, 3, 4, 5, 6

UTF8_TOKEN_KINDS = ("overlong", "surrogate", "too_large", "truncated", "stray")


def _cont(rng, lo=0x80, hi=0xBF) -> int:
    return int(rng.integers(lo, hi + 1))


def utf8_error_token(rng: np.random.Generator, kind: str) -> tuple[bytes, int]:
    if kind == "overlong":
        form = int(rng.integers(0, 3))
        if form == 0:      # two-byte lead C0/C1
            return bytes([int(rng.integers(0xC0, 0xC2)), _cont(rng)]), OVERLONG
        if form == 1:      # E0 then 80..9F
            return bytes([0xE0, _cont(rng, 0x80, 0x9F), _cont(rng)]), OVERLONG
        return bytes([0xF0, _cont(rng, 0x80, 0x8F), _cont(rng), _cont(rng)]), OVERLONG
    if kind == "surrogate":  # ED A0..BF xx encodes D800..DFFF
        return bytes([0xED, _cont(rng, 0xA0, 0xBF), _cont(rng)]), SURROGATE
    if kind == "too_large":
        if rng.integers(0, 2) == 0:   # F4 90..BF xx xx is above U+10FFFF
            return bytes([0xF4, _cont(rng, 0x90, 0xBF), _cont(rng), _cont(rng)]), TOO_LARGE
        return bytes([int(rng.integers(0xF5, 0xF8)), _cont(rng), _cont(rng), _cont(rng)]), TOO_LARGE
    if kind == "truncated":  # a multi-byte character missing its last byte
        cls = (CYRILLIC, CJK, SUPPLEMENTARY)[int(rng.integers(0, 3))]
        full = to_utf8(cls.draw(rng, 1)).tobytes()
        return full[:-1], TOO_SHORT
    if kind == "stray":
        return bytes([_cont(rng)]), TOO_LONG
    if kind == "header":
        return bytes([int(rng.integers(0xF8, 0x100))]), HEADER_BITS
    raise ValueError(kind)


def utf16_error_token(rng: np.random.Generator) -> tuple[list[int], int]:
    form = int(rng.integers(0, 3))
    if form == 0:   # lone high surrogate
        return [int(rng.integers(0xD800, 0xDC00))], SURROGATE
    if form == 1:   # lone low surrogate
        return [int(rng.integers(0xDC00, 0xE000))], SURROGATE
    # a pair in the wrong order: the low unit comes first and is the error
    return [int(rng.integers(0xDC00, 0xE000)), int(rng.integers(0xD800, 0xDC00))], SURROGATE


@dataclass
class ErrorText:
    data: np.ndarray                 # uint8 (UTF-8) or uint16 (UTF-16)
    tokens: list = field(default_factory=list)   # (offset, length, class)

    def repaired_before(self, k: int) -> np.ndarray:
        """A copy with tokens 0..k-1 overwritten by printable ASCII of the same
        length, so that token k holds the first error."""
        d = self.data.copy()
        for off, ln, _ in self.tokens[:k]:
            d[off:off + ln] = 0x41
        return d


def utf8_error_text(seed: int, nbytes: int, mix: Mix, mean_gap: int,
                    kinds=UTF8_TOKEN_KINDS) -> ErrorText:
    """UTF-8 of exactly `nbytes` bytes with error tokens at character
    boundaries, spaced by exponential gaps of mean `mean_gap` bytes."""
    rng = rng_for(seed)
    targets = []
    pos = 0.0
    while True:
        pos += rng.exponential(mean_gap)
        if pos >= nbytes - 8:
            break
        targets.append(int(pos))
    toks = [utf8_error_token(rng, kinds[int(rng.integers(0, len(kinds)))]) for _ in targets]
    tok_bytes = sum(len(t[0]) for t in toks)
    cps, lens = draw_chars(rng, mix, nbytes - tok_bytes, "utf8", with_sizes=True)
    # character start offsets of the clean text (from the per-class lengths)
    starts = np.concatenate([[0], np.cumsum(lens)])
    pieces, tokens = [], []
    prev_char, shift = 0, 0
    for t, (tb, cls) in zip(targets, toks):
        j = int(np.searchsorted(starts, max(t - shift, 0), side="left"))
        j = max(j, prev_char)
        pieces.append(to_utf8(cps[prev_char:j]).tobytes())
        off = int(starts[j]) + shift
        tokens.append((off, len(tb), cls))
        pieces.append(tb)
        shift += len(tb)
        prev_char = j
    pieces.append(to_utf8(cps[prev_char:]).tobytes())
    data = np.frombuffer(b"".join(pieces), dtype=np.uint8).copy()
    assert data.size == nbytes
    return ErrorText(data, tokens)


# ---------------------------------------------------------------------------
# Batched strings: many strings of uneven lengths, given as CSR offsets.
# ---------------------------------------------------------------------------
@dataclass
class StringBatch:
    directions: np.ndarray           # int8: 0 = UTF-8 -> UTF-16, 1 = UTF-16 -> UTF-8
    strings: list                    # np.uint8 or np.uint16 arrays
    invalid: np.ndarray              # bool: an error token was placed in the string

    def pack(self, direction: int):
        """Concatenated input of one direction and its CSR offsets (code units)."""
        idx = np.nonzero(self.directions == direction)[0]
        dtype = np.uint8 if direction == 0 else np.uint16
        parts = [self.strings[i] for i in idx]
        sizes = np.array([p.size for p in parts], dtype=np.uint64)
        offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
        data = np.concatenate(parts).astype(dtype) if parts else np.zeros(0, dtype)
        return idx, data, offsets


def string_batch(seed: int, n_strings: int, median_bytes: int = KiB, sigma: float = 1.0,
                 min_bytes: int = 16, max_bytes: int = 64 * KiB,
                 invalid_frac: float = 0.01) -> StringBatch:
    """Strings with log-normal byte lengths (clipped), a script drawn per
    string, a fair-coin direction and a fraction with one error token."""
    rng = rng_for(seed)
    lengths = np.clip(np.exp(rng.normal(np.log(median_bytes), sigma, n_strings)),
                      min_bytes, max_bytes).astype(np.int64)
    scripts = rng.integers(0, len(SCRIPTS), n_strings)
    directions = rng.integers(0, 2, n_strings).astype(np.int8)
    invalid = rng.random(n_strings) < invalid_frac
    strings = []
    for i in range(n_strings):
        mix = SCRIPTS[int(scripts[i])]
        if directions[i] == 0:
            cps = draw_chars(rng, mix, int(lengths[i]), "utf8")
            s = to_utf8(cps)
            if invalid[i]:
                s = _insert_utf8_token(rng, cps, s)
        else:
            cps = draw_chars(rng, mix, int(lengths[i]) // 2, "utf16")
            s = to_utf16(cps)
            if invalid[i]:
                s = _insert_utf16_token(rng, cps, s)
        strings.append(s)
    return StringBatch(directions, strings, invalid)


def _insert_utf8_token(rng, cps, s):
    j = int(rng.integers(0, cps.size + 1))
    tb, _ = utf8_error_token(rng, UTF8_TOKEN_KINDS[int(rng.integers(0, len(UTF8_TOKEN_KINDS)))])
    head = to_utf8(cps[:j]).tobytes()
    return np.frombuffer(head + tb + s.tobytes()[len(head):], dtype=np.uint8).copy()


def _insert_utf16_token(rng, cps, s):
    j = int(rng.integers(0, cps.size + 1))
    tu, _ = utf16_error_token(rng)
    head = to_utf16(cps[:j])
    return np.concatenate([head, np.array(tu, dtype=np.uint16), s[head.size:]]).astype(np.uint16)


# ---------------------------------------------------------------------------
# The benchmark configurations, by what they are.
# ---------------------------------------------------------------------------
def latin_cyrillic_utf8_1mib(seed: int = 0) -> np.ndarray:
    """1 MiB of UTF-8: 90% U+0020-007E, 10% U+0400-04FF."""
    return utf8_text(seed, MiB, MIX_LATIN_CYRILLIC)


def cjk_emoji_utf16_256mib(seed: int = 1, nbytes: int = 256 * MiB) -> np.ndarray:
    """256 MiB of UTF-16LE: 20% U+0020-007E, 70% U+4E00-9FFF, 10% U+1F300-1FAFF."""
    return utf16_text(seed, nbytes // 2, MIX_CJK_EMOJI)


def four_byte_heavy_utf8_64mib(seed: int = 2, nbytes: int = 64 * MiB,
                               mean_gap: int = MiB) -> ErrorText:
    """64 MiB of UTF-8: 40% U+10000-10FFFF, 30% U+0800-FFFF (no surrogates),
    30% ASCII, with error tokens about once per MiB."""
    return utf8_error_text(seed, nbytes, MIX_FOUR_BYTE_HEAVY, mean_gap)


# ---------------------------------------------------------------------------
# Served requests: a stream of requests of log-uniform sizes, each a slice of
# a pool text of its script and direction, cut at character boundaries.
# ---------------------------------------------------------------------------
@dataclass
class ServeWorkload:
    texts: list                 # index 2 * script + direction: uint8 (UTF-8) or uint16 (UTF-16) text
    payloads: list              # private inputs of the invalid requests
    direction: np.ndarray       # int8: 0 = UTF-8 -> UTF-16, 1 = UTF-16 -> UTF-8
    validate_only: np.ndarray   # bool: validate without transcoding
    invalid: np.ndarray         # bool: an error token was inserted
    source: np.ndarray          # int64: text index, or -1 - k for payloads[k]
    offset: np.ndarray          # int64: first unit within the text (0 for payloads)
    units: np.ndarray           # int64: input code units
    gaps: np.ndarray            # float64: inter-arrival gaps with mean 1 (exponential)

    def input_bytes(self) -> np.ndarray:
        return self.units * (1 + self.direction.astype(np.int64))


def serve_workload(seed: int, n_requests: int, min_bytes: int = 64, max_bytes: int = 16 * MiB,
                   validate_frac: float = 0.2, invalid_frac: float = 0.01,
                   text_bytes: int = 24 * MiB) -> ServeWorkload:
    """Requests with sizes log-uniform in [min_bytes, max_bytes] input bytes,
    script uniform over SCRIPTS, a fair-coin direction, a fraction validated
    only and a fraction carrying one error token, arriving with exponential
    gaps (a Poisson process once the gaps are scaled by the mean gap)."""
    assert text_bytes >= max_bytes
    rng = rng_for(seed)
    texts, starts = [], []
    for mix in SCRIPTS:
        for direction in (0, 1):
            unit = "utf8" if direction == 0 else "utf16"
            budget = text_bytes if direction == 0 else text_bytes // 2
            cps, lens = draw_chars(rng, mix, budget, unit, with_sizes=True)
            texts.append(to_utf8(cps) if direction == 0 else to_utf16(cps))
            starts.append(np.concatenate([[0], np.cumsum(lens)]).astype(np.int64))
    sizes = np.exp(rng.uniform(np.log(min_bytes), np.log(max_bytes), n_requests)).astype(np.int64)
    scripts = rng.integers(0, len(SCRIPTS), n_requests)
    direction = rng.integers(0, 2, n_requests).astype(np.int8)
    validate_only = rng.random(n_requests) < validate_frac
    invalid = rng.random(n_requests) < invalid_frac
    gaps = rng.exponential(1.0, n_requests)
    source = (2 * scripts + direction).astype(np.int64)
    offset = np.zeros(n_requests, np.int64)
    units = np.zeros(n_requests, np.int64)
    payloads = []
    for i in range(n_requests):
        t = int(source[i])
        st, total = starts[t], texts[t].size
        want = int(sizes[i]) if direction[i] == 0 else int(sizes[i]) // 2
        last = int(np.searchsorted(st, total - want, side="right"))     # starts that leave room
        k = int(rng.integers(0, max(last, 1)))
        a = int(st[k])
        b = int(st[np.searchsorted(st, a + want, side="right") - 1])    # whole characters only
        offset[i], units[i] = a, b - a
        if invalid[i]:
            piece = texts[t][a:b]
            inner = st[k:np.searchsorted(st, b, side="right")] - a     # boundaries inside the slice
            j = int(inner[int(rng.integers(0, inner.size))])
            if direction[i] == 0:
                tok, _ = utf8_error_token(rng, UTF8_TOKEN_KINDS[int(rng.integers(0, len(UTF8_TOKEN_KINDS)))])
                tok = np.frombuffer(tok, dtype=np.uint8)
            else:
                tok = np.array(utf16_error_token(rng)[0], dtype=np.uint16)
            # the token goes in at boundary j; the slice keeps its length
            p = np.concatenate([piece[:j], tok, piece[j:]])[:piece.size].astype(piece.dtype)
            source[i], offset[i] = -1 - len(payloads), 0
            payloads.append(p)
    return ServeWorkload(texts, payloads, direction, validate_only, invalid, source, offset, units, gaps)
