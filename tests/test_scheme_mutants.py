"""Planted mistakes in the kernels' own headers, each caught by the host proofs.

The CUDA path's per-byte and per-unit arithmetic lives in headers that also
compile for the host (utf8_scheme.h, utf8_tables.h, utf16_scheme.h), where
the proofs in test_scheme_proof.py, test_utf8_decode_proof.py,
test_u16_scheme_proof.py and test_u16_encode_proof.py check it against the
oracle.  Each case here copies the headers, plants one plausible mistake in
the copy (a shift or mask one off, a dropped flag, a range bound off by one,
transposed constants, a table bit flipped, the fix-up's back-up removed), builds
the proofs' checkers against the copy and runs the proofs, fastest first,
until one fails: every mistake must make some proof fail.  The unmodified
copy, built the same way, passes them all.
"""
import importlib.util
import inspect
import os
import shutil

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2109_10433_gb300", "csrc")
HEADERS = ("utf8_scheme.h", "utf8_tables.h", "utf16_scheme.h")
PROOFS = ("test_utf8_decode_proof", "test_u16_scheme_proof", "test_u16_encode_proof", "test_scheme_proof")
# proofs known to take seconds run after the others
SLOW = ("test_every_short_string[3]", "test_five_byte_strings", "test_four_byte_strings[3]",
        "test_every_boundary_combination_at_the_ends[0]", "test_every_boundary_combination_around_a_group_boundary",
        "test_corrupted_synthetic_text")

# (what the mistake is, header, text in it, the text that replaces it)
MISTAKES = [
    ("UTF-16 counts: U+0800 bound of the gathered high bytes", "utf16_scheme.h",
     "const uint32_t ge08 = (((H & 0x78787878u) + 0x78787878u) | H) & 0x80808080u;   /* >= U+0800 */",
     "const uint32_t ge08 = (((H & 0x70707070u) + 0x70707070u) | H) & 0x80808080u;   /* >= U+0800 */"),
    ("UTF-16 counts: surrogate mask", "utf16_scheme.h",
     "const uint32_t sur = gputf_zero_bytes((H & 0xF8F8F8F8u) ^ 0xD8D8D8D8u);        /* D800-DFFF */",
     "const uint32_t sur = gputf_zero_bytes((H & 0xFCFCFCFCu) ^ 0xD8D8D8D8u);        /* D800-DFFF */"),
    ("UTF-16 counts: low-surrogate bit shift", "utf16_scheme.h",
     "const uint32_t t = H << 5;   /* bit 2", "const uint32_t t = H << 6;   /* bit 2"),
    ("UTF-16 counts: previous-unit permute", "utf16_scheme.h",
     "const uint32_t ph = gputf_bperm(*hprev, *hi, 0x6543);", "const uint32_t ph = gputf_bperm(*hprev, *hi, 0x5432);"),
    ("UTF-16 counts: N flag drops the pair test", "utf16_scheme.h",
     "*N = ~(*lo & ph) & 0x80808080u;", "*N = ~(*lo) & 0x80808080u;"),
    ("UTF-16 counts: A flag drops N", "utf16_scheme.h",
     "*A = ~(hz & ~Lo) & ~*c3 & *N;", "*A = ~(hz & ~Lo) & ~*c3;"),
    ("UTF-16 counts: next-unit shift", "utf16_scheme.h",
     "const uint32_t nl = gputf_fshr(lo, next_lo, 8);", "const uint32_t nl = gputf_fshr(lo, next_lo, 16);"),
    ("UTF-16 counts: B weighs one", "utf16_scheme.h",
     "return (N >> 7) + (A >> 7) + (B >> 6);", "return (N >> 7) + (A >> 7) + (B >> 7);"),
    ("UTF-8 bytes: lead prefixes transposed (front to back)", "utf16_scheme.h",
     "gputf_fshr(0xF0E0C000u, 0u, 8 * l - 8)", "gputf_fshr(0xE0F0C000u, 0u, 8 * l - 8)"),
    ("UTF-8 bytes: lead prefixes transposed (back to front)", "utf16_scheme.h",
     "gputf_bperm(0xE0C00000u, 0xF0u, l)", "gputf_bperm(0xC0E00000u, 0xF0u, l)"),
    ("UTF-8 bytes: second group shift", "utf16_scheme.h",
     "    *b2 = ((y >> 6) & 0x3F) | 0x80;\n    *b3 = ((y >> 12) & 0x3F) | 0x80;",
     "    *b2 = ((y >> 5) & 0x3F) | 0x80;\n    *b3 = ((y >> 12) & 0x3F) | 0x80;"),
    ("UTF-16 pairing at the run's end: flag bit", "utf16_scheme.h",
     "return (hprev >> 31) ^ (gputf_is_low(nu) ? 1u : 0u);", "return (hprev >> 30) ^ (gputf_is_low(nu) ? 1u : 0u);"),
    ("UTF-16 validate pass: pairing against the wrong flag", "utf16_scheme.h",
     "const uint32_t bad = gputf_bperm(*hprev, hi, 0x6543) ^ lo;",
     "const uint32_t bad = gputf_bperm(*hprev, hi, 0x6543) ^ hi;"),
    ("UTF-8 length pass: three-byte units weigh two more", "utf16_scheme.h",
     "return (ge80 >> 7) + (c3 >> 7);", "return (ge80 >> 7) + (c3 >> 6);"),
    ("UTF-8 check: three-back lead shift", "utf8_scheme.h",
     "gputf_fshl(st->f0, c.f0, 24)", "gputf_fshl(st->f0, c.f0, 16)"),
    ("UTF-8 check: 0xE0 mask is 0xC0", "utf8_scheme.h",
     "s.e0 = w & (w << 1) & (w << 2);", "s.e0 = w & (w << 1);"),
    ("UTF-8 check: 0xF0 mask is 0xE8", "utf8_scheme.h",
     "s.f0 = s.e0 & (w << 3);", "s.f0 = s.e0 & (w << 4);"),
    ("UTF-8 check: previous-byte funnel shift", "utf8_scheme.h",
     "const uint32_t prev1 = gputf_fshl(st->w, w, 8);", "const uint32_t prev1 = gputf_fshl(st->w, w, 16);"),
    ("UTF-8 check: low-nibble mask shift", "utf8_scheme.h",
     "gputf_prmt(prev1 << 4, 0, 0xBA98)", "gputf_prmt(prev1 << 3, 0, 0xBA98)"),
    ("UTF-8 fix-up: C1 not overlong", "utf8_scheme.h",
     "if (L == 2 && b < 0xC2) return GPUTF_E_OVERLONG;", "if (L == 2 && b < 0xC1) return GPUTF_E_OVERLONG;"),
    ("UTF-8 fix-up: E0 overlong bound", "utf8_scheme.h", "b == 0xE0 && b1 < 0xA0", "b == 0xE0 && b1 < 0x9F"),
    ("UTF-8 fix-up: ED surrogate bound", "utf8_scheme.h", "b == 0xED && b1 >= 0xA0", "b == 0xED && b1 > 0xA0"),
    ("UTF-8 fix-up: F0 overlong bound", "utf8_scheme.h", "b == 0xF0 && b1 < 0x90", "b == 0xF0 && b1 < 0x8F"),
    ("UTF-8 fix-up: F4 too-large bound", "utf8_scheme.h", "(b == 0xF4 && b1 >= 0x90)", "(b == 0xF4 && b1 > 0x90)"),
    ("UTF-8 fix-up: no back-up over continuation bytes", "utf8_scheme.h",
     "for (int k = 0; k < 4 && q > 0 && (in[q] & 0xC0) == 0x80; k++) q--;",
     "for (int k = 0; k < 0 && q > 0 && (in[q] & 0xC0) == 0x80; k++) q--;"),
    ("UTF-8 decode: sequence length from the leading ones", "utf8_scheme.h",
     "const uint32_t n = clo > 1 ? clo : 1u;", "const uint32_t n = clo > 2 ? clo : 1u;"),
    ("UTF-8 decode: prefix mask", "utf8_scheme.h", "& 0x7F3F3F3Fu;", "& 0x7F7F3F3Fu;"),
    ("UTF-8 decode: 0x10000 not subtracted", "utf8_scheme.h",
     "const uint32_t x = code - 0x10000u;", "const uint32_t x = code;"),
    ("UTF-8 decode: low-surrogate mask", "utf8_scheme.h",
     "*u1 = 0xDC00u | (x & 0x3FFu);", "*u1 = 0xDC00u | (x & 0x1FFu);"),
    ("UTF-8 decode: three-byte characters as pairs", "utf8_scheme.h",
     "const int pair = n >= 4;", "const int pair = n >= 3;"),
    ("UTF-8 tables: T2 loses C0's overlong bit", "utf8_tables.h",
     "#define GPUTF_T2_W0 0x838387AFu", "#define GPUTF_T2_W0 0x838387ABu"),
    ("UTF-8 tables: T3 gains a too-short bit", "utf8_tables.h",
     "#define GPUTF_T3_W2 0xD6D6CEAEu", "#define GPUTF_T3_W2 0xD6D6CEAFu"),
    ("UTF-8 tables: T1 loses a too-short bit", "utf8_tables.h",
     "#define GPUTF_T1_W3 0x61190105u", "#define GPUTF_T1_W3 0x61190104u"),
]


def _module(name):
    spec = importlib.util.spec_from_file_location(f"_mut_{name}", os.path.join(HERE, name + ".py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.fixture(scope="module")
def proofs():
    """(proof module, its tests with parameters, fastest first) for each proof."""
    out = []
    for name in PROOFS:
        mod = _module(name)
        calls = []
        for tname in sorted(n for n in dir(mod) if n.startswith("test_")):
            fn = getattr(mod, tname)
            fixture = list(inspect.signature(fn).parameters)[0]
            marks = [m for m in getattr(fn, "pytestmark", []) if m.name == "parametrize"]
            if not marks:
                calls.append((tname, fn, fixture, {}))
                continue
            assert len(marks) == 1, tname
            argnames, argvalues = marks[0].args[:2]
            names = [a.strip() for a in argnames.split(",")] if isinstance(argnames, str) else list(argnames)
            for k, vals in enumerate(argvalues):
                vals = tuple(vals) if len(names) > 1 else (vals,)
                label = f"{tname}[{vals[0]}]" if tname in ("test_every_short_string", "test_four_byte_strings") \
                    else f"{tname}[{k}]" if len(argvalues) > 1 else tname
                calls.append((label, fn, fixture, dict(zip(names, vals))))
        calls.sort(key=lambda c: c[0] in SLOW)
        out.append((mod, calls))
    return out


def header_copy(tmp_path, header=None, old=None, new=None):
    d = tmp_path / "csrc"
    d.mkdir()
    for h in HEADERS:
        shutil.copy(os.path.join(CSRC, h), d / h)
    if header is not None:
        text = (d / header).read_text()
        assert text.count(old) == 1, f"the text to change is not unique in {header}: {old!r}"
        (d / header).write_text(text.replace(old, new))
    return str(d)


def first_failing_proof(tmp_path, csrc, proofs, stop_at_first=True):
    failed = []
    for k, (mod, calls) in enumerate(proofs):
        out = tmp_path / f"build{k}"
        out.mkdir()
        checker = mod.build_checker(out, csrc=csrc)
        for label, fn, fixture, kw in calls:
            try:
                fn(**{fixture: checker}, **kw)
            except AssertionError:
                failed.append(f"{mod.__name__[5:]}::{label}")
                if stop_at_first:
                    return failed
    return failed


def test_unmodified_headers_pass_every_proof(tmp_path, proofs):
    assert first_failing_proof(tmp_path, header_copy(tmp_path), proofs, stop_at_first=False) == []
    assert sum(len(c) for _, c in proofs) >= 20


@pytest.mark.parametrize("what,header,old,new", MISTAKES, ids=[m[0] for m in MISTAKES])
def test_planted_mistake_fails_a_proof(tmp_path, proofs, what, header, old, new):
    by = {mod.__name__[5:]: entry for entry in proofs for mod in entry[:1]}
    names = (("test_u16_scheme_proof", "test_u16_encode_proof") if header == "utf16_scheme.h" else
             ("test_utf8_decode_proof", "test_scheme_proof", "test_u16_scheme_proof", "test_u16_encode_proof"))
    order = [by[n] for n in names]
    failed = first_failing_proof(tmp_path, header_copy(tmp_path, header, old, new), order)
    assert failed, f"no proof fails with the mistake: {what}"
