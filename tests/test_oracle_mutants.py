"""Planted mistakes in the oracle, each caught by its pins.

Each case copies oracle/oracle.c with one plausible mistake: a bound off by one
(among them the paper's own "less than -65" continuation test, read as
excluding 0xBF), a dropped term, a wrong shift or mask, transposed constants,
a wrong error class, offset or count.  The copy is built with gcc into a
temporary library, loaded in place of the oracle's library, and the pins of
test_oracle_pins.py run on it, fastest first, until one fails.  Every mistake
must make some pin fail.  The unmodified source, built and loaded the same
way, must pass them all, which shows that the harness itself does not fail
the pins.  No mistake reads or writes outside the buffers the wrappers pass.
"""
import importlib.util
import os
import subprocess

import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(os.path.dirname(HERE), "oracle", "oracle.c")

# (what the mistake is, text in oracle.c, the text that replaces it)
MISTAKES = [
    ("continuation test excludes 0xBF", "return b >= 0x80 && b <= 0xBF; }", "return b >= 0x80 && b < 0xBF; }"),
    ("stray-continuation bound off by one", "if (b <= 0xBF)                  /* 10xxxxxx",
     "if (b < 0xBF)                  /* 10xxxxxx"),
    ("five-leading-ones bound off by one", "if (b >= 0xF8)                  /* five",
     "if (b > 0xF8)                  /* five"),
    ("two-byte lead payload mask", "v = b & 0x1F;", "v = b & 0x0F;"),
    ("three-byte lead payload mask", "v = b & 0x0F;", "v = b & 0x07;"),
    ("four-byte lead payload mask", "v = b & 0x07;", "v = b & 0x03;"),
    ("continuation payload shift", "v = (v << 6) | (uint32_t)(in[p + k] & 0x3F);",
     "v = (v << 5) | (uint32_t)(in[p + k] & 0x3F);"),
    ("continuation payload mask", "v = (v << 6) | (uint32_t)(in[p + k] & 0x3F);",
     "v = (v << 6) | (uint32_t)(in[p + k] & 0x1F);"),
    ("two-byte overlong bound", "(L == 2 && v <= 0x7F)", "(L == 2 && v < 0x7F)"),
    ("three-byte overlong bound", "(L == 3 && v <= 0x7FF)", "(L == 3 && v < 0x7FF)"),
    ("four-byte overlong bound", "(L == 4 && v <= 0xFFFF)", "(L == 4 && v < 0xFFFF)"),
    ("too-large bound", "if (v > 0x10FFFF)\n        return ORC_TOO_LARGE;",
     "if (v >= 0x10FFFF)\n        return ORC_TOO_LARGE;"),
    ("encoded-surrogate range", "if (v >= 0xD800 && v <= 0xDFFF)\n        return ORC_SURROGATE;",
     "if (v >= 0xD800 && v < 0xDFFF)\n        return ORC_SURROGATE;"),
    ("class of a stray continuation byte", "return ORC_TOO_LONG;", "return ORC_TOO_SHORT;"),
    ("class of a missing continuation byte", "            return ORC_TOO_SHORT;\n    }",
     "            return ORC_TOO_LONG;\n    }"),
    ("class of an overlong form", "return ORC_OVERLONG;", "return ORC_TOO_LARGE;"),
    ("UTF-8 length: two/three-byte bound", "if (cp <= 0x7FF) return 2;", "if (cp < 0x7FF) return 2;"),
    ("UTF-8 length: three/four-byte bound", "if (cp <= 0xFFFF) return 3;", "if (cp < 0xFFFF) return 3;"),
    ("surrogate split: 0x10000 not subtracted", "uint32_t x = cp - 0x10000;", "uint32_t x = cp;"),
    ("surrogate split: high-unit shift", "(0xD800 | (x >> 10))", "(0xD800 | (x >> 11))"),
    ("surrogate split: low-unit mask", "(0xDC00 | (x & 0x3FF))", "(0xDC00 | (x & 0x1FF))"),
    ("UTF-16 writer: U+10000 as one unit", "if (cp < 0x10000) {\n        out[0] = (uint16_t)cp;",
     "if (cp <= 0x10000) {\n        out[0] = (uint16_t)cp;"),
    ("UTF-8 writer: continuation mask", "out[k] = (uint8_t)(0x80 | (cp & 0x3F));",
     "out[k] = (uint8_t)(0x80 | (cp & 0x7F));"),
    ("UTF-8 writer: lead prefixes transposed", "{0, 0, 0xC0, 0xE0, 0xF0}", "{0, 0, 0xC0, 0xF0, 0xE0}"),
    ("UTF-8 writer: payload shift", "cp >>= 6;", "cp >>= 5;"),
    ("UTF-8 -> UTF-16 error offset one past the start",
     "r->error = e;\n            r->position = p;\n            r->written = q;",
     "r->error = e;\n            r->position = p + 1;\n            r->written = q;"),
    ("UTF-8 -> UTF-16 written count on error",
     "r->error = e;\n            r->position = p;\n            r->written = q;",
     "r->error = e;\n            r->position = p;\n            r->written = q + 1;"),
    ("UTF-16 output capacity off by one", "if (q + (uint64_t)units > cap)", "if (q + (uint64_t)units >= cap)"),
    ("UTF-8 output capacity off by one", "if (q + (uint64_t)bytes > cap)", "if (q + (uint64_t)bytes >= cap)"),
    ("pair: low unit's upper bound dropped", "in[i + 1] >= 0xDC00 && in[i + 1] <= 0xDFFF)", "in[i + 1] >= 0xDC00)"),
    ("pair: 0x10000 not added", "*cp = ((hi10 << 10) | lo10) + 0x10000;", "*cp = ((hi10 << 10) | lo10);"),
    ("UTF-16: 0xDFFF outside the surrogates", "if (u < 0xD800 || u > 0xDFFF) {",
     "if (u < 0xD800 || u >= 0xDFFF) {"),
    ("UTF-16: a low unit opens a pair", "if (u <= 0xDBFF && i + 1 < n", "if (u <= 0xDFFF && i + 1 < n"),
    ("UTF-16 -> UTF-8 error offset one past the unit",
     "r->error = e;\n            r->position = i;\n            r->written = q;",
     "r->error = e;\n            r->position = i + 1;\n            r->written = q;"),
    ("UTF-16 length of UTF-8: four-byte lead bound", "if (b >= 0xF0) total += 1;", "if (b > 0xF0) total += 1;"),
    ("UTF-16 length of UTF-8: continuation test", "if (!is_continuation(b)) total += 1;",
     "if (b != 0x80) total += 1;"),
    ("UTF-8 length of UTF-16: surrogate units", "else if (u >= 0xD800 && u <= 0xDFFF) total += 2;",
     "else if (u >= 0xD800 && u <= 0xDFFF) total += 3;"),
    ("UTF-8 length of UTF-16: two/three-byte bound", "else if (u <= 0x7FF) total += 2;",
     "else if (u < 0x7FF) total += 2;"),
    ("UTF-8 validation offset one past the start",
     "r->error = e;\n            r->position = p;\n            return;",
     "r->error = e;\n            r->position = p + 1;\n            return;"),
    ("UTF-16 validation offset one past the unit",
     "r->error = e;\n            r->position = i;\n            return;",
     "r->error = e;\n            r->position = i + 1;\n            return;"),
]

# pins known to take seconds run last
SLOW = ("test_every_short_utf8_string[3]", "test_every_four_byte_string_with_a_four_byte_lead")


def _pins_module():
    spec = importlib.util.spec_from_file_location("_oracle_pins_for_mutants", os.path.join(HERE, "test_oracle_pins.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def pin_calls():
    """Every pin of test_oracle_pins.py with its parameters, fastest first."""
    mod = _pins_module()
    calls = []
    for name in sorted(n for n in dir(mod) if n.startswith("test_")):
        fn = getattr(mod, name)
        marks = [m for m in getattr(fn, "pytestmark", []) if m.name == "parametrize"]
        if not marks:
            calls.append((name, fn, {}))
            continue
        assert len(marks) == 1, name
        argnames, argvalues = marks[0].args[:2]
        names = [a.strip() for a in argnames.split(",")] if isinstance(argnames, str) else list(argnames)
        for k, vals in enumerate(argvalues):
            vals = tuple(vals) if len(names) > 1 else (vals,)
            label = f"{name}[{vals[0]}]" if name == "test_every_short_utf8_string" else f"{name}[{k}]"
            calls.append((label, fn, dict(zip(names, vals))))
    calls.sort(key=lambda c: c[0] in SLOW)
    return calls


@pytest.fixture(scope="module")
def pins():
    return pin_calls()


def build_variant(tmp_path, text, tag):
    src = tmp_path / f"oracle_{tag}.c"
    lib = tmp_path / f"liboracle_{tag}.so"
    src.write_text(text)
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", str(lib), str(src)])
    return str(lib)


def first_failing_pin(monkeypatch, lib_path, pins):
    """Loads the library at lib_path in place of the oracle's and runs the
    pins; returns the first one that fails, or None."""
    monkeypatch.setattr(oracle, "_lib", None)
    monkeypatch.setattr(oracle, "build", lambda force=False: lib_path)
    for label, fn, kw in pins:
        try:
            fn(**kw)
        except AssertionError:
            return label
        except (IndexError, ValueError, KeyError, OverflowError) as e:   # inconsistent results break a pin too
            return f"{label} ({type(e).__name__})"
    return None


def test_unmodified_source_passes_every_pin(tmp_path, monkeypatch, pins):
    lib = build_variant(tmp_path, open(SRC).read(), "same")
    assert first_failing_pin(monkeypatch, lib, pins) is None
    assert len(pins) >= 30


@pytest.mark.parametrize("what,old,new", MISTAKES, ids=[m[0] for m in MISTAKES])
def test_planted_mistake_fails_a_pin(tmp_path, monkeypatch, pins, what, old, new):
    text = open(SRC).read()
    assert text.count(old) == 1, f"the text to change is not unique in oracle.c: {old!r}"
    lib = build_variant(tmp_path, text.replace(old, new), "mut")
    caught = first_failing_pin(monkeypatch, lib, pins)
    assert caught is not None, f"no pin fails with the mistake: {what}"
