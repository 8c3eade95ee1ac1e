"""Proof, on the host, of the UTF-8 automaton of the validate-only pass.

tests/native/dfa_check.c compiles the CUDA path's own header (utf8_dfa.h)
for the CPU and checks it against the oracle: a run from ACCEPT over a
string and a zero byte rejects exactly the strings the oracle rejects, at a
position within three bytes after the oracle's error position, and the
resynchronising start (three bytes replayed from SYNC0) reaches the same
state as a run from the start at every position after a valid prefix.
Domains: every string of 1, 2 and 3 bytes; every string of 4 bytes over
two bytes from each class (the lowest and highest); strings of 5 and 6
bytes over one byte from each class; and random strings rich in leads and
continuation bytes.
"""
import ctypes
import itertools
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2109_10433_gb300", "csrc")

# the lowest and highest byte of each class of utf8_dfa.h
CLASS_EDGES = [0x00, 0x7F, 0x80, 0x8F, 0x90, 0x9F, 0xA0, 0xBF, 0xC0, 0xC1, 0xF5, 0xFF, 0xC2, 0xDF, 0xE0,
               0xE1, 0xEC, 0xEE, 0xEF, 0xED, 0xF0, 0xF1, 0xF3, 0xF4]
ONE_PER_CLASS = [0x41, 0x85, 0x95, 0xB5, 0xC1, 0xD0, 0xE0, 0xE5, 0xED, 0xF0, 0xF2, 0xF4, 0xF9]


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    out = os.path.join(str(tmp_path_factory.mktemp("dfa")), "dfa_check.so")
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-I" + os.path.join(ROOT, "oracle"),
                           "-I" + CSRC, "-o", out, os.path.join(ROOT, "tests", "native", "dfa_check.c")])
    lib = ctypes.CDLL(out)
    lib.dfa_check_all.restype = ctypes.c_uint64
    lib.dfa_check_all.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_uint64)]
    lib.dfa_check_list.restype = ctypes.c_uint64
    lib.dfa_check_list.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.POINTER(ctypes.c_uint64)]
    return lib


def _list(lib, strings, length):
    buf = np.ascontiguousarray(np.asarray(strings, dtype=np.uint8).reshape(-1, length))
    first = ctypes.c_uint64(0)
    fails = lib.dfa_check_list(buf.ctypes.data, buf.shape[0], length, ctypes.byref(first))
    return fails, (buf[first.value].tolist() if fails else None)


@pytest.mark.parametrize("length", [1, 2, 3])
def test_every_short_string(checker, length):
    first = ctypes.c_uint64(0)
    assert checker.dfa_check_all(length, ctypes.byref(first)) == 0, hex(first.value)


def test_four_bytes_over_class_edges(checker):
    strings = list(itertools.product(CLASS_EDGES, repeat=4))
    assert _list(checker, strings, 4) == (0, None)


@pytest.mark.parametrize("length", [5, 6])
def test_longer_strings_one_byte_per_class(checker, length):
    strings = list(itertools.product(ONE_PER_CLASS, repeat=length))
    assert _list(checker, strings, length) == (0, None)


def test_random_strings(checker):
    rng = np.random.default_rng(5)
    pool = np.array(CLASS_EDGES + list(range(0x80, 0xC0, 7)) + list(range(0xC2, 0xF5, 3)), np.uint8)
    for length in (8, 16, 33):
        strings = pool[rng.integers(0, pool.size, size=(20000, length))]
        assert _list(checker, strings, length) == (0, None)


# Planted mistakes in a copy of utf8_dfa.h, each of which the proof above
# must catch (the unmodified copy passes): wrong class edges, wrong second-
# byte ranges after E0 / ED / F0 / F4, a lead that needs the wrong number of
# continuation bytes, C0/C1 or F5-FF taken as leads, and resynchronisation
# that skips too many or too few continuation bytes.
MUTANTS = [
    ("if (b < 0xC2) return 4;", "if (b < 0xC0) return 4;"),
    ("if (b < 0x90) return 1;", "if (b < 0x88) return 1;"),
    ("if (b < 0xA0) return 2;", "if (b < 0xB0) return 2;"),
    ("if (b < 0xF4) return 10;", "if (b < 0xF5) return 10;"),
    ("    return 4;\n}", "    return 10;\n}"),
    ("return c == 3 ? GPUTF_DFA_NEED1 : GPUTF_DFA_REJECT;                /* A0-BF */",
     "return (c == 2 || c == 3) ? GPUTF_DFA_NEED1 : GPUTF_DFA_REJECT;"),
    ("return (c == 1 || c == 2) ? GPUTF_DFA_NEED1 : GPUTF_DFA_REJECT;   /* 80-9F */",
     "return cont ? GPUTF_DFA_NEED1 : GPUTF_DFA_REJECT;"),
    ("return (c == 2 || c == 3) ? GPUTF_DFA_NEED2 : GPUTF_DFA_REJECT;   /* 90-BF */",
     "return c == 3 ? GPUTF_DFA_NEED2 : GPUTF_DFA_REJECT;"),
    ("return c == 1 ? GPUTF_DFA_NEED2 : GPUTF_DFA_REJECT;                /* 80-8F */",
     "return (c == 1 || c == 2) ? GPUTF_DFA_NEED2 : GPUTF_DFA_REJECT;"),
    ("case 10: return GPUTF_DFA_NEED3;", "case 10: return GPUTF_DFA_NEED2;"),
    ("case 7: return GPUTF_DFA_NEED2;", "case 7: return GPUTF_DFA_NEED1;"),
    ("case GPUTF_DFA_NEED1: return cont ? GPUTF_DFA_ACCEPT : GPUTF_DFA_REJECT;",
     "case GPUTF_DFA_NEED1: return GPUTF_DFA_ACCEPT;"),
    ("if (cont) return s == GPUTF_DFA_SYNC2 ? GPUTF_DFA_ACCEPT : s + 1;",
     "if (cont) return GPUTF_DFA_SYNC0;"),
    ("if (cont) return s == GPUTF_DFA_SYNC2 ? GPUTF_DFA_ACCEPT : s + 1;",
     "if (cont) return s == GPUTF_DFA_SYNC1 ? GPUTF_DFA_ACCEPT : s + 1;"),
]


def _build_copy(tmp, header_text, name):
    d = os.path.join(str(tmp), name)
    os.makedirs(d, exist_ok=True)
    with open(os.path.join(CSRC, "utf8_scheme.h")) as f, open(os.path.join(d, "utf8_scheme.h"), "w") as g:
        g.write(f.read())
    with open(os.path.join(CSRC, "utf8_tables.h")) as f, open(os.path.join(d, "utf8_tables.h"), "w") as g:
        g.write(f.read())
    with open(os.path.join(d, "utf8_dfa.h"), "w") as g:
        g.write(header_text)
    out = os.path.join(d, "dfa_check.so")
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-I" + os.path.join(ROOT, "oracle"),
                           "-I" + d, "-o", out, os.path.join(ROOT, "tests", "native", "dfa_check.c")])
    lib = ctypes.CDLL(out)
    lib.dfa_check_all.restype = ctypes.c_uint64
    lib.dfa_check_all.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_uint64)]
    lib.dfa_check_list.restype = ctypes.c_uint64
    lib.dfa_check_list.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.POINTER(ctypes.c_uint64)]
    return lib


def _proof_fails(lib):
    first = ctypes.c_uint64(0)
    if lib.dfa_check_all(2, ctypes.byref(first)) or lib.dfa_check_all(3, ctypes.byref(first)):
        return True
    return _list(lib, list(itertools.product(CLASS_EDGES, repeat=4)), 4)[0] > 0


def test_planted_mistakes_fail_the_proof(tmp_path):
    with open(os.path.join(CSRC, "utf8_dfa.h")) as f:
        text = f.read()
    assert not _proof_fails(_build_copy(tmp_path, text, "unmodified"))
    for i, (old, new) in enumerate(MUTANTS):
        assert text.count(old) >= 1, old
        mutant = text.replace(old, new, 1)
        assert _proof_fails(_build_copy(tmp_path, mutant, f"m{i}")), (i, old, new)
