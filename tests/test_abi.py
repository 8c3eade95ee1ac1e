"""CPU checks of the boundary: the library builds for sm_103a, loads, and
exports every entry point that include/gputf.h declares; the binding declares
the same set; the committed UTF-8 tables are what their generator derives."""
import ctypes
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gputf.h")
CSRC = os.path.join(ROOT, "paper_2109_10433_gb300", "csrc")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gputf_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libgputf():
    import paper_2109_10433_gb300 as g
    g.build()
    return g


def test_library_exports_every_declared_function(libgputf):
    names = declared_functions()
    assert len(names) >= 14
    L = ctypes.CDLL(libgputf.LIB_PATH)
    for name in names:
        assert hasattr(L, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", libgputf.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (gputf_[a-z0-9_]+)$", out, flags=re.M))
    assert exported == set(names)
    assert set(libgputf.SIGNATURES) == set(names)


def test_binding_host_only_calls(libgputf):
    L = libgputf.lib()
    assert L.gputf_version() == 100
    assert L.gputf_error_name(0) == b"OK" and L.gputf_error_name(6) == b"SURROGATE"
    assert L.gputf_status_name(2) == b"WORKSPACE_TOO_SMALL"
    # workspace: header plus one word per 1024 units, growing with the input
    small, big = L.gputf_workspace_bytes(1), L.gputf_workspace_bytes(1 << 30)
    assert small >= 256 and big >= 256 + 8 * ((1 << 30) // 1024)


def test_library_is_built_for_sm_103a(libgputf):
    out = subprocess.run(["cuobjdump", "--list-elf", libgputf.LIB_PATH], capture_output=True, text=True)
    if out.returncode != 0:
        pytest.skip("cuobjdump unavailable")
    assert "sm_103a" in out.stdout


def test_utf8_tables_match_their_generator():
    sys.path.insert(0, CSRC)
    try:
        import gen_utf8_tables as gen
    finally:
        sys.path.pop(0)
    gen.check_terms()
    with open(os.path.join(CSRC, "utf8_tables.h")) as f:
        assert f.read() == gen.header_text()


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    import paper_2109_10433_gb300 as g
    monkeypatch.setattr(g, "_lib", None)
    monkeypatch.setattr(g, "LIB_PATH", str(tmp_path / "libgputf.so"))
    with pytest.raises(g.GputfError):
        g.lib()
