"""The CPU oracle and the host-compiled kernel headers under AddressSanitizer
and UndefinedBehaviorSanitizer.

tests/native/sanitize_driver.c calls the oracle's transcoders, validators and
length functions, and the headers' UTF-8 check, fix-up, decoder and UTF-16
classification and byte arithmetic, and the batched kernel's per-piece
arithmetic over every piece of random chunks, on every string of up to two bytes,
every scalar value, and 20,000 random inputs rich in continuation bytes,
leads and surrogates, each in a buffer of exactly the size the call is given
and with every capacity from none to ample.  Built with
-fsanitize=address,undefined and no recovery, any out-of-bounds access, shift
past the width or signed overflow fails the run."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def build_and_run(tmp_path, *defines):
    exe = str(tmp_path / ("sanitize_driver" + "".join(defines)))
    cmd = ["gcc", "-O1", "-g", "-std=gnu11", "-fno-omit-frame-pointer",
           "-fsanitize=address,undefined", "-fno-sanitize-recover=all", *[f"-D{d}" for d in defines],
           "-I" + os.path.join(ROOT, "oracle"), "-I" + os.path.join(ROOT, "paper_2109_10433_gb300", "csrc"),
           "-o", exe, os.path.join(ROOT, "tests", "native", "sanitize_driver.c")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0 and ("asan" in r.stderr.lower() or "ubsan" in r.stderr.lower()):
        pytest.skip("the sanitizer runtimes are not installed")
    assert r.returncode == 0, r.stderr
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0", UBSAN_OPTIONS="print_stacktrace=1")
    return subprocess.run([exe], capture_output=True, text=True, timeout=600, env=env)


def test_oracle_and_headers_are_clean_under_asan_and_ubsan(tmp_path):
    run = build_and_run(tmp_path)
    assert run.returncode == 0, run.stderr[-4000:]
    assert "runtime error" not in run.stderr and "ERROR: AddressSanitizer" not in run.stderr
    assert int(run.stdout.split()[0]) > 500000


def test_a_planted_overread_fails_the_run(tmp_path):
    """The same driver with one read a byte past a buffer: the sanitizers
    are live and the run fails."""
    run = build_and_run(tmp_path, "PLANT_OVERREAD")
    assert run.returncode != 0
    assert "AddressSanitizer: heap-buffer-overflow" in run.stderr
