"""The CPU oracle under the compiler's sanitizers.

tests/sanitize_driver.c drives the oracle's entry points (random and
edge-case pairs, tracebacks at end cells and at random cells, the threaded
batch driver) in a binary built with address + undefined-behaviour
sanitizers, and in one built with the thread sanitizer; any report fails the
run.  Skipped where the compiler's sanitizer runtimes are missing.
"""
import os
import subprocess
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = [os.path.join(ROOT, "oracle", "agatha_oracle.c"), os.path.join(HERE, "sanitize_driver.c")]


def _build_and_run(flags):
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "drv")
        r = subprocess.run(["gcc", "-std=c11", "-O1", "-g", "-fno-omit-frame-pointer", *flags, *SRC,
                            "-o", exe, "-pthread"], capture_output=True, text=True)
        if r.returncode != 0:
            pytest.skip(f"sanitizer build unavailable: {r.stderr.strip()[:200]}")
        env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0",
                   UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1", TSAN_OPTIONS="halt_on_error=1")
        return subprocess.run([exe], capture_output=True, text=True, env=env, timeout=600)


def test_oracle_clean_under_address_and_undefined_sanitizers():
    r = _build_and_run(["-fsanitize=address,undefined", "-fno-sanitize-recover=all"])
    assert r.returncode == 0, r.stdout + r.stderr[-3000:]
    assert " 0 bad" in r.stdout


def test_oracle_batch_driver_clean_under_thread_sanitizer():
    r = _build_and_run(["-fsanitize=thread"])
    if "unexpected memory mapping" in r.stderr or "FATAL: ThreadSanitizer" in r.stderr:
        pytest.skip("thread sanitizer cannot run in this environment")
    assert r.returncode == 0, r.stdout + r.stderr[-3000:]
