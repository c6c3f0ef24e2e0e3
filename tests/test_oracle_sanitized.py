"""The oracle's C code under AddressSanitizer and UndefinedBehaviorSanitizer: every
pin of tests/pins.py runs against a sanitized build of the oracle (out-of-bounds
reads or writes, overflowing arithmetic or undefined shifts abort the run)."""
import os
import subprocess
import sys
import textwrap

import pytest

from conftest import ROOT

CHILD = textwrap.dedent("""
    import os, sys
    sys.path.insert(0, os.environ["ORACLE_ROOT"])
    sys.path.insert(0, os.path.join(os.environ["ORACLE_ROOT"], "tests"))
    from oracle import Oracle
    import pins
    o = Oracle(os.environ["ORACLE_LIB"])
    for check in pins.ALL_CHECKS:
        check(o)
    print("sanitized pins ok", len(pins.ALL_CHECKS))
""")


def _runtime(name):
    try:
        p = subprocess.run(["gcc", f"-print-file-name={name}"], capture_output=True, text=True, check=True).stdout.strip()
    except (OSError, subprocess.CalledProcessError):
        return None
    return p if os.path.isabs(p) and os.path.exists(p) else None


def test_pins_pass_on_a_sanitized_oracle(tmp_path):
    asan = _runtime("libasan.so")
    if asan is None:
        pytest.skip("no AddressSanitizer runtime for gcc here")
    sys.path.insert(0, ROOT)
    from oracle import compile_oracle
    lib = str(tmp_path / "liboracle_san.so")
    compile_oracle(out=lib, extra=["-fsanitize=address,undefined", "-fno-sanitize-recover=all",
                                   "-fno-omit-frame-pointer", "-g"])
    env = dict(os.environ, ORACLE_ROOT=ROOT, ORACLE_LIB=lib, LD_PRELOAD=asan,
               ASAN_OPTIONS="detect_leaks=0:abort_on_error=1", UBSAN_OPTIONS="print_stacktrace=1")
    r = subprocess.run([sys.executable, "-c", CHILD], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, (r.stdout + r.stderr)[-4000:]
    assert "sanitized pins ok" in r.stdout
