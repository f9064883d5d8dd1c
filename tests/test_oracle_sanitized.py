"""The oracle under AddressSanitizer and UndefinedBehaviorSanitizer: its pins, the
independent NumPy restatement and the adjoint's finite-difference checks all run against
an oracle built with both sanitizers, every report fatal, in a child process that
preloads the ASan runtime.  An out-of-bounds read or write, a use after free, a signed
overflow or a misaligned access anywhere on those paths fails this test."""
import os
import subprocess
import sys

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_oracle_pins_under_sanitizers(tmp_path):
    libasan = subprocess.run(["gcc", "-print-file-name=libasan.so"], capture_output=True, text=True).stdout.strip()
    if not os.path.isabs(libasan) or not os.path.exists(libasan):
        pytest.skip("no ASan runtime for this gcc")
    so = oracle.build_sanitized(os.path.join(tmp_path, "liboracle_sanitized.so"))
    env = dict(os.environ, LD_PRELOAD=libasan, HMFSR_ORACLE_LIB=so,
               ASAN_OPTIONS="detect_leaks=0:exitcode=23", UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1",
               OMP_NUM_THREADS="4")
    files = ["tests/test_oracle_pins.py", "tests/test_oracle_restatement.py", "tests/test_oracle_adjoint.py"]
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", "-m", "not gpu",
                        *files], cwd=ROOT, env=env, capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, (r.stdout[-4000:], r.stderr[-4000:])
    assert " passed" in r.stdout
