"""The oracle under AddressSanitizer and UndefinedBehaviorSanitizer: a small C driver
(tests/oracle_sanitize.c) runs its 2D and 3D forward / back / COO export on small
geometries; any out-of-bounds access, leak or undefined behaviour fails the run."""
import os
import shutil
import subprocess
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_oracle_under_sanitizers():
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "oracle_sanitize")
        cmd = [cc, "-O1", "-g", "-fno-omit-frame-pointer", "-fsanitize=address,undefined",
               "-fno-sanitize-recover=all", os.path.join(ROOT, "oracle", "csm_oracle.c"),
               os.path.join(HERE, "oracle_sanitize.c"), "-lm", "-o", exe]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            if "sanitize" in r.stderr or "asan" in r.stderr.lower():
                pytest.skip("sanitizer runtime not available: " + r.stderr.strip()[:200])
            raise AssertionError(r.stderr)
        env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0",
                   UBSAN_OPTIONS="print_stacktrace=1:halt_on_error=1")
        run = subprocess.run([exe], capture_output=True, text=True, env=env, timeout=300)
        assert run.returncode == 0, run.stdout + run.stderr
        assert run.stdout.count(": ok") == 2, run.stdout
