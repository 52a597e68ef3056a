"""The CPU oracle under AddressSanitizer and UndefinedBehaviorSanitizer:
every entry point on ragged layouts (empty and single-SD cells, dead SDs,
multiplicities up to 2^62, SDs outside the domain, both kernels and
precisions, p far above 1), with no memory error, no undefined behaviour and
the conservation laws intact.  compute-sanitizer is not used on the GPU path;
that path is checked bit for bit against this oracle instead."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_oracle_clean_under_asan_and_ubsan(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    exe = tmp_path / "oracle_sanitized"
    src = os.path.join(ROOT, "oracle", "sanitize_main.c")
    build = subprocess.run([gcc, "-std=c11", "-O1", "-g", "-fsanitize=address,undefined",
                            "-fno-sanitize-recover=all", "-fno-omit-frame-pointer", "-ffp-contract=off",
                            src, "-lm", "-o", str(exe)], capture_output=True, text=True)
    if build.returncode != 0 and "sanitize" in build.stderr:
        pytest.skip("this compiler has no sanitizer runtime: " + build.stderr.strip().splitlines()[-1])
    assert build.returncode == 0, build.stderr
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0", UBSAN_OPTIONS="print_stacktrace=1")
    run = subprocess.run([str(exe)], capture_output=True, text=True, env=env, timeout=300)
    assert run.returncode == 0, run.stderr[-4000:]
    assert "runtime error" not in run.stderr and "ERROR: AddressSanitizer" not in run.stderr
    assert "cases ok" in run.stdout
