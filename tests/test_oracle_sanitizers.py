"""The C oracle built with AddressSanitizer and UndefinedBehaviorSanitizer and
driven through every function on small seeded inputs and edge cases
(`oracle_sanitize_main.c`): the oracle must be free of memory errors and
undefined behaviour before it can be trusted as the reference."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_oracle_under_asan_and_ubsan(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    exe = str(tmp_path / "oracle_san")
    cmd = [cc, "-std=c11", "-O1", "-g", "-fsanitize=address,undefined", "-fno-sanitize-recover=all",
           "-fno-omit-frame-pointer", "-I", os.path.join(ROOT, "oracle"),
           os.path.join(HERE, "oracle_sanitize_main.c"), os.path.join(ROOT, "oracle", "wt_oracle.c"), "-lm",
           "-o", exe]
    build = subprocess.run(cmd, capture_output=True, text=True)
    if build.returncode != 0:
        if "sanitize" in build.stderr or "asan" in build.stderr.lower():
            pytest.skip("sanitizer runtime not available: " + build.stderr.strip().splitlines()[-1])
        raise AssertionError(build.stderr)
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0", UBSAN_OPTIONS="print_stacktrace=1")
    res = subprocess.run([exe], capture_output=True, text=True, env=env, timeout=300)
    assert res.returncode == 0, res.stdout + res.stderr
    assert "oracle sanitizer run: ok" in res.stdout
