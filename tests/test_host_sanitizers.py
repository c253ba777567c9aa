"""Host code built with AddressSanitizer and UndefinedBehaviorSanitizer
(compute-sanitizer is not available for the device side): the C oracle driven
through every function on small seeded inputs and edge cases
(`oracle_sanitize_main.c`), and the serving planner driven through seeded
random request streams with its invariants checked (`planner_sanitize_main.cpp`)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


SAN = ["-O1", "-g", "-fsanitize=address,undefined", "-fno-sanitize-recover=all", "-fno-omit-frame-pointer"]


def _build_and_run(compiler, std, sources, includes, exe, marker):
    cc = shutil.which(compiler)
    if cc is None:
        pytest.skip(f"no {compiler}")
    cmd = [cc, std] + SAN + [a for i in includes for a in ("-I", i)] + sources + ["-lm", "-o", exe]
    build = subprocess.run(cmd, capture_output=True, text=True)
    if build.returncode != 0:
        if "sanitize" in build.stderr or "asan" in build.stderr.lower():
            pytest.skip("sanitizer runtime not available: " + build.stderr.strip().splitlines()[-1])
        raise AssertionError(build.stderr)
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0", UBSAN_OPTIONS="print_stacktrace=1")
    res = subprocess.run([exe], capture_output=True, text=True, env=env, timeout=300)
    assert res.returncode == 0, res.stdout + res.stderr
    assert marker in res.stdout


def test_oracle_under_asan_and_ubsan(tmp_path):
    _build_and_run("gcc", "-std=c11",
                   [os.path.join(HERE, "oracle_sanitize_main.c"), os.path.join(ROOT, "oracle", "wt_oracle.c")],
                   [os.path.join(ROOT, "oracle")], str(tmp_path / "oracle_san"), "oracle sanitizer run: ok")


def test_serving_planner_under_asan_and_ubsan(tmp_path):
    _build_and_run("g++", "-std=c++17", [os.path.join(HERE, "planner_sanitize_main.cpp")],
                   [os.path.join(ROOT, "include"), os.path.join(ROOT, "paper_2201_00094_gb300", "csrc")],
                   str(tmp_path / "planner_san"), "planner sanitizer run: ok")
