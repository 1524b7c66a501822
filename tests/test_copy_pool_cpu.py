"""The serving loop's host copy pool on the CPU (plain C++): a checker built with g++ runs many
parallel loops of random sizes and uneven item costs on pools of 0 to 8 workers and checks that
every index is handed out exactly once and that every call has returned when run() returns."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_copy_pool_every_index_once():
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    out_dir = os.path.join(ROOT, "paper_0809_0063_gb300", "_build")
    os.makedirs(out_dir, exist_ok=True)
    exe = os.path.join(out_dir, "copy_pool_check")
    cmd = ["g++", "-std=c++17", "-O1", "-pthread", "-Wall", "-Wextra", "-Werror",
           "-I", os.path.join(ROOT, "paper_0809_0063_gb300", "csrc"),
           os.path.join(ROOT, "tests", "copy_pool_check.cpp"), "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    run = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert run.returncode == 0 and run.stdout.strip() == "ok", run.stdout + run.stderr
