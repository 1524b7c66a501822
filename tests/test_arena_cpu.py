"""The serving loop's device-arena allocator on the CPU (its bookkeeping is plain C++): a
checker built with g++ replays random allocations and releases against a byte map of the
arena (first fit, every adjacent free run merged, exact failure when nothing fits)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_first_fit_arena_against_byte_map():
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    out_dir = os.path.join(ROOT, "paper_0809_0063_gb300", "_build")
    os.makedirs(out_dir, exist_ok=True)
    exe = os.path.join(out_dir, "arena_check")
    cmd = ["g++", "-std=c++17", "-O1", "-Wall", "-Wextra", "-Werror",
           "-I", os.path.join(ROOT, "paper_0809_0063_gb300", "csrc"),
           os.path.join(ROOT, "tests", "arena_check.cpp"), "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    run = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert run.returncode == 0 and run.stdout.strip() == "ok", run.stdout + run.stderr
