"""The C ABI used from C: a small C program (tests/abi_c_check.c) that includes only the
public header, compiled with gcc as C99 with warnings as errors, linked to libfpdqt.so, and run
on the CPU.  Its host-only planner answers must equal the Python binding's."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_0809_0063_gb300")


@pytest.fixture(scope="module")
def fp():
    import __graft_entry__ as g
    g.build()
    import paper_0809_0063_gb300 as m
    return m


def test_c_program_agrees_with_binding(fp):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    out_dir = os.path.join(PKG, "_build")
    os.makedirs(out_dir, exist_ok=True)
    exe = os.path.join(out_dir, "abi_c_check")
    cmd = ["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "abi_c_check.c"), "-o", exe, "-L", PKG, "-lfpdqt",
           "-Wl,-rpath," + PKG]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    env = dict(os.environ)
    env["LD_LIBRARY_PATH"] = os.pathsep.join([PKG, "/usr/local/cuda/lib64", env.get("LD_LIBRARY_PATH", "")])
    run = subprocess.run([exe], capture_output=True, text=True, env=env, timeout=120)
    assert run.returncode == 0, run.stderr
    lines = run.stdout.strip().splitlines()
    fields = ["kernel", "word", "blk_a", "blk_b", "b", "ndig", "L", "m"]
    n_plans = 0
    for ln in lines:
        t = ln.split()
        if t[0] == "plan":
            p, da, db, algo = (int(x) for x in t[1:5])
            if t[5] == "ok":
                want = fp.fp_polymul_plan(p, da, db, algo)
                assert [int(x) for x in t[6:]] == [want[f] for f in fields], ln
            else:
                with pytest.raises(fp.FpError) as ei:
                    fp.fp_polymul_plan(p, da, db, algo)
                assert ei.value.status == int(t[6]), ln
            n_plans += 1
        elif t[0] == "dqt":
            prm = fp.fp_dqt_choose(int(t[1]), 3, 1000, fp.FP_WORD_U64)
            assert [int(t[3]), int(t[4])] == [prm.b, prm.ndig], ln
        elif t[0] == "mm":
            assert tuple(int(x) for x in t[3:6]) == fp.fp_mm_choose(int(t[1]), 4096, fp.FP_MM_RIGHT_F64), ln
        elif t[0] == "bad":
            assert int(t[1]) == fp.FP_EINVAL and t[2] == "message", ln
    assert n_plans == 5 * 5 * 7
