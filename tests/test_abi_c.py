"""The C ABI used from C: small C programs that include only the public header (and the CUDA
runtime's C header), compiled with gcc as C99 with warnings as errors and linked to
libfpdqt.so.  tests/abi_c_check.c runs on the CPU: its host-only planner answers must equal the
Python binding's.  tests/abi_c_compute.c runs on a GPU: it allocates device memory itself,
copies seeded inputs in, runs a matrix product, a batched polynomial product and a dot product
through the C ABI and copies the results out; they must equal the oracle's."""
import os
import shutil
import subprocess

import numpy as np
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


def _cuda_include():
    for d in ("/usr/local/cuda/include", "/usr/local/cuda/targets/sbsa-linux/include",
              "/usr/local/cuda/targets/x86_64-linux/include"):
        if os.path.exists(os.path.join(d, "cuda_runtime_api.h")):
            return d
    return None


def _compile_compute(out_dir):
    inc = _cuda_include()
    if shutil.which("gcc") is None or inc is None:
        pytest.skip("gcc or the CUDA runtime header not available")
    exe = os.path.join(out_dir, "abi_c_compute")
    cmd = ["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
           "-isystem", inc, os.path.join(ROOT, "tests", "abi_c_compute.c"), "-o", exe, "-L", PKG, "-lfpdqt",
           "-L", "/usr/local/cuda/lib64", "-lcudart", "-Wl,-rpath," + PKG, "-Wl,-rpath,/usr/local/cuda/lib64"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_c_compute_program_builds(fp):
    """The GPU consumer compiles as strict C99 against the public header (no GPU needed)."""
    out_dir = os.path.join(PKG, "_build")
    os.makedirs(out_dir, exist_ok=True)
    _compile_compute(out_dir)


@pytest.mark.gpu
def test_c_program_computes_on_device_buffers(fp, tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import workloads
    from oracle import field
    out_dir = os.path.join(PKG, "_build")
    os.makedirs(out_dir, exist_ok=True)
    exe = _compile_compute(out_dir)
    p, m, n, k, batch, deg, nd = 3, 200, 333, 517, 4099, 2, 100003
    a, b = workloads.matmul_inputs(31, p, m, k, n)
    pa, pb = workloads.polymul_inputs(32, p, batch, deg, deg)
    u, v = workloads.dot_inputs(33, p, nd)
    for name, x in (("A", a), ("B", b), ("Pa", pa), ("Pb", pb), ("U", u), ("V", v)):
        np.ascontiguousarray(x, dtype=np.uint8).tofile(str(tmp_path / f"{name}.bin"))
    env = dict(os.environ)
    env["LD_LIBRARY_PATH"] = os.pathsep.join([PKG, "/usr/local/cuda/lib64", env.get("LD_LIBRARY_PATH", "")])
    run = subprocess.run([exe, str(tmp_path), str(p), str(m), str(n), str(k), str(batch), str(deg), str(nd)],
                         capture_output=True, text=True, env=env, timeout=300)
    assert run.returncode == 0, run.stderr
    C = np.fromfile(str(tmp_path / "C.bin"), dtype=np.uint8).reshape(m, n)
    Pc = np.fromfile(str(tmp_path / "Pc.bin"), dtype=np.uint8).reshape(batch, 2 * deg + 1)
    dot = int(np.fromfile(str(tmp_path / "dot.bin"), dtype=np.uint32)[0])
    np.testing.assert_array_equal(C, field.matmul_mod(a, b, p))
    np.testing.assert_array_equal(Pc, field.polymul_mod(pa, pb, p))
    assert dot == field.dot_mod(u, v, p)
    assert "range_status %d" % fp.FP_EINVAL in run.stdout
