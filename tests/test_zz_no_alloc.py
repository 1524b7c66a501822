"""GPU test of fp_dot_noalloc, the allocation-free dot product for callers that cannot
allocate device memory (its scratch is a fixed array inside the library's device image).

It is called through the C ABI and compared with the context-based fp_dot on the same
inputs; results are integers, so the tolerance is exact equality.  Two calls run back to back
on each case, since every call reuses the same fixed scratch.  This file is collected last so
that a run stopping at the first failure has already run every other test."""
import numpy as np
import pytest

import workloads
from oracle import field
from tests._gpu import to_dev, torch_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch, dev = torch_dev()
    import __graft_entry__ as g
    g.build()
    import paper_0809_0063_gb300 as fp
    ctx = fp.fp_ctx_create(0)
    yield fp, torch, dev, ctx
    fp.fp_ctx_destroy(ctx)


@pytest.mark.parametrize("algo", ["AUTO", "PLAIN", "DQT_U64"])
@pytest.mark.parametrize("p,n", [(3, 1 << 20), (7, 100003), (251, 4096), (2, 17), (31, 1 << 24)])
def test_noalloc_matches_fp_dot_twice(env, algo, p, n):
    fp, torch, dev, ctx = env
    a = getattr(fp, "FP_ALGO_" + algo)
    for call in range(2):
        u, v = workloads.dot_inputs(1000 * call + n + p, p, n)
        U, V = to_dev(torch, dev, u), to_dev(torch, dev, v)
        ref = torch.zeros((1,), dtype=torch.int32, device=dev)
        got = torch.full((1,), -7, dtype=torch.int32, device=dev)
        fp.fp_dot(ctx, p, U, V, n, ref, a)
        fp.fp_ctx_status(ctx)
        fp.fp_dot_noalloc(p, U, V, n, got, a)
        torch.cuda.synchronize()
        assert int(got.item()) == int(ref.item())
        assert int(got.item()) == field.dot_mod(u, v, p)


@pytest.mark.parametrize("algo", ["AUTO", "DQT_U64", "PLAIN"])
@pytest.mark.parametrize("p,n", [(3, 100003), (7, 17), (2, 4096 + 5), (13, 1 << 20)])
def test_noalloc_offset_views(env, algo, p, n):
    """Arrays that start one byte past a 16-byte line (the entry-by-entry route) and lengths
    that are not a multiple of 16 (the tail that block 0 adds), against fp_dot and the oracle."""
    fp, torch, dev, ctx = env
    a = getattr(fp, "FP_ALGO_" + algo)
    for call in range(2):
        u, v = workloads.dot_inputs(77 * call + n + p, p, n + 1)
        U, V = to_dev(torch, dev, u)[1:], to_dev(torch, dev, v)[1:]
        assert U.data_ptr() % 16 == 1
        want = field.dot_mod(u[1:], v[1:], p)
        ref = torch.zeros((1,), dtype=torch.int32, device=dev)
        got = torch.full((1,), -7, dtype=torch.int32, device=dev)
        fp.fp_dot(ctx, p, U, V, n, ref, a)
        fp.fp_ctx_status(ctx)
        fp.fp_dot_noalloc(p, U, V, n, got, a)
        torch.cuda.synchronize()
        assert int(got.item()) == int(ref.item()) == want


def test_noalloc_flags_bad_input_then_recovers(env):
    fp, torch, dev, ctx = env
    p, n = 5, 5000
    u, v = workloads.dot_inputs(3, p, n)
    U, V = to_dev(torch, dev, u), to_dev(torch, dev, v)
    out = torch.zeros((1,), dtype=torch.int32, device=dev)
    U[17] = 9
    fp.fp_dot_noalloc(p, U, V, n, out)
    torch.cuda.synchronize()
    assert int(out.item()) & 0xFFFFFFFF == 0xFFFFFFFF
    U[17] = int(u[17])
    ref = torch.zeros((1,), dtype=torch.int32, device=dev)
    fp.fp_dot(ctx, p, U, V, n, ref)
    fp.fp_dot_noalloc(p, U, V, n, out)
    fp.fp_ctx_status(ctx)
    assert int(out.item()) == int(ref.item())
    with pytest.raises(fp.FpError) as ei:
        fp.fp_dot_noalloc(p, U, V, (1 << 40) + 1, out)
    assert ei.value.status == fp.FP_EINVAL
