"""GPU parity of the matrix product over GF(p^k) (Algorithm FGDP on every entry, fp_gf_matmul)
against the oracle's field matrix product (field.gf_matmul), bit-exact: the three fields of the
GF configuration and small fields, ragged shapes spanning several 64 x 64 tiles and inner
lengths around the chunk and the 32-step staging tile, both element forms, leading dimensions
larger than the width, all-(p-1) elements at the digit bound, and the range check."""
import numpy as np
import pytest

import workloads
from oracle import field
from tests._gpu import torch_dev

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


def _dev(torch, dev, x, dt):
    x = np.ascontiguousarray(x.astype(dt))
    return torch.from_numpy(x.view(np.int16) if dt == np.uint16 else x).to(dev)


def gf_mm(fp, torch, dev, ctx, gf, a, b, dt, form, pad=(0, 0, 0)):
    m, k = a.shape
    n = b.shape[1]
    lda, ldb, ldc = k + pad[0], n + pad[1], n + pad[2]
    A = np.zeros((m, lda), dt)
    A[:, :k] = a
    B = np.zeros((k, ldb), dt)
    B[:, :n] = b
    sentinel = 7
    C = _dev(torch, dev, np.full((m, ldc), sentinel), dt)
    fp.fp_gf_matmul(ctx, gf, m, n, k, _dev(torch, dev, A, dt), lda, _dev(torch, dev, B, dt), ldb, C, ldc, form)
    fp.fp_ctx_status(ctx)
    out = C.cpu().numpy()
    out = (out.view(np.uint16) if dt == np.uint16 else out).astype(np.int64)
    if pad[2]:
        assert (out[:, n:] == sentinel).all(), "write past the n columns of C"
    return out[:, :n]


@pytest.mark.parametrize("p,k", [(3, 5), (7, 4), (2, 8), (3, 2), (5, 1), (2, 3), (13, 2)])
@pytest.mark.parametrize("m,n,kk", [(70, 65, 33), (1, 1, 1), (64, 128, 31), (5, 200, 100)])
def test_gf_matmul_matches_oracle(env, p, k, m, n, kk):
    fp, torch, dev, ctx = env
    gf = fp.fp_gf_create(ctx, p, k)
    try:
        mod = field.smallest_monic_irreducible(p, k)
        q = p ** k
        dt = workloads.gf_index_dtype(p, k)
        rng = np.random.default_rng(q * 131 + m + n + kk)
        a, b = rng.integers(0, q, (m, kk)), rng.integers(0, q, (kk, n))
        want = field.gf_matmul(a, b, p, k, mod)
        got = gf_mm(fp, torch, dev, ctx, gf, a, b, dt, fp.FP_GF_INDEX, pad=(3, 1, 2))
        np.testing.assert_array_equal(got, want)
        antilog, log = field.log_tables(p, k, mod)
        got_l = gf_mm(fp, torch, dev, ctx, gf, log[a], log[b], dt, fp.FP_GF_LOG)
        np.testing.assert_array_equal(got_l, log[want])
    finally:
        fp.fp_gf_destroy(gf)


@pytest.mark.parametrize("p,k", [(3, 5), (7, 4), (2, 8)])
def test_gf_matmul_entry_is_the_dot_product(env, p, k):
    """Every entry equals the oracle's field dot product of its row and column (a 256 x 256 x 300
    product, rows and columns sampled), and the chunked accumulation is exercised at every
    length around the chunk."""
    fp, torch, dev, ctx = env
    gf = fp.fp_gf_create(ctx, p, k)
    try:
        mod = field.smallest_monic_irreducible(p, k)
        q, nc = p ** k, fp.fp_gf_dot_info(gf)["chunk"]
        dt = workloads.gf_index_dtype(p, k)
        rng = np.random.default_rng(q + 5)
        m = n = 256
        kk = 300
        a, b = rng.integers(0, q, (m, kk)), rng.integers(0, q, (kk, n))
        got = gf_mm(fp, torch, dev, ctx, gf, a, b, dt, fp.FP_GF_INDEX)
        for r, c in [(0, 0), (255, 255), (17, 200), (128, 64), (63, 64), (64, 63)]:
            assert got[r, c] == field.gf_dot(a[r], b[:, c], p, k, mod)
        for kk in sorted({nc - 1, nc, nc + 1, 2 * nc + 1, 32, 33} - {0}):
            a, b = rng.integers(0, q, (3, kk)), rng.integers(0, q, (kk, 4))
            got = gf_mm(fp, torch, dev, ctx, gf, a, b, dt, fp.FP_GF_INDEX)
            np.testing.assert_array_equal(got, field.gf_matmul(a, b, p, k, mod))
        # all elements p^k - 1: every chunk's digits at the bound's edge
        a = np.full((9, 3 * nc + 5), q - 1)
        got = gf_mm(fp, torch, dev, ctx, gf, a, a.T.copy(), dt, fp.FP_GF_INDEX)
        np.testing.assert_array_equal(got, field.gf_matmul(a, a.T, p, k, mod))
    finally:
        fp.fp_gf_destroy(gf)


def test_gf_matmul_bad_code_and_arguments(env):
    fp, torch, dev, ctx = env
    gf = fp.fp_gf_create(ctx, 3, 5)
    try:
        a = np.zeros((4, 10), np.uint8)
        a[2, 3] = 243
        A = torch.from_numpy(a).to(dev)
        C = torch.empty((4, 4), dtype=torch.uint8, device=dev)
        fp.fp_gf_matmul(ctx, gf, 4, 4, 10, A, 10, A.t().contiguous(), 4, C, 4)
        with pytest.raises(fp.FpError) as ei:
            fp.fp_ctx_status(ctx)
        assert ei.value.status == fp.FP_EINVAL
        with pytest.raises(fp.FpError) as ei:
            fp.fp_gf_matmul(ctx, gf, 4, 4, 10, A, 9, A, 4, C, 4)      # lda < k
        assert ei.value.status == fp.FP_EINVAL
        with pytest.raises(fp.FpError):
            fp.fp_gf_matmul(ctx, gf, 4, 4, 10, A, 10, A, 4, C, 4, 2)  # no such form
    finally:
        fp.fp_gf_destroy(gf)


@pytest.mark.parametrize("p,k", [(3, 5), (7, 4), (2, 8)])
def test_gf_matmul_long_inner_all_max(env, p, k):
    """Inner dimension 2000 with every element p^k - 1 (every REDQ at its digit bound, many folds
    of the deferred coefficient sums) and a random 2000-term product, in both forms."""
    fp, torch, dev, ctx = env
    gf = fp.fp_gf_create(ctx, p, k)
    try:
        mod = field.smallest_monic_irreducible(p, k)
        q = p ** k
        dt = workloads.gf_index_dtype(p, k)
        antilog, log = field.log_tables(p, k, mod)
        a = np.full((5, 2000), q - 1)
        want = field.gf_matmul(a, a.T, p, k, mod)
        np.testing.assert_array_equal(gf_mm(fp, torch, dev, ctx, gf, a, a.T.copy(), dt, fp.FP_GF_INDEX), want)
        np.testing.assert_array_equal(gf_mm(fp, torch, dev, ctx, gf, log[a], log[a.T].copy(), dt, fp.FP_GF_LOG),
                                      log[want])
        rng = np.random.default_rng(q + 77)
        a, b = rng.integers(0, q, (6, 2000)), rng.integers(0, q, (2000, 70))
        want = field.gf_matmul(a, b, p, k, mod)
        np.testing.assert_array_equal(gf_mm(fp, torch, dev, ctx, gf, a, b, dt, fp.FP_GF_INDEX), want)
        np.testing.assert_array_equal(gf_mm(fp, torch, dev, ctx, gf, log[a], log[b], dt, fp.FP_GF_LOG), log[want])
    finally:
        fp.fp_gf_destroy(gf)


@pytest.mark.parametrize("form", ["INDEX", "LOG"])
@pytest.mark.parametrize("p,k,bad", [(3, 5, (243, 255)), (7, 4, (2401, 4096 + 3, 65535))])
def test_gf_matmul_bad_codes_count_as_zero(env, p, k, bad, form):
    """Codes >= p^k in A and B (GF(7^4) codes among them whose low 12 bits are a valid code)
    count as zero and set the range error, in both forms."""
    fp, torch, dev, ctx = env
    gf = fp.fp_gf_create(ctx, p, k)
    try:
        mod = field.smallest_monic_irreducible(p, k)
        q = p ** k
        dt = workloads.gf_index_dtype(p, k)
        antilog, log = field.log_tables(p, k, mod)
        rng = np.random.default_rng(q + 91)
        m, n, kk = 70, 66, 45
        a, b = rng.integers(0, q, (m, kk)), rng.integers(0, q, (kk, n))
        ca, cb = (log[a], log[b]) if form == "LOG" else (a.copy(), b.copy())
        za, zb = a.copy(), b.copy()
        for i, (r, c) in enumerate(((0, 0), (69, 44), (33, 7))):
            ca[r, c] = bad[i % len(bad)]
            za[r, c] = 0
        for i, (r, c) in enumerate(((44, 65), (3, 64))):
            cb[r, c] = bad[(i + 1) % len(bad)]
            zb[r, c] = 0
        want = field.gf_matmul(za, zb, p, k, mod)
        if form == "LOG":
            want = log[want]
        C = _dev(torch, dev, np.zeros((m, n)), dt)
        fp.fp_gf_matmul(ctx, gf, m, n, kk, _dev(torch, dev, ca, dt), kk, _dev(torch, dev, cb, dt), n, C, n,
                        getattr(fp, "FP_GF_" + form))
        torch.cuda.synchronize()
        got = C.cpu().numpy()
        got = (got.view(np.uint16) if dt == np.uint16 else got).astype(np.int64)
        with pytest.raises(fp.FpError) as ei:
            fp.fp_ctx_status(ctx)
        assert ei.value.status == fp.FP_EINVAL
        np.testing.assert_array_equal(got, want)
    finally:
        fp.fp_gf_destroy(gf)
