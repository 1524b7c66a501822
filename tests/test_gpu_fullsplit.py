"""GPU parity of full compression (Sec. 7.5, FP_MM_FULL_F64) and of right compression with a split
inner dimension (Sec. 7.6, FP_MM_SPLIT_F64) against the oracle, bit-exact: the oracle's own
compressed products (oracle/dqt.py full_compressed_product, split_right_compressed_product) at
the planner's parameters, the plain definition (field.matmul_mod) on ragged shapes spanning
several tiles, the all-(p-1) inputs at the edge of the digit bound (one piece and just past
it), sampled rows at the matrix configuration's n = 4096, and the range check."""
import numpy as np
import pytest

import workloads
from oracle import dqt as odqt
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


def run(fp, torch, dev, ctx, p, a, b, algo, ldc_extra=0):
    m, k = a.shape
    n = b.shape[1]
    ldc = n + ldc_extra
    C = torch.full((m, ldc), 255, dtype=torch.uint8, device=dev)
    fp.fp_matmul(ctx, p, m, n, k, to_dev(torch, dev, a), k, to_dev(torch, dev, b), n, C, ldc, algo)
    fp.fp_ctx_status(ctx)
    out = C.cpu().numpy()
    if ldc_extra:
        assert (out[:, n:] == 255).all(), "write past the n columns of C"
    return out[:, :n]


@pytest.mark.parametrize("p,m,n,k", [(3, 37, 45, 200), (2, 64, 129, 127), (5, 20, 31, 60), (3, 1, 1, 1),
                                     (7, 9, 11, 100), (13, 16, 17, 40), (3, 130, 67, 1000)])
def test_full_vs_oracle_full_compression(env, p, m, n, k):
    """One piece: the GPU equals the oracle's full compression at the planner's (Q, dq, dt)."""
    fp, torch, dev, ctx = env
    b, dq1, dt1, piece = fp.fp_mm_full_choose(p, k)
    assert piece == k and dq1 >= 2 and dt1 >= 2
    a, bb = workloads.matmul_inputs(p * 7919 + m * 31 + k, p, m, k, n)
    got = run(fp, torch, dev, ctx, p, a, bb, fp.FP_MM_FULL_F64, ldc_extra=5)
    want = odqt.full_compressed_product(a, bb, p, dq1 - 1, dt1 - 1, 2 ** b, dq1)
    np.testing.assert_array_equal(got, want)
    np.testing.assert_array_equal(got, field.matmul_mod(a, bb, p))


@pytest.mark.parametrize("p,m,n,k", [(3, 70, 90, 4100), (7, 33, 47, 1000), (2, 40, 41, 20000), (23, 17, 19, 100)])
def test_full_split_pieces(env, p, m, n, k):
    """Inner dimension split into pieces: equals the plain definition (the unique C)."""
    fp, torch, dev, ctx = env
    b, dq1, dt1, piece = fp.fp_mm_full_choose(p, k)
    assert piece < k and piece * (p - 1) ** 2 < 2 ** b
    a, bb = workloads.matmul_inputs(p * 104729 + k, p, m, k, n)
    got = run(fp, torch, dev, ctx, p, a, bb, fp.FP_MM_FULL_F64)
    np.testing.assert_array_equal(got, field.matmul_mod(a, bb, p))


@pytest.mark.parametrize("k", [2047, 2048, 4096])
def test_full_all_max_entries_at_the_bound(env, k):
    """All entries p-1 = 2 over F_3: at k = 2047 every digit is 8188, the largest below Q = 2^13
    (one piece); from 2048 on the planner must split."""
    fp, torch, dev, ctx = env
    p, m, n = 3, 10, 14
    a = np.full((m, k), p - 1, dtype=np.uint8)
    bb = np.full((k, n), p - 1, dtype=np.uint8)
    got = run(fp, torch, dev, ctx, p, a, bb, fp.FP_MM_FULL_F64)
    np.testing.assert_array_equal(got, np.full((m, n), (k * (p - 1) ** 2) % p, dtype=np.uint8))
    b, dq1, dt1, piece = fp.fp_mm_full_choose(p, k)
    assert (b, dq1, dt1) == (13, 2, 2) and (piece == k) == (k <= 2047)


@pytest.mark.parametrize("p,m,n,k", [(2, 30, 57, 2000), (3, 20, 33, 4100), (7, 12, 25, 4096), (3, 9, 10, 300)])
def test_split_vs_oracle_split(env, p, m, n, k):
    """Right compression with the planner's pieces equals the oracle's split product over the same
    pieces (each piece at its own Q, reduced, added mod p) and the plain definition."""
    fp, torch, dev, ctx = env
    b, e, piece = fp.fp_mm_choose(p, k, fp.FP_MM_SPLIT_F64)
    a, bb = workloads.matmul_inputs(p * 15485863 + k + m, p, m, k, n)
    got = run(fp, torch, dev, ctx, p, a, bb, fp.FP_MM_SPLIT_F64, ldc_extra=3)
    want = odqt.split_right_compressed_product(a, bb, p, piece, 52)
    np.testing.assert_array_equal(got, want)
    np.testing.assert_array_equal(got, field.matmul_mod(a, bb, p))


def test_split_keeps_compression_four_past_2048(env):
    """Sec. 7.6: over F_3 the split product keeps e = 4 (Q = 2^13) past k = 2047 where the
    unsplit right compression drops to e = 3; every piece then satisfies Eq. lower."""
    fp, torch, dev, ctx = env
    for k in (2048, 2049, 4096, 10000):
        b, e, piece = fp.fp_mm_choose(3, k, fp.FP_MM_SPLIT_F64)
        assert (b, e) == (13, 4) and piece * 4 < 2 ** 13 and piece % 4 == 0
        assert fp.fp_mm_choose(3, k, fp.FP_MM_RIGHT_F64)[1] == 3
    p, m, n, k = 3, 8, 16, 4096
    a = np.full((m, k), 2, dtype=np.uint8)
    bb = np.full((k, n), 2, dtype=np.uint8)
    got = run(fp, torch, dev, ctx, p, a, bb, fp.FP_MM_SPLIT_F64)
    np.testing.assert_array_equal(got, np.full((m, n), (k * 4) % 3, dtype=np.uint8))


def test_split_many_pieces_rereduce(env):
    """Enough pieces that R's fields are re-reduced several times (F_2 at e = 5: fields of 12 bits,
    pieces add up to 1023 each, a re-reduction every 4 pieces)."""
    fp, torch, dev, ctx = env
    p, m, n, k = 2, 16, 20, 30000
    b, e, piece = fp.fp_mm_choose(p, k, fp.FP_MM_SPLIT_F64)
    assert e == 5 and k // piece >= 20
    a = np.ones((m, k), dtype=np.uint8)
    bb = np.ones((k, n), dtype=np.uint8)
    a[:, ::7] = 0
    got = run(fp, torch, dev, ctx, p, a, bb, fp.FP_MM_SPLIT_F64)
    np.testing.assert_array_equal(got, field.matmul_mod(a, bb, p))


@pytest.mark.parametrize("algo", ["FULL_F64", "SPLIT_F64"])
@pytest.mark.parametrize("p", [3, 7])
def test_matrix_config_n4096_sampled_rows(env, algo, p):
    """The matrix configuration's n = 4096 products, rows sampled across every tile row."""
    fp, torch, dev, ctx = env
    n = 4096
    a, bb = workloads.matmul_inputs(p * 7 + n, p, n, n, n)
    C = torch.empty((n, n), dtype=torch.uint8, device=dev)
    fp.fp_matmul(ctx, p, n, n, n, to_dev(torch, dev, a), n, to_dev(torch, dev, bb), n, C, n,
                 getattr(fp, "FP_MM_" + algo))
    fp.fp_ctx_status(ctx)
    rows = np.array([0, 1, 63, 64, 127, 1000, 2047, 2048, 3001, 4094, 4095])
    np.testing.assert_array_equal(C[rows].cpu().numpy(), field.matmul_mod_rows(a, bb, p, rows))


@pytest.mark.parametrize("algo", ["FULL_F64", "SPLIT_F64"])
def test_range_error(env, algo):
    fp, torch, dev, ctx = env
    p, m, n, k = 3, 8, 9, 50
    a, bb = workloads.matmul_inputs(5, p, m, k, n)
    a[3, 7] = 3
    C = torch.empty((m, n), dtype=torch.uint8, device=dev)
    fp.fp_matmul(ctx, p, m, n, k, to_dev(torch, dev, a), k, to_dev(torch, dev, bb), n, C, n,
                 getattr(fp, "FP_MM_" + algo))
    with pytest.raises(fp.FpError) as ex:
        fp.fp_ctx_status(ctx)
    assert ex.value.status == fp.FP_EINVAL


def test_full_refuses_large_p(env):
    fp, torch, dev, ctx = env
    A = torch.zeros((16, 16), dtype=torch.uint8, device=dev)
    with pytest.raises(fp.FpError) as ex:   # 16 (31-1)^2 >= 2^13: no 2 x 2 packing of any piece
        fp.fp_matmul(ctx, 31, 16, 16, 16, A, 16, A, 16, A, 16, fp.FP_MM_FULL_F64)
    assert ex.value.status == fp.FP_EBOUND
