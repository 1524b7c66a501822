"""GPU parity of the compressed matrix product C = A B mod p (every algorithm) against the
oracle, bit-exact: ragged sizes spanning several tiles, the paper's configurations (full
compare at n = 1024, sampled rows at n = 4096 in the launch configuration the benchmark
times), adversarial all-(p-1) inputs at the bound's edge, and error paths."""
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


ALL = ["AUTO", "RIGHT_F64", "RIGHT_F32", "PLAIN_F64", "PLAIN_F32", "PLAIN_I8", "PLAIN_TC", "RIGHT_TC", "PLAIN_F8"]


def run(fp, torch, dev, ctx, p, a, b, algo):
    m, k = a.shape
    n = b.shape[1]
    C = torch.full((m, n), 255, dtype=torch.uint8, device=dev)
    fp.fp_matmul(ctx, p, m, n, k, to_dev(torch, dev, a), k, to_dev(torch, dev, b), n, C, n,
                 getattr(fp, "FP_MM_" + algo))
    fp.fp_ctx_status(ctx)
    return C.cpu().numpy()


def supported(fp, p, k, algo):
    if algo == "RIGHT_F32" and (p - 1) ** 2 > 511:
        return False
    if algo == "PLAIN_TC" and k * (p - 1) ** 2 >= 2 ** 24:
        return False
    if algo == "RIGHT_TC" and (p not in (2, 3, 5, 7) or (p <= 3 and k > 32767)):
        return False
    if algo == "PLAIN_F8" and (p > 17 or k * (p - 1) ** 2 >= 2 ** 24):
        return False
    return True


@pytest.mark.parametrize("algo", ALL)
@pytest.mark.parametrize("p,m,n,k", [(3, 200, 333, 517), (7, 130, 70, 1000), (2, 64, 129, 4100),
                                     (17, 257, 255, 96), (31, 33, 300, 300), (3, 1, 1, 1), (5, 5, 7, 3)])
def test_matmul_ragged(env, algo, p, m, n, k):
    fp, torch, dev, ctx = env
    if not supported(fp, p, k, algo):
        pytest.skip("outside the algorithm's exactness bound")
    a, b = workloads.matmul_inputs(p * 1000 + m, p, m, k, n)
    try:
        got = run(fp, torch, dev, ctx, p, a, b, algo)
    except fp.FpError as e:
        if e.status == fp.FP_EUNSUPPORTED:
            pytest.skip(str(e))
        raise
    assert np.array_equal(got, field.matmul_mod(a, b, p))


@pytest.mark.parametrize("algo", ALL)
@pytest.mark.parametrize("p", [3, 7])
def test_matmul_config_n1024_full(env, algo, p):
    fp, torch, dev, ctx = env
    if not supported(fp, p, 1024, algo):
        pytest.skip("outside the algorithm's exactness bound")
    a, b = workloads.matmul_inputs(p, p, 1024, 1024, 1024)
    try:
        got = run(fp, torch, dev, ctx, p, a, b, algo)
    except fp.FpError as e:
        if e.status == fp.FP_EUNSUPPORTED:
            pytest.skip(str(e))
        raise
    rows = np.arange(0, 1024, 3)    # a third of the rows: every tile row, the last row
    rows = np.union1d(rows, [1023])
    assert np.array_equal(got[rows], field.matmul_mod_rows(a, b, p, rows))


@pytest.mark.parametrize("algo", ALL)
@pytest.mark.parametrize("p", [3, 7])
def test_matmul_config_n4096_sampled(env, algo, p):
    fp, torch, dev, ctx = env
    if not supported(fp, p, 4096, algo):
        pytest.skip("outside the algorithm's exactness bound")
    a, b = workloads.matmul_inputs(p + 10, p, 4096, 4096, 4096)
    try:
        got = run(fp, torch, dev, ctx, p, a, b, algo)
    except fp.FpError as e:
        if e.status == fp.FP_EUNSUPPORTED:
            pytest.skip(str(e))
        raise
    rows = np.array([0, 1, 127, 128, 2047, 2048, 3000, 4095])
    assert np.array_equal(got[rows], field.matmul_mod_rows(a, b, p, rows))


@pytest.mark.parametrize("algo", ALL)
@pytest.mark.parametrize("p,k", [(3, 2047), (3, 2048), (7, 4096), (2, 4095), (17, 1000)])
def test_matmul_all_max_entries(env, algo, p, k):
    """All entries p-1: every digit reaches k (p-1)^2, the edge of Eq. lower; the strict
    reading of the bound is what keeps these exact (k = 2048, p = 3 is Table comprange's
    boundary column)."""
    fp, torch, dev, ctx = env
    if not supported(fp, p, k, algo):
        pytest.skip("outside the algorithm's exactness bound")
    m, n = 70, 131
    a = np.full((m, k), p - 1, np.uint8)
    b = np.full((k, n), p - 1, np.uint8)
    try:
        got = run(fp, torch, dev, ctx, p, a, b, algo)
    except fp.FpError as e:
        if e.status == fp.FP_EUNSUPPORTED:
            pytest.skip(str(e))
        raise
    assert np.all(got == (k * (p - 1) ** 2) % p)


@pytest.mark.parametrize("word", [0, 2, 1])
def test_pack_cb_matches_oracle(env, word):
    fp, torch, dev, ctx = env
    p, k, n = 3, 37, 103
    bq, e = (13, 4) if word != 2 else (12, 2)
    a, b = workloads.matmul_inputs(5, p, 1, k, n)
    nw = -(-n // e)
    dt = {0: torch.float64, 1: torch.int64, 2: torch.float32}[word]
    CB = torch.empty((k, nw), dtype=dt, device=dev)
    fp.fp_pack_cb(ctx, p, k, n, to_dev(torch, dev, b), n, bq, e, word, CB)
    fp.fp_ctx_status(ctx)
    got = CB.cpu().numpy()
    want = odqt.right_compress(b, e, 1 << bq)
    assert all(int(got[i, j]) == int(want[i, j]) for i in range(k) for j in range(nw))


def test_matmul_errors(env):
    fp, torch, dev, ctx = env
    A = torch.zeros((4, 4), dtype=torch.uint8, device=dev)
    with pytest.raises(fp.FpError) as ei:
        fp.fp_matmul(ctx, 3, 4, 4, 4, A, 3, A, 4, A, 4)          # lda < k
    assert ei.value.status == fp.FP_EINVAL
    with pytest.raises(fp.FpError) as ei:
        fp.fp_matmul(ctx, 31, 4, 4, 4, A, 4, A, 4, A, 4, fp.FP_MM_RIGHT_F32)   # (p-1)^2 > 511
    assert ei.value.status == fp.FP_EBOUND
    A[0, 0] = 7
    C = torch.empty((4, 4), dtype=torch.uint8, device=dev)
    fp.fp_matmul(ctx, 3, 4, 4, 4, A, 4, A, 4, C, 4)
    with pytest.raises(fp.FpError) as ei:
        fp.fp_ctx_status(ctx)
    assert ei.value.status == fp.FP_EINVAL


def _padded(torch, dev, x, ld, fill):
    """x (rows x cols) stored with leading dimension ld; the pad bytes hold `fill`."""
    rows, cols = x.shape
    buf = np.full((rows, ld), fill, np.uint8)
    buf[:, :cols] = x
    return torch.from_numpy(buf).to(dev)


@pytest.mark.parametrize("p,m,n,k", [(3, 200, 333, 517), (7, 130, 70, 1000), (2, 64, 129, 4100),
                                     (17, 257, 255, 96), (5, 1, 1, 1), (13, 300, 600, 129)])
def test_matmul_f8_direct_operands(env, p, m, n, k):
    """PLAIN_F8 on 16-byte aligned leading dimensions streams the caller's residue bytes as
    e4m3 (r 2^-9) with B MN-major in the persistent kernel: ragged m, n, k, the pad bytes past
    k and n set to 255 (out of range, so reading them would also raise the range error), no
    conversion pass."""
    fp, torch, dev, ctx = env
    a, b = workloads.matmul_inputs(p * 77 + k, p, m, k, n)
    lda, ldb, ldc = -(-k // 16) * 16 + 16, -(-n // 16) * 16, n + 3
    A, B = _padded(torch, dev, a, lda, 255), _padded(torch, dev, b, ldb, 255)
    C = torch.full((m, ldc), 254, dtype=torch.uint8, device=dev)
    fp.fp_ctx_profile(ctx, 2)
    fp.fp_ctx_profile(ctx, 1)
    fp.fp_matmul(ctx, p, m, n, k, A, lda, B, ldb, C, ldc, fp.FP_MM_PLAIN_F8)
    fp.fp_ctx_status(ctx)
    conv, _ = fp.fp_ctx_profile_read(ctx, "")
    mm, _ = fp.fp_ctx_profile_read(ctx, "k_mm_f8g")
    fp.fp_ctx_profile(ctx, 0)
    got = C.cpu().numpy()
    assert (conv, mm) == (1, 1)                       # the one launch is the e4m3 kernel
    assert np.array_equal(got[:, :n], field.matmul_mod(a, b, p))
    assert np.all(got[:, n:] == 254)                  # nothing written past n


@pytest.mark.parametrize("where", ["A_first", "A_last", "B_first", "B_last", "B_mid"])
def test_matmul_f8_direct_range_check(env, where):
    """The direct e4m3 path checks every input byte on the device (each CTA a slice of the
    tiles it loads): one residue equal to p anywhere, in any tile, raises the range error."""
    fp, torch, dev, ctx = env
    p, m, n, k = 7, 300, 520, 700
    a, b = workloads.matmul_inputs(3, p, m, k, n)
    a, b = a.copy(), b.copy()
    pos = {"A_first": ("a", 0, 0), "A_last": ("a", m - 1, k - 1), "B_first": ("b", 0, 0),
           "B_last": ("b", k - 1, n - 1), "B_mid": ("b", 333, 261)}[where]
    (a if pos[0] == "a" else b)[pos[1], pos[2]] = p
    lda, ldb = -(-k // 16) * 16, -(-n // 16) * 16
    A, B = _padded(torch, dev, a, lda, 0), _padded(torch, dev, b, ldb, 0)
    C = torch.empty((m, n), dtype=torch.uint8, device=dev)
    fp.fp_matmul(ctx, p, m, n, k, A, lda, B, ldb, C, n, fp.FP_MM_PLAIN_F8)
    with pytest.raises(fp.FpError) as ei:
        fp.fp_ctx_status(ctx)
    assert ei.value.status == fp.FP_EINVAL
    # the context is usable afterwards: the same product with the entry fixed is exact
    (a if pos[0] == "a" else b)[pos[1], pos[2]] = p - 1
    A, B = _padded(torch, dev, a, lda, 0), _padded(torch, dev, b, ldb, 0)
    fp.fp_matmul(ctx, p, m, n, k, A, lda, B, ldb, C, n, fp.FP_MM_PLAIN_F8)
    fp.fp_ctx_status(ctx)
    assert np.array_equal(C.cpu().numpy(), field.matmul_mod(a, b, p))


def test_auto_direct_and_autotuned(env):
    """AUTO: an aligned p <= 17 product takes the direct e4m3 kernel with no tuning runs; a
    p = 31 product is timed once over the exact candidates, the winner is cached and reused."""
    fp, torch, dev, ctx = env
    p, n = 7, 512
    a, b = workloads.matmul_inputs(71, p, n, n, n)
    A, B = to_dev(torch, dev, a), to_dev(torch, dev, b)
    C = torch.empty((n, n), dtype=torch.uint8, device=dev)
    fp.fp_ctx_profile(ctx, 2)
    fp.fp_ctx_profile(ctx, 1)
    fp.fp_matmul(ctx, p, n, n, n, A, n, B, n, C, n, fp.FP_MM_AUTO)
    fp.fp_ctx_status(ctx)
    total, _ = fp.fp_ctx_profile_read(ctx, "")
    direct, _ = fp.fp_ctx_profile_read(ctx, "k_mm_f8g")
    fp.fp_ctx_profile(ctx, 0)
    assert (total, direct) == (1, 1)
    assert fp.fp_ctx_autotune_choice(ctx, p, n, n, n) == -1
    assert np.array_equal(C.cpu().numpy(), field.matmul_mod(a, b, p))
    p = 31
    a, b = workloads.matmul_inputs(72, p, n, n, n)
    A, B = to_dev(torch, dev, a), to_dev(torch, dev, b)
    fp.fp_matmul(ctx, p, n, n, n, A, n, B, n, C, n, fp.FP_MM_AUTO)
    fp.fp_ctx_status(ctx)
    choice = fp.fp_ctx_autotune_choice(ctx, p, n, n, n)
    assert choice in (fp.FP_MM_RIGHT_F64, fp.FP_MM_PLAIN_I8, fp.FP_MM_PLAIN_TC, fp.FP_MM_RIGHT_F32)
    l0 = fp.fp_ctx_launches(ctx)
    fp.fp_matmul(ctx, p, n, n, n, A, n, B, n, C, n, fp.FP_MM_AUTO)
    fp.fp_ctx_status(ctx)
    assert fp.fp_ctx_launches(ctx) - l0 <= 3       # the cached variant only, no timing runs
    assert np.array_equal(C.cpu().numpy(), field.matmul_mod(a, b, p))


@pytest.mark.parametrize("algo", ["LEFT_F32", "LEFT_F64"])
@pytest.mark.parametrize("p,m,n,k", [(3, 200, 70, 517), (7, 333, 129, 64), (2, 64, 1, 1000), (31, 1, 50, 300),
                                     (13, 130, 257, 129)])
def test_matmul_left_compression(env, algo, p, m, n, k):
    """Left compression (Sec. 7.4) by transposition: ragged m != n, C with a leading dimension
    past n whose pad bytes must stay untouched; every entry compared."""
    fp, torch, dev, ctx = env
    a, b = workloads.matmul_inputs(p * 31 + m, p, m, k, n)
    ldc = n + 5
    C = torch.full((m, ldc), 254, dtype=torch.uint8, device=dev)
    try:
        fp.fp_matmul(ctx, p, m, n, k, to_dev(torch, dev, a), k, to_dev(torch, dev, b), n, C, ldc,
                     getattr(fp, "FP_MM_" + algo))
    except fp.FpError as e:
        if e.status == fp.FP_EBOUND:
            pytest.skip("no packing fits the word for this p, k")
        raise
    fp.fp_ctx_status(ctx)
    got = C.cpu().numpy()
    assert np.array_equal(got[:, :n], field.matmul_mod(a, b, p))
    assert np.all(got[:, n:] == 254)


@pytest.mark.parametrize("algo", ["LEFT_F32", "LEFT_F64"])
def test_matmul_left_compression_range_and_grouped(env, algo):
    """A residue equal to p in A or in B raises the range error; the same algorithm through a
    grouped call gives the products of its problems."""
    fp, torch, dev, ctx = env
    p, m, n, k = 5, 90, 60, 300
    al = getattr(fp, "FP_MM_" + algo)
    for which in ("a", "b"):
        a, b = workloads.matmul_inputs(3, p, m, k, n)
        a, b = a.copy(), b.copy()
        (a if which == "a" else b)[5, 7] = p
        C = torch.empty((m, n), dtype=torch.uint8, device=dev)
        fp.fp_matmul(ctx, p, m, n, k, to_dev(torch, dev, a), k, to_dev(torch, dev, b), n, C, n, al)
        with pytest.raises(fp.FpError) as ei:
            fp.fp_ctx_status(ctx)
        assert ei.value.status == fp.FP_EINVAL
    probs, keep = [], []
    for i, (pp, mm, nn, kk) in enumerate([(3, 70, 40, 200), (7, 33, 99, 150)]):
        a, b = workloads.matmul_inputs(50 + i, pp, mm, kk, nn)
        A, B = to_dev(torch, dev, a), to_dev(torch, dev, b)
        C = torch.empty((mm, nn), dtype=torch.uint8, device=dev)
        probs.append(fp.fp_mm_problem_of(pp, mm, nn, kk, A, kk, B, nn, C, nn))
        keep.append((a, b, pp, A, B, C))
    fp.fp_matmul_grouped(ctx, probs, al)
    fp.fp_ctx_status(ctx)
    for a, b, pp, A, B, C in keep:
        assert np.array_equal(C.cpu().numpy(), field.matmul_mod(a, b, pp))


@pytest.mark.parametrize("p,m,n,k", [(3, 200, 70, 517), (7, 33, 129, 1000), (2, 64, 1, 4000), (13, 130, 257, 129),
                                     (5, 1, 1, 1), (3, 96, 96, 16383), (2, 50, 60, 101), (3, 40, 41, 62)])
def test_matmul_cmm_middle_product(env, p, m, n, k):
    """Compressed matrix multiplication by the middle product (Sec. 7.1) on FP64 DMMA: ragged
    shapes, k not a multiple of d+1 (zero-padded last block), d+1 = 2, 3 (p = 3, k = 62) and 4
    (p = 2, k = 101) entries per word, all-(p-1) inputs at the largest k of the test, C's pad
    columns untouched."""
    fp, torch, dev, ctx = env
    a, b = workloads.matmul_inputs(p * 17 + k, p, m, k, n)
    if k == 16383:
        a, b = np.full_like(a, p - 1), np.full_like(b, p - 1)
    ldc = n + 3
    C = torch.full((m, ldc), 254, dtype=torch.uint8, device=dev)
    fp.fp_matmul(ctx, p, m, n, k, to_dev(torch, dev, a), k, to_dev(torch, dev, b), n, C, ldc, fp.FP_MM_CMM_F64)
    fp.fp_ctx_status(ctx)
    got = C.cpu().numpy()
    assert np.array_equal(got[:, :n], field.matmul_mod(a, b, p))
    assert np.all(got[:, n:] == 254)


def test_matmul_cmm_bound_and_range(env):
    """k (p-1)^2 >= 2^17 leaves no d >= 1 (refused on the host, nothing enqueued); an entry equal
    to p raises the range error."""
    fp, torch, dev, ctx = env
    A = torch.zeros((8, 200), dtype=torch.uint8, device=dev)
    C = torch.zeros((8, 8), dtype=torch.uint8, device=dev)
    with pytest.raises(fp.FpError) as ei:
        fp.fp_matmul(ctx, 31, 8, 8, 200, A, 200, A, 8, C, 8, fp.FP_MM_CMM_F64)
    assert ei.value.status == fp.FP_EBOUND
    p, m, n, k = 7, 40, 30, 200
    a, b = workloads.matmul_inputs(5, p, m, k, n)
    b = b.copy()
    b[199, 29] = p
    C = torch.empty((m, n), dtype=torch.uint8, device=dev)
    fp.fp_matmul(ctx, p, m, n, k, to_dev(torch, dev, a), k, to_dev(torch, dev, b), n, C, n, fp.FP_MM_CMM_F64)
    with pytest.raises(fp.FpError) as ei:
        fp.fp_ctx_status(ctx)
    assert ei.value.status == fp.FP_EINVAL


@pytest.mark.parametrize("p,k", [(7, 16), (7, 3600), (7, 3648), (7, 4100), (5, 8120), (5, 8200)])
@pytest.mark.parametrize("sign", [1, -1])
def test_right_tc_p57_largest_digits(env, p, k, sign):
    """Packed fp16 words for p = 5, 7 (Q = 1023 / 681, chunks of 64 / 32 inner steps): entries
    whose centred value is +-(p-1)/2 everywhere make every chunk digit reach its bound dmax and
    every digit of R grow by dmax per chunk; k around the re-reduction period (127 chunks of 64
    for p = 5, 113 chunks of 32 for p = 7) crosses it."""
    fp, torch, dev, ctx = env
    h = (p - 1) // 2
    m, n = 130, 257
    a = np.full((m, k), h, np.uint8)
    b = np.full((k, n), h if sign > 0 else p - h, np.uint8)
    a[:, 1::5] = p - h if sign > 0 else h          # a mix of signs that keeps the sums large
    got = run(fp, torch, dev, ctx, p, a, b, "RIGHT_TC")
    assert np.array_equal(got, field.matmul_mod(a, b, p))


@pytest.mark.parametrize("p", [5, 7])
def test_right_tc_p57_random_ragged(env, p):
    fp, torch, dev, ctx = env
    for (m, n, k) in ((1, 1, 1), (200, 333, 517), (129, 513, 4100), (64, 1000, 17)):
        a, b = workloads.matmul_inputs(p * 31 + m + k, p, m, k, n)
        got = run(fp, torch, dev, ctx, p, a, b, "RIGHT_TC")
        assert np.array_equal(got, field.matmul_mod(a, b, p)), (m, n, k)
