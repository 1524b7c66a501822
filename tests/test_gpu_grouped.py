"""GPU parity of fp_matmul_grouped (several independent products C_i = A_i B_i mod p_i in
persistent tensor-core launches) against the oracle, bit-exact: mixed groups where some
problems take the grouped e4m3 kernel and others the single-product path, more problems than
one launch holds, many tiles per CTA (both accumulator buffers reused many times), the
exactness edge k (p-1)^2 just below 2^24, range errors, and host-side argument checks."""
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


def _store(torch, dev, x, ld, fill=0):
    rows, cols = x.shape
    buf = np.full((rows, ld), fill, np.uint8)
    buf[:, :cols] = x
    return torch.from_numpy(buf).to(dev)


class Prob:
    """One product with its device buffers; `align` picks leading dimensions that are (or are
    not) multiples of 16."""

    def __init__(self, fp, torch, dev, seed, p, m, n, k, align=True, pad_fill=255):
        self.p, self.m, self.n, self.k = p, m, n, k
        self.a, self.b = workloads.matmul_inputs(seed, p, m, k, n)
        r16 = lambda x: -(-x // 16) * 16
        self.lda = r16(k) if align else k
        self.ldb = r16(n) if align else n
        self.ldc = n + 5
        self.A = _store(torch, dev, self.a, self.lda, pad_fill if self.lda > k else 0)
        self.B = _store(torch, dev, self.b, self.ldb, pad_fill if self.ldb > n else 0)
        self.C = torch.full((m, self.ldc), 253, dtype=torch.uint8, device=dev)
        self.desc = fp.fp_mm_problem_of(p, m, n, k, self.A, self.lda, self.B, self.ldb, self.C, self.ldc)

    def check(self, rows=None):
        got = self.C.cpu().numpy()
        assert np.all(got[:, self.n:] == 253)
        if rows is None:
            assert np.array_equal(got[:, :self.n], field.matmul_mod(self.a, self.b, self.p))
        else:
            assert np.array_equal(got[rows, :self.n], field.matmul_mod_rows(self.a, self.b, self.p, rows))


def _launches(fp, ctx, fn):
    fp.fp_ctx_profile(ctx, 2)
    fp.fp_ctx_profile(ctx, 1)
    fn()
    fp.fp_ctx_status(ctx)
    out = {name: fp.fp_ctx_profile_read(ctx, name)[0] for name in ("k_mm_f8g", "")}
    fp.fp_ctx_profile(ctx, 0)
    return out


def test_grouped_mixed(env):
    """Eligible problems (p <= 17, aligned) share one launch; p = 31, an unaligned layout and
    p = 17 beyond the fp8 bound go through fp_matmul (AUTO) one by one; every result is exact."""
    fp, torch, dev, ctx = env
    probs = [Prob(fp, torch, dev, 1, 3, 200, 333, 517), Prob(fp, torch, dev, 2, 7, 130, 70, 1000),
             Prob(fp, torch, dev, 3, 2, 64, 129, 4100), Prob(fp, torch, dev, 4, 17, 257, 255, 96),
             Prob(fp, torch, dev, 5, 31, 33, 300, 300), Prob(fp, torch, dev, 6, 5, 77, 91, 333, align=False),
             Prob(fp, torch, dev, 7, 13, 1, 1, 1), Prob(fp, torch, dev, 8, 17, 40, 50, 70000)]
    n = _launches(fp, ctx, lambda: fp.fp_matmul_grouped(ctx, [q.desc for q in probs]))
    assert n["k_mm_f8g"] == 2          # the group, and the unaligned p = 5 product (padded copy)
    for q in probs:
        q.check()


def test_grouped_more_than_one_launch(env):
    """More problems than one launch holds: ceil(count / FP_GROUP_MAX) launches."""
    fp, torch, dev, ctx = env
    cnt = fp.FP_GROUP_MAX + 5
    rng = np.random.default_rng(11)
    primes = [2, 3, 5, 7, 11, 13, 17]
    probs = [Prob(fp, torch, dev, 100 + i, primes[i % 7], int(rng.integers(1, 300)), int(rng.integers(1, 600)),
                  int(rng.integers(1, 900))) for i in range(cnt)]
    n = _launches(fp, ctx, lambda: fp.fp_matmul_grouped(ctx, [q.desc for q in probs], fp.FP_MM_PLAIN_F8))
    assert n["k_mm_f8g"] == 2 and n[""] == 2         # nothing but the two grouped launches
    for q in probs:
        q.check()


def test_grouped_benchmark_configuration(env):
    """The four products of the benchmark (p in {3, 7} x n in {1024, 4096}) in one launch:
    full comparison at n = 1024, sampled rows (every tile row boundary) at n = 4096."""
    fp, torch, dev, ctx = env
    probs = [Prob(fp, torch, dev, 21, 3, 1024, 1024, 1024), Prob(fp, torch, dev, 22, 7, 1024, 1024, 1024),
             Prob(fp, torch, dev, 23, 3, 4096, 4096, 4096), Prob(fp, torch, dev, 24, 7, 4096, 4096, 4096)]
    n = _launches(fp, ctx, lambda: fp.fp_matmul_grouped(ctx, [q.desc for q in probs]))
    assert n["k_mm_f8g"] == 1
    probs[0].check()
    probs[1].check()
    rows = np.array([0, 1, 127, 128, 1000, 2047, 2048, 4095])
    probs[2].check(rows)
    probs[3].check(rows)


def test_grouped_many_tiles_per_cta(env):
    """Short inner dimension, many output tiles: each CTA reuses both TMEM buffers many times
    and the epilogue, not the MMA, sets the pace."""
    fp, torch, dev, ctx = env
    q = Prob(fp, torch, dev, 31, 11, 2048, 8192, 200)
    fp.fp_matmul_grouped(ctx, [q.desc])
    fp.fp_ctx_status(ctx)
    rows = np.array([0, 5, 127, 128, 129, 1023, 1024, 2047])
    q.check(rows)


@pytest.mark.parametrize("p,k", [(17, 65535), (2, 1 << 20), (3, 4194303), (17, 32767), (17, 32768), (13, 58253)])
def test_grouped_exactness_edge(env, p, k):
    """All entries p-1 with k (p-1)^2 just below 2^24 (p = 3: k = 2^22 - 1 is beyond the
    fp_matmul size limit, so it must be refused): every fp32 sum is the largest exact one.
    k (p-1)^2 = 2^23 - 256 (p = 17, k = 32767) and 2^23 - 176 (p = 13, k = 58253) are at the
    edge of the sums the epilogue reduces by FDIV (Table fdiv case 3 in binary32); 2^23
    (k = 32768) takes the integer reduction."""
    fp, torch, dev, ctx = env
    m, n = 40, 300
    if k > (1 << 20):
        A = torch.zeros((1, 16), dtype=torch.uint8, device=dev)
        d = fp.fp_mm_problem_of(p, 1, 1, k, A, k, A, 16, A, 16)
        with pytest.raises(fp.FpError) as ei:
            fp.fp_matmul_grouped(ctx, [d])
        assert ei.value.status == fp.FP_EINVAL
        return
    lda = -(-k // 16) * 16
    A = torch.full((m, lda), p - 1, dtype=torch.uint8, device=dev)
    B = torch.full((k, 304), p - 1, dtype=torch.uint8, device=dev)
    C = torch.empty((m, n), dtype=torch.uint8, device=dev)
    d = fp.fp_mm_problem_of(p, m, n, k, A, lda, B, 304, C, n)
    n_l = _launches(fp, ctx, lambda: fp.fp_matmul_grouped(ctx, [d]))
    assert n_l["k_mm_f8g"] == 1
    assert np.all(C.cpu().numpy() == (k * (p - 1) ** 2) % p)


def test_grouped_range_error_and_recovery(env):
    fp, torch, dev, ctx = env
    good = Prob(fp, torch, dev, 41, 5, 300, 400, 500)
    bad = Prob(fp, torch, dev, 42, 7, 260, 520, 700)
    bad.b[699, 519] = 7
    bad.B[699, 519] = 7
    fp.fp_matmul_grouped(ctx, [good.desc, bad.desc])
    with pytest.raises(fp.FpError) as ei:
        fp.fp_ctx_status(ctx)
    assert ei.value.status == fp.FP_EINVAL
    bad.b[699, 519] = 6
    bad.B[699, 519] = 6
    fp.fp_matmul_grouped(ctx, [good.desc, bad.desc])
    fp.fp_ctx_status(ctx)
    good.check()
    bad.check()


def test_grouped_host_checks(env):
    fp, torch, dev, ctx = env
    fp.fp_matmul_grouped(ctx, [])                  # no-op
    A = torch.zeros((4, 16), dtype=torch.uint8, device=dev)
    ok = fp.fp_mm_problem_of(3, 4, 4, 4, A, 16, A, 16, A, 16)
    for bad in (fp.fp_mm_problem_of(4, 4, 4, 4, A, 16, A, 16, A, 16),     # p not prime
                fp.fp_mm_problem_of(3, 4, 4, 20, A, 16, A, 16, A, 16),    # lda < k
                fp.fp_mm_problem_of(3, 0, 4, 4, A, 16, A, 16, A, 16)):    # empty
        with pytest.raises(fp.FpError) as ei:
            fp.fp_matmul_grouped(ctx, [ok, bad])
        assert ei.value.status == fp.FP_EINVAL
    with pytest.raises(fp.FpError) as ei:
        fp.fp_matmul_grouped(ctx, [ok], fp.FP_MM_LEFT_F32 + 10)
    assert ei.value.status == fp.FP_EINVAL


def test_grouped_range_check_covers_every_position(env):
    """One out-of-range byte at each of 80 random positions of A and B (one at a time, in a
    group of two products of different shapes): each is caught, so the slices the tiles check
    cover the whole of both inputs, including partial 16-byte chunks at row ends."""
    fp, torch, dev, ctx = env
    other = Prob(fp, torch, dev, 51, 13, 100, 200, 300)
    q = Prob(fp, torch, dev, 52, 11, 300, 600, 333, pad_fill=0)
    rng = np.random.default_rng(5)
    spots = [("A", int(rng.integers(q.m)), int(rng.integers(q.k))) for _ in range(40)] + \
            [("B", int(rng.integers(q.k)), int(rng.integers(q.n))) for _ in range(40)]
    spots += [("A", q.m - 1, q.k - 1), ("B", q.k - 1, q.n - 1), ("A", 0, 0), ("B", 0, 0)]
    for which, r, c in spots:
        T = q.A if which == "A" else q.B
        old = int(T[r, c].item())
        T[r, c] = 200 if r % 2 else q.p
        fp.fp_matmul_grouped(ctx, [other.desc, q.desc])
        with pytest.raises(fp.FpError) as ei:
            fp.fp_ctx_status(ctx)
        assert ei.value.status == fp.FP_EINVAL, (which, r, c)
        T[r, c] = old
    fp.fp_matmul_grouped(ctx, [other.desc, q.desc])
    fp.fp_ctx_status(ctx)
    other.check()
    q.check()


@pytest.mark.parametrize("algo", ["RIGHT_TC", "PLAIN_TC"])
def test_grouped_16bit(env, algo):
    """RIGHT_TC (packed fp16, two residues per MMA column) and PLAIN_TC (bf16) groups: ragged
    shapes, odd n (a last word with one residue), several chunks of 448 inner steps, unaligned
    leading dimensions (the conversions read any layout); one persistent launch each."""
    fp, torch, dev, ctx = env
    if algo == "RIGHT_TC":
        shapes = [(3, 200, 333, 517), (2, 64, 129, 4100), (3, 130, 71, 1000), (3, 1, 1, 1), (2, 257, 600, 448),
                  (3, 100, 513, 449), (7, 130, 257, 4100), (5, 65, 63, 200)]
    else:
        shapes = [(7, 200, 333, 517), (251, 64, 129, 200), (31, 130, 71, 1000), (3, 1, 1, 1), (13, 257, 600, 4096)]
    probs = [Prob(fp, torch, dev, 60 + i, p, m, n, k, align=(i % 2 == 0)) for i, (p, m, n, k) in enumerate(shapes)]
    name = "k_mm_t16_packed" if algo == "RIGHT_TC" else "k_mm_t16_plain"
    fp.fp_ctx_profile(ctx, 2)
    fp.fp_ctx_profile(ctx, 1)
    fp.fp_matmul_grouped(ctx, [q.desc for q in probs], getattr(fp, "FP_MM_" + algo))
    fp.fp_ctx_status(ctx)
    launches, _ = fp.fp_ctx_profile_read(ctx, name)
    fp.fp_ctx_profile(ctx, 0)
    assert launches == (2 if algo == "RIGHT_TC" else 1)     # p <= 3 and p = 5, 7 run in one launch each
    for q in probs:
        q.check()


def test_grouped_bound_refused_before_enqueue(env):
    """A group whose forced algorithm is inexact for one problem (RIGHT_TC with p = 11) is
    refused with FP_EBOUND and nothing runs, not even the problems that would fit."""
    fp, torch, dev, ctx = env
    fine = Prob(fp, torch, dev, 81, 3, 64, 64, 64)
    bad = Prob(fp, torch, dev, 82, 11, 64, 64, 64)
    l0 = fp.fp_ctx_launches(ctx)
    with pytest.raises(fp.FpError) as ei:
        fp.fp_matmul_grouped(ctx, [fine.desc, bad.desc], fp.FP_MM_RIGHT_TC)
    assert ei.value.status == fp.FP_EBOUND
    fp.fp_ctx_status(ctx)
    assert fp.fp_ctx_launches(ctx) == l0
    assert np.all(fine.C.cpu().numpy() == 253)


@pytest.mark.parametrize("c_off", [0, 1, 2, 4])
@pytest.mark.parametrize("ldc_extra", [0, 1, 2, 4, 8, 16])
def test_plain_f8_stores_any_c_alignment(env, c_off, ldc_extra):
    """The e4m3 epilogue stores rows of C 16 bytes per lane when they are 16-byte aligned, else
    4, 2 or 1 bytes per lane as C's address and ldc allow: a product with C starting 0, 1, 2 or 4
    bytes past an aligned address and ldc = n + 0 .. 16 reaches every path, with ragged row and
    column blocks; every entry against the oracle, and nothing written outside the n columns."""
    fp, torch, dev, ctx = env
    p, m, n, k = 7, 150, 304, 208          # A and B rows 16-byte aligned: read in place by TMA
    a, b = workloads.matmul_inputs(900 + c_off * 31 + ldc_extra, p, m, k, n)
    ldc = n + ldc_extra
    A = torch.from_numpy(a).to(dev)
    B = torch.from_numpy(b).to(dev)
    buf = torch.full((c_off + m * ldc + 64,), 251, dtype=torch.uint8, device=dev)
    C = buf[c_off:c_off + m * ldc]
    fp.fp_matmul(ctx, p, m, n, k, A, k, B, n, C, ldc, fp.FP_MM_PLAIN_F8)
    fp.fp_ctx_status(ctx)
    out = buf.cpu().numpy()
    assert (out[:c_off] == 251).all() and (out[c_off + m * ldc:] == 251).all()
    got = out[c_off:c_off + m * ldc].reshape(m, ldc)
    np.testing.assert_array_equal(got[:, :n], field.matmul_mod(a, b, p))
    assert (got[:, n:] == 251).all()
