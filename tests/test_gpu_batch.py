"""GPU parity of the uneven batch (matmul and dot instances of mixed p and size: the large
products on the tensor-core kernels, the rest in one persistent launch): every result bit-exact
against the oracle, and identical to the same instance run alone through fp_matmul / fp_dot."""
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


def make_instances(fp, torch, dev, insts):
    bufs, arr = [], []
    for x in insts:
        A = to_dev(torch, dev, x.a)
        B = to_dev(torch, dev, x.b)
        if x.kind == "matmul":
            C = torch.full((x.m, x.n), 255, dtype=torch.uint8, device=dev)
            arr.append(fp.fp_instance(kind=0, p=x.p, m=x.m, n=x.n, k=x.k, reserved=0,
                                      A=A.data_ptr(), B=B.data_ptr(), C=C.data_ptr()))
        else:
            C = torch.full((4,), 255, dtype=torch.uint8, device=dev)
            arr.append(fp.fp_instance(kind=1, p=x.p, m=1, n=1, k=x.k, reserved=0,
                                      A=A.data_ptr(), B=B.data_ptr(), C=C.data_ptr()))
        bufs.append((A, B, C))
    return bufs, arr


def result(x, C):
    if x.kind == "matmul":
        return C.cpu().numpy()
    return int(C.cpu().numpy().view(np.uint32)[0])


def oracle(x):
    return field.matmul_mod(x.a, x.b, x.p) if x.kind == "matmul" else field.dot_mod(x.a, x.b, x.p)


def test_batch_small_uneven(env):
    fp, torch, dev, ctx = env
    insts = workloads.uneven_batch(7, count=96, lo=1, hi=300)
    bufs, arr = make_instances(fp, torch, dev, insts)
    fp.fp_batch_run(ctx, arr)
    fp.fp_ctx_status(ctx)
    for x, (A, B, C) in zip(insts, bufs):
        got = result(x, C)
        assert np.array_equal(got, oracle(x)), (x.kind, x.p, x.m, x.n, x.k)


@pytest.mark.parametrize("p", [2, 3, 5, 7, 17, 31])
def test_batch_ragged_edges_each_p(env, p):
    fp, torch, dev, ctx = env
    shapes = [(1, 1, 1), (1, 65, 33), (65, 1, 700), (63, 129, 449), (130, 255, 896), (64, 64, 32), (3, 7, 2049)]
    g = np.random.default_rng(p)
    insts = []
    for (m, n, k) in shapes:
        x = workloads.Instance("matmul", p, m, k, n)
        x.a = g.integers(0, p, (m, k), dtype=np.uint8)
        x.b = g.integers(0, p, (k, n), dtype=np.uint8)
        insts.append(x)
    for n in (1, 31, 1000):
        x = workloads.Instance("dot", p, 1, n, 1)
        x.a = g.integers(0, p, n, dtype=np.uint8)
        x.b = g.integers(0, p, n, dtype=np.uint8)
        insts.append(x)
    bufs, arr = make_instances(fp, torch, dev, insts)
    fp.fp_batch_run(ctx, arr)
    fp.fp_ctx_status(ctx)
    for x, (A, B, C) in zip(insts, bufs):
        assert np.array_equal(result(x, C), oracle(x)), (x.kind, p, x.m, x.n, x.k)


def test_batch_all_max_entries(env):
    fp, torch, dev, ctx = env
    insts = []
    for p, k in [(3, 2048), (2, 2047), (7, 2048), (31, 2048), (3, 449)]:
        x = workloads.Instance("matmul", p, 70, k, 130)
        x.a = np.full((70, k), p - 1, np.uint8)
        x.b = np.full((k, 130), p - 1, np.uint8)
        insts.append(x)
    bufs, arr = make_instances(fp, torch, dev, insts)
    fp.fp_batch_run(ctx, arr)
    fp.fp_ctx_status(ctx)
    for x, (A, B, C) in zip(insts, bufs):
        assert np.all(result(x, C) == (x.k * (x.p - 1) ** 2) % x.p)


def test_batch_equals_alone_config_sample(env):
    """The uneven-batch configuration (4096 instances, sizes log-uniform in [16, 2048]):
    every instance's result in the batch equals the same instance run alone, and a sample is
    checked against the oracle."""
    fp, torch, dev, ctx = env
    insts = workloads.uneven_batch(11, count=4096)
    bufs, arr = make_instances(fp, torch, dev, insts)
    fp.fp_batch_run(ctx, arr)
    fp.fp_ctx_status(ctx)
    batch_res = [result(x, C) for x, (A, B, C) in zip(insts, bufs)]
    alone = []
    for x, (A, B, C) in zip(insts, bufs):
        if x.kind == "matmul":
            C2 = torch.empty_like(C)
            fp.fp_matmul(ctx, x.p, x.m, x.n, x.k, A, x.k, B, x.n, C2, x.n, fp.FP_MM_PLAIN_TC
                         if x.k * (x.p - 1) ** 2 < 2 ** 24 else fp.FP_MM_PLAIN_I8)
        else:
            C2 = torch.empty_like(C)
            fp.fp_dot(ctx, x.p, A, B, x.k, C2, fp.FP_ALGO_PLAIN)
        alone.append(C2)
    fp.fp_ctx_status(ctx)
    for x, r, C2 in zip(insts, batch_res, alone):
        assert np.array_equal(r, result(x, C2))
    # every instance against the oracle: one sampled row of each product (a different row per
    # instance, across every tile row), every dot product whole; three rows of 24 of them
    g = np.random.default_rng(0)
    for i, x in enumerate(insts):
        if x.kind == "matmul":
            rows = np.array([int(g.integers(0, x.m))])
            assert np.array_equal(batch_res[i][rows], field.matmul_mod_rows(x.a, x.b, x.p, rows)), i
        else:
            assert batch_res[i] == field.dot_mod(x.a, x.b, x.p), i
    for i in g.choice(len(insts), 24, replace=False):
        x = insts[i]
        if x.kind == "matmul":
            rows = np.unique(np.array([0, x.m - 1, x.m // 2]))
            assert np.array_equal(batch_res[i][rows], field.matmul_mod_rows(x.a, x.b, x.p, rows))


def test_batch_captured_in_a_cuda_graph(env):
    """A warm batch captured into a CUDA graph replays its own instances after eager batches of
    other instances (other sizes, so the context's scratch grows) ran on the same context: the
    captured plan and operand copies live in the graph and in scratch that is kept for it."""
    fp, torch, dev, ctx = env
    insts = workloads.uneven_batch(21, count=300, lo=16, hi=700)
    assert any(x.kind == "matmul" and min(x.m, x.n) >= 64 and x.m * x.n * x.k >= 2 ** 21 for x in insts)
    bufs, arr = make_instances(fp, torch, dev, insts)
    fp.fp_batch_run(ctx, arr)                      # warm: scratch sized, packing degrees tuned
    fp.fp_ctx_status(ctx)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        fp.fp_batch_run(ctx, arr)
    for A, B, C in bufs:
        C.fill_(255)
    other = workloads.uneven_batch(22, count=200, lo=200, hi=2048)
    bufs2, arr2 = make_instances(fp, torch, dev, other)
    fp.fp_batch_run(ctx, arr2)                     # eager, larger: scratch grows, plans differ
    fp.fp_ctx_status(ctx)
    for rep in range(2):
        graph.replay()
        torch.cuda.synchronize()
        fp.fp_ctx_status(ctx)
        for x, (A, B, C) in zip(insts, bufs):
            assert np.array_equal(result(x, C), oracle(x)), (rep, x.kind, x.p, x.m, x.n, x.k)
        for A, B, C in bufs:
            C.fill_(255)
    for i in range(0, len(other), 9):
        x, (A, B, C) = other[i], bufs2[i]
        if x.kind == "matmul":
            rows = np.array([0, x.m - 1])
            assert np.array_equal(result(x, C)[rows], field.matmul_mod_rows(x.a, x.b, x.p, rows))
        else:
            assert result(x, C) == field.dot_mod(x.a, x.b, x.p)
    del graph


def test_batch_capture_refuses_scratch_growth(env):
    """Inside a capture a batch that would need more scratch than the context holds is refused
    (FP_EUNSUPPORTED) instead of freeing and allocating memory."""
    fp, torch, dev, ctx = env
    fresh = fp.fp_ctx_create(0)
    try:
        insts = workloads.uneven_batch(23, count=40, lo=16, hi=300)
        bufs, arr = make_instances(fp, torch, dev, insts)
        graph = torch.cuda.CUDAGraph()
        with pytest.raises(fp.FpError) as ei:
            with torch.cuda.graph(graph):
                fp.fp_batch_run(fresh, arr)
        assert ei.value.status == fp.FP_EUNSUPPORTED
        del graph
        torch.cuda.synchronize()
        fp.fp_batch_run(fresh, arr)               # the same call outside a capture works
        fp.fp_ctx_status(fresh)
        for x, (A, B, C) in zip(insts, bufs):
            assert np.array_equal(result(x, C), oracle(x))
    finally:
        fp.fp_ctx_destroy(fresh)


def test_batch_rejects_bad_instances(env):
    fp, torch, dev, ctx = env
    with pytest.raises(fp.FpError) as ei:
        fp.fp_batch_run(ctx, [fp.fp_instance(kind=0, p=4, m=1, n=1, k=1, reserved=0, A=1, B=1, C=1)])
    assert ei.value.status == fp.FP_EINVAL
    with pytest.raises(fp.FpError) as ei:
        fp.fp_batch_run(ctx, [fp.fp_instance(kind=0, p=3, m=1, n=1, k=1, reserved=0, A=0, B=1, C=1)])
    assert ei.value.status == fp.FP_EINVAL


def _mm(p, m, k, n, seed):
    g = np.random.default_rng(seed)
    x = workloads.Instance("matmul", p, m, k, n)
    x.a = g.integers(0, p, (m, k), dtype=np.uint8)
    x.b = g.integers(0, p, (k, n), dtype=np.uint8)
    return x


@pytest.mark.parametrize("off_a,off_b", [(0, 0), (1, 2), (3, 1), (2, 3)])
def test_batch_tensor_core_share_unaligned(env, off_a, off_b):
    """Large products with p <= 31 run on the e4m3 kernel after their operands are laid out as
    swizzled tiles of centred residues, those with 31 < p <= 127 on the bf16 kernel after a
    conversion; operands starting 1-3 bytes past an aligned address and inner dimensions / widths
    that are not multiples of 4 exercise every shift of those copies (k (p-1)^2 up to 0.86 x 2^24
    for p = 61).  Mixed with products (p = 131, small shapes) and dots that stay on the batch kernel;
    every entry compared."""
    fp, torch, dev, ctx = env
    shapes = [(3, 130, 449, 257), (17, 200, 1021, 67), (5, 64, 512, 64), (2, 333, 2047, 129), (7, 96, 33, 700),
              (31, 150, 300, 200), (3, 40, 900, 900), (127, 100, 500, 90), (61, 64, 4000, 64), (131, 80, 700, 80)]
    insts = [_mm(p, m, k, n, 100 + i) for i, (p, m, k, n) in enumerate(shapes)]
    d = workloads.Instance("dot", 7, 1, 999, 1)
    g = np.random.default_rng(5)
    d.a = g.integers(0, 7, 999, dtype=np.uint8)
    d.b = g.integers(0, 7, 999, dtype=np.uint8)
    insts.append(d)
    bufs, arr = [], []
    for x in insts:
        if x.kind == "matmul":
            ra = torch.zeros(x.a.size + 16, dtype=torch.uint8, device=dev)
            rb = torch.zeros(x.b.size + 16, dtype=torch.uint8, device=dev)
            A = ra[off_a:off_a + x.a.size]
            B = rb[off_b:off_b + x.b.size]
            A.copy_(torch.from_numpy(x.a.reshape(-1)).to(dev))
            B.copy_(torch.from_numpy(x.b.reshape(-1)).to(dev))
            C = torch.full((x.m, x.n), 255, dtype=torch.uint8, device=dev)
            arr.append(fp.fp_instance(kind=0, p=x.p, m=x.m, n=x.n, k=x.k, reserved=0,
                                      A=A.data_ptr(), B=B.data_ptr(), C=C.data_ptr()))
        else:
            A, B = to_dev(torch, dev, x.a), to_dev(torch, dev, x.b)
            C = torch.full((4,), 255, dtype=torch.uint8, device=dev)
            arr.append(fp.fp_instance(kind=1, p=x.p, m=1, n=1, k=x.k, reserved=0,
                                      A=A.data_ptr(), B=B.data_ptr(), C=C.data_ptr()))
        bufs.append((A, B, C))
    fp.fp_batch_run(ctx, arr)
    fp.fp_ctx_status(ctx)
    for x, (A, B, C) in zip(insts, bufs):
        assert np.array_equal(result(x, C), oracle(x)), (x.kind, x.p, x.m, x.n, x.k)


@pytest.mark.parametrize("p,where", [(5, "a"), (31, "a"), (31, "b"), (127, "b")])
def test_batch_tensor_core_share_range_error(env, p, where):
    """An entry equal to p inside a product routed to the tensor cores (e4m3 for p = 5, 31, bf16
    for p = 127) raises the range error."""
    fp, torch, dev, ctx = env
    x = _mm(p, 128, 300, 129, 7)
    if where == "a":
        x.a = x.a.copy()
        x.a[77, 250] = p
    else:
        x.b = x.b.copy()
        x.b[299, 128] = p
    bufs, arr = make_instances(fp, torch, dev, [x, _mm(3, 10, 10, 10, 8)])
    fp.fp_batch_run(ctx, arr)
    with pytest.raises(fp.FpError) as ei:
        fp.fp_ctx_status(ctx)
    assert ei.value.status == fp.FP_EINVAL


def test_batch_invalid_instance_enqueues_nothing(env):
    """A rejected instance anywhere in the batch: the call fails before any launch, so the
    outputs of the valid instances (including one bound for the tensor cores) stay untouched."""
    fp, torch, dev, ctx = env
    good = [_mm(3, 256, 256, 256, 9), _mm(7, 20, 20, 20, 10)]
    bufs, arr = make_instances(fp, torch, dev, good)
    bad = fp.fp_instance(kind=0, p=9, m=4, n=4, k=4, reserved=0, A=arr[0].A, B=arr[0].B, C=arr[0].C)
    with pytest.raises(fp.FpError) as ei:
        fp.fp_batch_run(ctx, arr + [bad])
    assert ei.value.status == fp.FP_EINVAL
    torch.cuda.synchronize()
    fp.fp_ctx_status(ctx)
    for A, B, C in bufs:
        assert int(C.min().item()) == 255 and int(C.max().item()) == 255


def _mm_const(p, m, k, n, ra, rb):
    x = workloads.Instance("matmul", p, m, k, n)
    x.a = np.full((m, k), ra, dtype=np.uint8)
    x.b = np.full((k, n), rb, dtype=np.uint8)
    return x


@pytest.mark.parametrize("k", [2, 31, 32, 33, 97, 127, 128, 129, 255, 385])
def test_batch_pretiled_ragged_inner(env, k):
    """The e4m3 share at inner lengths around the 128-byte k tile and its four K = 32 steps (the
    last k tile issues only the steps that hold some of k, the rest of the tile is zero): ragged
    row and column blocks, every entry against the oracle."""
    fp, torch, dev, ctx = env
    m, n = (1400, 1500) if k < 40 else (200, 330)
    assert m * n * k >= 2 ** 21
    x = _mm(7, m, k, n, 1000 + k)
    bufs, arr = make_instances(fp, torch, dev, [x])
    fp.fp_batch_run(ctx, arr)
    fp.fp_ctx_status(ctx)
    assert np.array_equal(result(x, bufs[0][2]), oracle(x))


@pytest.mark.parametrize("ra,rb", [(15, 15), (15, 16), (16, 16), (30, 30), (0, 17)])
@pytest.mark.parametrize("k", [18641, 18642])
def test_batch_pretiled_fdiv_bound_p31(env, ra, rb, k):
    """p = 31 at the largest k the e4m3 route takes (2 k 15^2 + 31 < 2^23 holds for k = 18641, not
    for 18642, which goes elsewhere): all entries of A equal ra and of B rb, so the centred
    values +-15 (or -1) make every sum +-k 225 (or k), the ends of FDIV's range once the offset
    is added.  Every entry equals k ra rb mod 31."""
    fp, torch, dev, ctx = env
    p, m, n = 31, 64, 70
    x = _mm_const(p, m, k, n, ra, rb)
    bufs, arr = make_instances(fp, torch, dev, [x])
    fp.fp_batch_run(ctx, arr)
    fp.fp_ctx_status(ctx)
    assert np.array_equal(result(x, bufs[0][2]), np.full((m, n), k * ra * rb % p, dtype=np.uint8))


def test_batch_pretiled_more_than_one_launch(env):
    """4100 products routed to the e4m3 kernel (64 x 512 x 64, p cycling over the primes up to
    31): the share takes two launches (4096 + 4 products).  The first and last rows of every
    product against the oracle, all of the products around the boundary in full."""
    fp, torch, dev, ctx = env
    primes = [2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31]
    insts = [_mm(primes[i % len(primes)], 64, 512, 64, 20000 + i) for i in range(4100)]
    bufs, arr = make_instances(fp, torch, dev, insts)
    fp.fp_batch_run(ctx, arr)
    fp.fp_ctx_status(ctx)
    rows = np.array([0, 63])
    for i, (x, (A, B, C)) in enumerate(zip(insts, bufs)):
        got = result(x, C)
        if 4090 <= i or i < 4:
            assert np.array_equal(got, oracle(x)), i
        else:
            assert np.array_equal(got[rows], field.matmul_mod_rows(x.a, x.b, x.p, rows)), i


@pytest.mark.parametrize("m,n,k", [(8, 256, 1024), (20, 1500, 300), (1500, 17, 700), (63, 63, 2048), (4, 2048, 512)])
def test_batch_pretiled_thin_products(env, m, n, k):
    """Products with fewer than 64 rows or columns whose 128 x 256 x 32-padded MACs are at most 32
    times their own run on the e4m3 kernel (most of each tile is zero padding); every entry
    against the oracle, alone and beside a product that fills its tiles."""
    fp, torch, dev, ctx = env
    pad = -(-m // 128) * 128 * -(-n // 256) * 256 * -(-k // 32) * 32
    assert 2 ** 21 <= pad <= 32 * m * n * k
    insts = [_mm(13, m, k, n, m * 7 + n), _mm(29, 300, 400, 500, 3)]
    bufs, arr = make_instances(fp, torch, dev, insts)
    fp.fp_batch_run(ctx, arr)
    fp.fp_ctx_status(ctx)
    for x, (A, B, C) in zip(insts, bufs):
        assert np.array_equal(result(x, C), oracle(x)), (x.p, x.m, x.n, x.k)


@pytest.mark.parametrize("k", [32767, 32768])
@pytest.mark.parametrize("r", [16, 9, 8])
def test_batch_pretiled_unsigned_to_centred_p17(env, k, r):
    """p = 17: residues go to the e4m3 kernel as they stand while k 16^2 < 2^23 (k = 32767, every
    sum up to 32767 x 256, just below FDIV's 2^23), centred past it (k = 32768: 16 -> -1, 9 -> -8).
    All entries of A and B equal r; every entry equals k r^2 mod 17."""
    fp, torch, dev, ctx = env
    p, m, n = 17, 64, 80
    x = _mm_const(p, m, k, n, r, r)
    bufs, arr = make_instances(fp, torch, dev, [x])
    fp.fp_batch_run(ctx, arr)
    fp.fp_ctx_status(ctx)
    assert np.array_equal(result(x, bufs[0][2]), np.full((m, n), k * r * r % p, dtype=np.uint8))
