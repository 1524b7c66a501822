"""GPU parity of GF(p^k) multiplication (Algorithm FGDP, n = 1) and of the modular dot
product against the oracle, bit-exact."""
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


def gf_run(fp, torch, dev, ctx, gf, a, b):
    dt = torch.uint8 if a.dtype == np.uint8 else torch.int16
    A = torch.from_numpy(a.view(np.int16) if a.dtype == np.uint16 else a).to(dev)
    B = torch.from_numpy(b.view(np.int16) if b.dtype == np.uint16 else b).to(dev)
    C = torch.empty(len(a), dtype=dt, device=dev)
    fp.fp_gf_mul_batched(ctx, gf, A, B, C, len(a))
    fp.fp_ctx_status(ctx)
    out = C.cpu().numpy()
    return out.view(np.uint16) if a.dtype == np.uint16 else out


@pytest.mark.parametrize("p,k", [(3, 5), (7, 4), (2, 8), (2, 3), (5, 2), (3, 1), (13, 2), (2, 1)])
def test_gf_mul_matches_oracle(env, p, k):
    fp, torch, dev, ctx = env
    gf = fp.fp_gf_create(ctx, p, k)
    try:
        info = fp.fp_gf_info(gf, k)
        modulus = field.smallest_monic_irreducible(p, k) if k > 1 else [0, 1]
        assert info["modulus"] == modulus
        order = p ** k
        if order * order <= 70000:            # exhaustive: every pair
            a = np.repeat(np.arange(order), order)
            b = np.tile(np.arange(order), order)
        else:
            a, b = workloads.gf_inputs(p + k, p, k, 300001)
        dt = workloads.gf_index_dtype(p, k)
        a, b = a.astype(dt), b.astype(dt)
        got = gf_run(fp, torch, dev, ctx, gf, a, b)
        want = field.gf_mul(a.astype(np.int64), b.astype(np.int64), p, k, modulus)
        assert np.array_equal(got.astype(np.int64), want)
    finally:
        fp.fp_gf_destroy(gf)


@pytest.mark.parametrize("p,k", [(3, 5), (7, 4), (2, 8)])
def test_gf_config_2_24_sampled(env, p, k):
    """2^24 random pairs (the benchmark's batch); every 97th result checked, plus the tail."""
    fp, torch, dev, ctx = env
    n = 1 << 24
    a, b = workloads.gf_inputs(0, p, k, n)
    gf = fp.fp_gf_create(ctx, p, k)
    try:
        got = gf_run(fp, torch, dev, ctx, gf, a, b)
    finally:
        fp.fp_gf_destroy(gf)
    idx = np.union1d(np.arange(0, n, 97), np.arange(n - 64, n))
    m = field.smallest_monic_irreducible(p, k)
    want = field.gf_mul(a[idx].astype(np.int64), b[idx].astype(np.int64), p, k, m)
    assert np.array_equal(got[idx].astype(np.int64), want)


def test_gf_7_4_every_pair(env):
    """GF(7^4): all 2401^2 products (1407 full tiles of the word-level kernel and a ragged tail),
    checked against the oracle in slices."""
    fp, torch, dev, ctx = env
    p, k = 7, 4
    order = p ** k
    a = np.repeat(np.arange(order, dtype=np.uint16), order)
    b = np.tile(np.arange(order, dtype=np.uint16), order)
    gf = fp.fp_gf_create(ctx, p, k)
    try:
        got = gf_run(fp, torch, dev, ctx, gf, a, b)
    finally:
        fp.fp_gf_destroy(gf)
    m = field.smallest_monic_irreducible(p, k)
    step = 600 * order
    for s in range(0, len(a), step):
        want = field.gf_mul(a[s:s + step].astype(np.int64), b[s:s + step].astype(np.int64), p, k, m)
        assert np.array_equal(got[s:s + step].astype(np.int64), want), s


def test_gf_bad_index(env):
    fp, torch, dev, ctx = env
    gf = fp.fp_gf_create(ctx, 3, 5)
    try:
        a = np.array([0, 1, 250, 3], np.uint8)            # 250 >= 243
        with pytest.raises(fp.FpError) as ei:
            gf_run(fp, torch, dev, ctx, gf, a, a)
        assert ei.value.status == fp.FP_EINVAL
    finally:
        fp.fp_gf_destroy(gf)


@pytest.mark.parametrize("algo", ["AUTO", "PLAIN", "DQT_U64"])
@pytest.mark.parametrize("p,n", [(3, 1), (3, 17), (2, 4096), (3, 65536 + 3), (7, 100000), (31, 12345),
                                 (251, 1 << 20), (5, 0), (3, 1 << 26)])
def test_dot_matches_oracle(env, algo, p, n):
    fp, torch, dev, ctx = env
    u, v = workloads.dot_inputs(n + p, p, n)
    out = torch.full((1,), 12345, dtype=torch.int32, device=dev)
    U = to_dev(torch, dev, u) if n else torch.empty(0, dtype=torch.uint8, device=dev)
    V = to_dev(torch, dev, v) if n else torch.empty(0, dtype=torch.uint8, device=dev)
    fp.fp_dot(ctx, p, U, V, n, out, getattr(fp, "FP_ALGO_" + algo))
    fp.fp_ctx_status(ctx)
    assert int(out.item()) == field.dot_mod(u, v, p)


def test_dot_unaligned_and_all_max(env):
    fp, torch, dev, ctx = env
    p, n = 7, 100003
    buf = torch.full((n + 1,), p - 1, dtype=torch.uint8, device=dev)
    out = torch.zeros((1,), dtype=torch.int32, device=dev)
    for algo in (fp.FP_ALGO_PLAIN, fp.FP_ALGO_DQT_U64):
        fp.fp_dot(ctx, p, buf[1:], buf[1:], n, out, algo)    # 1-byte offset: unaligned path
        fp.fp_ctx_status(ctx)
        assert int(out.item()) == (n * (p - 1) ** 2) % p


@pytest.mark.parametrize("p,k,pos,bad", [(3, 5, 5000, 243), (3, 5, 6001, 255), (7, 4, 4095, 2401),
                                         (7, 4, 4094, 4096 + 5), (7, 4, 9000, 32768), (7, 4, 9001, 65535),
                                         (3, 5, 3 * 4096 + 7, 243)])
def test_gf_bad_index_in_full_tiles(env, p, k, pos, bad):
    """An index >= p^k inside a full tile of the word-level kernel (including values whose low
    12 bits are a valid index, and values with the top bit set), or in the tail, raises the
    range error."""
    fp, torch, dev, ctx = env
    n = 3 * 4096 + 100
    a, b = workloads.gf_inputs(17, p, k, n)
    a = a.copy()
    a[pos] = bad
    gf = fp.fp_gf_create(ctx, p, k)
    try:
        with pytest.raises(fp.FpError) as ei:
            gf_run(fp, torch, dev, ctx, gf, a, b)
        assert ei.value.status == fp.FP_EINVAL
    finally:
        fp.fp_gf_destroy(gf)


@pytest.mark.parametrize("p", [2, 3, 5, 7, 31, 251])
@pytest.mark.parametrize("algo", ["AUTO", "DQT_U64"])
def test_dot_vector_path_all_max_and_range(env, p, algo):
    """Aligned arrays take the 16-byte vector middle product: all entries p-1 (every digit at
    its bound, accumulated F blocks at a time) with a ragged tail of 7 entries; then one entry
    equal to p inside a vector raises the range error."""
    fp, torch, dev, ctx = env
    n = 16 * 5003 + 7
    u = torch.full((n,), p - 1, dtype=torch.uint8, device=dev)
    out = torch.zeros((1,), dtype=torch.int32, device=dev)
    fp.fp_dot(ctx, p, u, u, n, out, getattr(fp, "FP_ALGO_" + algo))
    fp.fp_ctx_status(ctx)
    assert int(out.item()) == (n * (p - 1) ** 2) % p
    a, b = workloads.dot_inputs(p, p, n)
    A, B = torch.from_numpy(a).to(dev), torch.from_numpy(b).to(dev)
    fp.fp_dot(ctx, p, A, B, n, out, getattr(fp, "FP_ALGO_" + algo))
    fp.fp_ctx_status(ctx)
    assert int(out.item()) == field.dot_mod(a, b, p)
    u[12345] = p
    fp.fp_dot(ctx, p, u, u, n, out, getattr(fp, "FP_ALGO_" + algo))
    with pytest.raises(fp.FpError) as ei:
        fp.fp_ctx_status(ctx)
    assert ei.value.status == fp.FP_EINVAL


def _dev_elems(torch, dev, x, dt):
    x = np.ascontiguousarray(x.astype(dt))
    return torch.from_numpy(x.view(np.int16) if dt == np.uint16 else x).to(dev)


def _gf_dot_run(fp, torch, dev, ctx, gf, a, b, form, dt, offset=0):
    A = _dev_elems(torch, dev, np.concatenate([np.zeros(offset, dt), a.astype(dt)]), dt)[offset:]
    B = _dev_elems(torch, dev, np.concatenate([np.zeros(offset, dt), b.astype(dt)]), dt)[offset:]
    out = torch.full((1,), 7, dtype=torch.uint8 if dt == np.uint8 else torch.int16, device=dev)
    fp.fp_gf_dot(ctx, gf, A, B, len(a), out, form)
    fp.fp_ctx_status(ctx)
    v = out.cpu().numpy()
    return int((v.view(np.uint16) if dt == np.uint16 else v)[0])


@pytest.mark.parametrize("p,k", [(3, 5), (7, 4), (2, 8), (3, 2), (5, 1), (13, 2), (251, 1), (2, 4), (3, 3)])
def test_gf_dot_matches_oracle_both_forms(env, p, k):
    """Algorithm FGDP with n > 1: index and discrete-log forms, lengths around the chunk size and
    the 16-byte vector, 2^20 + 3 terms, and arrays that start one element past a 16-byte line."""
    fp, torch, dev, ctx = env
    gf = fp.fp_gf_create(ctx, p, k)
    try:
        m = field.smallest_monic_irreducible(p, k)
        info = fp.fp_gf_dot_info(gf)
        assert info["generator"] == field.primitive_element(p, k, m)
        antilog, log = field.log_tables(p, k, m)
        q, nc = p ** k, info["chunk"]
        assert nc >= 1 and nc * k * (p - 1) ** 2 < (1 << info["b_dot"])
        dt = workloads.gf_index_dtype(p, k)
        rng = np.random.default_rng(q + 11)
        for n in sorted({0, 1, 5, 16, 17, min(nc, 5000), min(nc + 1, 5001), 4096 * 16 + 5, (1 << 20) + 3}):
            a, b = rng.integers(0, q, n), rng.integers(0, q, n)
            want = field.gf_dot(a, b, p, k, m) if n else 0
            assert _gf_dot_run(fp, torch, dev, ctx, gf, a, b, fp.FP_GF_INDEX, dt) == want, n
            assert _gf_dot_run(fp, torch, dev, ctx, gf, log[a], log[b], fp.FP_GF_LOG, dt) == log[want], n
            if n > 1:
                assert _gf_dot_run(fp, torch, dev, ctx, gf, a, b, fp.FP_GF_INDEX, dt, offset=1) == want, n
        # every element p^k - 1 (all coefficients p - 1): every chunk's digits at the bound's edge
        n = min(3 * nc + 1, 1 << 20)
        a = np.full(n, q - 1)
        assert _gf_dot_run(fp, torch, dev, ctx, gf, a, a, fp.FP_GF_INDEX, dt) == field.gf_dot(a, a, p, k, m)
    finally:
        fp.fp_gf_destroy(gf)


def test_gf_dot_whole_field_and_bad_code(env):
    """Sum of x^2 over all of GF(3^5) is 0 and over GF(3) is 2 (power sums); a code >= p^k is
    reported through the context status."""
    fp, torch, dev, ctx = env
    for p, k, want in [(3, 5, 0), (3, 1, 2), (7, 4, 0)]:
        gf = fp.fp_gf_create(ctx, p, k)
        try:
            x = np.arange(p ** k)
            dt = workloads.gf_index_dtype(p, k)
            assert _gf_dot_run(fp, torch, dev, ctx, gf, x, x, fp.FP_GF_INDEX, dt) == want
        finally:
            fp.fp_gf_destroy(gf)
    gf = fp.fp_gf_create(ctx, 3, 5)
    try:
        a = np.zeros(1000, np.uint8)
        a[500] = 243
        A = torch.from_numpy(a).to(dev)
        out = torch.empty(1, dtype=torch.uint8, device=dev)
        fp.fp_gf_dot(ctx, gf, A, A, 1000, out, fp.FP_GF_INDEX)
        with pytest.raises(fp.FpError) as ei:
            fp.fp_ctx_status(ctx)
        assert ei.value.status == fp.FP_EINVAL
        with pytest.raises(fp.FpError):
            fp.fp_gf_dot(ctx, gf, A, A, 1000, out, 2)        # no such form: host check
    finally:
        fp.fp_gf_destroy(gf)


@pytest.mark.parametrize("form", ["INDEX", "LOG"])
@pytest.mark.parametrize("p,k,bad", [(3, 5, (243, 250, 255)), (7, 4, (2401, 4096 + 5, 32768 + 1, 65535))])
def test_gf_dot_bad_codes_count_as_zero(env, p, k, bad, form):
    """Codes >= p^k inside 16-byte vectors and in the ragged tail of the word-level dot product
    (GF(7^4) codes among them whose low 12 bits are a valid code), in index and in log form,
    count as zero and set the range error; arrays one element past a 16-byte line (the generic
    kernel) give the same."""
    fp, torch, dev, ctx = env
    gf = fp.fp_gf_create(ctx, p, k)
    try:
        m = field.smallest_monic_irreducible(p, k)
        _, log = field.log_tables(p, k, m)
        dt = workloads.gf_index_dtype(p, k)
        q = p ** k
        rng = np.random.default_rng(q + 5)
        n = 4096 * 16 + 5
        a, b = rng.integers(0, q, n), rng.integers(0, q, n)
        if form == "LOG":
            a, b = log[a], log[b]
        pos = (3, 777, 40000, n - 2)
        for i, j in enumerate(pos):
            a[j] = bad[i % len(bad)]
            b[j + 1] = bad[(i + 1) % len(bad)]
        keep_a = np.ones(n, bool)
        keep_b = np.ones(n, bool)
        keep_a[list(pos)] = False
        keep_b[[j + 1 for j in pos]] = False
        if form == "LOG":
            antilog = np.zeros(q, np.int64)
            antilog[log[np.arange(q)]] = np.arange(q)
            ia, ib = np.where(keep_a, antilog[np.where(keep_a, a, 0)], 0), np.where(keep_b, antilog[np.where(keep_b, b, 0)], 0)
        else:
            ia, ib = np.where(keep_a, a, 0), np.where(keep_b, b, 0)
        want = field.gf_dot(ia, ib, p, k, m)
        if form == "LOG":
            want = int(log[want])
        for offset in (0, 1):
            A = _dev_elems(torch, dev, np.concatenate([np.zeros(offset, dt), a.astype(dt)]), dt)[offset:]
            B = _dev_elems(torch, dev, np.concatenate([np.zeros(offset, dt), b.astype(dt)]), dt)[offset:]
            out = torch.full((1,), 7, dtype=torch.uint8 if dt == np.uint8 else torch.int16, device=dev)
            fp.fp_gf_dot(ctx, gf, A, B, n, out, getattr(fp, "FP_GF_" + form))
            torch.cuda.synchronize()
            v = out.cpu().numpy()
            got = int((v.view(np.uint16) if dt == np.uint16 else v)[0])
            with pytest.raises(fp.FpError) as ei:
                fp.fp_ctx_status(ctx)
            assert ei.value.status == fp.FP_EINVAL
            assert got == want, offset
    finally:
        fp.fp_gf_destroy(gf)


@pytest.mark.parametrize("p,k", [(3, 5), (7, 4)])
def test_gf_dot_long_enough_for_three_vector_trips(env, p, k):
    """n large enough that every thread of the one-wave grid (one 1024-thread block per SM) takes
    the three-vectors-per-trip loop at least once, then per-vector trips and the ragged tail:
    random codes in both forms and all-(p^k - 1) codes (every REDQ at its digit bound, every
    fold), against the oracle."""
    fp, torch, dev, ctx = env
    gf = fp.fp_gf_create(ctx, p, k)
    try:
        m = field.smallest_monic_irreducible(p, k)
        _, log = field.log_tables(p, k, m)
        dt = workloads.gf_index_dtype(p, k)
        q = p ** k
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        epv = 16 // np.dtype(dt).itemsize
        n = (5 * sms * 1024 + 1000) * epv + 5
        rng = np.random.default_rng(q + 29)
        a, b = rng.integers(0, q, n), rng.integers(0, q, n)
        want = field.gf_dot(a, b, p, k, m)
        assert _gf_dot_run(fp, torch, dev, ctx, gf, a, b, fp.FP_GF_INDEX, dt) == want
        assert _gf_dot_run(fp, torch, dev, ctx, gf, log[a], log[b], fp.FP_GF_LOG, dt) == log[want]
        full = np.full(n, q - 1)
        assert _gf_dot_run(fp, torch, dev, ctx, gf, full, full, fp.FP_GF_INDEX, dt) == \
            field.gf_dot(full, full, p, k, m)
    finally:
        fp.fp_gf_destroy(gf)
