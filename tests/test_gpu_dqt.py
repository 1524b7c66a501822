"""GPU parity of DQT pack, REDQ unpack and the batched polynomial product against the oracle
(bit-exact).  Calls go through the C ABI via the thin binding."""
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


WORDS = {0: (np.float64, 52), 1: (np.uint64, 64), 2: (np.float32, 23), 3: (np.uint32, 32)}


def _as_int(arr):
    return [int(x) for x in np.asarray(arr).astype(np.float64 if arr.dtype.kind == "f" else arr.dtype)] \
        if arr.dtype.kind == "f" else [int(x) for x in arr]


@pytest.mark.parametrize("word", [0, 1, 2, 3])
@pytest.mark.parametrize("p,k", [(2, 5), (3, 3), (5, 4), (7, 2), (31, 2), (37, 1), (251, 1)])
def test_pack_matches_oracle(env, word, p, k):
    fp, torch, dev, ctx = env
    dt, beta = WORDS[word]
    b = max(1, (p - 1).bit_length())
    while (p - 1) * sum(1 << (j * b) for j in range(k)) >= 2 ** beta:
        k -= 1
    prm = fp.fp_dqt_params(p=p, k=k, b=b, ndig=1, word=word, qform=0, n_accum=1)
    count = 3 * 256 + 17                              # several tiles and a ragged tail
    c = workloads.uniform_mod(k * 100 + p, p, (count, k))
    words = torch.empty(count, dtype=getattr(torch, np.dtype(dt).name), device=dev)
    fp.fp_dqt_pack(ctx, prm, to_dev(torch, dev, c), words, count)
    fp.fp_ctx_status(ctx)
    got = words.cpu().numpy()
    want = odqt.dqt(c, 1 << b)
    assert [int(x) for x in got] == [int(x) for x in want]


@pytest.mark.parametrize("word", [0, 1, 2, 3])
@pytest.mark.parametrize("p", [2, 3, 5, 7, 13, 31, 37, 251])
def test_unpack_redq_matches_radix_conversion(env, word, p):
    """Words r = sum mu~_i q^i with lower digits < q and a free top digit, below the word's
    exact range; REDQ must give the digits mod p (inverse DQT by radix conversion)."""
    fp, torch, dev, ctx = env
    dt, beta = WORDS[word]
    g = np.random.default_rng(p * 7 + word)
    for b in sorted({(p - 1).bit_length() + 1, (p - 1).bit_length() + 4, 12}):
        ndig = max(1, min(9, (beta - 1) // b))
        count = 2 * 256 + 5
        lo = g.integers(0, 1 << b, size=(count, ndig - 1)) if ndig > 1 else np.zeros((count, 0), np.int64)
        top_max = (2 ** beta - 1) >> (b * (ndig - 1))
        top = g.integers(0, min(top_max, 2 ** 62) + 1, size=count)
        r = [int(odqt.dqt(list(lo[i]) + [int(top[i])], 1 << b)) for i in range(count)]
        r[0] = 0
        r[1] = min(2 ** beta - 1, r[1])
        words = torch.tensor(np.array(r, dtype=np.uint64).astype(dt), device=dev)
        out = torch.empty((count, ndig), dtype=torch.uint8, device=dev)
        prm = fp.fp_dqt_params(p=p, k=1, b=b, ndig=ndig, word=word, qform=0, n_accum=1)
        fp.fp_dqt_unpack_redq(ctx, prm, words, out, count)
        fp.fp_ctx_status(ctx)
        got = out.cpu().numpy()
        for i in range(count):
            assert list(got[i]) == odqt.dqt_inverse(r[i], 1 << b, ndig, p), (p, b, ndig, r[i])


@pytest.mark.parametrize("word", [0, 1, 2, 3])
@pytest.mark.parametrize("p,t", [(3, 3), (2, 4), (5, 2), (7, 5), (3, 0), (13, 1), (251, 2)])
def test_q_p_times_pow2_pack_unpack(env, word, p, t):
    """q = p 2^t (the conclusion's alternative, FP_Q_P_POW2): packing equals the oracle's DQT at
    that q; unpacking (no correction step, divisions by p only) equals the oracle's radix
    conversion and its REDQ for words whose lower digits are below q and whose top digit is free."""
    fp, torch, dev, ctx = env
    dt, beta = WORDS[word]
    q = p << t
    k = 6
    while k > 1 and (p - 1) * sum(q ** j for j in range(k)) >= 2 ** beta:
        k -= 1
    if (p - 1) * sum(q ** j for j in range(k)) >= 2 ** beta:
        pytest.skip("q too large for this word")
    tdt = getattr(torch, np.dtype(dt).name)
    prm = fp.fp_dqt_params(p=p, k=k, b=t, ndig=1, word=word, qform=fp.FP_Q_P_POW2, n_accum=1)
    count = 2 * 256 + 9
    c = workloads.uniform_mod(k * 1000 + p + t, p, (count, k))
    c[0, :] = p - 1
    words = torch.empty(count, dtype=tdt, device=dev)
    fp.fp_dqt_pack(ctx, prm, to_dev(torch, dev, c), words, count)
    fp.fp_ctx_status(ctx)
    assert [int(x) for x in words.cpu().numpy()] == [int(x) for x in odqt.dqt(c, q)]
    g = np.random.default_rng(p * 31 + t + word)
    ndig = 1
    while ndig < 8 and q ** ndig < 2 ** beta:
        ndig += 1
    lo = g.integers(0, q, size=(count, ndig - 1)) if ndig > 1 else np.zeros((count, 0), np.int64)
    top_max = (2 ** beta - 1) // q ** (ndig - 1)
    top = g.integers(0, min(top_max, 2 ** 62) + 1, size=count)
    r = [int(odqt.dqt(list(lo[i]) + [int(top[i])], q)) for i in range(count)]
    r = [min(x, 2 ** beta - 1) for x in r]
    r[0] = 0
    words = torch.tensor(np.array(r, dtype=np.uint64).astype(dt), device=dev)
    out = torch.empty((count, ndig), dtype=torch.uint8, device=dev)
    prm = fp.fp_dqt_params(p=p, k=1, b=t, ndig=ndig, word=word, qform=fp.FP_Q_P_POW2, n_accum=1)
    fp.fp_dqt_unpack_redq(ctx, prm, words, out, count)
    fp.fp_ctx_status(ctx)
    got = out.cpu().numpy()
    for i in range(count):
        want = odqt.dqt_inverse(r[i], q, ndig, p)
        assert list(got[i]) == want == list(odqt.redq(r[i], p, q, ndig - 1)), (p, t, ndig, r[i])


def test_q_24_degree_2_products_over_f3(env):
    """The degree-2 products over F_3 at q = 24 = 3 2^3 (the smallest q = p 2^t above the digit
    bound 12): operands packed on the device, word products formed exactly (Python integers),
    REDQ_5 on the device; equals the schoolbook product mod 3."""
    fp, torch, dev, ctx = env
    count = 4099
    a, b = workloads.polymul_inputs(24, 3, count, 2, 2)
    prm = fp.fp_dqt_params(p=3, k=3, b=3, ndig=1, word=0, qform=fp.FP_Q_P_POW2, n_accum=1)
    wa = torch.empty(count, dtype=torch.float64, device=dev)
    wb = torch.empty(count, dtype=torch.float64, device=dev)
    fp.fp_dqt_pack(ctx, prm, to_dev(torch, dev, a), wa, count)
    fp.fp_dqt_pack(ctx, prm, to_dev(torch, dev, b), wb, count)
    prod = (wa * wb).contiguous()              # exact: below 24^5 < 2^23
    out = torch.empty((count, 5), dtype=torch.uint8, device=dev)
    prm5 = fp.fp_dqt_params(p=3, k=1, b=3, ndig=5, word=0, qform=fp.FP_Q_P_POW2, n_accum=1)
    fp.fp_dqt_unpack_redq(ctx, prm5, prod, out, count)
    fp.fp_ctx_status(ctx)
    np.testing.assert_array_equal(out.cpu().numpy(), field.polymul_mod(a, b, 3))


def test_qform_rejected(env):
    fp, torch, dev, ctx = env
    w = torch.zeros(4, dtype=torch.float64, device=dev)
    c = torch.zeros((4, 2), dtype=torch.uint8, device=dev)
    with pytest.raises(fp.FpError) as ei:
        fp.fp_dqt_pack(ctx, fp.fp_dqt_params(p=3, k=2, b=3, ndig=1, word=0, qform=2, n_accum=1), c, w, 4)
    assert ei.value.status == fp.FP_EINVAL


ALGOS = ["AUTO", "PLAIN", "DQT_F64", "DQT_U64", "DQT_F32", "DQT_U32"]


@pytest.mark.parametrize("algo", ALGOS)
def test_polymul_config_f3_degree2(env, algo):
    """2^20 independent pairs of degree-2 polynomials over F_3 (the batched single-word case)."""
    fp, torch, dev, ctx = env
    batch = 1 << 20
    a, b = workloads.polymul_inputs(0, 3, batch, 2, 2)
    C = torch.empty((batch, 5), dtype=torch.uint8, device=dev)
    fp.fp_polymul_batched(ctx, 3, to_dev(torch, dev, a), 2, to_dev(torch, dev, b), 2, C, batch,
                          getattr(fp, "FP_ALGO_" + algo))
    fp.fp_ctx_status(ctx)
    assert np.array_equal(C.cpu().numpy(), field.polymul_mod(a, b, 3))


@pytest.mark.parametrize("p,da,db,batch", [(2, 7, 3, 1000), (3, 4, 4, 257), (5, 1, 6, 3000), (7, 3, 3, 999),
                                           (31, 2, 1, 4097), (251, 0, 2, 300), (3, 0, 0, 5)])
@pytest.mark.parametrize("algo", ["AUTO", "PLAIN", "DQT_U64"])
def test_polymul_small_degrees(env, p, da, db, batch, algo):
    fp, torch, dev, ctx = env
    a, b = workloads.polymul_inputs(p + da, p, batch, da, db)
    C = torch.empty((batch, da + db + 1), dtype=torch.uint8, device=dev)
    fp.fp_polymul_batched(ctx, p, to_dev(torch, dev, a), da, to_dev(torch, dev, b), db, C, batch,
                          getattr(fp, "FP_ALGO_" + algo))
    fp.fp_ctx_status(ctx)
    assert np.array_equal(C.cpu().numpy(), field.polymul_mod(a, b, p))


@pytest.mark.parametrize("p,da,db", [(3, 512, 512), (7, 100, 333), (5, 64, 1), (2, 1023, 1023), (31, 40, 50)])
@pytest.mark.parametrize("algo", ["AUTO", "PLAIN"])
def test_polymul_large_degrees_fqt(env, p, da, db, algo):
    fp, torch, dev, ctx = env
    batch = 37
    a, b = workloads.polymul_inputs(da, p, batch, da, db)
    C = torch.empty((batch, da + db + 1), dtype=torch.uint8, device=dev)
    fp.fp_polymul_batched(ctx, p, to_dev(torch, dev, a), da, to_dev(torch, dev, b), db, C, batch,
                          getattr(fp, "FP_ALGO_" + algo))
    fp.fp_ctx_status(ctx)
    assert np.array_equal(C.cpu().numpy(), field.polymul_mod(a, b, p))


@pytest.mark.parametrize("p,da,db,batch", [(3, 512, 512, 37), (3, 1023, 1023, 9), (2, 1023, 1023, 9),
                                           (251, 1023, 1023, 5), (127, 592, 794, 5), (7, 100, 333, 37),
                                           (5, 64, 1, 37), (3, 1023, 0, 37), (3, 0, 1023, 37), (31, 40, 50, 37),
                                           (3, 0, 0, 37), (2, 1, 2, 37), (17, 299, 298, 37), (3, 63, 63, 37),
                                           (61, 260, 1014, 7), (3, 40, 40, 5000)])
def test_polymul_karatsuba(env, p, da, db, batch):
    """Karatsuba FQT: leaf counts 3 to 81, unequal and one-word operands, a grid-stride batch."""
    fp, torch, dev, ctx = env
    a, b = workloads.polymul_inputs(da + 7 * db, p, batch, da, db)
    C = torch.empty((batch, da + db + 1), dtype=torch.uint8, device=dev)
    fp.fp_polymul_batched(ctx, p, to_dev(torch, dev, a), da, to_dev(torch, dev, b), db, C, batch,
                          fp.FP_ALGO_KARATSUBA)
    fp.fp_ctx_status(ctx)
    assert np.array_equal(C.cpu().numpy(), field.polymul_mod(a, b, p))


def test_polymul_karatsuba_all_max_and_bad_input(env):
    """Every coefficient p-1 (every result word at the digit bound's edge), then one residue out
    of range, which the kernel reports through the context status."""
    fp, torch, dev, ctx = env
    for p, d in [(3, 1023), (7, 511), (251, 700), (2, 5)]:
        a = np.full((19, d + 1), p - 1, np.uint8)
        C = torch.empty((19, 2 * d + 1), dtype=torch.uint8, device=dev)
        A = to_dev(torch, dev, a)
        fp.fp_polymul_batched(ctx, p, A, d, A, d, C, 19, fp.FP_ALGO_KARATSUBA)
        fp.fp_ctx_status(ctx)
        assert np.array_equal(C.cpu().numpy(), field.polymul_mod(a, a, p))
    A = torch.zeros((4, 600), dtype=torch.uint8, device=dev)
    A[2, 599] = 3
    C = torch.empty((4, 1199), dtype=torch.uint8, device=dev)
    fp.fp_polymul_batched(ctx, 3, A, 599, A, 599, C, 4, fp.FP_ALGO_KARATSUBA)
    with pytest.raises(fp.FpError) as ei:
        fp.fp_ctx_status(ctx)
    assert ei.value.status == fp.FP_EINVAL


def test_polymul_all_max_coefficients(env):
    """Every coefficient p-1: the largest digit of every word (the bound's edge)."""
    fp, torch, dev, ctx = env
    for p, d in [(3, 2), (7, 5), (251, 1), (3, 300)]:
        a = np.full((513, d + 1), p - 1, np.uint8)
        C = torch.empty((513, 2 * d + 1), dtype=torch.uint8, device=dev)
        A = to_dev(torch, dev, a)
        fp.fp_polymul_batched(ctx, p, A, d, A, d, C, 513, fp.FP_ALGO_AUTO)
        fp.fp_ctx_status(ctx)
        assert np.array_equal(C.cpu().numpy(), field.polymul_mod(a, a, p))


def test_polymul_empty_batch_and_bad_input(env):
    fp, torch, dev, ctx = env
    A = torch.zeros((4, 3), dtype=torch.uint8, device=dev)
    C = torch.empty((4, 5), dtype=torch.uint8, device=dev)
    fp.fp_polymul_batched(ctx, 3, A, 2, A, 2, C, 0, fp.FP_ALGO_AUTO)   # empty: no-op
    A[1, 1] = 3                                                          # out of range for p = 3
    fp.fp_polymul_batched(ctx, 3, A, 2, A, 2, C, 4, fp.FP_ALGO_AUTO)
    with pytest.raises(fp.FpError) as ei:
        fp.fp_ctx_status(ctx)
    assert ei.value.status == fp.FP_EINVAL
    fp.fp_ctx_status(ctx)                                                # flag was cleared
    with pytest.raises(fp.FpError):
        fp.fp_polymul_batched(ctx, 4, A, 2, A, 2, C, 4, fp.FP_ALGO_AUTO)  # not prime: host check


@pytest.mark.parametrize("p,d", [(2, 1), (3, 2), (5, 1), (3, 3), (7, 2), (2, 3), (3, 1)])
@pytest.mark.parametrize("algo", ["AUTO", "DQT_U32"])
def test_polymul_word_granular_path(env, p, d, algo):
    """Full tiles of 2048 pairs on the word-granular small-degree kernel (p = 2: no correction,
    p = 3: two residues per table lookup, p = 5: one; p = 7 takes the shared-table path) plus a
    ragged tail on the per-pair kernel; every coefficient compared."""
    fp, torch, dev, ctx = env
    batch = 3 * 2048 + 777
    a, b = workloads.polymul_inputs(40 + p * d, p, batch, d, d)
    a[-1], b[0] = p - 1, p - 1                        # bound edges in the tail and the first tile
    C = torch.empty((batch, 2 * d + 1), dtype=torch.uint8, device=dev)
    try:
        fp.fp_polymul_batched(ctx, p, to_dev(torch, dev, a), d, to_dev(torch, dev, b), d, C, batch,
                              getattr(fp, "FP_ALGO_" + algo))
    except fp.FpError as e:
        if e.status == fp.FP_EBOUND:
            pytest.skip("the product does not fit a 32-bit word")
        raise
    fp.fp_ctx_status(ctx)
    assert np.array_equal(C.cpu().numpy(), field.polymul_mod(a, b, p))


@pytest.mark.parametrize("p,d", [(2, 2), (3, 2), (5, 3)])
def test_polymul_word_granular_staged(env, p, d):
    """Above 512 full tiles (2^20 pairs) the word-granular kernel stages tiles through shared
    memory by bulk copies instead of reading in place; 600 tiles plus a ragged tail, every
    coefficient compared, plus a coefficient equal to p in the last full tile."""
    fp, torch, dev, ctx = env
    batch = 600 * 2048 + 333
    a, b = workloads.polymul_inputs(7 + p * d, p, batch, d, d)
    C = torch.empty((batch, 2 * d + 1), dtype=torch.uint8, device=dev)
    try:
        fp.fp_polymul_batched(ctx, p, to_dev(torch, dev, a), d, to_dev(torch, dev, b), d, C, batch, fp.FP_ALGO_AUTO)
    except fp.FpError as e:
        if e.status == fp.FP_EBOUND:
            pytest.skip("the product does not fit a 32-bit word")
        raise
    fp.fp_ctx_status(ctx)
    assert np.array_equal(C.cpu().numpy(), field.polymul_mod(a, b, p))
    a[600 * 2048 - 5, 1] = p
    fp.fp_polymul_batched(ctx, p, to_dev(torch, dev, a), d, to_dev(torch, dev, b), d, C, batch, fp.FP_ALGO_AUTO)
    with pytest.raises(fp.FpError) as ei:
        fp.fp_ctx_status(ctx)
    assert ei.value.status == fp.FP_EINVAL


@pytest.mark.parametrize("pos", [0, 1000, 2047, 4095, 6143, 6144 + 700])
def test_polymul_word_granular_range_check(env, pos):
    """A coefficient equal to p anywhere (each full tile, the tail) raises the range error."""
    fp, torch, dev, ctx = env
    p, d, batch = 3, 2, 3 * 2048 + 777
    a, b = workloads.polymul_inputs(91, p, batch, d, d)
    a[pos, pos % 3] = p
    C = torch.empty((batch, 5), dtype=torch.uint8, device=dev)
    fp.fp_polymul_batched(ctx, p, to_dev(torch, dev, a), d, to_dev(torch, dev, b), d, C, batch, fp.FP_ALGO_AUTO)
    with pytest.raises(fp.FpError) as ei:
        fp.fp_ctx_status(ctx)
    assert ei.value.status == fp.FP_EINVAL


@pytest.mark.parametrize("p,k", [(2, 5), (3, 3), (5, 4), (7, 2), (3, 2), (13, 2)])
def test_pack_u32_word_granular(env, p, k):
    """32-bit DQT pack through the word-granular kernel (full tiles of 4096 words) and the
    per-word kernel (the ragged tail); a residue equal to p in a full tile is caught."""
    fp, torch, dev, ctx = env
    b = max(1, (p - 1).bit_length())
    count = 2 * 4096 + 123
    prm = fp.fp_dqt_params(p=p, k=k, b=b, ndig=1, word=3, qform=0, n_accum=1)
    c = workloads.uniform_mod(k * 1000 + p, p, (count, k))
    c[0] = p - 1
    words = torch.empty(count, dtype=torch.int32, device=dev)
    C = to_dev(torch, dev, c)
    fp.fp_dqt_pack(ctx, prm, C, words, count)
    fp.fp_ctx_status(ctx)
    got = words.cpu().numpy().view(np.uint32)
    assert np.array_equal(got.astype(np.int64), np.array([int(x) for x in odqt.dqt(c, 1 << b)], np.int64))
    C[5000, k - 1] = p
    fp.fp_dqt_pack(ctx, prm, C, words, count)
    with pytest.raises(fp.FpError) as ei:
        fp.fp_ctx_status(ctx)
    assert ei.value.status == fp.FP_EINVAL


@pytest.mark.parametrize("p", [2, 3, 5, 7])
@pytest.mark.parametrize("ndig", [3, 5, 7])
def test_unpack_u32_word_granular(env, p, ndig):
    """32-bit REDQ unpack through the word-granular kernel (ndig in {3, 5, 7}; p = 2 no
    correction, 3 two residues per lookup, 5 one, 7 the shared-table fallback) and the tail."""
    fp, torch, dev, ctx = env
    b = 32 // ndig
    count = 2 * 4096 + 99
    g = np.random.default_rng(p * 31 + ndig)
    lo = g.integers(0, 1 << b, size=(count, ndig - 1))
    top = g.integers(0, ((1 << 32) - 1) >> (b * (ndig - 1)), size=count)
    r = [int(odqt.dqt(list(lo[i]) + [int(top[i])], 1 << b)) for i in range(count)]
    words = torch.tensor(np.array(r, dtype=np.uint64).astype(np.uint32).view(np.int32), device=dev)
    out = torch.empty((count, ndig), dtype=torch.uint8, device=dev)
    prm = fp.fp_dqt_params(p=p, k=1, b=b, ndig=ndig, word=3, qform=0, n_accum=1)
    fp.fp_dqt_unpack_redq(ctx, prm, words, out, count)
    fp.fp_ctx_status(ctx)
    got = out.cpu().numpy()
    for i in list(range(0, count, 7)) + list(range(count - 110, count)):
        assert list(got[i]) == odqt.dqt_inverse(r[i], 1 << b, ndig, p), (p, b, ndig, i)
