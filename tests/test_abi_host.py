"""CPU checks of the C ABI: the library loads, exports every entry point the header declares,
its host-only planner agrees with the oracle's bounds, and device calls fail loudly (with a
status, not a fallback) when no GPU is present."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fp():
    import __graft_entry__ as g
    g.build()
    import paper_0809_0063_gb300 as m
    return m


def header_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(fp_\w+)\s*\(", txt))
    return names


def test_library_exports_every_header_symbol(fp):
    L = fp.lib()
    names = header_functions()
    assert len(names) >= 15
    missing = [n for n in sorted(names) if not hasattr(L, n)]
    assert not missing, missing
    # and the binding wraps each of them under the same name
    assert all(n in fp._SIGS for n in names), sorted(names - set(fp._SIGS))


def test_dqt_choose_matches_theorem_bounds(fp):
    """q is the Theorem's (Eq. bounds) smallest power of two above n k (p-1)^2; the word is
    accepted exactly when the largest packed result n DQT(all p-1)^2 fits the word's exact
    range (the Theorem's (2k-1) log2 q <= beta is a sufficient form of that condition)."""
    from oracle import bounds, dqt
    for p in (2, 3, 5, 7, 31, 251):
        for k in (1, 2, 3, 5, 8):
            for n in (1, 7, 1000):
                for word, beta in ((fp.FP_WORD_F64, 52), (fp.FP_WORD_U64, 64), (fp.FP_WORD_F32, 23), (fp.FP_WORD_U32, 32)):
                    q = max(bounds.smallest_pow2_q(n * k * (p - 1) ** 2), 2)
                    largest = n * dqt.dqt([p - 1] * k, q) ** 2
                    theorem_ok = bounds.thm_bounds_ok(q, n, k, p, beta)
                    try:
                        prm = fp.fp_dqt_choose(p, k, n, word)
                    except fp.FpError as e:
                        assert e.status == fp.FP_EBOUND
                        assert largest >= 2 ** beta and not theorem_ok
                        continue
                    assert (1 << prm.b) == q and prm.ndig == 2 * k - 1
                    assert largest < 2 ** beta


def _q_for(p, digit_max):
    """Smallest q = 2^b (b >= 1) above the largest digit and at least p (Eq. bounds, strict)."""
    from oracle import bounds
    return max(bounds.smallest_pow2_q(digit_max), bounds.smallest_pow2_q(p - 1), 2)


def test_polymul_plan_matches_bounds(fp):
    """The polynomial product's plan against the oracle's bounds: one word per operand when
    the exact largest product DQT(p-1, ..)^2 fits the word (AUTO takes the first of u32, f32,
    u64, f64 that fits), else blocks of d+1 coefficients in u64 words with q above the largest
    digit min(#blocks) (d+1) (p-1)^2 and the largest result word min(#blocks) DQT(p-1..)^2 below
    2^64; the Karatsuba form pads the block words to m 2^L with L >= 1."""
    from oracle import dqt
    beta = {fp.FP_WORD_F64: 52, fp.FP_WORD_U64: 64, fp.FP_WORD_F32: 23, fp.FP_WORD_U32: 32}
    auto_order = [fp.FP_WORD_U32, fp.FP_WORD_F32, fp.FP_WORD_U64, fp.FP_WORD_F64]
    forced = {fp.FP_ALGO_DQT_F64: fp.FP_WORD_F64, fp.FP_ALGO_DQT_U64: fp.FP_WORD_U64,
              fp.FP_ALGO_DQT_F32: fp.FP_WORD_F32, fp.FP_ALGO_DQT_U32: fp.FP_WORD_U32}
    algos = [fp.FP_ALGO_AUTO, fp.FP_ALGO_PLAIN, fp.FP_ALGO_KARATSUBA] + list(forced)
    for p in (2, 3, 5, 7, 31, 251):
        for da, db in ((0, 0), (2, 2), (1, 6), (10, 10), (31, 32), (100, 333), (511, 511), (1023, 1023),
                       (1023, 0)):
            ka, kb = da + 1, db + 1
            q1 = _q_for(p, min(ka, kb) * (p - 1) ** 2)
            largest1 = dqt.dqt([p - 1] * ka, q1) * dqt.dqt([p - 1] * kb, q1)
            fits = {w: ka + kb - 1 <= 64 and largest1 < 2 ** bt for w, bt in beta.items()}
            for algo in algos:
                try:
                    pl = fp.fp_polymul_plan(p, da, db, algo)
                except fp.FpError as e:
                    assert e.status == fp.FP_EBOUND
                    assert algo in forced and forced[algo] != fp.FP_WORD_U64 and not fits[forced[algo]]
                    continue
                if algo == fp.FP_ALGO_PLAIN:
                    assert pl["kernel"] == fp.FP_PM_PLAIN
                    continue
                if pl["kernel"] == fp.FP_PM_SINGLE_WORD:
                    assert algo != fp.FP_ALGO_KARATSUBA
                    w = pl["word"]
                    assert fits[w] and (1 << pl["b"]) == q1
                    assert (pl["blk_a"], pl["blk_b"], pl["ndig"]) == (ka, kb, ka + kb - 1)
                    if algo == fp.FP_ALGO_AUTO:
                        assert w == next(x for x in auto_order if fits[x])
                    else:
                        assert w == forced[algo]
                    continue
                # blocked FQT or its Karatsuba form, u64 words
                assert pl["kernel"] == (fp.FP_PM_KARATSUBA if algo == fp.FP_ALGO_KARATSUBA else fp.FP_PM_FQT)
                if algo in (fp.FP_ALGO_AUTO, fp.FP_ALGO_DQT_U64):
                    assert not fits[fp.FP_WORD_U64] if algo == fp.FP_ALGO_DQT_U64 else not any(fits.values())
                d1 = pl["blk_a"]
                assert pl["word"] == fp.FP_WORD_U64 and pl["blk_b"] == d1 and pl["ndig"] == 2 * d1 - 1
                na, nb = -(-ka // d1), -(-kb // d1)
                q = 1 << pl["b"]
                assert q == _q_for(p, min(na, nb) * d1 * (p - 1) ** 2)
                assert min(na, nb) * dqt.dqt([p - 1] * d1, q) ** 2 < 2 ** 64
                if pl["kernel"] == fp.FP_PM_KARATSUBA:
                    L, m = pl["L"], pl["m"]
                    assert L >= 1 and m == -(-max(na, nb) // (1 << L))
                else:
                    assert pl["L"] == 0 and pl["m"] == 0


def test_mm_choose_matches_eq_lower_upper(fp):
    from oracle import bounds
    for p in (2, 3, 7, 17, 31):
        for kdim in (16, 255, 256, 1024, 2047, 2048, 4096, 32767):
            b, e, _ = fp.fp_mm_choose(p, kdim, fp.FP_MM_RIGHT_F64)
            Q = bounds.cmm_Q(kdim, p)
            assert (1 << b) == max(Q, 2)
            D = kdim * (p - 1) ** 2
            # the largest packed word fits below 2^52 and one more residue would not
            assert D * sum(Q ** t for t in range(e)) < 2 ** 52
            assert D * sum(Q ** t for t in range(e + 1)) >= 2 ** 52
            assert e <= bounds.compression_factor(53, Q) + 1
    # Table "comprange" column n <= 2047 (strict reading of the 2048 column): Q = 2^13, e = 4
    assert fp.fp_mm_choose(3, 2047, fp.FP_MM_RIGHT_F64)[:2] == (13, 4)
    assert fp.fp_mm_choose(3, 2048, fp.FP_MM_RIGHT_F64)[:2] == (14, 3)
    # FP32 words: two residues at 2^12 per chunk, chunk digit bound below 2^12
    b, e, c = fp.fp_mm_choose(3, 4096, fp.FP_MM_RIGHT_F32)
    assert (b, e) == (12, 2) and c * 4 < 4096 and c % 8 == 0
    with pytest.raises(fp.FpError):
        fp.fp_mm_choose(31, 4096, fp.FP_MM_RIGHT_F32)


def test_full_and_split_planners_match_the_bounds(fp):
    """Full compression (Sec. 7.5): Q = 2^b strict for the piece (Eq. lower), Theta = Q^dq1
    (Eq. qtheta), Eq. dq at the paper's beta = 53 and the exact FP64 range (largest packed product
    below 2^52), and no larger balanced packing fits.  Splitting (Sec. 7.6): every piece of the
    oracle's split plan at the planner's piece length keeps at least the planner's compression."""
    from oracle import bounds, dqt
    for p in (2, 3, 5, 7, 13, 23):
        for kdim in (1, 16, 100, 255, 1000, 2047, 2048, 4096, 100000):
            b, dq1, dt1, piece = fp.fp_mm_full_choose(p, kdim)
            Q = 1 << b
            assert piece <= kdim and (piece == kdim or piece % 4 == 0)
            assert Q == bounds.cmm_Q(piece, p) or (piece * (p - 1) ** 2 < Q <= 2 * max(1, piece * (p - 1) ** 2))
            assert dq1 >= 2 and dt1 >= dq1
            assert bounds.full_compression_ok(Q, Q ** dq1, dq1 - 1, dt1 - 1, 53)
            D = piece * (p - 1) ** 2
            assert D * sum(Q ** t for t in range(dq1 * dt1)) < 2 ** 52
            if piece == kdim:   # one piece: no larger two-sided packing (both sides >= 2) fits
                for prod in range(dq1 * dt1 + 1, 17):
                    if any(prod % q == 0 and prod // q >= 2 for q in range(2, prod)):
                        assert D * sum(Q ** t for t in range(prod)) >= 2 ** 52
            if kdim > piece:
                npieces = -(-kdim // piece)
                assert -(-kdim // npieces) <= piece      # balanced
            b2, e2, c2 = fp.fp_mm_choose(p, kdim, fp.FP_MM_FULL_F64)
            assert (b2, e2, c2) == (b, dq1 * dt1, piece)
        for kdim in (16, 300, 2047, 2048, 4096, 30000):
            b, e, piece = fp.fp_mm_choose(p, kdim, fp.FP_MM_SPLIT_F64)
            for l0, kc, Q, e_piece in dqt.split_plan(kdim, piece, p, 52):
                assert e_piece >= e and Q <= (1 << b)
            # never below the unsplit right compression
            assert e >= fp.fp_mm_choose(p, kdim, fp.FP_MM_RIGHT_F64)[1]
    with pytest.raises(fp.FpError) as ei:
        fp.fp_mm_full_choose(29, 16)
    assert ei.value.status == fp.FP_EBOUND


def test_bad_arguments_are_rejected_on_host(fp):
    with pytest.raises(fp.FpError) as ei:
        fp.fp_dqt_choose(4, 3, 1, fp.FP_WORD_F64)       # not prime
    assert ei.value.status == fp.FP_EINVAL
    with pytest.raises(fp.FpError) as ei:
        fp.fp_dqt_choose(251, 40, 10 ** 6, fp.FP_WORD_F32)
    assert ei.value.status == fp.FP_EBOUND
    assert "exceeds" in fp.fp_last_error()


def test_device_calls_fail_loudly_without_gpu(fp):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(fp.FpError) as ei:
        fp.fp_ctx_create(0)
    assert ei.value.status in (fp.FP_ECUDA, fp.FP_EINVAL)
