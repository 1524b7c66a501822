"""Pins of the oracle's DQT, inverse DQT and REDQ against the paper's worked examples,
Theorem REDQ, Lemma flfl and exhaustive brute force on tiny p, q, k."""
import itertools

import numpy as np
import pytest

from oracle import dqt, field
from tests._golden import paper_examples

EX = paper_examples()


def test_kronecker_example():
    e = EX["kronecker"]
    q, p = e["q"], e["p"]
    wa, wb = dqt.dqt(e["a"], q), dqt.dqt(e["b"], q)
    assert (wa, wb) == (e["word_a"], e["word_b"])
    assert wa * wb == e["product"]
    assert dqt.radix_digits(wa * wb, q, 3) == e["digits"]
    assert dqt.dqt_inverse(wa * wb, q, 3, p) == e["result"]
    # and the plain definition agrees
    assert list(field.polymul_mod(np.array(e["a"]), np.array(e["b"]), p)) == e["result"]


def test_redq_p_divides_q_example():
    e = EX["redq_pdivq"]
    p, q = e["p"], e["q"]
    r = dqt.dqt(e["coeffs"], q)
    assert r == e["r"]
    assert dqt.dqt(e["a"], q) * dqt.dqt(e["b"], q) == r
    s = r // p
    # the quotient of each coefficient sits in s: floor(s/q^i) - q floor(s/q^(i+1)) is the
    # i-th base-q digit of s; for this example the digits printed in bold are the quotients
    # of the coefficients by p, up to the borrow of the lower digit's remainder.
    assert [c // p for c in reversed(e["coeffs"])] == e["qdigits_high_first"]
    assert dqt.redq_compression(r, p, q, 4) == e["result"]
    assert dqt.redq(r, p, q, 4) == e["result"]           # q = 0 mod p: no correction
    assert s == 8002600560054003


def test_redq_full_example():
    e = EX["redq_full"]
    p, q = e["p"], e["q"]
    r = dqt.dqt(e["coeffs"], q)
    assert r == e["r"] and r > 2 ** 64
    assert r // p == e["s"]
    u = dqt.redq_compression(r, p, q, 3)
    assert u == e["u"]
    assert dqt.redq_correction(u, p, q) == e["mu"]
    assert dqt.redq(r, p, q, 3) == e["mu"]
    assert [c % p for c in e["coeffs"]] == e["mu"]
    # matrix version (Sec. 3.4)
    Qk = dqt.correction_matrix(4, p, q)
    assert Qk[0, 1] == EX["correction_entry"]["entry"]
    assert list((Qk @ np.array(u)) % p) == e["mu"]


@pytest.mark.parametrize("p", [2, 3, 5, 7])
def test_redq_exhaustive(p):
    """Theorem REDQ by brute force: for every q in p+1..32 and every digit tuple the REDQ
    result equals radix conversion followed by mod p; 0 <= u_i < p (Theorem REDQ)."""
    for q in range(p + 1, 33):
        kmax = 4 if q <= 8 else (3 if q <= 16 else 2)
        for k in range(1, kmax + 1):
            digs = np.array(list(itertools.product(range(q), repeat=k)), dtype=np.int64)
            r = np.zeros(len(digs), dtype=np.int64)
            for i in range(k - 1, -1, -1):
                r = r * q + digs[:, i]
            u = dqt.redq_compression(r, p, q, k - 1)
            for ui in u:
                assert np.all((ui >= 0) & (ui < p))
            mu = dqt.redq(r, p, q, k - 1)
            for i in range(k):
                assert np.array_equal(mu[i] % p if q % p == 0 else mu[i], digs[:, i] % p), (p, q, k, i)
            inv = dqt.dqt_inverse(r, q, k, p)
            for i in range(k):
                assert np.array_equal(inv[i], digs[:, i] % p)


def test_redq_skipping_correction_is_wrong_when_p_does_not_divide_q():
    # the compression alone is not the answer when p does not divide q (Example "full")
    e = EX["redq_full"]
    assert dqt.redq_compression(e["r"], e["p"], e["q"], 3) != e["mu"]


def test_lemma_flfl_exhaustive():
    r = np.arange(0, 600)
    for a in range(1, 13):
        for b in range(1, 13):
            assert np.array_equal((r // b) // a, r // (a * b))
            assert np.array_equal((r // a) // b, r // (a * b))


def test_q6_by_q2_tables():
    """Example tmto: three lookups in the underline{Q}_2 table reproduce Q_6 u mod p; the
    table has p^3 entries; Proposition tmto's count floor((k-1)/(j-1)) is 3 for k=7, j=3."""
    from oracle.bounds import tmto_lookups
    for p, q in [(3, 16), (5, 32), (7, 64), (23, 10 ** 6)]:
        t = dqt.q2_table(p, q)
        assert len(t) == p ** 3
        Q7 = dqt.correction_matrix(7, p, q)
        g = np.random.default_rng(p)
        for _ in range(200):
            u = [int(x) for x in g.integers(0, p, 7)]
            assert dqt.q6_by_q2(u, p, t) == [int(x) for x in (Q7 @ np.array(u)) % p]
    assert tmto_lookups(7, 3) == 3


def test_right_compression_2x2_identity():
    """Sec. 7.4's 2x2 identity: [a b; c d] x [e+Qf; g+Qh] = [(ae+bg)+Q(af+bh); ...]."""
    Q = 1 << 10
    a, b, c, d, e, f, g, h = 2, 1, 0, 2, 1, 2, 2, 1
    A = np.array([[a, b], [c, d]])
    B = np.array([[e, f], [g, h]])
    CB = dqt.right_compress(B, 2, Q)
    assert list(CB[:, 0]) == [e + Q * f, g + Q * h]
    CC = A.astype(object) @ CB
    assert CC[0, 0] == (a * e + b * g) + Q * (a * f + b * h)
    assert CC[1, 0] == (c * e + d * g) + Q * (c * f + d * h)
    assert np.array_equal(dqt.right_compressed_product(A, B, 3, 2, Q), field.matmul_mod(A, B, 3))


def test_middle_product_2x2_identity():
    """Sec. 7.1: (Qa+b)(e+Qg) has (ae+bg) as coefficient of Q (d = 1)."""
    Q = 1 << 8
    a, b, e, g = 2, 1, 2, 2
    w = (Q * a + b) * (e + Q * g)
    assert (w // Q) % Q == a * e + b * g
    rng = np.random.default_rng(0)
    for p, d in [(3, 1), (3, 3), (7, 2)]:
        n = 37
        u = rng.integers(0, p, n)
        v = rng.integers(0, p, n)
        Qb = 1 << ((n * (p - 1) ** 2).bit_length())
        assert dqt.middle_product_dot(u, v, p, d, Qb) == field.dot_mod(u, v, p)


def test_right_compressed_product_random_ragged():
    rng = np.random.default_rng(1)
    for p, e in [(3, 4), (7, 3), (2, 5)]:
        m, k, n = 5, 9, 11           # n not a multiple of e: partial compression
        A = rng.integers(0, p, (m, k))
        B = rng.integers(0, p, (k, n))
        Q = 1 << ((k * (p - 1) ** 2).bit_length())
        assert np.array_equal(dqt.right_compressed_product(A, B, p, e, Q), field.matmul_mod(A, B, p))


def test_full_compression_2x2_identity():
    """Sec. 7.5's example: [a+Qc, b+Qd] x [e+Theta f; g+Theta h] =
    (ae+bg) + Q(ce+dg) + Theta(af+bh) + Q Theta(cf+dh), written out here term by term."""
    rng = np.random.default_rng(75)
    for _ in range(50):
        a, b, c, d, e, f, g, h = (int(x) for x in rng.integers(0, 1000, 8))
        Q = 1 << int(rng.integers(20, 24))
        Theta = Q * Q
        WA = dqt.full_compress_rows(np.array([[a, b], [c, d]]), 1, Q)
        WB = dqt.full_compress_cols(np.array([[e, f], [g, h]]), 1, Theta)
        assert WA.shape == (1, 2) and WB.shape == (2, 1)
        assert int((WA @ WB)[0, 0]) == (a * e + b * g) + Q * (c * e + d * g) + Theta * (a * f + b * h) \
            + Q * Theta * (c * f + d * h)


@pytest.mark.parametrize("p,m,k,n,dq,dt,extra", [(3, 7, 50, 5, 1, 1, 0), (2, 5, 9, 11, 2, 3, 0), (5, 6, 20, 7, 1, 2, 1),
                                                 (7, 3, 33, 4, 0, 2, 0), (3, 1, 1, 1, 2, 2, 0)])
def test_full_compressed_product_matches_plain(p, m, k, n, dq, dt, extra):
    """Full compression with Q > k (p-1)^2 (Eq. lower) and Theta = Q^(dq+1+extra) (Eq. qtheta)
    reproduces A B mod p on ragged shapes; all-(p-1) operands reach the digit bound's edge."""
    rng = np.random.default_rng(p * 100 + m)
    Q = 2
    while Q <= k * (p - 1) ** 2:
        Q *= 2
    for A, B in [(rng.integers(0, p, (m, k)), rng.integers(0, p, (k, n))),
                 (np.full((m, k), p - 1), np.full((k, n), p - 1))]:
        assert np.array_equal(dqt.full_compressed_product(A, B, p, dq, dt, Q, dq + 1 + extra),
                              field.matmul_mod(A, B, p))


def test_full_compression_non_strict_q_breaks():
    """At Q = k (p-1)^2 (the non-strict reading of Eq. lower) an all-(p-1) product carries into
    the next digit and the result is wrong; one more bit of Q fixes it."""
    p, k = 3, 16
    A, B = np.full((2, k), p - 1), np.full((k, 2), p - 1)
    want = field.matmul_mod(A, B, p)
    assert not np.array_equal(dqt.full_compressed_product(A, B, p, 1, 1, k * (p - 1) ** 2, 2), want)
    assert np.array_equal(dqt.full_compressed_product(A, B, p, 1, 1, 2 * k * (p - 1) ** 2, 2), want)


def test_split_inner_dimension_keeps_compression_four():
    """Sec. 7.6: over F_3 with 53-bit words the compression drops from 4 to 3 once n (p-1)^2
    reaches 2^13 (with the strict digit bound that is at n = 2048, one dimension before the
    paper's table); an inner dimension of 2049 cut into pieces of 1025 and 1024 keeps
    Q = 2^13 and compression 4 in each piece."""
    from oracle import bounds
    assert bounds.compression_factor(53, bounds.cmm_Q(2047, 3)) == 4
    assert bounds.compression_factor(53, bounds.cmm_Q(2048, 3)) == 3
    assert bounds.compression_factor(53, bounds.cmm_Q(2049, 3)) == 3
    plan = dqt.split_plan(2049, 1025, 3, 53)
    assert [(l0, kc) for l0, kc, _, _ in plan] == [(0, 1025), (1025, 1024)]
    assert all(Q == 1 << 13 and e == 4 for _, _, Q, e in plan)


@pytest.mark.parametrize("p,m,k,n,chunk", [(3, 5, 70, 9, 16), (7, 4, 33, 6, 10), (2, 3, 100, 13, 64), (5, 2, 9, 3, 1)])
def test_split_right_compressed_product_matches_plain(p, m, k, n, chunk):
    """Splitting the inner dimension (ragged last piece included) and adding the pieces' REDQ
    results mod p gives A B mod p; all-(p-1) operands reach each piece's digit bound."""
    rng = np.random.default_rng(p + k)
    for A, B in [(rng.integers(0, p, (m, k)), rng.integers(0, p, (k, n))),
                 (np.full((m, k), p - 1), np.full((k, n), p - 1))]:
        assert np.array_equal(dqt.split_right_compressed_product(A, B, p, chunk, 53), field.matmul_mod(A, B, p))
