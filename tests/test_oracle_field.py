"""Pins of the oracle's plain definitions: library routines, algebraic identities, closed
forms (Gauss's count of irreducibles), field axioms and an independent GF(2^8) multiply."""
import numpy as np
import pytest

from oracle import field, gfpk


def test_polymul_matches_numpy_convolve():
    rng = np.random.default_rng(0)
    for p in (2, 3, 7, 31, 251):
        a = rng.integers(0, p, (50, 6))
        b = rng.integers(0, p, (50, 4))
        c = field.polymul_mod(a, b, p)
        for i in range(50):
            assert np.array_equal(c[i], np.convolve(a[i], b[i]) % p)


def test_polymul_exhaustive_deg2_f3_identities():
    """All 3^6 pairs of degree-2 polynomials over F_3: commutativity, the product by X is a
    shift, and evaluation at every point of F_3 is a ring morphism."""
    import itertools
    allp = np.array(list(itertools.product(range(3), repeat=3)))
    A = np.repeat(allp, len(allp), axis=0)
    B = np.tile(allp, (len(allp), 1))
    C = field.polymul_mod(A, B, 3)
    assert np.array_equal(C, field.polymul_mod(B, A, 3))
    for x in range(3):
        ev = lambda P: (P * (x ** np.arange(P.shape[1]))).sum(1) % 3
        assert np.array_equal(ev(C), (ev(A) * ev(B)) % 3)
    X = np.tile(np.array([[0, 1, 0]]), (len(A), 1))
    assert np.array_equal(field.polymul_mod(A, X, 3)[:, 1:4], A)


def test_matmul_matches_float_blas_and_associates():
    rng = np.random.default_rng(1)
    for p in (2, 3, 7, 31):
        A = rng.integers(0, p, (33, 47))
        B = rng.integers(0, p, (47, 29))
        D = rng.integers(0, p, (29, 5))
        C = field.matmul_mod(A, B, p)
        ref = np.fmod(A.astype(np.float64) @ B.astype(np.float64), p).astype(np.int64)
        assert np.array_equal(C, ref)
        assert np.array_equal(field.matmul_mod(C, D, p), field.matmul_mod(A, field.matmul_mod(B, D, p), p))
        assert np.array_equal(field.matmul_mod_rows(A, B, p, [3, 7]), C[[3, 7]])
        I = np.eye(47, dtype=np.int64)
        assert np.array_equal(field.matmul_mod(I, B, p), B % p)


def test_dot_matches_python_sum():
    rng = np.random.default_rng(2)
    u = rng.integers(0, 31, 1001)
    v = rng.integers(0, 31, 1001)
    assert field.dot_mod(u, v, 31) == sum(int(a) * int(b) for a, b in zip(u, v)) % 31


def _mobius(n):
    res, m, d = 1, n, 2
    while d * d <= m:
        if m % d == 0:
            m //= d
            if m % d == 0:
                return 0
            res = -res
        d += 1
    return -res if m > 1 else res


@pytest.mark.parametrize("p,k", [(2, 2), (2, 3), (2, 4), (2, 5), (3, 2), (3, 3), (5, 2), (7, 2)])
def test_irreducible_count_gauss_formula(p, k):
    """The brute-force irreducibility test finds exactly (1/k) sum_{d|k} mu(d) p^(k/d)
    monic irreducibles of degree k (Gauss's formula)."""
    expect = sum(_mobius(d) * p ** (k // d) for d in range(1, k + 1) if k % d == 0) // k
    assert field.count_monic_irreducibles(p, k) == expect


def _gf2_8_mul_bitwise(a, b, poly_low):
    """Independent GF(2^8) multiply: shift-and-xor with reduction by x^8 + poly_low."""
    r = 0
    for _ in range(8):
        if b & 1:
            r ^= a
        b >>= 1
        carry = a & 0x80
        a = (a << 1) & 0xFF
        if carry:
            a ^= poly_low
    return r


def test_gf_moduli_and_gf2_8_cross_check():
    m28 = field.smallest_monic_irreducible(2, 8)
    # x^8 + x^4 + x^3 + x + 1
    assert m28 == [1, 1, 0, 1, 1, 0, 0, 0, 1]
    low = sum(c << i for i, c in enumerate(m28[:8]))
    a = np.arange(256).repeat(256)
    b = np.tile(np.arange(256), 256)
    got = field.gf_mul(a, b, 2, 8, m28)
    sel = np.random.default_rng(3).integers(0, 65536, 3000)
    for i in sel:
        assert got[i] == _gf2_8_mul_bitwise(int(a[i]), int(b[i]), low)
    for (p, k) in [(3, 5), (7, 4)]:
        m = field.smallest_monic_irreducible(p, k)
        assert field.is_irreducible(m, p)
        key = sum(c * p ** i for i, c in enumerate(m[:k]))
        for kk, f in field.monic_candidates(p, k):
            if kk >= key:
                break
            assert not field.is_irreducible(f, p)


@pytest.mark.parametrize("p,k", [(3, 5), (7, 4), (2, 8)])
def test_gf_field_axioms(p, k):
    m = field.smallest_monic_irreducible(p, k)
    rng = np.random.default_rng(p * 10 + k)
    a, b, c = (rng.integers(0, p ** k, 400) for _ in range(3))
    mul = lambda x, y: field.gf_mul(x, y, p, k, m)
    add = lambda x, y: field.gf_add(x, y, p, k)
    assert np.array_equal(mul(a, b), mul(b, a))
    assert np.array_equal(mul(mul(a, b), c), mul(a, mul(b, c)))
    assert np.array_equal(mul(a, add(b, c)), add(mul(a, b), mul(a, c)))
    assert np.array_equal(mul(a, np.ones_like(a)), a)
    assert np.all(mul(a, np.zeros_like(a)) == 0)
    nz = a[a != 0][:60]
    assert np.all(field.gf_pow(nz, p ** k - 1, p, k, m) == 1)
    # every nonzero element has an inverse: x^(p^k-2) * x = 1
    assert np.all(mul(nz, field.gf_pow(nz, p ** k - 2, p, k, m)) == 1)


@pytest.mark.parametrize("p,k,q", [(3, 2, 16), (3, 3, 32), (2, 4, 16), (5, 2, 64), (3, 5, 32)])
def test_fgdp_theorem(p, k, q):
    """Theorem fgdp: the L/H-table route of Algorithm FGDP equals the plain field dot."""
    m = field.smallest_monic_irreducible(p, k)
    tabs = gfpk.fgdp_tables(p, k, q, m)
    rng = np.random.default_rng(k)
    for n in (1, 2, 3):
        if q <= n * k * (p - 1) ** 2:
            continue
        for _ in range(30):
            v1 = rng.integers(0, p ** k, n)
            v2 = rng.integers(0, p ** k, n)
            plain = 0
            for x, y in zip(v1, v2):
                plain = int(field.gf_add(np.array(plain), field.gf_mul(np.array(x), np.array(y), p, k, m), p, k))
            assert gfpk.fgdp_dot(v1, v2, p, k, q, m, tabs) == plain


# Smallest primitive root modulo p (number-theory tables, OEIS A001918).
_SMALLEST_PRIMITIVE_ROOT = {2: 1, 3: 2, 5: 2, 7: 3, 11: 2, 13: 2, 17: 3, 19: 2, 23: 5, 29: 2, 31: 3, 37: 2,
                            41: 6, 43: 3, 47: 5, 71: 7, 73: 5, 97: 5}


def test_primitive_element_known_values():
    """The generator of the discrete-log form is the smallest index of full order: for k = 1
    the smallest primitive root mod p; in the AES field (x^8 + x^4 + x^3 + x + 1) x has order
    51 and x + 1 (index 3) generates the multiplicative group."""
    for p, g in _SMALLEST_PRIMITIVE_ROOT.items():
        assert field.primitive_element(p, 1, field.smallest_monic_irreducible(p, 1)) == g, p
    m = field.smallest_monic_irreducible(2, 8)
    assert field.primitive_element(2, 8, m) == 3
    powers = [int(field.gf_pow(np.array(2), e, 2, 8, m)) for e in range(1, 256)]
    assert powers.index(1) + 1 == 51


@pytest.mark.parametrize("p,k", [(3, 5), (7, 4), (2, 8), (3, 2), (5, 1), (2, 1)])
def test_log_tables_are_a_group_isomorphism(p, k):
    """antilog is a bijection from exponents 0..p^k-2 onto the nonzero elements with
    antilog(e1 + e2 mod p^k - 1) = antilog(e1) antilog(e2); p^k - 1 stands for zero."""
    m = field.smallest_monic_irreducible(p, k)
    antilog, log = field.log_tables(p, k, m)
    q = p ** k
    assert antilog[q - 1] == 0 and log[0] == q - 1
    assert sorted(antilog[: q - 1].tolist()) == list(range(1, q))
    assert np.array_equal(antilog[log], np.arange(q))
    rng = np.random.default_rng(q)
    e1, e2 = rng.integers(0, q - 1, 300), rng.integers(0, q - 1, 300)
    assert np.array_equal(antilog[(e1 + e2) % (q - 1)], field.gf_mul(antilog[e1], antilog[e2], p, k, m))


@pytest.mark.parametrize("p,k", [(3, 5), (7, 4), (2, 8), (2, 1), (3, 1), (2, 2), (5, 2), (3, 3)])
def test_gf_dot_closed_forms_and_fold(p, k):
    """Sum over all x of x^2 is -1 when p^k - 1 divides 2 and 0 otherwise; the sum over the
    nonzero x of x x^-1 is p^k - 1 = -1 (the constant p - 1); and gf_dot equals the fold of
    gf_mul and gf_add, and is additive in its second argument."""
    m = field.smallest_monic_irreducible(p, k)
    q = p ** k
    x = np.arange(q)
    assert field.gf_dot(x, x, p, k, m) == ((p - 1) if 2 % (q - 1) == 0 else 0)
    nz = np.arange(1, q)
    assert field.gf_dot(nz, field.gf_pow(nz, q - 2, p, k, m), p, k, m) == p - 1
    rng = np.random.default_rng(7 * q)
    a, b, c = (rng.integers(0, q, 50) for _ in range(3))
    fold = 0
    for s, t in zip(a, b):
        fold = int(field.gf_add(np.array(fold), field.gf_mul(np.array(s), np.array(t), p, k, m), p, k))
    assert field.gf_dot(a, b, p, k, m) == fold
    lhs = field.gf_dot(a, field.gf_add(b, c, p, k), p, k, m)
    rhs = field.gf_add(np.array(field.gf_dot(a, b, p, k, m)), np.array(field.gf_dot(a, c, p, k, m)), p, k)
    assert lhs == int(rhs)


@pytest.mark.parametrize("p,k", [(3, 5), (7, 2), (2, 8), (5, 1), (3, 2)])
def test_gf_matmul_ring_laws(p, k):
    """The GF(p^k) matrix product: the identity matrix is neutral, the product is associative
    and distributes over addition, every entry is the row-by-column field dot product, and for
    k = 1 it is the prime-field product mod p."""
    m = field.smallest_monic_irreducible(p, k)
    q = p ** k
    rng = np.random.default_rng(q + 3)
    A, B, C = rng.integers(0, q, (4, 6)), rng.integers(0, q, (6, 5)), rng.integers(0, q, (5, 3))
    mm = lambda x, y: field.gf_matmul(x, y, p, k, m)
    eye = np.eye(6, dtype=np.int64)                 # index 1 is the field's one
    assert np.array_equal(mm(A, eye), A)
    assert np.array_equal(mm(mm(A, B), C), mm(A, mm(B, C)))
    B2 = rng.integers(0, q, (6, 5))
    assert np.array_equal(mm(A, field.gf_add(B, B2, p, k)), field.gf_add(mm(A, B), mm(A, B2), p, k))
    AB = mm(A, B)
    for i in range(4):
        for j in range(5):
            assert AB[i, j] == field.gf_dot(A[i], B[:, j], p, k, m)
    if k == 1:
        assert np.array_equal(AB, field.matmul_mod(A, B, p))
