"""Property tests of the oracle at sizes the exhaustive pins cannot reach: Theorem REDQ for
large q, k and p, the exactness range of FDIV case 3 for any mantissa width, the middle-product
and right-compression identities of Sec. 7 on random shapes, and the GF(p^k) dot product's
bilinearity.  Each property compares two independently written computations (or a closed
form), so a wrong index, sign or bound in either fails it."""
import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

from oracle import dqt, fdiv, field  # noqa: E402

PRIMES = [2, 3, 5, 7, 11, 13, 17, 31, 61, 127, 251]
SETTINGS = dict(max_examples=150, deadline=None)


@settings(**SETTINGS)
@given(p=st.sampled_from(PRIMES), b=st.integers(1, 30), k=st.integers(1, 9), seed=st.integers(0, 2 ** 32 - 1))
def test_redq_equals_radix_conversion_for_any_digits_below_q(p, b, k, seed):
    """Theorem REDQ: for r = sum mu~_i q^i with every digit below q except the top one (which
    takes whatever is left), REDQ gives mu~_i mod p for every i, as radix conversion does."""
    q = 1 << b
    if q < p:
        q = 1 << p.bit_length()
    rng = np.random.default_rng(seed)
    d = 2 * k - 2
    digits = [int(x) for x in rng.integers(0, q, d)] + [int(rng.integers(0, 1 << 20))]
    r = sum(c * q ** i for i, c in enumerate(digits))
    assert dqt.redq(r, p, q, d) == [c % p for c in digits]
    assert dqt.dqt_inverse(r, q, d + 1, p) == [c % p for c in digits]


@settings(**SETTINGS)
@given(p=st.sampled_from(PRIMES), k=st.integers(1, 8), n=st.integers(1, 50), seed=st.integers(0, 2 ** 32 - 1))
def test_packed_dot_of_polynomials_matches_convolution(p, k, n, seed):
    """Eq. mult with delayed reduction: the sum of n packed products at the Theorem's q
    (q > n k (p-1)^2) carries every convolution coefficient in its own digit."""
    q = 2
    while q <= n * k * (p - 1) ** 2 or q < p:
        q *= 2
    rng = np.random.default_rng(seed)
    a = rng.integers(0, p, (n, k))
    b = rng.integers(0, p, (n, k))
    r = sum(int(dqt.dqt(a[i], q)) * int(dqt.dqt(b[i], q)) for i in range(n))
    want = field.polymul_mod(a, b, p).sum(axis=0) % p
    assert dqt.redq(r, p, q, 2 * k - 2) == [int(x) for x in want]


@settings(**SETTINGS)
@given(p=st.integers(2, 2 ** 20), beta=st.integers(8, 60), seed=st.integers(0, 2 ** 32 - 1))
def test_fdiv_case3_exact_below_half_mantissa_range(p, beta, seed):
    """Table fdiv, case 3 (1/p rounded up, the product rounded down): floor(r/p) exactly for
    every 0 <= r < 2^(beta-1), at any mantissa width; checked at random r and at the edges
    next to multiples of p."""
    rng = np.random.default_rng(seed)
    top = (1 << (beta - 1)) - 1
    rs = {0, top, max(0, top - 1)}
    rs |= {int(x) for x in rng.integers(0, top + 1, 20, dtype=np.uint64)} if top < 2 ** 63 else set()
    m = top // p
    rs |= {max(0, m * p - 1), m * p, min(top, m * p + p - 1)}
    for r in rs:
        assert fdiv.fdiv(r, p, beta, "up", "down") == r // p


@settings(**SETTINGS)
@given(p=st.sampled_from(PRIMES[:7]), n=st.integers(1, 200), d=st.integers(0, 6), seed=st.integers(0, 2 ** 32 - 1))
def test_middle_product_dot_matches_plain_dot(p, n, d, seed):
    """Sec. 7.1: blocks packed reversed on the left and forward on the right put the dot
    product in the coefficient of Q^d whenever Q > n (p-1)^2 (the digit bound)."""
    Q = 2
    while Q <= n * (p - 1) ** 2:
        Q *= 2
    rng = np.random.default_rng(seed)
    u = rng.integers(0, p, n)
    v = rng.integers(0, p, n)
    assert dqt.middle_product_dot(u, v, p, d, Q) == field.dot_mod(u, v, p)


@settings(max_examples=60, deadline=None)
@given(p=st.sampled_from(PRIMES[:6]), m=st.integers(1, 9), k=st.integers(1, 40), n=st.integers(1, 13),
       e=st.integers(1, 4), seed=st.integers(0, 2 ** 32 - 1))
def test_right_compressed_product_matches_plain_product(p, m, k, n, e, seed):
    """Sec. 7.4: right compression of B with e entries per word at Q > k (p-1)^2, then REDQ_e of
    every word of A CB, gives A B mod p for any shape, including a ragged last block."""
    Q = 2
    while Q <= k * (p - 1) ** 2:
        Q *= 2
    rng = np.random.default_rng(seed)
    A = rng.integers(0, p, (m, k))
    B = rng.integers(0, p, (k, n))
    assert np.array_equal(dqt.right_compressed_product(A, B, p, e, Q), field.matmul_mod(A, B, p))


@settings(max_examples=40, deadline=None)
@given(pk=st.sampled_from([(2, 3), (3, 2), (3, 5), (5, 2), (7, 2), (2, 8), (13, 1)]), n=st.integers(1, 60),
       seed=st.integers(0, 2 ** 32 - 1))
def test_gf_dot_is_symmetric_and_bilinear(pk, n, seed):
    """The GF(p^k) dot product is symmetric, additive in each argument, and homogeneous:
    dot(c a, b) = c dot(a, b) for a scalar c of the field."""
    p, k = pk
    m = field.smallest_monic_irreducible(p, k)
    q = p ** k
    rng = np.random.default_rng(seed)
    a, b, c = (rng.integers(0, q, n) for _ in range(3))
    s = int(rng.integers(0, q))
    dot = lambda x, y: field.gf_dot(x, y, p, k, m)
    assert dot(a, b) == dot(b, a)
    assert dot(field.gf_add(a, c, p, k), b) == int(field.gf_add(np.array(dot(a, b)), np.array(dot(c, b)), p, k))
    sa = field.gf_mul(np.full(n, s), a, p, k, m)
    assert dot(sa, b) == int(field.gf_mul(np.array(s), np.array(dot(a, b)), p, k, m))


@settings(max_examples=60, deadline=None)
@given(p=st.sampled_from(PRIMES[:5]), m=st.integers(1, 8), k=st.integers(1, 30), n=st.integers(1, 8),
       dq=st.integers(0, 3), dt=st.integers(0, 3), extra=st.integers(0, 2), seed=st.integers(0, 2 ** 32 - 1))
def test_full_compressed_product_matches_plain_product(p, m, k, n, dq, dt, extra, seed):
    """Sec. 7.5: compressing A's rows by Q and B's columns by Theta = Q^(dq+1+extra) (Eq.
    qtheta) with Q > k (p-1)^2 (Eq. lower) gives A B mod p for any shape and degrees."""
    Q = 2
    while Q <= k * (p - 1) ** 2:
        Q *= 2
    rng = np.random.default_rng(seed)
    A = rng.integers(0, p, (m, k))
    B = rng.integers(0, p, (k, n))
    assert np.array_equal(dqt.full_compressed_product(A, B, p, dq, dt, Q, dq + 1 + extra), field.matmul_mod(A, B, p))
