"""Plain definitions over F_p and GF(p^k) (oracle; test infrastructure only).

Every result of the packed hot path is an exact mathematical object with a plain definition;
this module writes those definitions out with numpy integer arithmetic and a final % p.
"""
from __future__ import annotations

import itertools

import numpy as np


# --------------------------------------------------------------------------- prime field
def polymul_mod(a, b, p):
    """Batched polynomial product over F_p.

    a: [batch, ka], b: [batch, kb] coefficient arrays (low degree first).
    Returns c: [batch, ka+kb-1] with c_j = (sum_i a_i b_{j-i}) mod p, the convolution sums of
    Eq. mult (Sec. 2.1) reduced mod p.
    """
    a = np.asarray(a, dtype=np.int64)
    b = np.asarray(b, dtype=np.int64)
    squeeze = a.ndim == 1
    if squeeze:
        a, b = a[None, :], b[None, :]
    batch, ka = a.shape
    kb = b.shape[1]
    c = np.zeros((batch, ka + kb - 1), dtype=np.int64)
    for i in range(ka):
        for j in range(kb):
            c[:, i + j] += a[:, i] * b[:, j]
    c %= p
    return c[0] if squeeze else c


def dot_mod(u, v, p):
    """(sum_i u_i v_i) mod p: Algorithm 1's ensured value for degree-0 polynomials."""
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    return int(np.sum(u * v) % p)


def matmul_mod(A, B, p):
    """C_ij = (sum_l A_il B_lj) mod p (Sec. 7: the product that compressed schemes compute)."""
    A = np.asarray(A, dtype=np.int64)
    B = np.asarray(B, dtype=np.int64)
    return (A @ B) % p


def matmul_mod_rows(A, B, p, rows):
    """Selected rows of matmul_mod, for sampled parity at sizes the full product is too slow."""
    A = np.asarray(A, dtype=np.int64)[rows]
    return (A @ np.asarray(B, dtype=np.int64)) % p


# --------------------------------------------------------------------------- polynomials
def poly_rem_mod(c, modulus, p):
    """Remainder of c (low degree first, [..., m]) by a monic modulus of degree k, mod p,
    by schoolbook long division.  Returns [..., k]."""
    c = np.array(c, dtype=np.int64) % p
    modulus = [int(x) % p for x in modulus]
    k = len(modulus) - 1
    assert modulus[k] == 1, "modulus must be monic"
    m = c.shape[-1]
    for deg in range(m - 1, k - 1, -1):
        lead = c[..., deg].copy()
        for i in range(k + 1):
            c[..., deg - k + i] = (c[..., deg - k + i] - lead * modulus[i]) % p
    out = np.zeros(c.shape[:-1] + (k,), dtype=np.int64)
    out[..., :min(k, m)] = c[..., :min(k, m)]
    return out


def index_to_coeffs(x, p, k):
    """Element index sum_i c_i p^i -> coefficients [..., k] (c_0 first)."""
    x = np.asarray(x, dtype=np.int64)
    out = np.zeros(x.shape + (k,), dtype=np.int64)
    for i in range(k):
        out[..., i] = x % p
        x = x // p
    return out


def coeffs_to_index(c, p):
    c = np.asarray(c, dtype=np.int64)
    k = c.shape[-1]
    x = np.zeros(c.shape[:-1], dtype=np.int64)
    for i in range(k - 1, -1, -1):
        x = x * p + c[..., i]
    return x


def is_irreducible(f, p):
    """Brute-force irreducibility of a monic polynomial f (coefficients low first) over F_p:
    f of degree k is irreducible iff no monic polynomial of degree 1..k//2 divides it."""
    k = len(f) - 1
    f = np.array(f, dtype=np.int64)
    for deg in range(1, k // 2 + 1):
        for low in itertools.product(range(p), repeat=deg):
            g = list(low) + [1]
            if not np.any(poly_rem_mod(f, g, p)[:deg]):
                return False
    return True


def monic_candidates(p, k):
    """Monic degree-k polynomials in increasing order of the key sum_{i<k} c_i p^i."""
    for key in range(p ** k):
        low = [(key // p ** i) % p for i in range(k)]
        yield key, low + [1]


def smallest_monic_irreducible(p, k):
    """The monic irreducible of degree k with the smallest key sum_{i<k} c_i p^i."""
    for _, f in monic_candidates(p, k):
        if is_irreducible(f, p):
            return f
    raise ValueError("no irreducible found")  # unreachable for prime p


def count_monic_irreducibles(p, k):
    return sum(1 for _, f in monic_candidates(p, k) if is_irreducible(f, p))


def gf_mul(a, b, p, k, modulus):
    """GF(p^k) product of element indices: schoolbook product mod p, then the remainder by
    the monic modulus (Sec. 6: polynomials modulo p and modulo an irreducible of degree k)."""
    ca = index_to_coeffs(a, p, k)
    cb = index_to_coeffs(b, p, k)
    prod = np.zeros(ca.shape[:-1] + (2 * k - 1,), dtype=np.int64)
    for i in range(k):
        for j in range(k):
            prod[..., i + j] += ca[..., i] * cb[..., j]
    prod %= p
    return coeffs_to_index(poly_rem_mod(prod, modulus, p), p)


def gf_add(a, b, p, k):
    return coeffs_to_index((index_to_coeffs(a, p, k) + index_to_coeffs(b, p, k)) % p, p)


def gf_pow(a, e, p, k, modulus):
    a = np.asarray(a, dtype=np.int64)
    r = np.ones_like(a)
    base = a.copy()
    while e:
        if e & 1:
            r = gf_mul(r, base, p, k, modulus)
        base = gf_mul(base, base, p, k, modulus)
        e >>= 1
    return r


def gf_dot(a, b, p, k, modulus):
    """Dot product over GF(p^k) (the value Algorithm FGDP returns, Sec. 6): sum_i a_i b_i in the
    field, for index vectors a, b.  Written as the sum over i of the coefficient convolutions of
    a_i(X) b_i(X), reduced mod p and then by the modulus once (reduction is a ring homomorphism,
    so this equals folding gf_mul with gf_add).  Returns the element index."""
    ca = index_to_coeffs(np.asarray(a, dtype=np.int64), p, k)
    cb = index_to_coeffs(np.asarray(b, dtype=np.int64), p, k)
    s = np.zeros(2 * k - 1, dtype=np.int64)
    for i in range(k):
        for j in range(k):
            s[i + j] = (s[i + j] + int((ca[..., i] * cb[..., j]).sum() % p)) % p
    return int(coeffs_to_index(poly_rem_mod(s, modulus, p), p))


def _prime_factors(n):
    out, d = [], 2
    while d * d <= n:
        if n % d == 0:
            out.append(d)
            while n % d == 0:
                n //= d
        d += 1
    if n > 1:
        out.append(n)
    return out


def primitive_element(p, k, modulus):
    """The generator used for the discrete-log element form: the smallest index g whose
    multiplicative order is p^k - 1, tested by g^((p^k - 1) / r) != 1 for every prime r of
    p^k - 1 (Lagrange)."""
    n = p ** k - 1
    if n == 1:
        return 1
    for g in range(2, p ** k):
        if all(int(gf_pow(np.array(g), n // r, p, k, modulus)) != 1 for r in _prime_factors(n)):
            return g
    raise ValueError("no primitive element")


def log_tables(p, k, modulus):
    """Discrete-log form of GF(p^k) (the element representation Algorithm FGDP assumes): the
    element g^e is written e, 0 <= e <= p^k - 2, and zero is written p^k - 1.  Returns
    (antilog, log): antilog[e] = index of g^e (antilog[p^k - 1] = 0) and log[x] = its inverse."""
    order = p ** k
    g = primitive_element(p, k, modulus)
    antilog = np.zeros(order, dtype=np.int64)
    x = 1
    for e in range(order - 1):
        antilog[e] = x
        x = int(gf_mul(np.array(x), np.array(g), p, k, modulus))
    antilog[order - 1] = 0
    log = np.zeros(order, dtype=np.int64)
    log[antilog] = np.arange(order)
    return antilog, log


def gf_matmul(A, B, p, k, modulus):
    """Matrix product over GF(p^k) (the matrix case of Algorithm FGDP's dot product, Sec. 6):
    C[i][j] = sum_l A[i][l] B[l][j] in the field, for index matrices.  Written as the coefficient
    convolutions of every product summed over l, reduced mod p and then by the modulus once."""
    ca = index_to_coeffs(np.asarray(A, dtype=np.int64), p, k)        # [m][kk][k]
    cb = index_to_coeffs(np.asarray(B, dtype=np.int64), p, k)        # [kk][n][k]
    m, n = ca.shape[0], cb.shape[1]
    s = np.zeros((m, n, 2 * k - 1), dtype=np.int64)
    for i in range(k):
        for j in range(k):
            s[:, :, i + j] = (s[:, :, i + j] + (ca[:, :, i] @ cb[:, :, j]) % p) % p
    return coeffs_to_index(poly_rem_mod(s, modulus, p), p)
