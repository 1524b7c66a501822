"""Discrete Q-adic Transform, its inverse and REDQ (oracle; test infrastructure only).

All functions take exact integers: Python ints (arbitrary precision, needed for the paper's
examples beyond 2^64) or numpy integer arrays (element-wise, for exhaustive tests).  Floor
division // and % are the mathematical ones for non-negative operands.
"""
from __future__ import annotations

import numpy as np


def dqt(coeffs, q):
    """Eq. dqt: sum_i alpha_i X^i -> sum_i alpha_i q^i, evaluated by Horner's rule from the
    highest coefficient (Sec. 2.1).  coeffs[..., i] is alpha_i."""
    coeffs = list(coeffs) if not isinstance(coeffs, np.ndarray) else coeffs
    if isinstance(coeffs, np.ndarray):
        c = coeffs.astype(object) if coeffs.dtype != object else coeffs
        r = np.zeros(c.shape[:-1], dtype=object)
        for i in range(c.shape[-1] - 1, -1, -1):
            r = r * q + c[..., i]
        return r
    r = 0
    for a in reversed(coeffs):
        r = r * q + int(a)
    return r


def radix_digits(r, q, ndig):
    """Radix conversion (the first inverse step of Algorithm 1): r = sum_{i<ndig} mu~_i q^i with 0 <= mu~_i < q
    for i < ndig-1; the top digit takes whatever is left (floor(r / q^(ndig-1)))."""
    out = []
    for i in range(ndig):
        if i < ndig - 1:
            out.append(r % q)
            r = r // q
        else:
            out.append(r)
    return out


def dqt_inverse(r, q, ndig, p):
    """Inverse DQT: radix conversion then each digit mod p (the inverse in Algorithm 1)."""
    return [d % p for d in radix_digits(r, q, ndig)]


def redq_compression(r, p, q, d):
    """REDQ COMPRESSION (Algorithm 2): s = floor(r/p); u_i = floor(r/q^i) - p floor(s/q^i),
    i = 0..d.  Theorem REDQ shows 0 <= u_i < p."""
    s = r // p
    return [r // q ** i - p * (s // q ** i) for i in range(d + 1)]


def redq_correction(u, p, q):
    """REDQ CORRECTION (Algorithm 2, needed when p does not divide q):
    mu_d = u_d and mu_i = (u_i - q u_{i+1}) mod p for i < d."""
    d = len(u) - 1
    mu = [None] * (d + 1)
    mu[d] = u[d]
    for i in range(d):
        mu[i] = (u[i] - q * u[i + 1]) % p
    return mu


def redq(r, p, q, d):
    """REDQ_{d+1} (Algorithm 2): the d+1 residues mu_i = mu~_i mod p of r = sum mu~_i q^i.
    When p divides q the correction is skipped (u_i is already mu_i)."""
    u = redq_compression(r, p, q, d)
    if q % p == 0:
        return u
    return redq_correction(u, p, q)


def correction_matrix(k, p, q):
    """Q_k (Sec. 3.4): the k x k upper bidiagonal matrix with 1 on the diagonal and -q mod p
    on the superdiagonal, so that mu = Q_k u mod p."""
    m = np.zeros((k, k), dtype=np.int64)
    for i in range(k):
        m[i, i] = 1
        if i + 1 < k:
            m[i, i + 1] = (-q) % p
    return m


def q2_table(p, q):
    """Table of the 2x3 map underline{Q}_2 (Example tmto): for every (u0,u1,u2) in F_p^3,
    the first two rows of Q_2 applied to it, (u0 - q u1 mod p, u1 - q u2 mod p).
    Indexed by u0 + u1 p + u2 p^2 (Note on Indexing)."""
    t = {}
    for u0 in range(p):
        for u1 in range(p):
            for u2 in range(p):
                t[u0 + u1 * p + u2 * p * p] = ((u0 - q * u1) % p, (u1 - q * u2) % p)
    return t


def q6_by_q2(u, p, table):
    """Example tmto's algorithm: Q_6 applied to [u_0..u_6] with three lookups in the
    underline{Q}_2 table (extra memory p^3)."""
    a = table[u[0] + u[1] * p + u[2] * p * p]
    b = table[u[2] + u[3] * p + u[4] * p * p]
    c = table[u[4] + u[5] * p + u[6] * p * p]
    return [a[0], a[1], b[0], b[1], c[0], c[1], u[6]]


# --------------------------------------------------------------------------- compressed mm
def right_compress(B, e, Q):
    """Right compression (Sec. 7.4): CB[l][j] = sum_{t<e} B[l][j e + t] Q^t, with missing
    columns of a ragged last block taken as zero (partial compression, Sec. 7.1).
    Returns an object array of exact integers, shape [k, ceil(n/e)]."""
    B = np.asarray(B, dtype=np.int64)
    k, n = B.shape
    nw = -(-n // e)
    CB = np.zeros((k, nw), dtype=object)
    for j in range(nw):
        for t in range(e - 1, -1, -1):
            col = j * e + t
            v = B[:, col].astype(object) if col < n else np.zeros(k, dtype=object)
            CB[:, j] = CB[:, j] * Q + v
    return CB


def right_compressed_product(A, B, p, e, Q):
    """Eq. LeftComp with an uncompressed A: CC = A x CB in exact integers, then each word
    reduced to its e residues by REDQ_e; returns C (m x n) mod p."""
    A = np.asarray(A, dtype=np.int64)
    m, k = A.shape
    n = np.asarray(B).shape[1]
    CB = right_compress(B, e, Q)
    CC = A.astype(object) @ CB
    C = np.zeros((m, n), dtype=np.int64)
    for i in range(m):
        for j in range(CB.shape[1]):
            mu = redq(int(CC[i, j]), p, Q, e - 1)
            for t in range(e):
                if j * e + t < n:
                    C[i, j * e + t] = mu[t]
    return C


def split_plan(k, chunk, p, beta):
    """Inner-dimension splitting (Sec. 7.6, after Table comprange): the inner dimension k is cut
    into pieces of at most `chunk`; each piece gets its own Q (Eq. lower for the piece's length)
    and compression e = floor(beta / log2 Q) (Sec. 7.6.1).  Returns [(start, length, Q, e)]."""
    from .bounds import cmm_Q, compression_factor
    plan = []
    for l0 in range(0, k, chunk):
        kc = min(chunk, k - l0)
        Q = cmm_Q(kc, p)
        plan.append((l0, kc, Q, compression_factor(beta, Q)))
    return plan


def split_right_compressed_product(A, B, p, chunk, beta):
    """Right-compressed product with the inner dimension split by split_plan: each piece is a
    right-compressed product reduced by REDQ (the extra modular reductions), and the pieces'
    results are added mod p.  Returns C (m x n) mod p."""
    A = np.asarray(A, dtype=np.int64)
    B = np.asarray(B, dtype=np.int64)
    C = np.zeros((A.shape[0], B.shape[1]), dtype=np.int64)
    for l0, kc, Q, e in split_plan(A.shape[1], chunk, p, beta):
        C = (C + right_compressed_product(A[:, l0:l0 + kc], B[l0:l0 + kc, :], p, e, Q)) % p
    return C


def full_compress_rows(A, dq, Q):
    """Full compression, left operand (Sec. 7.5): word [r][l] = sum_{i<=dq} A[r(dq+1)+i][l] Q^i,
    missing rows of a ragged last block taken as zero.  Exact integers, shape [ceil(m/(dq+1)), k]."""
    A = np.asarray(A, dtype=np.int64)
    m, k = A.shape
    nr = -(-m // (dq + 1))
    W = np.zeros((nr, k), dtype=object)
    for r in range(nr):
        for i in range(dq, -1, -1):
            row = r * (dq + 1) + i
            v = A[row, :].astype(object) if row < m else np.zeros(k, dtype=object)
            W[r, :] = W[r, :] * Q + v
    return W


def full_compress_cols(B, dt, Theta):
    """Full compression, right operand (Sec. 7.5): word [l][c] = sum_{j<=dt} B[l][c(dt+1)+j]
    Theta^j, missing columns of a ragged last block taken as zero.  Shape [k, ceil(n/(dt+1))]."""
    return right_compress(B, dt + 1, Theta)


def full_compressed_product(A, B, p, dq, dt, Q, s):
    """Full compression (Sec. 7.5) with Theta = Q^s, s >= dq + 1 (Eq. qtheta): the exact
    integer product of the compressed operands holds C[r(dq+1)+i][c(dt+1)+j] as the coefficient
    of Q^i Theta^j = Q^(i + s j); with every coefficient below Q (Eq. lower) the word is a base-Q
    number and REDQ over its s dt + dq + 1 digits gives them mod p.  Returns C (m x n) mod p."""
    assert s >= dq + 1
    A = np.asarray(A, dtype=np.int64)
    B = np.asarray(B, dtype=np.int64)
    m, n = A.shape[0], B.shape[1]
    WA = full_compress_rows(A, dq, Q)
    WB = full_compress_cols(B, dt, Q ** s)
    CC = WA @ WB
    C = np.zeros((m, n), dtype=np.int64)
    ndig = s * dt + dq + 1
    for r in range(CC.shape[0]):
        for c in range(CC.shape[1]):
            mu = redq(int(CC[r, c]), p, Q, ndig - 1)
            for i in range(dq + 1):
                for j in range(dt + 1):
                    row, col = r * (dq + 1) + i, c * (dt + 1) + j
                    if row < m and col < n:
                        C[row, col] = mu[i + s * j]
    return C


def middle_product_dot(u, v, p, d, Q):
    """Middle-product dot product (Sec. 7.1): blocks of d+1 entries are packed reversed on
    the left (sum_t u_{l(d+1)+t} Q^{d-t}) and forward on the right; the coefficient of Q^d of
    the summed word products is the dot product.  Exact integers; returns it mod p."""
    u = [int(x) for x in u]
    v = [int(x) for x in v]
    n = len(u)
    nb = -(-n // (d + 1))
    acc = 0
    for blk in range(nb):
        cu = 0
        cv = 0
        for t in range(d + 1):
            idx = blk * (d + 1) + t
            uu = u[idx] if idx < n else 0
            vv = v[idx] if idx < n else 0
            cu += uu * Q ** (d - t)
            cv += vv * Q ** t
        acc += cu * cv
    return (acc // Q ** d) % Q % p
