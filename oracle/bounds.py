"""Exactness bounds and cost model of the packed representation (oracle; tests only).

Notation: p prime, q = Q = 2^b, beta = mantissa bits of the word, n = accumulated products,
k = coefficients per packed operand, e = compression factor.
"""
from __future__ import annotations

import math


def thm_bounds_ok(q, n, k, p, beta):
    """Theorem (Eq. bounds, Sec. 2.3): Algorithm 1 is correct when q > n k (p-1)^2 and
    (2k-1) log2(q) <= beta."""
    return q > n * k * (p - 1) ** 2 and (2 * k - 1) * math.log2(q) <= beta


def smallest_pow2_q(bound):
    """Smallest q = 2^b with q > bound (the strict reading of Eq. bounds / Eq. lower)."""
    b = 0
    while (1 << b) <= bound:
        b += 1
    return 1 << b


def delayed_nd(p, beta):
    """Eq. delayed with the centered representation: n_d = floor(2^(beta+1) / (p-1)^2)."""
    return (2 ** (beta + 1)) // ((p - 1) ** 2)


def compression_factor(beta, Q):
    """Sec. 7.6.1: e = floor(beta / log2(Q))."""
    return int(beta // math.log2(Q))


def cmm_Q(kdim, p):
    """Eq. lower, strict: smallest power of two Q with k (p-1)^2 < Q."""
    return smallest_pow2_q(kdim * (p - 1) ** 2)


def cmm_upper_ok(Q, d, beta):
    """Eq. upper: Q^(d+1) < 2^beta."""
    return Q ** (d + 1) < 2 ** beta


def full_compression_ok(Q, Theta, dq, dtheta, beta):
    """Eq. qtheta and Eq. dq (Sec. 7.5): Q^(dq+1) <= Theta and Q^((dq+1)(dtheta+1)) < 2^beta."""
    return Q ** (dq + 1) <= Theta and Q ** ((dq + 1) * (dtheta + 1)) < 2 ** beta


def fqt_Dq(N, d):
    """Sec. 5.3: D_q = ceil((N+1)/(d+1)) - 1."""
    return -(-(N + 1) // (d + 1)) - 1


def mulpol_costs(p, N, d, beta, qbits_real=None):
    """Table "mulpol": (mul&add, reductions) of the delayed and the (d+1)-FQT products.
    n_q uses q = 2^(beta/(2d+1)) (real exponent) as in Sec. 5.3."""
    nd = delayed_nd(p, beta)
    delayed = ((2 * N + 1) ** 2, (2 * N + 1) * -(-(2 * N + 1) // nd))
    Dq = fqt_Dq(N, d)
    qb = beta / (2 * d + 1) if qbits_real is None else qbits_real
    nq = int(math.floor(2 ** qb / ((d + 1) * (p - 1) ** 2)))
    fqt = ((2 * Dq + 1) ** 2, (2 * Dq + 1) * -(-(2 * Dq + 1) // nq))
    return {"nd": nd, "Dq": Dq, "nq": nq, "delayed": delayed, "fqt": fqt}


def redq_axpy_count(k):
    """Proposition redqcost: REDQ_k compression costs ceil((k+1)/2) multiply-adds (q = 2^b)."""
    return -(-(k + 1) // 2)


def tmto_lookups(k, j):
    """Proposition (time-memory trade-off): with a table of size p^j, a REDQ_k correction
    takes floor((k-1)/(j-1)) table accesses (j >= 2)."""
    return (k - 1) // (j - 1)
