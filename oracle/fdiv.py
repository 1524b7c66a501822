"""Euclidean division by floating-point routines (Sec. 4), in exact software arithmetic
(oracle; test infrastructure only).

A "beta-bit float" here is m * 2^E with an integer significand m < 2^beta; rounding of an
exact rational to beta significant bits is done with integers only, in the three IEEE
directions: 'up' (towards +inf), 'down' (towards -inf) and 'near' (to nearest, ties to even).
All operands are positive, as in Algorithm FDIV.
"""
from __future__ import annotations

import numpy as np

MODES = ("up", "near", "down")
# (circ_1, circ_2) of the nine cases of Table "fdiv", in the paper's order.
CASES = {1: ("up", "up"), 2: ("up", "near"), 3: ("up", "down"),
         4: ("near", "up"), 5: ("near", "near"), 6: ("near", "down"),
         7: ("down", "up"), 8: ("down", "near"), 9: ("down", "down")}


def _round_shift(N, s, mode):
    """Round N / 2^s (N >= 0 integer, s >= 0) to an integer in the given direction."""
    if s <= 0:
        return N << (-s)
    m = N >> s
    rem = N - (m << s)
    if mode == "down":
        return m
    if mode == "up":
        return m + (1 if rem else 0)
    half = 1 << (s - 1)
    if rem > half or (rem == half and (m & 1)):
        return m + 1
    return m


def round_to_beta(num, den, beta, mode):
    """Round the positive rational num/den to beta significant bits.
    Returns (m, E) with value m * 2^E (m may equal 2^beta after rounding up)."""
    assert num > 0 and den > 0
    # exponent so that 2^(beta-1) <= num/den * 2^(-E) < 2^beta
    E = num.bit_length() - den.bit_length() - beta
    while (num << max(0, -E)) < ((den << max(0, E)) << (beta - 1)):
        E -= 1
    while (num << max(0, -E)) >= ((den << max(0, E)) << beta):
        E += 1
    # significand = num / (den 2^E), rounded
    if E >= 0:
        n2, d2 = num, den << E
    else:
        n2, d2 = num << (-E), den
    m, rem = divmod(n2, d2)
    if rem:
        if mode == "up":
            m += 1
        elif mode == "near":
            if 2 * rem > d2 or (2 * rem == d2 and (m & 1)):
                m += 1
    return m, E


def fdiv(r, p, beta, c1, c2):
    """Algorithm FDIV: invp = circ_1(1/p); x = circ_2(r * invp); return floor(x).
    Exact for any integers 0 <= r, 1 <= p (no overflow: Python ints)."""
    mi, ei = round_to_beta(1, p, beta, c1)
    if r == 0:
        return 0
    N = r * mi                     # r * invp = N * 2^ei exactly
    L = N.bit_length()
    s = max(0, L - beta)
    m = _round_shift(N, s, c2)     # x = m * 2^(ei + s)
    e = ei + s
    return m << e if e >= 0 else m >> (-e)


def fdiv_table_numpy(beta, c1, c2, r_max=None, p_max=None):
    """Vectorised FDIV over all 0 <= r < r_max and 1 <= p < p_max (default 2^beta) for
    small beta (<= 14, so that r * significand fits in int64).
    Returns (floor_x, k) arrays of shape [p_max-1, r_max]."""
    assert beta <= 14
    r_max = r_max or (1 << beta)
    p_max = p_max or (1 << beta)
    r = np.arange(r_max, dtype=np.int64)
    fx = np.zeros((p_max - 1, r_max), dtype=np.int64)
    kk = np.zeros((p_max - 1, r_max), dtype=np.int64)
    for p in range(1, p_max):
        mi, ei = round_to_beta(1, p, beta, c1)
        N = r * mi
        L = np.zeros_like(N)
        nz = N > 0
        L[nz] = np.floor(np.log2(N[nz].astype(np.float64))).astype(np.int64) + 1
        # guard the float log2 near powers of two
        L[nz] += (N[nz] >> L[nz]) > 0
        L[nz] -= (N[nz] >> np.maximum(L[nz] - 1, 0)) == 0
        s = np.maximum(0, L - beta)
        m = N >> s
        rem = N - (m << s)
        if c2 == "up":
            m = m + (rem > 0)
        elif c2 == "near":
            half = np.where(s > 0, np.left_shift(np.int64(1), np.maximum(s - 1, 0)), 0)
            m = m + ((s > 0) & ((rem > half) | ((rem == half) & ((m & 1) == 1))))
        e = ei + s
        fx[p - 1] = np.where(e >= 0, m << np.maximum(e, 0), m >> np.maximum(-e, 0))
        kk[p - 1] = r // p
    return fx, kk


def table_bound(case, beta):
    """Strict upper bound on r from Table "fdiv" below which floor(x) <= k (None: always)."""
    from fractions import Fraction as F
    two_b = F(2) ** beta
    return {1: two_b / (4 + F(2) ** (2 - beta)),
            2: two_b / (3 + F(2) ** (1 - beta)),
            3: two_b / 2,
            4: two_b / (3 + F(2) ** (1 - beta)),
            5: F(2) ** (beta - 1) / (1 + F(2) ** (-1 - beta)),
            6: None, 7: two_b / 2, 8: None, 9: None}[case]


TABLE_RANGE = {1: (0, 1), 2: (0, 1), 3: (0, 1), 4: (0, 1), 5: (-1, 1),
               6: (-1, 0), 7: (-1, 1), 8: (-1, 0), 9: (-1, 0)}
"""Table "fdiv" column Range: floor(x) - k lies in this closed interval."""


def afdiv(r, p, beta, mode):
    """Algorithm AFDIV for the current rounding mode circ_2 = mode: multiply by the inverse
    precomputed for that mode, floor, and one correction test when r >= B_mode."""
    from fractions import Fraction as F
    B = {"up": F(2) ** beta / (3 + F(2) ** (1 - beta)),
         "near": F(2) ** beta / (3 + F(2) ** (1 - beta)),
         "down": F(2) ** (beta - 1)}[mode]
    c1 = {"up": "near", "near": "up", "down": "up"}[mode]
    y = fdiv(r, p, beta, c1, mode)
    if r >= B:
        if p * y > r:
            y -= 1
    return y
