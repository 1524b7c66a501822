"""Pins of the oracle's FDIV/AFDIV software float against Table "fdiv" (Sec. 4): the
guaranteed ranges and bounds on r checked exhaustively for small mantissas, the paper's
counterexample family for case 2, and AFDIV exact for every r."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import fdiv


def test_round_to_beta_matches_ieee_double():
    # With beta = 53 the three directions bracket Python's correctly rounded 1/p.
    import math
    for p in (3, 5, 7, 23, 1009, 65521, 2 ** 31 - 1):
        m_near, e = fdiv.round_to_beta(1, p, 53, "near")
        assert m_near * 2.0 ** e == 1.0 / p
        m_up, eu = fdiv.round_to_beta(1, p, 53, "up")
        m_dn, ed = fdiv.round_to_beta(1, p, 53, "down")
        assert m_dn * 2.0 ** ed == math.nextafter(m_up * 2.0 ** eu, 0.0)
        assert Fraction(m_dn) * Fraction(2) ** ed < Fraction(1, p) < Fraction(m_up) * Fraction(2) ** eu


@pytest.mark.parametrize("beta", [6, 8, 10])
@pytest.mark.parametrize("case", range(1, 10))
def test_fdiv_table_exhaustive(beta, case):
    """For every 0 <= r < 2^beta and 1 <= p < 2^beta: floor(x) - k lies in the Range column,
    and floor(x) <= k whenever r is below the 'Bound on r' column."""
    c1, c2 = fdiv.CASES[case]
    fx, k = fdiv.fdiv_table_numpy(beta, c1, c2)
    diff = fx - k
    lo, hi = fdiv.TABLE_RANGE[case]
    assert diff.min() >= lo and diff.max() <= hi
    B = fdiv.table_bound(case, beta)
    r = np.arange(1 << beta)
    if B is None:
        assert diff.max() <= 0
    else:
        below = r < float(B)     # B is not an integer for the odd denominators; r integer
        assert diff[:, below].max() <= 0
    if lo == 0:
        assert diff.min() >= 0   # cases 1-4 never fall below k


def test_fdiv_numpy_matches_exact_scalar():
    rng = np.random.default_rng(0)
    for case in range(1, 10):
        c1, c2 = fdiv.CASES[case]
        fx, _ = fdiv.fdiv_table_numpy(10, c1, c2)
        for _ in range(300):
            r = int(rng.integers(0, 1024))
            p = int(rng.integers(1, 1024))
            assert fx[p - 1, r] == fdiv.fdiv(r, p, 10, c1, c2)


def test_fdiv_off_by_at_most_one_double():
    """Lemma: never off by more than one (beta = 53, random r, several p)."""
    rng = np.random.default_rng(1)
    for case in range(1, 10):
        c1, c2 = fdiv.CASES[case]
        for p in (3, 5, 7, 17, 31, 65537):
            for _ in range(50):
                r = int(rng.integers(0, 2 ** 53 - 1, dtype=np.int64))
                assert abs(fdiv.fdiv(r, p, 53, c1, c2) - r // p) <= 1


@pytest.mark.parametrize("n", range(4, 13))
def test_case2_counterexample_family(n):
    """Sec. 4.3: beta = 2n+1, p = 2^n - 1, r = (3 2^(n-2) + 3) p - 1 gives floor(x) = k+1 in
    case 2, with r above the table's bound (so the table is not contradicted) and r/2^beta
    tending to 3/8."""
    beta = 2 * n + 1
    p = 2 ** n - 1
    r = (3 * 2 ** (n - 2) + 3) * p - 1
    assert fdiv.fdiv(r, p, beta, "up", "near") == r // p + 1
    assert r >= fdiv.table_bound(2, beta)
    assert abs(Fraction(r, 2 ** beta) - Fraction(3, 8)) < Fraction(3, 2 ** (n - 1))


@pytest.mark.parametrize("mode", fdiv.MODES)
def test_afdiv_exact_everywhere(mode):
    beta = 9
    for p in range(1, 1 << beta):
        for r in range(0, 1 << beta, 3):
            assert fdiv.afdiv(r, p, beta, mode) == r // p


def test_case3_exact_below_half_double():
    """Case 3 (invp rounded up, product rounded down) is exact for r < 2^(beta-1); this is
    the mode the packed words use.  Edge values around multiples of p up to 2^52."""
    for p in (2, 3, 5, 7, 17, 31, 251):
        for top in (2 ** 52 - 1, 2 ** 40, 298116, 2 ** 23 - 1):
            for r in range(max(0, top - 2 * p), top + 1):
                assert fdiv.fdiv(r, p, 53, "up", "down") == r // p
        for r in (2 ** 23 - 1, 2 ** 22 + 5, 12345):
            assert fdiv.fdiv(r, p, 24, "up", "down") == r // p
