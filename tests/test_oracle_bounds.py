"""Pins of the oracle's bounds and cost model: Table "comprange" recomputed, the two
numeric examples under Table "mulpol", Proposition redqcost, and the strict reading of the
digit bound shown necessary by an adversarial all-(p-1) input."""
import math

import numpy as np

from oracle import bounds, dqt, field
from tests._golden import comprange


def test_comprange_table_recomputed():
    dims, comp = comprange()
    p, beta = 3, 53
    for qb, dim in dims:
        Q = 1 << qb
        # the Dimensions row is Q / (p-1)^2: the table reads Eq. lower as k (p-1)^2 <= Q
        assert dim == Q // (p - 1) ** 2
        # under the strict Eq. lower the same Q serves dimensions up to dim - 1
        assert bounds.cmm_Q(dim - 1, p) <= Q
        assert bounds.cmm_Q(dim, p) == 2 * Q
    for qb, e in comp:
        assert bounds.compression_factor(beta, 1 << qb) == e
        assert bounds.cmm_upper_ok(1 << qb, e - 1, beta)
        assert not bounds.cmm_upper_ok(1 << qb, e, beta)
    # first three columns: the compression is capped by the dimension itself
    for qb, dim in dims[:3]:
        assert min(dim, bounds.compression_factor(beta, 1 << qb)) == dim


def test_non_strict_bound_breaks_on_all_max_input():
    """With k (p-1)^2 = Q exactly (the table's boundary) an all-(p-1) right-compressed
    product carries out of the lowest digit and REDQ returns a wrong residue; with the
    strict bound (Q doubled) it is exact."""
    p, n, e = 3, 256, 2
    A = np.full((1, n), p - 1)
    B = np.full((n, e), p - 1)
    truth = field.matmul_mod(A, B, p)
    Q = n * (p - 1) ** 2                    # 1024 = 2^10, non-strict
    assert not np.array_equal(dqt.right_compressed_product(A, B, p, e, Q), truth)
    Qs = bounds.cmm_Q(n, p)
    assert Qs == 2048
    assert np.array_equal(dqt.right_compressed_product(A, B, p, e, Qs), truth)


def test_mulpol_example_p3_N500():
    c = bounds.mulpol_costs(3, 500, 3, 53)
    assert c["delayed"] == (1001 ** 2, 1001)          # ~1e6 mul&add, ~1e3 REDC
    assert c["Dq"] == 125
    assert c["fqt"][0] == 251 ** 2 == 63001
    assert c["nq"] == 11
    assert c["fqt"][1] == 251 * 23 == 5773           # ~5.7e3 REDQ_7
    axpy = bounds.redq_axpy_count(7)
    assert axpy == 4
    total = c["fqt"][0] + axpy * c["fqt"][1]
    assert round(total / 1e3) == 86                  # ~8.6e4
    assert 11 <= c["delayed"][0] / total < 12        # "a factor close to 11"


def test_mulpol_example_p1009_d2_beta128():
    c = bounds.mulpol_costs(1009, 500, 2, 128)
    assert c["Dq"] == 166
    assert c["fqt"][0] == 333 ** 2
    assert c["nq"] == 16
    assert c["fqt"][1] == 333 * 21 == 6993           # ~7e3 divisions
    total = c["fqt"][0] + bounds.redq_axpy_count(5) * c["fqt"][1]
    assert round(total / 1e4) == 13                  # ~1.3e5
    assert 7 <= (1001 ** 2) / total < 8              # "reduced by a factor of 7"


def test_redq_axpy_count_prop():
    # Proposition redqcost: b_q k (k+1)/2 <= beta ceil((k+1)/2) whenever b_q k <= beta
    for beta in (24, 32, 53, 64):
        for bq in range(1, 20):
            for k in range(1, beta // bq + 1):
                assert bq * k * (k + 1) / 2 <= beta * bounds.redq_axpy_count(k)


def test_thm_bounds_config_polymul_f3():
    """Degree-2 x degree-2 over F_3 (one product per word): q > 1*3*4 = 12 gives q = 16,
    and 5 digits of 4 bits fit 53 (and 24) mantissa bits."""
    assert bounds.smallest_pow2_q(1 * 3 * 4) == 16
    assert bounds.thm_bounds_ok(16, 1, 3, 3, 53)
    assert bounds.thm_bounds_ok(16, 1, 3, 3, 24)
    assert not bounds.thm_bounds_ok(8, 1, 3, 3, 53)


def test_full_compression_constraints():
    # Eq. qtheta / Eq. dq: with Q = 2^6 and d_q = d_theta = 1, Theta = Q^2 = 2^12 works
    assert bounds.full_compression_ok(1 << 6, 1 << 12, 1, 1, 53)
    assert not bounds.full_compression_ok(1 << 6, 1 << 11, 1, 1, 53)
    assert not bounds.full_compression_ok(1 << 14, 1 << 28, 1, 1, 53)
