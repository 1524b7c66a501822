"""Algorithm FGDP (Sec. 6) restated over exact integers (oracle; test infrastructure only).

Elements of GF(p^k) are indices sum_i c_i p^i of their coefficient vectors modulo a monic
irreducible P of degree k.  FGDP computes a dot product (here of length n), in this order, by
  - mapping each element to its evaluation at q (a table in the paper),
  - one integer dot product r~ of those evaluations,
  - REDQ COMPRESSION of r~ into u_0..u_{2k-2},
  - two table lookups L[u_0..u_{k-1}] and H[u_{k-1}..u_{2k-2}] that fold the REDQ
    correction and the reduction modulo P,
  - one addition in the field.
The tables are built here from the plain field arithmetic of ``field``.
"""
from __future__ import annotations

import itertools

import numpy as np

from . import field
from .dqt import redq_compression


def fgdp_tables(p, k, q, modulus):
    """L and H as dicts keyed by the tuples (u_0..u_{k-1}) and (u_{k-1}..u_{2k-2}).
    Theorem fgdp: L = sum_{i=0}^{k-2} (u_i - q u_{i+1} mod p) X^i and
    H = u_{2k-2} X^{2k-2} + sum_{i=k-1}^{2k-3} (u_i - q u_{i+1} mod p) X^i, each reduced
    modulo P and returned as an element index."""
    L, H = {}, {}
    for tup in itertools.product(range(p), repeat=k):
        # L from (u_0..u_{k-1})
        poly = [0] * (2 * k - 1)
        for i in range(k - 1):
            poly[i] = (tup[i] - q * tup[i + 1]) % p
        L[tup] = int(field.coeffs_to_index(field.poly_rem_mod(np.array(poly), modulus, p), p))
        # H from (u_{k-1}..u_{2k-2}); tup[j] is u_{k-1+j}
        poly = [0] * (2 * k - 1)
        poly[2 * k - 2] = tup[k - 1] % p
        for j in range(k - 1):
            i = k - 1 + j
            poly[i] = (tup[j] - q * tup[j + 1]) % p
        H[tup] = int(field.coeffs_to_index(field.poly_rem_mod(np.array(poly), modulus, p), p))
    return L, H


def fgdp_dot(v1, v2, p, k, q, modulus, tables=None):
    """Dot product over GF(p^k) of two index vectors by the steps of Algorithm FGDP."""
    L, H = tables if tables is not None else fgdp_tables(p, k, q, modulus)
    def ev(x):
        c = field.index_to_coeffs(np.array(int(x)), p, k)
        return sum(int(c[i]) * q ** i for i in range(k))
    r = sum(ev(a) * ev(b) for a, b in zip(v1, v2))
    u = redq_compression(r, p, q, 2 * k - 2)
    lo = L[tuple(u[:k])]
    hi = H[tuple(u[k - 1:])]
    return int(field.gf_add(np.array(lo), np.array(hi), p, k))
