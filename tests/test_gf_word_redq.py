"""CPU pin of the arithmetic behind the 32-bit word GF(p^k) dot and matrix products
(Algorithm FGDP, Sec. 6, with the chunk q of reading 18): the word tables, REDQ compression in
SWAR form on 32-bit pieces, the L/H tables as wide coefficient fields, the deferred field
additions with their folds, and GF(2^8)'s XOR accumulation, restated here in plain Python
integers and compared with the oracle's field dot product.  A wrong lane mask, split point,
correction constant or fold bound changes some result below."""
import numpy as np
import pytest

from oracle import field

M32 = 0xFFFFFFFF


def umulhi(a, b):
    return ((a & M32) * (b & M32)) >> 32


def shr64(lo, hi, s):
    return (((hi << 32) | lo) >> s) & M32


def poly_rem(a, m, p):
    a = list(a)
    k = len(m) - 1
    for d in range(len(a) - 1, k - 1, -1):
        lead = a[d] % p
        if lead:
            for i in range(k + 1):
                a[d - k + i] = (a[d - k + i] + (p - lead) * m[i]) % p
    return a[:k]


def tables(p, k, mod):
    """Word table at the chunk's q, and L/H tables of reduced coefficients in wide fields."""
    q = p ** k
    bd, fw = (7, 6) if p == 3 else (9, 8)
    cq = (p - ((1 << bd) % p)) % p                     # -q mod p
    digs = lambda x: [(x // p ** i) % p for i in range(k)]
    W = [sum(c << (bd * i) for i, c in enumerate(digs(x))) if x < q else 0 for x in range(4096)]
    wide = lambda c: sum(v << (fw * i) for i, v in enumerate(c))
    L, H = [0] * 4096, [0] * 4096
    if p == 3:
        for il in range(4096):   # (u0 + 4 u1) + 16 (u2 + 4 u3) + 256 (u4 + 4 u5)
            u = []
            for j in range(3):
                pr = (il >> (4 * j)) & 15
                u += [pr & 3, pr >> 2]
            if max(u) < p:
                L[il] = wide([(u[i] + cq * u[i + 1]) % p for i in range(k)])
        for ih in range(256):    # (u5 + 4 u6) + 16 (u7 + 4 u8)
            u = [(ih >> (2 * t)) & 3 for t in range(4)]
            if max(u) < p:
                ph = [0] * 5 + [(u[i] + cq * u[i + 1]) % p for i in range(3)] + [u[3]]
                H[ih] = wide(poly_rem(ph, mod, p))
    else:
        for il in range(4096):   # sum_t u_t 8^t, t = 0..3
            u = [(il >> (3 * t)) & 7 for t in range(4)]
            if max(u) < p:
                L[il] = wide([(u[i] + cq * u[i + 1]) % p for i in range(3)] + [0])
        for ih in range(4096):   # sum_t u_{3+t} 8^t
            u = [(ih >> (3 * t)) & 7 for t in range(4)]
            if max(u) < p:
                ph = [0] * 3 + [(u[i] + cq * u[i + 1]) % p for i in range(3)] + [u[3]]
                H[ih] = wide(poly_rem(ph, mod, p))
    return W, L, H


def pairs(p, x, s):
    """u_i = (x_i - p s_i) mod q for even and odd digits in separate lanes, paired."""
    if p == 3:
        ME, CE, MU, sh, up = 0x001FC07F, 0x00600180, 0x0000C003, 7, 2
    else:
        ME, CE, MU, sh, up = 0x07FC01FF, 0x38000E00, 0x001C0007, 9, 3
    te = (((x & ME) | CE) - p * (s & ME)) & M32
    to = ((((x >> sh) & ME) | CE) - p * ((s >> sh) & ME)) & M32
    return (te & MU) | (((to & MU) << up) & M32)


def redq(p, r, L, H):
    lo, hi = r & M32, r >> 32
    if p == 3:
        rhh = hi >> 3                                          # digits 5..8
        yh = pairs(3, rhh, umulhi(rhh, 0x55555556))
        u5 = yh & 3
        t4 = (shr64(lo, hi, 28) & 0x7F) + (u5 << 7)
        u4 = t4 - 3 * umulhi(t4, 0x55555556)
        rl = (lo & 0x0FFFFFFF) + (u4 << 28)
        yl = pairs(3, rl, umulhi(rl, 0x55555556))
        il = ((yl + (yl >> 10)) & 0xFF) + ((u4 + 4 * u5) << 8)
        ih = (yh + (yh >> 10)) & 0xFF
    else:
        rhh = hi >> 4                                          # digits 4..6
        yh = pairs(7, rhh, umulhi(rhh, 0x24924925))
        t3 = (shr64(lo, hi, 27) & 0x1FF) + ((yh & 7) << 9)
        u3 = t3 - 7 * umulhi(t3, 0x24924925)
        rl = (lo & 0x07FFFFFF) + (u3 << 27)
        yl = pairs(7, rl, umulhi(rl, 0x24924925))
        il = (yl + (yl >> 12)) & 0xFFF
        ih = u3 + (((yh + (yh >> 12)) & 0x1FF) << 3)
    return (L[il] + H[ih]) & M32


def fold(p, x):
    if p == 3:
        return ((x >> 4) & 0x030C30C3) + (x & 0x0F3CF3CF)
    return ((x >> 3) & 0x1F1F1F1F) + (x & 0x07070707)


def word_dot(a, b, p, k, tabs):
    """The dot product as the word kernels take it: chunks of CH terms, REDQ, deferred sums,
    a fold after every eight REDQs; returns the element index."""
    W, L, H = tabs
    ch, fw = (6, 6) if p == 3 else (3, 8)
    acc, r, cnt, red = 0, 0, 0, 0
    for x, y in zip(a, b):
        r += W[min(int(x), 4095)] * W[min(int(y), 4095)]
        cnt += 1
        if cnt == ch:
            assert r < 1 << 63
            acc += redq(p, r, L, H)
            r, cnt, red = 0, 0, red + 1
            if red % 8 == 0:
                acc = fold(p, acc)
    if cnt:
        acc += redq(p, r, L, H)
    acc = fold(p, acc)
    return sum((((acc >> (fw * f)) & ((1 << fw) - 1)) % p) * p ** f for f in range(k))


def fields_never_carry(p, k, tabs, n):
    """Every field of the running sum stays below its width on all-(p^k - 1) inputs."""
    W, L, H = tabs
    ch, fw = (6, 6) if p == 3 else (3, 8)
    q = p ** k
    acc = 0
    for red in range(1, n // ch + 1):
        r = ch * W[q - 1] * W[q - 1]
        before = acc
        acc += redq(p, r, L, H)
        for f in range(k):   # no field overflowed into the next
            assert ((acc >> (fw * f)) & ((1 << fw) - 1)) == ((before >> (fw * f)) & ((1 << fw) - 1)) + \
                ((redq(p, r, L, H) >> (fw * f)) & ((1 << fw) - 1))
        if red % 8 == 0:
            acc = fold(p, acc)


@pytest.mark.parametrize("p,k", [(3, 5), (7, 4)])
def test_word_redq_dot_matches_field(p, k):
    mod = field.smallest_monic_irreducible(p, k)
    tabs = tables(p, k, mod)
    q = p ** k
    rng = np.random.default_rng(q + 3)
    for n in (1, 2, 3, 5, 6, 7, 12, 13, 48, 100, 400):
        for _ in range(4):
            a, b = rng.integers(0, q, n), rng.integers(0, q, n)
            assert word_dot(a, b, p, k, tabs) == field.gf_dot(a, b, p, k, mod), n
    # every digit of every chunk at its bound, over many folds
    a = np.full(600, q - 1)
    assert word_dot(a, a, p, k, tabs) == field.gf_dot(a, a, p, k, mod)
    fields_never_carry(p, k, tabs, 600)
    # single products (REDQ of one word product) against the field multiply
    for x, y in zip(rng.integers(0, q, 300), rng.integers(0, q, 300)):
        assert word_dot([x], [y], p, k, tabs) == field.gf_dot(np.array([x]), np.array([y]), p, k, mod)


def test_word_redq_codes_at_or_above_order_are_zero():
    """The word tables map codes >= p^k to the zero word (GF(7^4) clamps a uint16 to 2401)."""
    for p, k in [(3, 5), (7, 4)]:
        mod = field.smallest_monic_irreducible(p, k)
        tabs = tables(p, k, mod)
        q = p ** k
        assert tabs[0][q] == 0 and tabs[0][min(4095, 255 if p == 3 else 2401)] == 0
        a = np.array([q - 1, 5, q - 1])
        assert word_dot(a, np.array([q, q - 1, 7]), p, k, tabs) == \
            field.gf_dot(np.array([q - 1, 5, q - 1]), np.array([0, q - 1, 7]), p, k, mod)


def test_gf28_xor_accumulation_matches_field():
    """GF(2^8), q = 2^4: XOR of the word products, then one REDQ (bits 0, 4, .., 56) and the
    high part's table, equals the field dot product for any length."""
    p, k = 2, 8
    mod = field.smallest_monic_irreducible(p, k)
    W = [sum(((x >> i) & 1) << (4 * i) for i in range(8)) for x in range(256)]
    Ht = []
    for g in range(128):
        ph = [0] * 8 + [(g >> t) & 1 for t in range(7)]
        Ht.append(sum(v << i for i, v in enumerate(poly_rem(ph, mod, p))))

    def gather4(w):
        return sum(((w >> (4 * i)) & 1) << i for i in range(8))

    rng = np.random.default_rng(28)
    for n in (1, 2, 3, 17, 255, 1000):
        for _ in range(4):
            a, b = rng.integers(0, 256, n), rng.integers(0, 256, n)
            r = 0
            for x, y in zip(a, b):
                r ^= W[x] * W[y]
            assert r < 1 << 58
            assert gather4(r & M32) ^ Ht[gather4(r >> 32)] == field.gf_dot(a, b, p, k, mod), n
