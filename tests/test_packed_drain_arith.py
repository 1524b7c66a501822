"""CPU pin of the drain arithmetic of the packed fp16 product for p = 5, 7 (right compression on
the tensor cores, delayed reduction per chunk, Sec. 2.2 and Sec. 7.4): a chunk's fp32 sum
v = d0 + Q d1 (|d0|, |d1| <= dmax < Q / 2) is split by two magic-constant roundings,
y = bits(v + 1.5 2^23) = 0x4B400000 + v and t = bits(fma(v, 1/Q, 1.5 2^23)) = 0x4B400000 + d1,
and added into a wrapping 32-bit word as R += y + (2^16 - Q) t.  After cr chunks
R + off (1 + 2^16) - cr 0x4B400000 (1 + 2^16 - Q) (mod 2^32) must hold the two digit sums, each
offset by off = dmax cr, in its 16-bit halves.  Restated here with exact float32 rounding and
checked against the digit sums directly."""
import numpy as np
import pytest

M32 = (1 << 32) - 1
MAGIC = 12582912.0           # 1.5 * 2^23
MAGIC_BITS = 0x4B400000


def f32(x):
    return np.float32(x)


def bits(x):
    return int(np.array([x], dtype=np.float32).view(np.uint32)[0])


def fmaf(a, b, c):
    # a * b is exact in float64 (24-bit operands); one rounding to float32 gives the fused result
    return f32(float(a) * float(b) + float(c))


@pytest.mark.parametrize("p,Q,dmax,chunk", [(7, 681, 9 * 32, 32), (5, 1023, 4 * 64, 64)])
def test_drain_split_and_folded_constant(p, Q, dmax, chunk):
    assert dmax < Q / 2                                   # the separability bound of the chunk
    qinv = f32(1.0 / Q)
    qdec = 65536 - int(round(1.0 / float(qinv)))
    assert qdec == 65536 - Q
    cmag = (MAGIC_BITS * (1 + qdec)) & M32
    rng = np.random.default_rng(Q)
    for trial in range(40):
        nch = int(rng.integers(1, 113 if p == 7 else 127))
        d0 = rng.integers(-dmax, dmax + 1, nch)
        d1 = rng.integers(-dmax, dmax + 1, nch)
        if trial == 0:
            d0[:] = dmax
            d1[:] = dmax
        elif trial == 1:
            d0[:] = -dmax
            d1[:] = -dmax
        R = 0
        for a, b in zip(d0, d1):
            v = f32(int(a) + Q * int(b))                  # the exact fp32 chunk sum
            assert float(v) == int(a) + Q * int(b)
            y = bits(f32(v + f32(MAGIC)))
            t = bits(fmaf(v, qinv, MAGIC))
            assert y == MAGIC_BITS + int(a) + Q * int(b)
            assert t == MAGIC_BITS + int(b)               # round(v / Q) = d1
            R = (R + y + t * qdec) & M32
        off = dmax * nch
        fixed = (R + off * 65537 - nch * cmag) & M32
        assert fixed & 0xFFFF == int(d0.sum()) + off
        assert fixed >> 16 == int(d1.sum()) + off
        assert 0 <= int(d0.sum()) + off < 65536 and 0 <= int(d1.sum()) + off < 65536
