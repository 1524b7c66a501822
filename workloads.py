"""Seeded synthetic inputs for every workload of the packed F_p hot path.

This module only draws random numbers; it holds none of the method's arithmetic, so the
CPU oracle and the CUDA path can both consume exactly the same buffers.  Every generator
takes an explicit seed and uses numpy's PCG64 bit generator.

Recipes (shapes and distributions of the paper's workloads, Sections 5-7):
  * polymul  : A[batch][da+1], B[batch][db+1] uint8, coefficients uniform in [0, p-1]
  * matmul   : A[m][k], B[k][n] uint8, entries uniform in [0, p-1]
  * dot      : u[n], v[n] uint8, entries uniform in [0, p-1]
  * gf_mul   : element indices uniform in [0, p^k), uint8 when p^k <= 256 else uint16
  * uneven   : mixed matmul / dot instances, p from {2,3,5,7,17,31}, log-uniform sizes
  * serving  : Poisson arrivals mixing polymul, dot, GF batches and matmuls
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def uniform_mod(seed: int, p: int, shape) -> np.ndarray:
    """uint8 array of the given shape, entries uniform in [0, p-1]."""
    return rng(seed).integers(0, p, size=shape, dtype=np.uint8)


def polymul_inputs(seed: int, p: int, batch: int, da: int, db: int):
    g = rng(seed)
    a = g.integers(0, p, size=(batch, da + 1), dtype=np.uint8)
    b = g.integers(0, p, size=(batch, db + 1), dtype=np.uint8)
    return a, b


def matmul_inputs(seed: int, p: int, m: int, k: int, n: int):
    g = rng(seed)
    a = g.integers(0, p, size=(m, k), dtype=np.uint8)
    b = g.integers(0, p, size=(k, n), dtype=np.uint8)
    return a, b


def dot_inputs(seed: int, p: int, n: int):
    g = rng(seed)
    return (g.integers(0, p, size=n, dtype=np.uint8),
            g.integers(0, p, size=n, dtype=np.uint8))


def gf_index_dtype(p: int, k: int):
    return np.uint8 if p ** k <= 256 else np.uint16


def gf_inputs(seed: int, p: int, k: int, count: int):
    g = rng(seed)
    dt = gf_index_dtype(p, k)
    return (g.integers(0, p ** k, size=count, dtype=np.int64).astype(dt),
            g.integers(0, p ** k, size=count, dtype=np.int64).astype(dt))


def log_uniform_int(g: np.random.Generator, lo: int, hi: int, size=None):
    """Integers log-uniform on [lo, hi] (inclusive)."""
    u = g.random(size)
    return np.minimum(hi, np.floor(np.exp(math.log(lo) + u * (math.log(hi + 1) - math.log(lo))))).astype(np.int64)


UNEVEN_PRIMES = (2, 3, 5, 7, 17, 31)


@dataclass
class Instance:
    kind: str            # "matmul" or "dot"
    p: int
    m: int = 1
    k: int = 1
    n: int = 1
    a: np.ndarray = field(default=None, repr=False)
    b: np.ndarray = field(default=None, repr=False)


def uneven_batch(seed: int, count: int = 4096, lo: int = 16, hi: int = 2048,
                 matmul_frac: float = 0.5, with_data: bool = True):
    """Uneven batch of modular matmul / dot-product instances.

    p uniform over {2,3,5,7,17,31}; matmul with m, k, n independently log-uniform on
    [lo, hi]; dot with length log-uniform on [lo, hi]; entries uniform in [0, p-1].
    """
    g = rng(seed)
    out = []
    for _ in range(count):
        p = int(g.choice(UNEVEN_PRIMES))
        if g.random() < matmul_frac:
            m, k, n = (int(x) for x in log_uniform_int(g, lo, hi, 3))
            inst = Instance("matmul", p, m, k, n)
            if with_data:
                inst.a = g.integers(0, p, size=(m, k), dtype=np.uint8)
                inst.b = g.integers(0, p, size=(k, n), dtype=np.uint8)
        else:
            n = int(log_uniform_int(g, lo, hi))
            inst = Instance("dot", p, 1, n, 1)
            if with_data:
                inst.a = g.integers(0, p, size=n, dtype=np.uint8)
                inst.b = g.integers(0, p, size=n, dtype=np.uint8)
        out.append(inst)
    return out


@dataclass
class Request:
    t_arrival: float     # seconds from the start of the stream
    kind: str            # "polymul", "dot", "gf", "matmul"
    p: int
    size: int            # degree (polymul), length (dot), batch (gf), n (matmul)
    gf_k: int = 0
    seed: int = 0


GF_FIELDS = ((3, 5), (7, 4), (2, 8))


def serving_stream(seed: int, rate: float = 20000.0, duration: float = 1.0):
    """Poisson request stream: 50% polymul (degree log-U 2..512, p in {3,5,7}), 30% dot
    (length log-U 64..65536), 15% GF(p^k) batches (size log-U 1..4096, field uniform over
    GF(3^5), GF(7^4), GF(2^8)), 5% matmul (n log-U 64..1024)."""
    g = rng(seed)
    t = 0.0
    out = []
    i = 0
    while True:
        t += g.exponential(1.0 / rate)
        if t >= duration:
            break
        u = g.random()
        if u < 0.50:
            r = Request(t, "polymul", int(g.choice((3, 5, 7))), int(log_uniform_int(g, 2, 512)))
        elif u < 0.80:
            r = Request(t, "dot", int(g.choice((3, 5, 7))), int(log_uniform_int(g, 64, 65536)))
        elif u < 0.95:
            p, k = GF_FIELDS[int(g.integers(0, 3))]
            r = Request(t, "gf", p, int(log_uniform_int(g, 1, 4096)), gf_k=k)
        else:
            r = Request(t, "matmul", int(g.choice((3, 5, 7))), int(log_uniform_int(g, 64, 1024)))
        r.seed = seed * 1000003 + i
        i += 1
        out.append(r)
    return out


def request_arrays(req: Request, matmul_cap: int = 0):
    """Seeded operands of one serving request: (kind code, sizes (a, b, c), A, B, out array).
    polymul: degrees (size, independent log-uniform 2..512); dot: length size; GF: count size
    in the request's field; matmul: square n = size (capped at matmul_cap when given)."""
    g = rng(req.seed)
    if req.kind == "polymul":
        da = req.size
        db = int(log_uniform_int(g, 2, 512))
        A = g.integers(0, req.p, da + 1, dtype=np.uint8)
        B = g.integers(0, req.p, db + 1, dtype=np.uint8)
        return 0, (da, db, 0), A, B, np.zeros(da + db + 1, np.uint8)
    if req.kind == "dot":
        A = g.integers(0, req.p, req.size, dtype=np.uint8)
        B = g.integers(0, req.p, req.size, dtype=np.uint8)
        return 1, (req.size, 0, 0), A, B, np.zeros(1, np.uint32)
    if req.kind == "gf":
        dt = gf_index_dtype(req.p, req.gf_k)
        A = g.integers(0, req.p ** req.gf_k, req.size, dtype=np.int64).astype(dt)
        B = g.integers(0, req.p ** req.gf_k, req.size, dtype=np.int64).astype(dt)
        return 2, (req.size, 0, 0), A, B, np.zeros(req.size, dt)
    n = min(req.size, matmul_cap) if matmul_cap else req.size
    A = g.integers(0, req.p, (n, n), dtype=np.uint8)
    B = g.integers(0, req.p, (n, n), dtype=np.uint8)
    return 3, (n, n, n), A, B, np.zeros((n, n), np.uint8)
