"""GPU test of the serving loop (continuous batching): a mixed Poisson request stream is
served while requests keep arriving; every result is bit-exact against the oracle and equal
to the same request run alone through the direct calls."""
import time

import numpy as np
import pytest

import workloads
from oracle import field
from tests._gpu import to_dev, torch_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch, dev = torch_dev()
    import __graft_entry__ as g
    g.build()
    import paper_0809_0063_gb300 as fp
    ctx = fp.fp_ctx_create(0)
    gfs = {(p, k): fp.fp_gf_create(ctx, p, k) for p, k in workloads.GF_FIELDS}
    yield fp, torch, dev, ctx, gfs
    for g in gfs.values():
        fp.fp_gf_destroy(g)
    fp.fp_ctx_destroy(ctx)


def oracle(req, code, A, B, moduli):
    if code == 0:
        return field.polymul_mod(A.astype(np.int64), B.astype(np.int64), req.p)
    if code == 1:
        return np.array([field.dot_mod(A, B, req.p)])
    if code == 2:
        return field.gf_mul(A.astype(np.int64), B.astype(np.int64), req.p, req.gf_k, moduli[(req.p, req.gf_k)])
    return field.matmul_mod(A, B, req.p)


def alone(fp, torch, dev, ctx, gfs, req, code, sz, A, B, out):
    if code == 0:
        C = torch.empty(out.shape, dtype=torch.uint8, device=dev)
        fp.fp_polymul_batched(ctx, req.p, to_dev(torch, dev, A), sz[0], to_dev(torch, dev, B), sz[1], C, 1)
    elif code == 1:
        C = torch.empty((1,), dtype=torch.int32, device=dev)
        fp.fp_dot(ctx, req.p, to_dev(torch, dev, A), to_dev(torch, dev, B), sz[0], C)
    elif code == 2:
        v = (lambda x: x.view(np.int16) if x.dtype == np.uint16 else x)
        C = torch.empty(out.shape, dtype=torch.uint8 if out.dtype == np.uint8 else torch.int16, device=dev)
        fp.fp_gf_mul_batched(ctx, gfs[(req.p, req.gf_k)], torch.from_numpy(v(A)).to(dev),
                             torch.from_numpy(v(B)).to(dev), C, sz[0])
    else:
        n = sz[0]
        C = torch.empty((n, n), dtype=torch.uint8, device=dev)
        fp.fp_matmul(ctx, req.p, n, n, n, to_dev(torch, dev, A), n, to_dev(torch, dev, B), n, C, n)
    fp.fp_ctx_status(ctx)
    r = C.cpu().numpy()
    return r.view(out.dtype) if r.dtype.itemsize == out.dtype.itemsize else r.astype(out.dtype)


@pytest.mark.parametrize("streams,window", [(4, 100), (1, 0)])
def test_serving_mix_equals_alone_and_oracle(env, streams, window):
    fp, torch, dev, ctx, gfs = env
    moduli = {pk: field.smallest_monic_irreducible(*pk) for pk in workloads.GF_FIELDS}
    reqs = workloads.serving_stream(5 + streams, rate=20000.0, duration=0.03)
    assert len(reqs) > 300
    srv = fp.fp_server_create(ctx, arena_bytes=256 << 20, streams=streams, max_batch=128, window_us=window)
    keep, tickets = [], []
    t0 = time.perf_counter()
    for r in reqs:
        code, sz, A, B, out = workloads.request_arrays(r, matmul_cap=160)
        while time.perf_counter() - t0 < r.t_arrival:       # submit at the arrival times
            pass
        q = fp.fp_request(kind=code, p=r.p, a=sz[0], b=sz[1], c=sz[2], reserved=0,
                          gf=gfs[(r.p, r.gf_k)].value if code == 2 else None,
                          host_a=A.ctypes.data, host_b=B.ctypes.data, host_out=out.ctypes.data)
        tickets.append(fp.fp_server_submit(srv, q))
        keep.append((r, code, sz, A, B, out))
    fp.fp_server_drain(srv, 60.0)
    st = fp.fp_server_stats_get(srv)
    lats = fp.fp_server_latencies(srv, tickets[0], len(tickets))
    fp.fp_server_destroy(srv)
    fp.fp_ctx_status(ctx)
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert st["batches"] < len(reqs)                         # requests were batched together
    assert all(l >= 0 for l in lats)
    for (r, code, sz, A, B, out) in keep:
        want = oracle(r, code, A, B, moduli)
        got = out if code != 1 else out.astype(np.int64)
        assert np.array_equal(got.astype(np.int64), np.asarray(want).astype(np.int64)), (r.kind, r.p, sz)
    for (r, code, sz, A, B, out) in keep[::7]:
        assert np.array_equal(alone(fp, torch, dev, ctx, gfs, r, code, sz, A, B, out), out), (r.kind, sz)


def test_serving_full_size_matmuls(env):
    """The serving configuration's matmul sizes uncapped (n log-uniform 64..1024, plus requests
    of n = 1024 and 777 placed in the stream): every result equals the oracle -- the large
    products on sampled rows, everything else whole -- and a sample equals the request alone."""
    fp, torch, dev, ctx, gfs = env
    moduli = {pk: field.smallest_monic_irreducible(*pk) for pk in workloads.GF_FIELDS}
    reqs = workloads.serving_stream(41, rate=20000.0, duration=0.02)
    for i, (t, n) in enumerate(((0.001, 1024), (0.005, 777), (0.011, 1024), (0.015, 513))):
        reqs.append(workloads.Request(t, "matmul", (3, 5, 7)[i % 3], n, seed=990000 + i))
    reqs.sort(key=lambda r: r.t_arrival)
    big = [r for r in reqs if r.kind == "matmul" and r.size > 160]
    assert len(big) >= 4
    srv = fp.fp_server_create(ctx, arena_bytes=256 << 20, streams=4, max_batch=128, window_us=100)
    keep, tickets = [], []
    t0 = time.perf_counter()
    for r in reqs:
        code, sz, A, B, out = workloads.request_arrays(r)
        while time.perf_counter() - t0 < r.t_arrival:
            pass
        q = fp.fp_request(kind=code, p=r.p, a=sz[0], b=sz[1], c=sz[2], reserved=0,
                          gf=gfs[(r.p, r.gf_k)].value if code == 2 else None,
                          host_a=A.ctypes.data, host_b=B.ctypes.data, host_out=out.ctypes.data)
        tickets.append(fp.fp_server_submit(srv, q))
        keep.append((r, code, sz, A, B, out))
    fp.fp_server_drain(srv, 120.0)
    st = fp.fp_server_stats_get(srv)
    fp.fp_server_destroy(srv)
    fp.fp_ctx_status(ctx)
    assert st["completed"] == len(reqs) and st["failed"] == 0
    for (r, code, sz, A, B, out) in keep:
        if code == 3 and sz[0] > 160:
            n = sz[0]
            rows = np.unique(np.array([0, 1, n // 3, n // 2, n - 2, n - 1]))
            assert np.array_equal(out[rows], field.matmul_mod_rows(A, B, r.p, rows)), (r.p, n)
            continue
        want = oracle(r, code, A, B, moduli)
        got = out if code != 1 else out.astype(np.int64)
        assert np.array_equal(got.astype(np.int64), np.asarray(want).astype(np.int64)), (r.kind, r.p, sz)
    for (r, code, sz, A, B, out) in [k for k in keep if k[1] == 3] + keep[::11]:
        assert np.array_equal(alone(fp, torch, dev, ctx, gfs, r, code, sz, A, B, out), out), (r.kind, sz)


def test_server_rejects_bad_requests(env):
    fp, torch, dev, ctx, gfs = env
    srv = fp.fp_server_create(ctx, arena_bytes=64 << 20, streams=2)
    A = np.zeros(8, np.uint8)
    try:
        with pytest.raises(fp.FpError):
            fp.fp_server_submit(srv, fp.fp_request(kind=9, p=3, a=1, host_a=A.ctypes.data, host_b=A.ctypes.data,
                                                   host_out=A.ctypes.data))
        with pytest.raises(fp.FpError):
            fp.fp_server_submit(srv, fp.fp_request(kind=0, p=4, a=1, b=1, host_a=A.ctypes.data,
                                                   host_b=A.ctypes.data, host_out=A.ctypes.data))
    finally:
        fp.fp_server_destroy(srv)


def test_submit_many_whole_stream_and_all_or_nothing(env):
    """A whole request stream in one fp_server_submit_many call (large batches: the gather and
    scatter copies run on the server's copy threads): consecutive tickets, every result equals
    the oracle.  A stream with one invalid request in the middle is refused and queues nothing."""
    fp, torch, dev, ctx, gfs = env
    moduli = {pk: field.smallest_monic_irreducible(*pk) for pk in workloads.GF_FIELDS}
    reqs = workloads.serving_stream(77, rate=20000.0, duration=0.05)
    srv = fp.fp_server_create(ctx, arena_bytes=512 << 20, streams=4, max_batch=512, window_us=100)
    keep, qs = [], []
    for r in reqs:
        code, sz, A, B, out = workloads.request_arrays(r, matmul_cap=300)
        qs.append(fp.fp_request(kind=code, p=r.p, a=sz[0], b=sz[1], c=sz[2], reserved=0,
                                gf=gfs[(r.p, r.gf_k)].value if code == 2 else None,
                                host_a=A.ctypes.data, host_b=B.ctypes.data, host_out=out.ctypes.data))
        keep.append((r, code, sz, A, B, out))
    bad = list(qs)
    bad[len(bad) // 2] = fp.fp_request(kind=0, p=4, a=2, b=2, c=0, reserved=0, gf=None,
                                       host_a=keep[0][3].ctypes.data, host_b=keep[0][4].ctypes.data,
                                       host_out=keep[0][5].ctypes.data)
    with pytest.raises(fp.FpError) as ei:
        fp.fp_server_submit_many(srv, bad)
    assert ei.value.status == fp.FP_EINVAL
    assert fp.fp_server_stats_get(srv)["submitted"] == 0
    first = fp.fp_server_submit_many(srv, (fp.fp_request * len(qs))(*qs))   # a prebuilt array
    assert first == 0
    fp.fp_server_drain(srv, 120.0)
    st = fp.fp_server_stats_get(srv)
    lats = fp.fp_server_latencies(srv, first, len(qs))
    fp.fp_server_destroy(srv)
    fp.fp_ctx_status(ctx)
    assert st["submitted"] == len(qs) and st["completed"] == len(qs) and st["failed"] == 0
    assert all(l >= 0 for l in lats)
    for (r, code, sz, A, B, out) in keep:
        want = oracle(r, code, A, B, moduli)
        got = out if code != 1 else out.astype(np.int64)
        assert np.array_equal(got.astype(np.int64), np.asarray(want).astype(np.int64)), (r.kind, r.p, sz)
