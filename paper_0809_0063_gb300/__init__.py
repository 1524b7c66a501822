"""Python binding of libfpdqt (packed small-prime-field arithmetic on GB300, sm_103a).

Argument marshalling only: every function here forwards to the C ABI entry point of the same
name declared in include/fpdqt.h.  Arrays are torch tensors on the CUDA device (their
data_ptr() is passed); streams default to torch's current stream.  A non-FP_OK status raises
FpError with the library's message.  There is no CPU fallback: if libfpdqt.so is missing or
cannot be loaded, importing the compute functions raises.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfpdqt.so")

# status codes (fp_status)
FP_OK, FP_EINVAL, FP_EBOUND, FP_ENOMEM, FP_ECUDA, FP_ETIMEOUT, FP_EUNSUPPORTED = range(7)
STATUS_NAMES = ["FP_OK", "FP_EINVAL", "FP_EBOUND", "FP_ENOMEM", "FP_ECUDA", "FP_ETIMEOUT", "FP_EUNSUPPORTED"]
# word types (fp_word)
FP_WORD_F64, FP_WORD_U64, FP_WORD_F32, FP_WORD_U32 = range(4)
# forms of q (fp_dqt_params.qform)
FP_Q_POW2, FP_Q_P_POW2 = range(2)
# polymul / dot algorithms
FP_ALGO_AUTO, FP_ALGO_PLAIN, FP_ALGO_DQT_F64, FP_ALGO_DQT_U64, FP_ALGO_DQT_F32, FP_ALGO_DQT_U32, \
    FP_ALGO_KARATSUBA = range(7)
# matmul algorithms
(FP_MM_AUTO, FP_MM_RIGHT_F64, FP_MM_RIGHT_F32, FP_MM_PLAIN_F64, FP_MM_PLAIN_F32, FP_MM_PLAIN_I8,
 FP_MM_PLAIN_TC, FP_MM_RIGHT_TC, FP_MM_LEFT_F32, FP_MM_PLAIN_F8, FP_MM_LEFT_F64, FP_MM_CMM_F64,
 FP_MM_FULL_F64, FP_MM_SPLIT_F64) = range(14)
FP_GROUP_MAX = 16
# GF(p^k) element forms for fp_gf_dot
FP_GF_INDEX, FP_GF_LOG = range(2)
# polynomial-product kernels (fp_polymul_plan)
FP_PM_SINGLE_WORD, FP_PM_FQT, FP_PM_KARATSUBA, FP_PM_PLAIN = range(4)


class FpError(RuntimeError):
    def __init__(self, status: int, msg: str):
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {msg}")
        self.status = status


class fp_dqt_params(ctypes.Structure):
    _fields_ = [("p", ctypes.c_uint32), ("k", ctypes.c_uint32), ("b", ctypes.c_uint32),
                ("ndig", ctypes.c_uint32), ("word", ctypes.c_uint32), ("qform", ctypes.c_uint32),
                ("n_accum", ctypes.c_uint64)]


class fp_polymul_plan_t(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_uint32), ("word", ctypes.c_uint32), ("blk_a", ctypes.c_uint32),
                ("blk_b", ctypes.c_uint32), ("b", ctypes.c_uint32), ("ndig", ctypes.c_uint32),
                ("L", ctypes.c_uint32), ("m", ctypes.c_uint32)]


class fp_instance(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_uint32), ("p", ctypes.c_uint32), ("m", ctypes.c_uint32),
                ("n", ctypes.c_uint32), ("k", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("A", ctypes.c_void_p), ("B", ctypes.c_void_p), ("C", ctypes.c_void_p)]


class fp_mm_problem(ctypes.Structure):
    _fields_ = [("p", ctypes.c_uint32), ("m", ctypes.c_int), ("n", ctypes.c_int), ("k", ctypes.c_int),
                ("A", ctypes.c_void_p), ("lda", ctypes.c_int), ("B", ctypes.c_void_p), ("ldb", ctypes.c_int),
                ("C", ctypes.c_void_p), ("ldc", ctypes.c_int)]


class fp_request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_uint32), ("p", ctypes.c_uint32), ("a", ctypes.c_uint32), ("b", ctypes.c_uint32),
                ("c", ctypes.c_uint32), ("reserved", ctypes.c_uint32), ("gf", ctypes.c_void_p),
                ("host_a", ctypes.c_void_p), ("host_b", ctypes.c_void_p), ("host_out", ctypes.c_void_p)]


class fp_server_config(ctypes.Structure):
    _fields_ = [("arena_bytes", ctypes.c_uint64), ("streams", ctypes.c_uint32), ("max_batch", ctypes.c_uint32),
                ("window_us", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class fp_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("batches", ctypes.c_uint64),
                ("launches", ctypes.c_uint64), ("failed", ctypes.c_uint64)]


FP_REQ_POLYMUL, FP_REQ_DOT, FP_REQ_GF, FP_REQ_MATMUL = range(4)

_lib = None
_V, _U32, _U64, _SZ, _I = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_size_t, ctypes.c_int
_SIGS = {
    "fp_ctx_create": (_I, [ctypes.POINTER(_V), _I]),
    "fp_ctx_destroy": (None, [_V]),
    "fp_ctx_status": (_I, [_V, _V]),
    "fp_last_error": (ctypes.c_char_p, []),
    "fp_ctx_profile": (_I, [_V, _I]),
    "fp_ctx_profile_read": (_I, [_V, ctypes.c_char_p, ctypes.POINTER(_U64), ctypes.POINTER(ctypes.c_double)]),
    "fp_ctx_launches": (_I, [_V, ctypes.POINTER(_U64)]),
    "fp_ctx_autotune": (_I, [_V, _I]),
    "fp_ctx_autotune_choice": (_I, [_V, _U32, _I, _I, _I, ctypes.POINTER(_I)]),
    "fp_dqt_choose": (_I, [_U32, _U32, _U64, _U32, ctypes.POINTER(fp_dqt_params)]),
    "fp_polymul_plan": (_I, [_U32, _U32, _U32, ctypes.c_int, ctypes.POINTER(fp_polymul_plan_t)]),
    "fp_mm_choose": (_I, [_U32, _U64, _U32, ctypes.POINTER(_U32), ctypes.POINTER(_U32), ctypes.POINTER(_U32)]),
    "fp_mm_full_choose": (_I, [_U32, _U64, ctypes.POINTER(_U32), ctypes.POINTER(_U32), ctypes.POINTER(_U32),
                               ctypes.POINTER(_U32)]),
    "fp_dqt_pack": (_I, [_V, ctypes.POINTER(fp_dqt_params), _V, _V, _SZ, _V]),
    "fp_dqt_unpack_redq": (_I, [_V, ctypes.POINTER(fp_dqt_params), _V, _V, _SZ, _V]),
    "fp_polymul_batched": (_I, [_V, _U32, _V, _U32, _V, _U32, _V, _SZ, _I, _V]),
    "fp_dot": (_I, [_V, _U32, _V, _V, _SZ, _V, _I, _V]),
    "fp_dot_noalloc": (_I, [_U32, _V, _V, _SZ, _V, _I, _V]),
    "fp_matmul": (_I, [_V, _U32, _I, _I, _I, _V, _I, _V, _I, _V, _I, _I, _V]),
    "fp_pack_cb": (_I, [_V, _U32, _I, _I, _V, _I, _U32, _U32, _U32, _V, _V]),
    "fp_gf_create": (_I, [_V, _U32, _U32, ctypes.POINTER(_V)]),
    "fp_gf_destroy": (None, [_V]),
    "fp_gf_info": (_I, [_V, ctypes.POINTER(_U32), ctypes.POINTER(_U32), ctypes.POINTER(_U32), ctypes.POINTER(_U32)]),
    "fp_gf_mul_batched": (_I, [_V, _V, _V, _V, _V, _SZ, _V]),
    "fp_gf_dot": (_I, [_V, _V, _V, _V, _SZ, _V, ctypes.c_int, _V]),
    "fp_gf_matmul": (_I, [_V, _V, ctypes.c_int, ctypes.c_int, ctypes.c_int, _V, ctypes.c_int, _V, ctypes.c_int, _V,
                          ctypes.c_int, ctypes.c_int, _V]),
    "fp_gf_dot_info": (_I, [_V, ctypes.POINTER(_U32), ctypes.POINTER(_U32), ctypes.POINTER(_U32)]),
    "fp_batch_run": (_I, [_V, ctypes.POINTER(fp_instance), _SZ, _V]),
    "fp_matmul_grouped": (_I, [_V, ctypes.POINTER(fp_mm_problem), _SZ, _I, _V]),
    "fp_selftest_bounded_wait": (_I, [_V, _U32, _V]),
    "fp_server_create": (_I, [_V, ctypes.POINTER(fp_server_config), ctypes.POINTER(_V)]),
    "fp_server_submit": (_I, [_V, ctypes.POINTER(fp_request), ctypes.POINTER(_U64)]),
    "fp_server_submit_many": (_I, [_V, ctypes.POINTER(fp_request), _SZ, ctypes.POINTER(_U64)]),
    "fp_server_poll": (_I, [_V, _U64, ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_double)]),
    "fp_server_drain": (_I, [_V, ctypes.c_double]),
    "fp_server_latencies": (_I, [_V, _U64, _SZ, ctypes.POINTER(ctypes.c_double)]),
    "fp_server_stats_get": (_I, [_V, ctypes.POINTER(fp_server_stats)]),
    "fp_server_destroy": (None, [_V]),
}


def lib():
    """Load libfpdqt.so (built in-tree by build.build()).  Raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libfpdqt.so not built at {LIB_PATH}; run paper_0809_0063_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(status: int):
    if status != FP_OK:
        raise FpError(status, lib().fp_last_error().decode())


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ------------------------------------------------------------------ context

def fp_ctx_create(device: int = 0):
    h = _V()
    _check(lib().fp_ctx_create(ctypes.byref(h), device))
    return h


def fp_ctx_destroy(ctx):
    lib().fp_ctx_destroy(ctx)


def fp_ctx_status(ctx, stream=None):
    _check(lib().fp_ctx_status(ctx, _stream(stream)))


def fp_last_error() -> str:
    return lib().fp_last_error().decode()


def fp_ctx_profile(ctx, mode: int):
    _check(lib().fp_ctx_profile(ctx, mode))


def fp_ctx_profile_read(ctx, prefix: str = ""):
    n, ms = _U64(), ctypes.c_double()
    _check(lib().fp_ctx_profile_read(ctx, prefix.encode(), ctypes.byref(n), ctypes.byref(ms)))
    return n.value, ms.value


def fp_ctx_autotune(ctx, enable: int):
    _check(lib().fp_ctx_autotune(ctx, enable))


def fp_ctx_autotune_choice(ctx, p: int, m: int, n: int, k: int) -> int:
    a = _I()
    _check(lib().fp_ctx_autotune_choice(ctx, p, m, n, k, ctypes.byref(a)))
    return a.value


def fp_ctx_launches(ctx) -> int:
    n = _U64()
    _check(lib().fp_ctx_launches(ctx, ctypes.byref(n)))
    return n.value


# ------------------------------------------------------------------ planner

def fp_polymul_plan(p: int, dega: int, degb: int, algo: int = FP_ALGO_AUTO) -> dict:
    out = fp_polymul_plan_t()
    _check(lib().fp_polymul_plan(p, dega, degb, algo, ctypes.byref(out)))
    return {name: getattr(out, name) for name, _ in fp_polymul_plan_t._fields_}


def fp_dqt_choose(p: int, k: int, n_accum: int, word: int) -> fp_dqt_params:
    out = fp_dqt_params()
    _check(lib().fp_dqt_choose(p, k, n_accum, word, ctypes.byref(out)))
    return out


def fp_mm_choose(p: int, kdim: int, algo: int):
    b, e, c = _U32(), _U32(), _U32()
    _check(lib().fp_mm_choose(p, kdim, algo, ctypes.byref(b), ctypes.byref(e), ctypes.byref(c)))
    return b.value, e.value, c.value


def fp_mm_full_choose(p: int, kdim: int):
    """(b, dq1, dt1, piece) of the full-compression product (Sec. 7.5)."""
    b, q1, t1, pc = _U32(), _U32(), _U32(), _U32()
    _check(lib().fp_mm_full_choose(p, kdim, ctypes.byref(b), ctypes.byref(q1), ctypes.byref(t1), ctypes.byref(pc)))
    return b.value, q1.value, t1.value, pc.value


# ------------------------------------------------------------------ compute

def fp_dqt_pack(ctx, prm: fp_dqt_params, coeffs, words, count: int, stream=None):
    _check(lib().fp_dqt_pack(ctx, ctypes.byref(prm), _ptr(coeffs), _ptr(words), count, _stream(stream)))


def fp_dqt_unpack_redq(ctx, prm: fp_dqt_params, words, coeffs, count: int, stream=None):
    _check(lib().fp_dqt_unpack_redq(ctx, ctypes.byref(prm), _ptr(words), _ptr(coeffs), count, _stream(stream)))


def fp_polymul_batched(ctx, p: int, A, dega: int, B, degb: int, C, batch: int, algo: int = FP_ALGO_AUTO,
                       stream=None):
    _check(lib().fp_polymul_batched(ctx, p, _ptr(A), dega, _ptr(B), degb, _ptr(C), batch, algo, _stream(stream)))


def fp_dot(ctx, p: int, u, v, n: int, out, algo: int = FP_ALGO_AUTO, stream=None):
    _check(lib().fp_dot(ctx, p, _ptr(u), _ptr(v), n, _ptr(out), algo, _stream(stream)))


def fp_dot_noalloc(p: int, u, v, n: int, out, algo: int = FP_ALGO_AUTO, stream=None):
    """Allocation-free dot product: no context, scratch in a fixed array of the library's
    device image (see include/fpdqt.h); *out = 0xFFFFFFFF flags an out-of-range residue."""
    _check(lib().fp_dot_noalloc(p, _ptr(u), _ptr(v), n, _ptr(out), algo, _stream(stream)))


def fp_matmul(ctx, p: int, m: int, n: int, k: int, A, lda: int, B, ldb: int, C, ldc: int,
              algo: int = FP_MM_AUTO, stream=None):
    _check(lib().fp_matmul(ctx, p, m, n, k, _ptr(A), lda, _ptr(B), ldb, _ptr(C), ldc, algo, _stream(stream)))


def fp_mm_problem_of(p: int, m: int, n: int, k: int, A, lda: int, B, ldb: int, C, ldc: int) -> fp_mm_problem:
    return fp_mm_problem(p=p, m=m, n=n, k=k, A=_ptr(A), lda=lda, B=_ptr(B), ldb=ldb, C=_ptr(C), ldc=ldc)


def fp_matmul_grouped(ctx, problems, algo: int = FP_MM_AUTO, stream=None):
    """problems: sequence of fp_mm_problem (see fp_mm_problem_of); the tensors they point to
    must stay alive until the work has run."""
    arr = (fp_mm_problem * len(problems))(*problems)
    _check(lib().fp_matmul_grouped(ctx, arr, len(problems), algo, _stream(stream)))


def fp_pack_cb(ctx, p: int, k: int, n: int, B, ldb: int, b: int, e: int, word: int, CB, stream=None):
    _check(lib().fp_pack_cb(ctx, p, k, n, _ptr(B), ldb, b, e, word, _ptr(CB), _stream(stream)))


def fp_gf_create(ctx, p: int, k: int):
    h = _V()
    _check(lib().fp_gf_create(ctx, p, k, ctypes.byref(h)))
    return h


def fp_gf_destroy(gf):
    lib().fp_gf_destroy(gf)


def fp_gf_info(gf, k: int):
    mod = (_U32 * (k + 1))()
    b, w, eb = _U32(), _U32(), _U32()
    _check(lib().fp_gf_info(gf, mod, ctypes.byref(b), ctypes.byref(w), ctypes.byref(eb)))
    return {"modulus": list(mod), "b": b.value, "word": w.value, "elem_bytes": eb.value}


def fp_gf_mul_batched(ctx, gf, a, b, c, count: int, stream=None):
    _check(lib().fp_gf_mul_batched(ctx, gf, _ptr(a), _ptr(b), _ptr(c), count, _stream(stream)))


def fp_gf_dot(ctx, gf, a, b, n: int, out, form: int = FP_GF_INDEX, stream=None):
    _check(lib().fp_gf_dot(ctx, gf, _ptr(a), _ptr(b), n, _ptr(out), form, _stream(stream)))


def fp_gf_matmul(ctx, gf, m: int, n: int, k: int, A, lda: int, B, ldb: int, C, ldc: int,
                 form: int = FP_GF_INDEX, stream=None):
    _check(lib().fp_gf_matmul(ctx, gf, m, n, k, _ptr(A), lda, _ptr(B), ldb, _ptr(C), ldc, form, _stream(stream)))


def fp_gf_dot_info(gf):
    g, b, c = _U32(), _U32(), _U32()
    _check(lib().fp_gf_dot_info(gf, ctypes.byref(g), ctypes.byref(b), ctypes.byref(c)))
    return {"generator": g.value, "b_dot": b.value, "chunk": c.value}


def fp_selftest_bounded_wait(ctx, polls: int, stream=None):
    _check(lib().fp_selftest_bounded_wait(ctx, polls, _stream(stream)))


def fp_instances(instances):
    """A contiguous fp_instance array (what fp_batch_run reads) from a sequence of fp_instance.
    Building it costs a few microseconds per instance: a caller that submits the same batch
    descriptors again keeps the array and passes it to fp_batch_run as it is."""
    return (fp_instance * len(instances))(*instances)


def fp_batch_run(ctx, instances, stream=None):
    """instances: a ctypes array of fp_instance (passed as it is) or a sequence of fp_instance."""
    arr = instances if isinstance(instances, ctypes.Array) else fp_instances(instances)
    _check(lib().fp_batch_run(ctx, arr, len(arr), _stream(stream)))


# ------------------------------------------------------------------ serving loop

def fp_server_create(ctx, arena_bytes: int = 1 << 30, streams: int = 4, max_batch: int = 256, window_us: int = 100):
    cfg = fp_server_config(arena_bytes=arena_bytes, streams=streams, max_batch=max_batch, window_us=window_us, reserved=0)
    h = _V()
    _check(lib().fp_server_create(ctx, ctypes.byref(cfg), ctypes.byref(h)))
    return h


def fp_server_submit(server, req: fp_request) -> int:
    t = _U64()
    _check(lib().fp_server_submit(server, ctypes.byref(req), ctypes.byref(t)))
    return t.value


def fp_server_submit_many(server, reqs) -> int:
    """reqs: a ctypes array of fp_request (passed as it is) or a sequence; returns the first ticket."""
    arr = reqs if isinstance(reqs, ctypes.Array) else (fp_request * len(reqs))(*reqs)
    t = _U64()
    _check(lib().fp_server_submit_many(server, arr, len(arr), ctypes.byref(t)))
    return t.value


def fp_server_poll(server, ticket: int):
    d, lat = _I(), ctypes.c_double()
    _check(lib().fp_server_poll(server, ticket, ctypes.byref(d), ctypes.byref(lat)))
    return d.value, lat.value


def fp_server_drain(server, timeout_s: float = 60.0):
    _check(lib().fp_server_drain(server, timeout_s))


def fp_server_latencies(server, first: int, n: int):
    out = (ctypes.c_double * n)()
    _check(lib().fp_server_latencies(server, first, n, out))
    return list(out)


def fp_server_stats_get(server) -> dict:
    s = fp_server_stats()
    _check(lib().fp_server_stats_get(server, ctypes.byref(s)))
    return {k: getattr(s, k) for k, _ in fp_server_stats._fields_}


def fp_server_destroy(server):
    lib().fp_server_destroy(server)
