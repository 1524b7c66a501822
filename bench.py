"""Benchmark of the packed F_p hot path on GB300: exact F_p MACs/s of the compressed matrix
product C = A B mod p (p in {3, 7}, n in {1024, 4096}), packed DQT + REDQ against the plain
mod-p kernels, with the roofline of the dominant kernel, an end-to-end number through the
C ABI with host buffers, and the CPU oracle timed beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--algo NAME]

One step = the four products of the configuration in one grouped call (AUTO: the e4m3
tensor-core product).  The same line carries the packed DQT + REDQ arm on the same inputs
(right compression: fp16 words on the tensor cores for p = 3, FP32 words on FFMA for p = 7),
graph-timed with its own roofline, and -- on one GPU, unless --no-configs -- the other
configurations nested under "configs": batched F_3 polynomial products, GF(p^k) products, the
4096-instance uneven batch and the serving loop, each with its roofline, end-to-end number and
the CPU oracle on one core and on all cores.  Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import hashlib
import gc
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads  # noqa: E402

PROBLEMS = [(3, 1024), (7, 1024), (3, 4096), (7, 4096)]
WORKLOAD = "compressed matmul C=A*B mod p, square uint8, p in {3,7} x n in {1024,4096}"
MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
L2_FLUSH_BYTES = 512 << 20

# Peaks (per GPU).  FP32 FFMA: 152 SMs x 128 lanes x 2 flops x 2.07 GHz (unit counts and
# maximum clock); FP64: measured bf16 dense peak x the nominal FP64:bf16 ratio 1.25/2250;
# u8 IMMA via mma.sync has no separate figure: measured bf16 peak x nominal int8:bf16 dense of
# the legacy path is unknown, so the probe's measured 150.6 TOP/s is used and labelled so.
FFMA_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


METRIC = "exact F_p MACs/s, packed DQT+REDQ vs plain mod-p on GB300"


def peaks():
    try:
        with open(MEASURED_PEAKS) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6792.7), d.get("bf16_tflops", 1928.9), d.get("bf16_tflops_sustained", 1750.5), "measured"
    except OSError:
        return 6800.0, 1900.0, 1700.0, "fallback"


def kernel_table(bf16_tf):
    """name -> (bound, peak TFLOP/s, peak label, algorithmic flops of one launch for (p, n, e))."""
    fp64 = bf16_tf * 1.25 / 2250.0
    return {
        "k_mm_ffma": ("alu", FFMA_PEAK_TFLOPS, "FFMA peak from unit counts and 2.07 GHz",
                      lambda n, e: 2.0 * n * n * (-(-n // e))),
        "k_mm_dmma": ("tensor", fp64, "FP64 = measured bf16 x 1.25/2250",
                      lambda n, e: 2.0 * n * n * (-(-n // e))),
        "k_mm_imma": ("tensor", 150.6, "u8 mma.sync measured by the pipe probe",
                      lambda n, e: 2.0 * n * n * n),
        "k_mm_t16_packed": ("tensor", bf16_tf, "measured bf16 dense (fp16 runs at the bf16 rate)",
                            lambda n, e: 2.0 * n * n * (-(-n // e))),
        "k_mm_t16_plain": ("tensor", bf16_tf, "measured bf16 dense",
                           lambda n, e: 2.0 * n * n * n),
        "k_mm_f8g": ("tensor", 2.0 * bf16_tf, "fp8 = measured bf16 x 2 (nominal 4.5/2.25)",
                     lambda n, e: 2.0 * n * n * n),
    }


def kernel_source_hash(name):
    """Hash of the CUDA file holding `name`, used to invalidate stored ncu traffic."""
    csrc = os.path.join(ROOT, "paper_0809_0063_gb300", "csrc")
    for fn in sorted(os.listdir(csrc)):
        path = os.path.join(csrc, fn)
        with open(path, "rb") as f:
            data = f.read()
        if (name + "(").encode() in data or (name + "<").encode() in data or ('"' + name + '"').encode() in data:
            return hashlib.sha256(data).hexdigest()[:16]
    return None


def stored_traffic(name, shapes, launches):
    """Average DRAM bytes per launch of `name` from a committed ncu capture of the same step:
    `shapes` lists the (variant, n) of every product the kernel ran in one step, and the
    capture is keyed by that list (traffic does not grow in proportion to n^3, so nothing is
    scaled across sizes).  None when the step has no capture or the kernel's source changed
    since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f).get(name)
    except (OSError, ValueError):
        return None
    if not d or d.get("source_hash") != kernel_source_hash(name) or not shapes:
        return None
    key = ",".join(sorted(f"{a}:{n}" for a, n in shapes))
    per_step = d.get("bytes_per_step", {}).get(key)
    return None if per_step is None else per_step / max(1, launches)


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        # raw samples: the package's build folder unless FPDQT_CLOCKS_DIR names another one
        folder = os.environ.get("FPDQT_CLOCKS_DIR") or os.path.join(ROOT, "paper_0809_0063_gb300", "_build")
        self.path = os.path.join(folder, f"clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def max_over_ranks(ms: float, device=None) -> float:
    """Largest timed region over all ranks (the job finishes when its slowest replica does)."""
    import torch
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        t = torch.tensor([ms], dtype=torch.float64, device=device if device is not None else "cpu")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())
    return ms


def whole_job_rate(units_per_step: float, steps: int, world_size: int, max_ms: float) -> float:
    """Whole-job throughput: every replica processes units_per_step per step."""
    return world_size * units_per_step * steps / (max_ms / 1e3)


def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ------------------------------------------------------------------ CPU oracle baselines
#
# The oracle as it stands, on the host cores: one process alone, then one process per core the
# bench may use (sched_getaffinity), each on its own bounded sample of the workload.  Processes
# are started with "spawn" (a fork after CUDA initialisation can hang).  A worker builds its
# inputs, then works until its time budget is spent, and returns (units, seconds).

def _cpu_work(kind, budget_s, wid):
    sys.path.insert(0, ROOT)
    from oracle import field
    g = np.random.default_rng(9000 + wid)
    units = 0.0
    if kind == "matmul":
        inputs = [(p, n) + workloads.matmul_inputs(100 + p + n, p, n, n, n) for p, n in PROBLEMS]
        t0 = time.perf_counter()
        i = 0
        while time.perf_counter() - t0 < budget_s:
            p, n, a, b = inputs[i % len(inputs)]
            r0 = int(g.integers(0, n - 16))
            field.matmul_mod_rows(a, b, p, np.arange(r0, r0 + 16))
            units += 16 * n * n
            i += 1
    elif kind == "polymul":
        a, b = workloads.polymul_inputs(900 + wid, 3, 1 << 20, 2, 2)
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < budget_s:
            field.polymul_mod(a, b, 3)
            units += (1 << 20) * 9
    elif kind == "gf":
        data = []
        for p, k in workloads.GF_FIELDS:
            a, b = workloads.gf_inputs(700 + p + wid, p, k, 1 << 17)
            data.append((p, k, a.astype(np.int64), b.astype(np.int64), field.smallest_monic_irreducible(p, k)))
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < budget_s:
            for p, k, a, b, mod in data:
                field.gf_mul(a, b, p, k, mod)
                units += k * k * len(a)
    elif kind == "batch":
        insts = workloads.uneven_batch(2024, count=4096)
        order = g.permutation(len(insts))
        t0 = time.perf_counter()
        i = 0
        while time.perf_counter() - t0 < budget_s:
            x = insts[order[i % len(insts)]]
            if x.kind == "matmul":
                rows = np.arange(0, min(x.m, 8))
                field.matmul_mod_rows(x.a, x.b, x.p, rows)
                units += len(rows) * x.k * x.n
            else:
                field.dot_mod(x.a, x.b, x.p)
                units += x.k
            i += 1
    elif kind == "serve":
        reqs = workloads.serving_stream(77, rate=20000.0, duration=1.0)
        mods = {pk: field.smallest_monic_irreducible(*pk) for pk in workloads.GF_FIELDS}
        order = g.permutation(len(reqs))
        t0 = time.perf_counter()
        i = 0
        while time.perf_counter() - t0 < budget_s:
            r = reqs[order[i % len(reqs)]]
            code, sz, A, B, out = workloads.request_arrays(r)
            if code == 0:
                field.polymul_mod(A, B, r.p)
            elif code == 1:
                field.dot_mod(A, B, r.p)
            elif code == 2:
                field.gf_mul(A.astype(np.int64), B.astype(np.int64), r.p, r.gf_k, mods[(r.p, r.gf_k)])
            else:
                field.matmul_mod(A, B, r.p)
            units += 1
            i += 1
    else:
        raise ValueError(kind)
    return units, time.perf_counter() - t0


_POOL = None


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline(kind, unit, sample, budget_s=6.0):
    """The oracle on one core and on all cores (a bounded sample, `budget_s` of work per process)."""
    global _POOL
    import multiprocessing as mp
    n = cpu_cores()
    if _POOL is None:
        _POOL = mp.get_context("spawn").Pool(n)
    u1, t1 = _POOL.apply(_cpu_work, (kind, budget_s, 0))
    res = _POOL.starmap(_cpu_work, [(kind, budget_s, w + 1) for w in range(n)])
    un = sum(u for u, _ in res)
    tn = max(t for _, t in res)
    return {"value": un / tn, "unit": unit, "cores": n, "kind": "oracle",
            "sample": f"{sample}; {budget_s:.0f} s of work per process, one process per core (spawn pool)",
            "single_core": {"value": u1 / t1, "cores": 1, "seconds": t1},
            "cores_source": "os.sched_getaffinity"}


def close_pool():
    global _POOL
    if _POOL is not None:
        _POOL.close()
        _POOL.join()
        _POOL = None


def run_reference(args, ws, rank):
    """Reference arm: the CPU oracle as it stands, each step a bounded sample of the
    workload (4 rows of each of the four products)."""
    if rank != 0:
        return
    from oracle import field
    inputs = [(p, n) + workloads.matmul_inputs(100 + p + n, p, n, n, n) for p, n in PROBLEMS]

    def step(s):
        macs = 0
        for p, n, a, b in inputs:
            rows = np.arange((4 * s) % n, (4 * s) % n + 4)
            field.matmul_mod_rows(a, b, p, rows)
            macs += 4 * n * n
        return macs

    for s in range(args.warmup):
        step(s)
    t0 = time.perf_counter()
    macs = 0
    for s in range(args.steps):
        macs += step(args.warmup + s)
    dt = time.perf_counter() - t0
    val = macs / dt
    sample = "per step: 4 rows of each of the four products (p in {3,7} x n in {1024,4096})"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": "F_p MAC/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "algo": "oracle (numpy int64 matmul, % p)"},
        "cpu_baseline": {"value": val, "unit": "F_p MAC/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": "F_p MAC/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def _timed(torch, stream, fn, reps, flush=None):
    ts = []
    for _ in range(reps):
        if flush is not None:
            flush.zero_()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        fn()
        a1.record(stream)
        torch.cuda.synchronize()
        ts.append(a0.elapsed_time(a1))
    return ts


def run_polymul(args, ws, rank, local, emit=True):
    """Batched polynomial products over F_3, degree 2 x degree 2 (the paper's Kronecker
    example size), DQT-packed: a step is 2^20 pairs; 48 input/output sets rotate so every step
    reads cold data (48 x 11.5 MB > 4 x L2), plus a scaled row of 2^26 pairs in one call."""
    import torch
    import __graft_entry__ as g
    g.build()
    import paper_0809_0063_gb300 as fp
    from oracle import field
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    hbm, bf16, _, peak_src = peaks()
    ctx = fp.fp_ctx_create(local)
    stream = torch.cuda.current_stream()
    p, da, db, batch, nsets = 3, 2, 2, 1 << 20, 48
    bpp = (da + 1) + (db + 1) + (da + db + 1)          # algorithmic bytes per pair (11)
    mpp = (da + 1) * (db + 1)                          # F_p MACs per pair (9)
    sets = []
    for i in range(nsets):
        a, b = workloads.polymul_inputs(500 + i, p, batch, da, db)
        sets.append((a, b, torch.from_numpy(a).to(dev), torch.from_numpy(b).to(dev),
                     torch.empty((batch, da + db + 1), dtype=torch.uint8, device=dev)))
    algo = getattr(fp, "FP_ALGO_" + (args.algo if args.algo != "AUTO" else "AUTO"))
    it = [0]

    def step(al=algo):
        a, b, A, B, C = sets[it[0] % nsets]
        it[0] += 1
        fp.fp_polymul_batched(ctx, p, A, da, B, db, C, batch, al)

    for i in range(nsets):                             # parity gate: every set, sampled pairs
        step()
    torch.cuda.synchronize()
    fp.fp_ctx_status(ctx)
    rows = np.random.default_rng(3).choice(batch, 4096, replace=False)
    for a, b, A, B, C in sets[:4]:
        assert np.array_equal(C[torch.from_numpy(rows).to(dev)].cpu().numpy(), field.polymul_mod(a[rows], b[rows], p))
    for _ in range(max(3, args.warmup)):
        step()
    # a step is ~2 us of device work: one CUDA graph holds a pass over the nsets rotating sets
    # (one library call each) and the step time is a replay's time / nsets
    torch.cuda.synchronize()
    l_a = fp.fp_ctx_launches(ctx)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        for _ in range(nsets):
            step()
    per_pass = fp.fp_ctx_launches(ctx) - l_a
    graph.replay()
    torch.cuda.synchronize()
    fp.fp_ctx_status(ctx)
    t_pass = statistics.median(_timed(torch, stream, graph.replay, 3))
    passes = max(3, args.steps // 4, int(1000.0 / max(t_pass, 1e-3)))   # about a second under load (clocks)
    clk = Clocks(local).__enter__()
    ts = [t / nsets for t in _timed(torch, stream, graph.replay, passes)]
    clk.__exit__(None, None, None)
    launches = per_pass * passes
    # per-kernel times from the library's own events over plain calls
    fp.fp_ctx_profile(ctx, 2)
    fp.fp_ctx_profile(ctx, 1)
    for _ in range(nsets):
        step()
    torch.cuda.synchronize()
    fp.fp_ctx_profile(ctx, 0)
    names = ["k_polymul_small", "k_polymul_word_bulk", "k_polymul_word", "k_polymul_plain_small", "k_polymul_fqt",
             "k_polymul_kara", "k_polymul_plain_big"]
    dom, dms, dn = None, 0.0, 0
    for nm in names:
        c, ms = fp.fp_ctx_profile_read(ctx, nm)
        if nm == "k_polymul_word":   # prefix of k_polymul_word_bulk: subtract the bulk launches
            cb, msb = fp.fp_ctx_profile_read(ctx, "k_polymul_word_bulk")
            c, ms = c - cb, ms - msb
        if c and ms > dms:
            dom, dms, dn = nm, ms, c
    t_ms = statistics.median(ts)
    value = ws * batch * mpp / (t_ms / 1e3)
    # scaled row: 2^26 pairs in one call
    big = 1 << 26
    ab, bb = workloads.polymul_inputs(900, p, big, da, db)
    Ab, Bb = torch.from_numpy(ab).to(dev), torch.from_numpy(bb).to(dev)
    Cb = torch.empty((big, da + db + 1), dtype=torch.uint8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    fn_big = lambda al=algo: fp.fp_polymul_batched(ctx, p, Ab, da, Bb, db, Cb, big, al)
    fn_big()
    torch.cuda.synchronize()
    fp.fp_ctx_status(ctx)
    rb = np.random.default_rng(4).choice(big, 4096, replace=False)
    assert np.array_equal(Cb[torch.from_numpy(rb).to(dev)].cpu().numpy(), field.polymul_mod(ab[rb], bb[rb], p))
    tb = statistics.median(_timed(torch, stream, fn_big, 5, flush))
    compare = {}
    if not args.no_compare:
        for nm in ("PLAIN", "DQT_U32", "DQT_F32", "DQT_U64", "DQT_F64"):
            al = getattr(fp, "FP_ALGO_" + nm)
            try:
                fn_big(al)
                torch.cuda.synchronize()
                fp.fp_ctx_status(ctx)
                compare[nm] = big * mpp / (statistics.median(_timed(torch, stream, lambda: fn_big(al), 3, flush)) / 1e3)
            except fp.FpError as ex:
                compare[nm] = f"unavailable: {ex.args[0][:60]}"
        if isinstance(compare.get("PLAIN"), float):
            compare["best_packed_over_plain"] = max(v for k, v in compare.items()
                                                    if k.startswith("DQT") and isinstance(v, float)) / compare["PLAIN"]
    # large degrees (blocked FQT, Sec. 5.2): the schoolbook over the u64 block words against the
    # Karatsuba splitting of the same words and the plain product, same inputs, L2 flushed
    large = {}
    if not args.no_compare:
        nl = 1 << 14
        for dl in (511, 1023):
            al_, bl_ = workloads.polymul_inputs(1000 + dl, p, nl, dl, dl)
            Al, Bl = torch.from_numpy(al_).to(dev), torch.from_numpy(bl_).to(dev)
            Cl = torch.empty((nl, 2 * dl + 1), dtype=torch.uint8, device=dev)
            rl = np.random.default_rng(dl).choice(nl, 8, replace=False)
            want = field.polymul_mod(al_[rl], bl_[rl], p)
            row = {}
            for nm in ("PLAIN", "DQT_U64", "KARATSUBA"):
                al = getattr(fp, "FP_ALGO_" + nm)
                fn = lambda al=al: fp.fp_polymul_batched(ctx, p, Al, dl, Bl, dl, Cl, nl, al)
                Cl.zero_()
                fn()
                torch.cuda.synchronize()
                fp.fp_ctx_status(ctx)
                assert np.array_equal(Cl[torch.from_numpy(rl).to(dev)].cpu().numpy(), want), f"parity {nm} deg {dl}"
                t = statistics.median(_timed(torch, stream, fn, 5, flush))
                row[nm] = {"ms": t, "F_p MAC/s": nl * (dl + 1) ** 2 / (t / 1e3)}
            row["karatsuba_over_schoolbook_fqt"] = row["DQT_U64"]["ms"] / row["KARATSUBA"]["ms"]
            row["karatsuba_over_plain"] = row["PLAIN"]["ms"] / row["KARATSUBA"]["ms"]
            large[f"2^14 pairs, degree {dl} x {dl}"] = row
            del Al, Bl, Cl
    # the other HBM-bound steps of the path on their own (a2 DQT pack, a4-a5 REDQ unpack, and
    # the dot product): GB/s of algorithmic bytes, L2 flushed before each call
    hbm_rows = {}
    if not args.no_compare:
        prm = fp.fp_dqt_choose(p, da + 1, 1, fp.FP_WORD_U32)            # 3 coefficients per u32 word at q = 16
        W = torch.empty(big, dtype=torch.int32, device=dev)
        fn = lambda: fp.fp_dqt_pack(ctx, prm, Ab, W, big)
        fn()
        torch.cuda.synchronize()
        t = statistics.median(_timed(torch, stream, fn, 5, flush))
        hbm_rows["dqt_pack (2^26 x 3 residues -> u32)"] = {"ms": t, "GB/s": big * (3 + 4) / (t / 1e3) / 1e9,
                                                            "frac_hbm": big * (3 + 4) / (t / 1e3) / 1e9 / hbm}
        prm5 = fp.fp_dqt_choose(p, da + 1, 1, fp.FP_WORD_U32)
        prm5.ndig = 2 * (da + 1) - 1                                   # unpack the 5 digits of a product word
        fn = lambda: fp.fp_dqt_unpack_redq(ctx, prm5, W, Cb, big)
        fn()
        torch.cuda.synchronize()
        t = statistics.median(_timed(torch, stream, fn, 5, flush))
        hbm_rows["dqt_unpack_redq (2^26 u32 -> 5 residues)"] = {"ms": t, "GB/s": big * (4 + 5) / (t / 1e3) / 1e9,
                                                                 "frac_hbm": big * (4 + 5) / (t / 1e3) / 1e9 / hbm}
        nd = 1 << 28
        u = torch.randint(0, p, (nd,), dtype=torch.uint8, device=dev)
        vv = torch.randint(0, p, (nd,), dtype=torch.uint8, device=dev)
        out = torch.empty(1, dtype=torch.int32, device=dev)
        for nm in ("AUTO", "PLAIN"):
            fn = lambda nm=nm: fp.fp_dot(ctx, p, u, vv, nd, out, getattr(fp, "FP_ALGO_" + nm))
            fn()
            torch.cuda.synchronize()
            t = statistics.median(_timed(torch, stream, fn, 5, flush))
            hbm_rows[f"dot {nm} (2^28 residue pairs)"] = {"ms": t, "GB/s": 2 * nd / (t / 1e3) / 1e9,
                                                          "frac_hbm": 2 * nd / (t / 1e3) / 1e9 / hbm}
        fp.fp_ctx_status(ctx)
        want = int((u.to(torch.int64) * vv.to(torch.int64)).sum().item()) % p
        fp.fp_dot(ctx, p, u, vv, nd, out, fp.FP_ALGO_AUTO)
        fp.fp_ctx_status(ctx)
        assert int(out.item()) == want, "dot parity"
        del u, vv, W
    # end to end: pinned host inputs in, results out, each step
    ha, hb = torch.from_numpy(sets[0][0]).pin_memory(), torch.from_numpy(sets[0][1]).pin_memory()
    hc = torch.empty((batch, da + db + 1), dtype=torch.uint8).pin_memory()
    A0, B0, C0 = sets[0][2], sets[0][3], sets[0][4]

    def e2e():
        A0.copy_(ha, non_blocking=True)
        B0.copy_(hb, non_blocking=True)
        fp.fp_polymul_batched(ctx, p, A0, da, B0, db, C0, batch, algo)
        hc.copy_(C0, non_blocking=True)

    e2e()
    torch.cuda.synchronize()
    te = statistics.median(_timed(torch, stream, e2e, 10))
    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline("polymul", "F_p MAC/s", "2^20 F_3 degree-2 pairs per pass, numpy int64 schoolbook + % p")
    roof = None
    if dom:
        # One launch per step: the timed graph replays give the launch's duration directly (their
        # events bracket only library launches; a plain call's own events would also count the
        # host's launch gap at this size).  Otherwise the library's per-launch events.
        one_per_step = per_pass == nsets and dn == nsets
        per_launch_ms = t_ms if one_per_step else dms / dn
        achieved = batch * bpp / (per_launch_ms / 1e3) / 1e9
        roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm,
                "traffic": stored_traffic(dom, [(args.algo, batch)], 1) if dom == "k_polymul_small" else None,
                "peak_source": f"HBM copy ({peak_src})", "launches": launches if one_per_step else dn,
                "avg_launch_ms": per_launch_ms,
                "launch_timing": "graph replay, one launch per step" if one_per_step else "library events per plain call",
                "scaled_2^26": {"achieved": big * bpp / (tb / 1e3) / 1e9, "frac": big * bpp / (tb / 1e3) / 1e9 / hbm,
                                "ms": tb}}
    res = None
    if rank == 0:
        res = {
            "metric": METRIC, "value": value, "unit": "F_p MAC/s", "n_gpus": ws, "steps": len(ts) * nsets,
            "warmup": max(3, args.warmup), "ms_per_step": t_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "packed word (planner: u32/f32/u64/f64)", "data": "synthetic",
            "timing": f"CUDA graph of {nsets} steps (one per rotating set), replayed {len(ts)} times",
            "config": {"workload": "batched polynomial product over F_3, 2^20 pairs of degree 2 x degree 2 per step",
                       "algo": args.algo, "l2": f"{nsets} rotating input/output sets ({nsets * batch * bpp / 1e6:.0f} MB)",
                       "scaled_row": "2^26 pairs per call, L2 flushed between calls",
                       "value_scaled_2^26": big * mpp / (tb / 1e3)},
            "roofline": roof, "cpu_baseline": cpu,
            "e2e": {"value": ws * batch * mpp / (te / 1e3), "unit": "F_p MAC/s",
                    "h2d_bytes_per_step": batch * (da + db + 2), "d2h_bytes_per_step": batch * (da + db + 1)},
            "gpu_launches": launches, "clocks": clk.summary(), "compare_same_inputs_2^26": compare,
            "other_hbm_steps": hbm_rows, "large_degree_same_inputs": large,
        }
        if emit:
            print(json.dumps(res))
    fp.fp_ctx_destroy(ctx)
    return res


def run_gf(args, ws, rank, local, emit=True):
    """GF(p^k) multiplication (Algorithm FGDP with n = 1): 2^24 random pairs in each of
    GF(3^5), GF(7^4), GF(2^8) per step (201 MB of indices moved, L2 flushed between steps).
    F_p MACs per multiply = k^2 (the schoolbook product; the reduction is not counted)."""
    import torch
    import __graft_entry__ as g
    g.build()
    import paper_0809_0063_gb300 as fp
    from oracle import field
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    hbm, bf16, _, peak_src = peaks()
    ctx = fp.fp_ctx_create(local)
    stream = torch.cuda.current_stream()
    count = 1 << 24
    fields = []
    for p, k in workloads.GF_FIELDS:
        a, b = workloads.gf_inputs(700 + p, p, k, count)
        gfh = fp.fp_gf_create(ctx, p, k)
        A, B = torch.from_numpy(a).to(dev), torch.from_numpy(b).to(dev)
        fields.append((p, k, a, b, gfh, A, B, torch.empty_like(A)))
    macs = sum(k * k for _, k in workloads.GF_FIELDS) * count
    nbytes = sum(3 * workloads.gf_index_dtype(p, k)(0).itemsize for p, k in workloads.GF_FIELDS) * count
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def step():
        for p, k, a, b, gfh, A, B, C in fields:
            fp.fp_gf_mul_batched(ctx, gfh, A, B, C, count)

    step()
    torch.cuda.synchronize()
    fp.fp_ctx_status(ctx)
    idx = np.random.default_rng(5).choice(count, 8192, replace=False)
    for p, k, a, b, gfh, A, B, C in fields:
        mod = field.smallest_monic_irreducible(p, k)
        want = field.gf_mul(a[idx].astype(np.int64), b[idx].astype(np.int64), p, k, mod)
        assert np.array_equal(C.cpu().numpy()[idx].astype(np.int64), want), f"GF({p}^{k}) parity"
    for _ in range(max(3, args.warmup)):
        step()
    l0 = fp.fp_ctx_launches(ctx)
    fp.fp_ctx_profile(ctx, 2)
    fp.fp_ctx_profile(ctx, 1)
    clk = Clocks(local).__enter__()
    ts = _timed(torch, stream, step, max(args.steps, 10), flush)
    clk.__exit__(None, None, None)
    fp.fp_ctx_profile(ctx, 0)
    launches = fp.fp_ctx_launches(ctx) - l0
    t_ms = statistics.median(ts)
    nk, kms = fp.fp_ctx_profile_read(ctx, "k_gf_mul")
    per_field = {}
    for p, k, a, b, gfh, A, B, C in fields:
        fn = lambda gfh=gfh, A=A, B=B, C=C: fp.fp_gf_mul_batched(ctx, gfh, A, B, C, count)
        t = statistics.median(_timed(torch, stream, fn, 5, flush))
        eb = 3 * A.element_size() * count
        per_field[f"GF({p}^{k})"] = {"ms": t, "GB/s": eb / (t / 1e3) / 1e9, "frac_hbm": eb / (t / 1e3) / 1e9 / hbm,
                                     "F_p MAC/s": k * k * count / (t / 1e3)}
    # Algorithm FGDP with n > 1: the dot product of 2^26 terms per field, index and discrete-log
    # forms, L2 flushed; parity on a 2^20-term prefix against the oracle's plain field dot.
    dot_rows = {}
    if not args.no_compare:
        nd = 1 << 26
        for p, k, a, b, gfh, A, B, C in fields:
            q = p ** k
            mod = field.smallest_monic_irreducible(p, k)
            _, log = field.log_tables(p, k, mod)
            dt = workloads.gf_index_dtype(p, k)
            ga = torch.randint(0, q, (nd,), dtype=torch.int32, device=dev)
            gb = torch.randint(0, q, (nd,), dtype=torch.int32, device=dev)
            tdt = torch.uint8 if dt == np.uint8 else torch.int16
            out = torch.empty(1, dtype=tdt, device=dev)
            row = {"products_per_redq": {(2, 8): "all (XOR)", (3, 5): 6, (7, 4): 3}.get((p, k), fp.fp_gf_dot_info(gfh)["chunk"])}
            for form, nm in ((fp.FP_GF_INDEX, "index"), (fp.FP_GF_LOG, "log")):
                if form == fp.FP_GF_LOG:
                    lt = torch.from_numpy(log.astype(np.int32)).to(dev)
                    xa, xb = lt[ga.long()].to(tdt), lt[gb.long()].to(tdt)
                else:
                    xa, xb = ga.to(tdt), gb.to(tdt)
                pre = 1 << 20
                fp.fp_gf_dot(ctx, gfh, xa, xb, pre, out, form)
                torch.cuda.synchronize()
                fp.fp_ctx_status(ctx)
                ha = ga[:pre].cpu().numpy().astype(np.int64)
                hb = gb[:pre].cpu().numpy().astype(np.int64)
                want = field.gf_dot(ha, hb, p, k, mod)
                got = int(out.cpu().numpy().view(np.uint16)[0]) if tdt == torch.int16 else int(out.item())
                assert got == (log[want] if form == fp.FP_GF_LOG else want), f"GF({p}^{k}) dot parity ({nm})"
                fn = lambda xa=xa, xb=xb, form=form: fp.fp_gf_dot(ctx, gfh, xa, xb, nd, out, form)
                t = statistics.median(_timed(torch, stream, fn, 5, flush))
                eb = 2 * nd * xa.element_size()
                word_kernel = {(2, 8): "k_gf_dot_w28", (3, 5): "k_gf_dot_wsum", (7, 4): "k_gf_dot_wsum"}.get((p, k))
                row[nm] = {"ms": t, "F_p MAC/s": k * k * nd / (t / 1e3), "GB/s": eb / (t / 1e3) / 1e9,
                           "frac_hbm": eb / (t / 1e3) / 1e9 / hbm, "kernel": word_kernel or "k_gf_dot"}
            dot_rows[f"GF({p}^{k})"] = row
            del ga, gb, xa, xb
    # GF(p^k) matrix product (Algorithm FGDP on every entry): 1024 x 1024 x 1024 per field,
    # sampled entries against the oracle's field dot product first
    mm_rows = {}
    if not args.no_compare:
        nm_ = 1024
        for p, k, a, b, gfh, A, B, C in fields:
            q = p ** k
            mod = field.smallest_monic_irreducible(p, k)
            dt = workloads.gf_index_dtype(p, k)
            g_ = np.random.default_rng(q)
            ha = g_.integers(0, q, (nm_, nm_)).astype(dt)
            hb = g_.integers(0, q, (nm_, nm_)).astype(dt)
            tdt = torch.uint8 if dt == np.uint8 else torch.int16
            to = lambda x: torch.from_numpy(x.view(np.int16) if x.dtype == np.uint16 else x).to(dev)
            Am, Bm = to(ha), to(hb)
            Cm = torch.empty((nm_, nm_), dtype=tdt, device=dev)
            fn = lambda Am=Am, Bm=Bm, Cm=Cm, gfh=gfh: fp.fp_gf_matmul(ctx, gfh, nm_, nm_, nm_, Am, nm_, Bm, nm_, Cm, nm_)
            fn()
            torch.cuda.synchronize()
            fp.fp_ctx_status(ctx)
            got = Cm.cpu().numpy()
            got = got.view(np.uint16) if dt == np.uint16 else got
            for r_, c_ in ((0, 0), (511, 1023), (1023, 7)):
                assert int(got[r_, c_]) == field.gf_dot(ha[r_].astype(np.int64), hb[:, c_].astype(np.int64), p, k, mod), \
                    f"GF({p}^{k}) matmul parity"
            t = statistics.median(_timed(torch, stream, fn, 3, flush))
            word_field = (p, k) in ((2, 8), (3, 5), (7, 4))
            mm_rows[f"GF({p}^{k})"] = {"ms": t, "GF MAC/s": nm_ ** 3 / (t / 1e3), "F_p MAC/s": k * k * nm_ ** 3 / (t / 1e3),
                                        "kernel": "k_gf_matmul_w" if word_field else "k_gf_matmul",
                                        "products_per_redq": {(2, 8): nm_, (3, 5): 6, (7, 4): 3}.get((p, k)) if word_field
                                        else fp.fp_gf_dot_info(gfh)["chunk"]}
            del Am, Bm, Cm
    hin = [(torch.from_numpy(a).pin_memory(), torch.from_numpy(b).pin_memory(), torch.empty(count, dtype=A.dtype).pin_memory())
           for p, k, a, b, gfh, A, B, C in fields]

    def e2e():
        for (p, k, a, b, gfh, A, B, C), (ha, hb, hc) in zip(fields, hin):
            A.copy_(ha, non_blocking=True)
            B.copy_(hb, non_blocking=True)
            fp.fp_gf_mul_batched(ctx, gfh, A, B, C, count)
            hc.copy_(C, non_blocking=True)

    e2e()
    torch.cuda.synchronize()
    te = statistics.median(_timed(torch, stream, e2e, 5))
    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline("gf", "F_p MAC/s", "2^17 pairs per field per pass, numpy schoolbook + remainder by the modulus")
    kper = kms / max(1, nk)
    # The kernel is bound by the integer ALU pipe (shifts, masks, logic): its roof is that pipe's
    # rate from unit counts, 152 SMs x 64 lanes x 2.07 GHz, and `achieved` the ALU-pipe operations
    # of the committed ncu capture (per product, per field) over the live launch time.  Null when
    # the kernel's source changed since the capture.  The HBM view stays in per_field.
    alu_peak = 152 * 64 * 2.07e9
    alu_ops = None
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            tg = json.load(f).get("k_gf_mul_fixed", {})
        if tg.get("source_hash") == kernel_source_hash("k_gf_mul_fixed") and "alu_ops_per_product" in tg:
            alu_ops = sum(tg["alu_ops_per_product"][f"GF({p}^{k})"] * count for p, k in workloads.GF_FIELDS)
    except (OSError, ValueError, KeyError):
        alu_ops = None
    ach = alu_ops / len(fields) / (kper / 1e3) if alu_ops else None
    roof = {"bound": "alu", "kernel": "k_gf_mul_fixed", "achieved": ach / 1e12 if ach else None,
            "peak": alu_peak / 1e12, "unit": "T int32 ops/s", "frac": ach / alu_peak if ach else None,
            "traffic": stored_traffic("k_gf_mul_fixed", [(f"GF({p}^{k})", count) for p, k in workloads.GF_FIELDS],
                                      len(fields)),
            "peak_source": "integer ALU pipe from unit counts: 152 SMs x 64 lanes x 2.07 GHz",
            "launches": nk, "avg_launch_ms": kper,
            "hbm_frac": nbytes / len(fields) / (kper / 1e3) / 1e9 / hbm,
            "note": "achieved = ALU-pipe operations per launch (committed ncu capture) / average launch time"}
    res = None
    if rank == 0:
        res = {
            "metric": METRIC, "value": ws * macs / (t_ms / 1e3), "unit": "F_p MAC/s", "n_gpus": ws,
            "steps": len(ts), "warmup": max(3, args.warmup), "ms_per_step": t_ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32 DQT words, u64 products",
            "data": "synthetic",
            "config": {"workload": "GF(p^k) multiply, 2^24 pairs each in GF(3^5), GF(7^4), GF(2^8) per step",
                       "l2": "flushed between steps (512 MiB write)", "per_field": per_field},
            "roofline": roof, "cpu_baseline": cpu,
            "e2e": {"value": ws * macs / (te / 1e3), "unit": "F_p MAC/s", "h2d_bytes_per_step": 2 * nbytes // 3,
                    "d2h_bytes_per_step": nbytes // 3},
            "gpu_launches": launches, "clocks": clk.summary(),
            "dot_2^26_terms": dot_rows, "matmul_1024^3": mm_rows,
        }
        if emit:
            print(json.dumps(res))
    fp.fp_ctx_destroy(ctx)
    return res


def run_batch(args, ws, rank, local, emit=True):
    """Uneven batch: 4096 matmul / dot instances (p in {2,3,5,7,17,31}, sizes log-uniform in
    [16, 2048]) in one fp_batch_run call (large products on the tensor-core kernels, the rest in
    one persistent launch), against one fp_matmul / fp_dot call per instance.  All operands live
    in one device arena (inputs, then outputs), so the end-to-end step is one host-to-device copy
    of every input, the call, and one device-to-host copy of every result."""
    import torch
    import __graft_entry__ as g
    g.build()
    import paper_0809_0063_gb300 as fp
    from oracle import field
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    ctx = fp.fp_ctx_create(local)          # the batch: packing degrees from the autotuner
    ctx1 = fp.fp_ctx_create(local)         # the per-instance arm: the fixed AUTO rule
    fp.fp_ctx_autotune(ctx1, 0)
    insts = workloads.uneven_batch(2024, count=4096)
    up = lambda x: (x + 255) & ~255
    off, in_bytes = [], 0
    for x in insts:
        oa = in_bytes
        in_bytes = up(in_bytes + x.a.nbytes)
        ob = in_bytes
        in_bytes = up(in_bytes + x.b.nbytes)
        off.append([oa, ob, 0])
    out_bytes = 0
    for x, o in zip(insts, off):
        o[2] = out_bytes
        out_bytes = up(out_bytes + (x.m * x.n if x.kind == "matmul" else 4))
    h_in = torch.zeros(in_bytes, dtype=torch.uint8).pin_memory()
    hv = h_in.numpy()
    for x, (oa, ob, _) in zip(insts, off):
        hv[oa:oa + x.a.nbytes] = x.a.reshape(-1)
        hv[ob:ob + x.b.nbytes] = x.b.reshape(-1)
    d_in = h_in.to(dev)
    d_out = torch.full((out_bytes,), 255, dtype=torch.uint8, device=dev)
    h_out = torch.empty(out_bytes, dtype=torch.uint8).pin_memory()
    bi, bo = d_in.data_ptr(), d_out.data_ptr()
    arr, macs = [], 0
    for x, (oa, ob, oc) in zip(insts, off):
        kind = 0 if x.kind == "matmul" else 1
        m, n = (x.m, x.n) if kind == 0 else (1, 1)
        arr.append(fp.fp_instance(kind=kind, p=x.p, m=m, n=n, k=x.k, reserved=0, A=bi + oa, B=bi + ob, C=bo + oc))
        macs += x.m * x.n * x.k if kind == 0 else x.k

    def c_of(i):
        x, oc = insts[i], off[i][2]
        if x.kind == "matmul":
            return d_out[oc:oc + x.m * x.n].view(x.m, x.n)
        return d_out[oc:oc + 4]

    stream = torch.cuda.current_stream()
    carr = fp.fp_instances(arr)      # the batch descriptors, built once (reused by every call)

    def batched():
        fp.fp_batch_run(ctx, carr)

    def per_instance():
        for x, a in zip(insts, arr):
            if x.kind == "matmul":
                fp.fp_matmul(ctx1, x.p, x.m, x.n, x.k, a.A, x.k, a.B, x.n, a.C, x.n, fp.FP_MM_AUTO)
            else:
                fp.fp_dot(ctx1, x.p, a.A, a.B, x.k, a.C, fp.FP_ALGO_PLAIN)

    batched()                        # planner + the packing-degree autotuner run once here
    fp.fp_ctx_status(ctx)
    for i in np.random.default_rng(1).choice(len(insts), 16, replace=False):   # parity gate
        x, C = insts[i], c_of(i)
        if x.kind == "matmul":
            rows = np.array([0, x.m - 1])
            assert np.array_equal(C[rows].cpu().numpy(), field.matmul_mod_rows(x.a, x.b, x.p, rows))
        else:
            assert int(C.cpu().numpy().view(np.uint32)[0]) == field.dot_mod(x.a, x.b, x.p)
    if not args.no_compare:
        per_instance()
        torch.cuda.synchronize()
        fp.fp_ctx_status(ctx1)

    def timed(fn, reps):
        # `reps` consecutive steps between two synchronisations (the inputs exceed L2), so one
        # step's host planning overlaps the previous step's kernels as in a running job; the
        # per-step time is the total over reps
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(reps):
            fn()
        a1.record(stream)
        torch.cuda.synchronize()
        return [a0.elapsed_time(a1) / reps]

    for _ in range(max(3, args.warmup)):
        batched()
    torch.cuda.synchronize()
    l0 = fp.fp_ctx_launches(ctx)
    clk = Clocks(local).__enter__()
    tb = timed(batched, args.steps)
    clk.__exit__(None, None, None)
    launches = fp.fp_ctx_launches(ctx) - l0
    # per-kernel times from the library's own events over separate steps
    fp.fp_ctx_profile(ctx, 2)
    fp.fp_ctx_profile(ctx, 1)
    for _ in range(args.steps):
        batched()
    torch.cuda.synchronize()
    fp.fp_ctx_profile(ctx, 0)
    names = ["k_mm_f8g_pre", "k_tile_pack", "k_mm_t16_plain", "k_t16_convert_jobs", "k_batch", "k_put_bytes"]
    kern = {}
    for nm in names:
        c, ms = fp.fp_ctx_profile_read(ctx, nm)
        if c:
            kern[nm] = {"launches_per_step": c / args.steps, "ms_per_step": ms / args.steps}
    tp = None if args.no_compare else timed(per_instance, max(2, args.steps // 5))
    fp.fp_ctx_status(ctx)
    fp.fp_ctx_status(ctx1)
    # the same call captured once into a CUDA graph (plans written by kernels inside the graph)
    # and replayed: no host work per step
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        batched()
    for _ in range(2):
        graph.replay()
    tg = timed(graph.replay, args.steps)
    fp.fp_ctx_status(ctx)
    del graph
    v_b = macs / (statistics.median(tb) / 1e3)
    v_p = None if tp is None else macs / (statistics.median(tp) / 1e3)

    # end to end: every input in, the call, every result out (one copy each way per step)
    def e2e():
        d_in.copy_(h_in, non_blocking=True)
        fp.fp_batch_run(ctx, carr)
        h_out.copy_(d_out, non_blocking=True)

    e2e()
    torch.cuda.synchronize()
    te = timed(e2e, max(3, args.steps // 2))
    fp.fp_ctx_status(ctx)
    hv_out = h_out.numpy()
    for i in np.random.default_rng(2).choice(len(insts), 8, replace=False):   # results read back
        x, oc = insts[i], off[i][2]
        if x.kind == "matmul":
            got = hv_out[oc:oc + x.m * x.n].reshape(x.m, x.n)[[0]]
            assert np.array_equal(got, field.matmul_mod_rows(x.a, x.b, x.p, np.array([0])))
        else:
            assert int(hv_out[oc:oc + 4].view(np.uint32)[0]) == field.dot_mod(x.a, x.b, x.p)
    # The library's routing (fp_batch_run's documented rule): products with p <= 17 and
    # k (p-1)^2 < 2^23 or p <= 31 and 2 k (p/2)^2 + p < 2^23 whose 128 x 256 x 32-padded MACs
    # are >= 2^21 and <= 32 x their own (or any such with k >= 128) on the pre-tiled e4m3
    # kernel, large ones with 31 < p <= 127 and k (p-1)^2 < 2^24 on the bf16 kernel, the rest
    # in the batch kernel.  Roofline of the kernel with the most time
    # per step, on its own MACs.
    def route(x):
        if x.kind != "matmul" or x.p > 127:
            return "k_batch"
        if (x.p <= 17 and x.k * (x.p - 1) ** 2 < (1 << 23)) or (x.p <= 31 and 2 * x.k * (x.p // 2) ** 2 + x.p < (1 << 23)):
            padded = -(-x.m // 128) * 128 * -(-x.n // 256) * 256 * -(-x.k // 32) * 32
            return "k_mm_f8g_pre" if padded >= (1 << 21) and (padded <= 32 * x.m * x.n * x.k or x.k >= 128) \
                else "k_batch"
        big = x.m >= 64 and x.n >= 64 and x.m * x.n * x.k >= (1 << 21)
        return "k_mm_t16_plain" if big and x.k * (x.p - 1) ** 2 < (1 << 24) else "k_batch"
    kmacs = {nm: 0 for nm in ("k_mm_f8g_pre", "k_mm_t16_plain", "k_batch")}
    for x in insts:
        kmacs[route(x)] += x.m * x.n * x.k if x.kind == "matmul" else x.k
    hbm, bf16, _, peak_src = peaks()
    peaks_k = {"k_mm_f8g_pre": (2.0 * bf16, f"fp8 = measured bf16 x 2 ({peak_src})"),
               "k_mm_t16_plain": (bf16, f"measured bf16 dense ({peak_src})"),
               "k_batch": (603.2, "mma.sync bf16 measured by the pipe probe (packed words count as 2 MACs)")}
    dom = max((nm for nm in kmacs if nm in kern), key=lambda nm: kern[nm]["ms_per_step"])
    achieved = 2.0 * kmacs[dom] / (kern[dom]["ms_per_step"] / 1e3) / 1e12
    for nm in kern:
        if nm in kmacs:
            kern[nm]["fp_macs_per_step"] = kmacs[nm]
            kern[nm]["frac_of_roof"] = 2.0 * kmacs[nm] / (kern[nm]["ms_per_step"] / 1e3) / 1e12 / peaks_k[nm][0]
    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline("batch", "F_p MAC/s", "instances of the same 4096-instance batch in random order: up to "
                           "8 rows of each product (numpy int64 matmul + % p), whole dot products")
    out = {"metric": "exact F_p MACs/s (uneven batch, one call)", "value": v_b, "unit": "F_p MAC/s",
           "n_gpus": 1, "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": statistics.median(tb),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "e4m3/bf16/f16",
           "data": "synthetic",
           "config": {"workload": "4096 instances: 50% matmul, 50% dot, p in {2,3,5,7,17,31}, sizes log-uniform [16,2048]",
                      "macs_per_step": macs, "instances": len(insts), "input_bytes": in_bytes, "output_bytes": out_bytes,
                      "autotuner": "on for the batch (packing degree per (p, k class) timed once on the first call); "
                                   "the per-instance arm uses a second context with the fixed rule"},
           "per_instance_launches": None if tp is None else {
               "value": v_p, "unit": "F_p MAC/s", "ms_per_step": statistics.median(tp),
               "launches": "one fp_matmul / fp_dot call per instance (fixed AUTO rule)"},
           "speedup_vs_per_instance": None if v_p is None else v_b / v_p,
           "timing": "consecutive steps between two synchronisations, inputs larger than L2",
           "graph_replay": {"value": macs / (statistics.median(tg) / 1e3), "unit": "F_p MAC/s",
                            "ms_per_step": statistics.median(tg),
                            "note": "the same call captured once in a CUDA graph, replayed"},
           "gpu_launches": launches,
           "clocks": clk.summary(),
           "kernels": kern,
           "roofline": {"bound": "tensor", "kernel": dom, "achieved": achieved, "peak": peaks_k[dom][0],
                        "unit": "TFLOP/s", "frac": achieved / peaks_k[dom][0], "peak_source": peaks_k[dom][1],
                        "traffic": stored_traffic(dom, [("uneven_batch", len(insts))], 1),
                        "traffic_source": "profiles/traffic.json (ncu capture of the same step; null if the "
                                          "kernel's source changed since)",
                        "note": "achieved = 2 x the kernel's own F_p MACs per step / its time per step"},
           "cpu_baseline": cpu,
           "e2e": {"value": macs / (statistics.median(te) / 1e3), "unit": "F_p MAC/s", "h2d_bytes_per_step": in_bytes,
                   "d2h_bytes_per_step": out_bytes}}
    if emit:
        print(json.dumps(out))
    fp.fp_ctx_destroy(ctx)
    fp.fp_ctx_destroy(ctx1)
    return out


def req_macs(code, sz, gf_k):
    if code == 0:
        return (sz[0] + 1) * (sz[1] + 1)
    if code == 1:
        return sz[0]
    if code == 2:
        return sz[0] * gf_k * gf_k
    return sz[0] ** 3


def run_serve(args, ws, rank, local, duration=1.0, rate=20000.0, emit=True):
    """Serving: a Poisson stream (20k requests/s offered for `duration` s; 50% polymul, 30% dot,
    15% GF(p^k) batches, 5% matmul) through the continuous-batching server.  Reports latency
    percentiles at the offered load, and capacity (the stream submitted at once) against a
    per-request-launch server (one direct call per request, in order, synchronised)."""
    import torch
    import __graft_entry__ as g
    g.build()
    import paper_0809_0063_gb300 as fp
    from oracle import field
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    ctx = fp.fp_ctx_create(local)
    gfs = {pk: fp.fp_gf_create(ctx, *pk) for pk in workloads.GF_FIELDS}
    moduli = {pk: field.smallest_monic_irreducible(*pk) for pk in workloads.GF_FIELDS}
    reqs = workloads.serving_stream(77, rate=rate, duration=duration)
    data = [workloads.request_arrays(r) for r in reqs]
    macs = sum(req_macs(c, sz, r.gf_k) for r, (c, sz, A, B, out) in zip(reqs, data))

    def make_req(r, d):
        code, sz, A, B, out = d
        return fp.fp_request(kind=code, p=r.p, a=sz[0], b=sz[1], c=sz[2], reserved=0,
                             gf=gfs[(r.p, r.gf_k)].value if code == 2 else None,
                             host_a=A.ctypes.data, host_b=B.ctypes.data, host_out=out.ctypes.data)

    def serve(paced):
        srv = fp.fp_server_create(ctx, arena_bytes=8 << 30, streams=4, max_batch=512, window_us=args.serve_window_us)
        if paced:
            # one submission per request at its arrival time
            t0 = time.perf_counter()
            first = None
            for r, d in zip(reqs, data):
                while time.perf_counter() - t0 < r.t_arrival:
                    pass
                t = fp.fp_server_submit(srv, make_req(r, d))
                first = t if first is None else first
        else:
            # capacity: the whole stream in one fp_server_submit_many call (descriptors built
            # before the clock starts, as a client holding a queue of requests would)
            arr = (fp.fp_request * len(reqs))(*[make_req(r, d) for r, d in zip(reqs, data)])
            t0 = time.perf_counter()
            first = fp.fp_server_submit_many(srv, arr)
        fp.fp_server_drain(srv, 120.0)
        wall = time.perf_counter() - t0
        lat = np.array(fp.fp_server_latencies(srv, first, len(reqs)))
        st = fp.fp_server_stats_get(srv)
        fp.fp_server_destroy(srv)
        return wall, lat, st

    # warm-up (first-use costs: module load, tables), then the paced run and the capacity run;
    # the collector is run once and held off during the paced run (a collection in the
    # submitting thread would delay arrivals by milliseconds)
    serve(False)
    gc.collect()
    gc.disable()
    try:
        wall_p, lat_p, st_p = serve(True)
    finally:
        gc.enable()
    fp.fp_ctx_profile(ctx, 2)
    fp.fp_ctx_profile(ctx, 1)
    wall_c, lat_c, st_c = serve(False)
    fp.fp_ctx_profile(ctx, 0)
    fp.fp_ctx_status(ctx)
    kern = {}
    for nm in ("k_polymul_var", "k_gf_mul_seg", "k_batch", "k_mm_f8g"):
        c, ms = fp.fp_ctx_profile_read(ctx, nm)
        if c:
            kern[nm] = {"launches": c, "ms": ms}
    # parity gate on a sample of the served results
    for i in np.random.default_rng(3).choice(len(reqs), 40, replace=False):
        r, (code, sz, A, B, out) = reqs[i], data[i]
        if code == 0:
            want = field.polymul_mod(A, B, r.p)
        elif code == 1:
            want = np.array([field.dot_mod(A, B, r.p)])
        elif code == 2:
            want = field.gf_mul(A.astype(np.int64), B.astype(np.int64), r.p, r.gf_k, moduli[(r.p, r.gf_k)])
        else:
            rows = np.array([0, sz[0] - 1])
            assert np.array_equal(out[rows], field.matmul_mod_rows(A, B, r.p, rows))
            continue
        assert np.array_equal(out.astype(np.int64), np.asarray(want).astype(np.int64))

    # per-request launches: one direct call per request, in arrival order, each synchronised
    n_base = min(len(reqs), 3000)
    to = lambda x: torch.from_numpy(x.view(np.int16) if x.dtype == np.uint16 else x).to(dev, non_blocking=False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    base_lat = []
    for r, (code, sz, A, B, out) in list(zip(reqs, data))[:n_base]:
        if code == 0:
            C = torch.empty(out.shape, dtype=torch.uint8, device=dev)
            fp.fp_polymul_batched(ctx, r.p, to(A), sz[0], to(B), sz[1], C, 1)
        elif code == 1:
            C = torch.empty((1,), dtype=torch.int32, device=dev)
            fp.fp_dot(ctx, r.p, to(A), to(B), sz[0], C)
        elif code == 2:
            C = torch.empty(out.shape, dtype=torch.uint8 if out.dtype == np.uint8 else torch.int16, device=dev)
            fp.fp_gf_mul_batched(ctx, gfs[(r.p, r.gf_k)], to(A), to(B), C, sz[0])
        else:
            C = torch.empty(out.shape, dtype=torch.uint8, device=dev)
            fp.fp_matmul(ctx, r.p, sz[0], sz[0], sz[0], to(A), sz[0], to(B), sz[0], C, sz[0])
        C.cpu()
        base_lat.append(time.perf_counter() - t0 - r.t_arrival)
    base_wall = time.perf_counter() - t0
    base_rps = n_base / base_wall
    cap_rps = len(reqs) / wall_c
    pct = lambda a, q: float(np.percentile(a[a >= 0], q))
    # roofline of the kernel with the most device time in the capacity run.  The server's rule:
    # matmul requests with p <= 17, m, n >= 64, k (p-1)^2 < 2^24 and m n k >= 2^21 run on the e4m3
    # kernel k_mm_f8g; other matmuls and the dots on k_batch (legacy mma.sync bf16 tiles);
    # k_polymul_var the blocked-FQT products (integer issue); k_gf_mul_seg the field products
    def tc_req(r, c, sz):
        return c == 3 and r.p <= 17 and sz[0] >= 64 and sz[1] >= 64 and sz[2] * (r.p - 1) ** 2 < (1 << 24) \
            and sz[0] * sz[1] * sz[2] >= (1 << 21)
    f8_macs = sum(req_macs(c, sz, r.gf_k) for r, (c, sz, A, B, out) in zip(reqs, data) if tc_req(r, c, sz))
    mm_macs = sum(req_macs(c, sz, r.gf_k) for r, (c, sz, A, B, out) in zip(reqs, data)
                  if c in (1, 3) and not tc_req(r, c, sz))
    roof = None
    if kern:
        dom = max(kern, key=lambda nm: kern[nm]["ms"])
        hbm_, bf16_, _, psrc_ = peaks()
        if dom in ("k_batch", "k_mm_f8g"):
            mac, pk_, src_ = (mm_macs, 603.2, "mma.sync bf16 measured by the pipe probe") if dom == "k_batch" else \
                (f8_macs, 2.0 * bf16_, f"fp8 = measured bf16 x 2 ({psrc_})")
            ach = 2.0 * mac / (kern[dom]["ms"] / 1e3) / 1e12
            roof = {"bound": "tensor", "kernel": dom, "achieved": ach, "peak": pk_, "unit": "TFLOP/s",
                    "frac": ach / pk_, "traffic": None, "peak_source": src_,
                    "note": "achieved = 2 x the F_p MACs of the requests this kernel ran / its device time"}
        else:
            # the polynomial and field kernels stream their requests' bytes: HBM roof
            code = 0 if dom == "k_polymul_var" else 2
            nb = sum(A.nbytes + B.nbytes + out.nbytes for r, (c, sz, A, B, out) in zip(reqs, data) if c == code)
            ach = nb / (kern[dom]["ms"] / 1e3) / 1e9
            roof = {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": hbm_, "unit": "GB/s", "frac": ach / hbm_,
                    "traffic": None, "peak_source": f"HBM copy ({psrc_})",
                    "note": "achieved = the requests' input and output bytes this kernel handled / its device time "
                            "(many small launches, one per batch: latency-bound)"}
        share = sum(v["ms"] for v in kern.values())
        for nm in kern:
            kern[nm]["share"] = kern[nm]["ms"] / share
    in_b = sum(A.nbytes + B.nbytes for (c, sz, A, B, out) in data)
    out_b = sum(out.nbytes for (c, sz, A, B, out) in data)
    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline("serve", "requests/s", "requests of the same stream in random order, the full oracle "
                           "per request (schoolbook polymul, dot, field product, plain matmul)")
    out = {"metric": "served requests/s (continuous batching) with p50/p99 latency", "value": cap_rps,
           "unit": "requests/s", "n_gpus": 1, "steps": 1, "warmup": 1, "ms_per_step": wall_c * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "mixed", "data": "synthetic",
           "config": {"workload": f"Poisson {rate:.0f} req/s for {duration} s: 50% polymul (deg 2-512, p in 3,5,7), "
                                  "30% dot (64-65536), 15% GF(3^5)/GF(7^4)/GF(2^8) batches (1-4096), 5% matmul (64-1024)",
                      "requests": len(reqs), "fp_macs": macs, "server": f"4 streams, 8 GiB arena, max_batch 512, {args.serve_window_us} us window"},
           "latency_us_at_offered_load": {"p50": pct(lat_p, 50), "p99": pct(lat_p, 99), "p999": pct(lat_p, 99.9),
                                          "max": float(lat_p.max()), "wall_s": wall_p, "batches": st_p["batches"]},
           "capacity": {"requests_per_s": cap_rps, "fp_macs_per_s": macs / wall_c, "batches": st_c["batches"],
                        "p50_us": pct(lat_c, 50), "p99_us": pct(lat_c, 99)},
           "per_request_launches": {"requests_per_s": base_rps, "requests": n_base,
                                    "p50_latency_us_at_offered_load": float(np.percentile(base_lat, 50)) * 1e6,
                                    "p99_latency_us_at_offered_load": float(np.percentile(base_lat, 99)) * 1e6},
           "capacity_vs_per_request": cap_rps / base_rps,
           "kernels_capacity_run": kern, "roofline": roof, "cpu_baseline": cpu,
           "e2e": {"value": cap_rps, "unit": "requests/s", "h2d_bytes_per_step": in_b, "d2h_bytes_per_step": out_b,
                   "note": "the server is end to end: host buffers in, host buffers out; a step is the whole stream"}}
    if emit:
        print(json.dumps(out))
    for g2 in gfs.values():
        fp.fp_gf_destroy(g2)
    fp.fp_ctx_destroy(ctx)
    return out


def graph_steps(torch, stream, step, flush, steps):
    """Per-step device times (ms) of `steps` replays of one CUDA graph of `step`, the L2 flushed
    (outside the events) before each; plain launches if the step cannot be captured."""
    graph = torch.cuda.CUDAGraph()
    try:
        with torch.cuda.graph(graph):
            step()
        run = graph.replay
        run()
    except Exception:           # not capturable: time plain launches
        torch.cuda.synchronize()
        graph, run = None, step
    torch.cuda.synchronize()
    ts = _timed(torch, stream, run, steps, flush)
    return ts, graph is not None


def packed_arm(args, fp, torch, ctx, prob, flush, stream, ktab, peak_src, plain_value, local):
    """Packed DQT + REDQ on the same resident inputs as the headline step: the right-compressed
    product (Sec. 7.4) of every problem on the tensor cores -- fp16 words with two centred
    residues (RIGHT_TC: Q = 2^10 in chunks of 448 inner steps for p = 3, Q = 2^9 in chunks of 16
    for p = 7), one grouped call -- timed as a graph-replayed step like the headline.  The
    dominant packed kernel's roofline counts its word operations 2 m ceil(n/2) k; the plain
    bf16 products on the same pipe (PLAIN_TC) are timed the same way for the same-pipe ratio."""
    from oracle import field
    macs = sum(q["n"] ** 3 for q in prob)
    descs = [fp.fp_mm_problem_of(q["p"], q["n"], q["n"], q["n"], q["A"], q["n"], q["B"], q["n"], q["C"], q["n"])
             for q in prob]
    arms = {}
    for label, algo in (("packed", fp.FP_MM_RIGHT_TC), ("plain_same_pipe", fp.FP_MM_PLAIN_TC)):
        def step(algo=algo):
            fp.fp_matmul_grouped(ctx, descs, algo)

        for q in prob:
            q["C"].fill_(255)
        step()
        torch.cuda.synchronize()
        fp.fp_ctx_status(ctx)
        for q in prob:          # parity gate: rows across the tile rows against the oracle
            rows = np.array([0, q["n"] // 3, q["n"] - 1])
            assert np.array_equal(q["C"][rows].cpu().numpy(), field.matmul_mod_rows(q["a"], q["b"], q["p"], rows)), \
                f"{label} parity p={q['p']} n={q['n']}"
        for _ in range(args.warmup):
            flush.zero_()
            step()
        ts, graphed = graph_steps(torch, stream, step, flush, args.steps)
        fp.fp_ctx_status(ctx)
        t_ms = statistics.median(ts)
        # per-kernel device time from the library's events over plain steps
        fp.fp_ctx_profile(ctx, 2)
        fp.fp_ctx_profile(ctx, 1)
        for _ in range(args.steps):
            flush.zero_()
            step()
        torch.cuda.synchronize()
        fp.fp_ctx_profile(ctx, 0)
        kern = {}
        for nm in ("k_mm_t16_packed_p57", "k_mm_t16_packed", "k_mm_t16_plain", "k_t16_convert"):
            c, ms = fp.fp_ctx_profile_read(ctx, nm)
            if nm == "k_mm_t16_packed":            # prefix of the p = 5, 7 kernel's name
                c2, ms2 = fp.fp_ctx_profile_read(ctx, "k_mm_t16_packed_p57")
                c, ms = c - c2, ms - ms2
            if c:
                kern[nm] = {"launches_per_step": c / args.steps, "ms_per_step": ms / args.steps}
        arms[label] = {"value": macs / (t_ms / 1e3), "ms_per_step": t_ms, "kernels": kern,
                       "timing": "CUDA graph replay of the step" if graphed else "plain launches"}
    pk = arms["packed"]
    cand = {"k_mm_t16_packed": [q for q in prob if q["p"] <= 3], "k_mm_t16_packed_p57": [q for q in prob if q["p"] > 3]}
    roofs = {}
    kt = ktab["k_mm_t16_packed"]
    for nm, qs in cand.items():
        if nm not in pk["kernels"] or not qs:
            continue
        flops = sum(2.0 * q["n"] * q["n"] * (-(-q["n"] // 2)) for q in qs)
        k_ms = pk["kernels"][nm]["ms_per_step"]
        ach = flops / (k_ms / 1e3) / 1e12
        roofs[nm] = {"bound": kt[0], "kernel": nm, "achieved": ach, "peak": kt[1], "unit": "TFLOP/s",
                     "frac": ach / kt[1], "traffic": None, "peak_source": kt[2] + f" ({peak_src})",
                     "avg_launch_ms": k_ms / pk["kernels"][nm]["launches_per_step"],
                     "problems": [f"p={q['p']} n={q['n']}" for q in qs],
                     "note": "achieved = word flops 2 m ceil(n/2) k of its problems / the kernel's device time per step"}
    dom = max(roofs, key=lambda nm: pk["kernels"][nm]["ms_per_step"]) if roofs else None
    return {"value": pk["value"], "unit": "F_p MAC/s", "ms_per_step": pk["ms_per_step"],
            "algo": "RIGHT_TC (grouped): fp16 pair words, Q = 2^10 (p = 3) / 681 (p = 7)",
            "timing": pk["timing"], "roofline": roofs.get(dom), "roofline_per_kernel": roofs, "kernels": pk["kernels"],
            "packed_over_plain": pk["value"] / plain_value,
            "packed_over_plain_note": "same inputs; plain = the headline step (e4m3 tensor cores, AUTO)",
            "plain_same_pipe": {"value": arms["plain_same_pipe"]["value"], "algo": "PLAIN_TC (bf16, grouped)",
                                "ms_per_step": arms["plain_same_pipe"]["ms_per_step"],
                                "kernels": arms["plain_same_pipe"]["kernels"]},
            "packed_over_plain_same_pipe": pk["value"] / arms["plain_same_pipe"]["value"]}


def run_matmul(args, ws, rank, local):
    """The default line: the compressed matrix product configuration (p in {3, 7} x n in
    {1024, 4096}); returns the JSON object rank 0 prints (None on other ranks)."""
    import torch
    import __graft_entry__ as g
    g.build()
    import paper_0809_0063_gb300 as fp

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    hbm, bf16, bf16s, peak_src = peaks()
    ktab = kernel_table(bf16)
    algo = getattr(fp, "FP_MM_" + args.algo)
    ctx = fp.fp_ctx_create(local)
    if args.no_autotune:
        fp.fp_ctx_autotune(ctx, 0)

    # resident inputs (seeded, identical on every rank: replicas)
    prob = []
    for p, n in PROBLEMS:
        a, b = workloads.matmul_inputs(p * 7 + n, p, n, n, n)
        prob.append(dict(p=p, n=n, a=a, b=b, A=torch.from_numpy(a).to(dev), B=torch.from_numpy(b).to(dev),
                         C=torch.empty((n, n), dtype=torch.uint8, device=dev)))
    macs_per_step = sum(n ** 3 for _, n in PROBLEMS)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    # one grouped call per step: the products that fit the e4m3 tensor-core path share one
    # persistent launch, any other goes through fp_matmul with the same algo
    descs = [fp.fp_mm_problem_of(q["p"], q["n"], q["n"], q["n"], q["A"], q["n"], q["B"], q["n"], q["C"], q["n"])
             for q in prob]

    def step(al=algo):
        fp.fp_matmul_grouped(ctx, descs, al)

    # parity gate on the resident buffers before timing (sampled rows against the oracle)
    from oracle import field
    step()
    fp.fp_ctx_status(ctx)
    for q in prob:
        rows = np.array([0, q["n"] // 2 + 1, q["n"] - 1])
        assert np.array_equal(q["C"][rows].cpu().numpy(), field.matmul_mod_rows(q["a"], q["b"], q["p"], rows)), \
            f"parity failure p={q['p']} n={q['n']}"

    # algorithm actually used per problem (the autotuner's cached choice under AUTO)
    chosen = {}
    for q in prob:
        grouped = args.algo in ("AUTO", "PLAIN_F8") and q["p"] <= 17 and q["n"] * (q["p"] - 1) ** 2 < 2 ** 24
        if grouped:
            chosen[(q["p"], q["n"])] = fp.FP_MM_PLAIN_F8
            continue
        a = fp.fp_ctx_autotune_choice(ctx, q["p"], q["n"], q["n"], q["n"]) if args.algo == "AUTO" else algo
        if a < 0 and args.algo == "AUTO":       # fixed rule (autotuning off): first exact candidate
            a = fp.FP_MM_PLAIN_F8 if q["p"] <= 17 else fp.FP_MM_PLAIN_TC
        chosen[(q["p"], q["n"])] = a if a >= 0 else algo
    names = {getattr(fp, k): k[6:] for k in dir(fp) if k.startswith("FP_MM_")}
    clk = Clocks(local).__enter__()
    t_w = time.perf_counter()
    nw_steps = 0
    while nw_steps < args.warmup or time.perf_counter() - t_w < args.min_warmup_s:   # >= W steps, >= 1 s loaded
        flush.zero_()
        step()
        nw_steps += 1
        if nw_steps % 8 == 0:
            torch.cuda.synchronize()
    torch.cuda.synchronize()
    # the step as one CUDA graph: every library call is capture-safe once warm (no host syncs,
    # no scratch growth, AUTO choices cached), so a step replays all its kernels with one launch
    graph = None
    launches_per_step = None
    if not args.no_graph:
        l_a = fp.fp_ctx_launches(ctx)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            step()
        launches_per_step = fp.fp_ctx_launches(ctx) - l_a
        graph.replay()
        torch.cuda.synchronize()
        fp.fp_ctx_status(ctx)
        for q in prob:   # parity of the replayed graph
            rows = np.array([2, q["n"] - 3])
            assert np.array_equal(q["C"][rows].cpu().numpy(), field.matmul_mod_rows(q["a"], q["b"], q["p"], rows))
    run_step = graph.replay if graph is not None else step
    # plain launches timed too (reported beside the graph number)
    ev0 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for i in range(args.steps):
        flush.zero_()
        ev0[i][0].record(stream)
        step()
        ev0[i][1].record(stream)
    torch.cuda.synchronize()
    plain_ms = sum(a.elapsed_time(b) for a, b in ev0)
    if ws > 1:
        torch.distributed.barrier()
    l0 = fp.fp_ctx_launches(ctx)
    fp.fp_ctx_profile(ctx, 2)
    fp.fp_ctx_profile(ctx, 1)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for i in range(args.steps):
        flush.zero_()                   # L2 flushed between steps (outside the events)
        ev[i][0].record(stream)
        run_step()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    clk.__exit__(None, None, None)
    fp.fp_ctx_profile(ctx, 0)
    fp.fp_ctx_status(ctx)
    launches = fp.fp_ctx_launches(ctx) - l0
    if graph is not None:          # graph replays do not pass through the library's counter
        launches = launches_per_step * args.steps
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(sum(step_ms), dev)
    value = whole_job_rate(macs_per_step, args.steps, ws, total_ms)

    if graph is not None:
        # per-kernel events need the library's own launches: one profiled pass of plain steps
        fp.fp_ctx_profile(ctx, 2)
        fp.fp_ctx_profile(ctx, 1)
        for i in range(args.steps):
            flush.zero_()
            step()
        torch.cuda.synchronize()
        fp.fp_ctx_profile(ctx, 0)
    # dominant kernel and its roofline from the library's own per-launch events
    dominant, dom_ms, dom_n = None, 0.0, 0
    for name in ktab:
        n_l, ms = fp.fp_ctx_profile_read(ctx, name)
        if ms > dom_ms:
            dominant, dom_ms, dom_n = name, ms, n_l
    roof = None
    if dominant:
        bound, peak, peak_label, flops_fn = ktab[dominant]
        flops = 0.0
        shapes = []
        kernel_of = {"RIGHT_F32": "k_mm_ffma", "PLAIN_F32": "k_mm_ffma", "RIGHT_F64": "k_mm_dmma",
                     "PLAIN_F64": "k_mm_dmma", "PLAIN_I8": "k_mm_imma", "PLAIN_TC": "k_mm_t16_plain", "RIGHT_TC": "k_mm_t16_packed",
                     "PLAIN_F8": "k_mm_f8g"}
        for p, n in PROBLEMS:
            an = names[chosen[(p, n)]]
            if kernel_of.get(an) != dominant:
                continue
            if an == "RIGHT_F64" or an == "PLAIN_F64":
                e = fp.fp_mm_choose(p, n, getattr(fp, "FP_MM_" + an))[1]
            elif an in ("RIGHT_F32", "RIGHT_TC"):
                e = 2
            else:
                e = 1
            f = flops_fn(n, e) * args.steps
            flops += f / args.steps
            shapes.append((an, n))
        flops *= args.steps
        achieved = flops / (dom_ms / 1e3) / 1e12
        traffic = stored_traffic(dominant, shapes, max(1, dom_n // args.steps))
        roof = {"bound": bound, "kernel": dominant, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic, "peak_source": peak_label + f" ({peak_src})",
                "launches": dom_n, "avg_launch_ms": dom_ms / max(1, dom_n)}

    packed_res = None
    if not args.no_packed and args.algo == "AUTO":
        packed_res = packed_arm(args, fp, torch, ctx, prob, flush, stream, ktab, peak_src, value, local)
    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    hA = [torch.from_numpy(q["a"]).pin_memory() for q in prob]
    hB = [torch.from_numpy(q["b"]).pin_memory() for q in prob]
    hC = [torch.empty((q["n"], q["n"]), dtype=torch.uint8).pin_memory() for q in prob]
    h2d = sum(q["a"].nbytes + q["b"].nbytes for q in prob)
    d2h = sum(q["n"] * q["n"] for q in prob)

    # Three streams (host-to-device copies, compute, device-to-host copies) and two device buffer
    # sets: step s+1's inputs are copied while step s computes and step s-1's results are read
    # back; within a step, product i computes as soon as its own inputs have landed.  Every step
    # copies all its inputs in and all its results out; the time of K steps / K is the step time.
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
    sets = [[(q["A"], q["B"], q["C"]) for q in prob],
            [(torch.empty_like(q["A"]), torch.empty_like(q["B"]), torch.empty_like(q["C"])) for q in prob]]
    ev_in = [[torch.cuda.Event() for _ in prob] for _ in range(2)]
    ev_c = [[torch.cuda.Event() for _ in prob] for _ in range(2)]
    ev_out = [[torch.cuda.Event() for _ in prob] for _ in range(2)]
    ev_used = [torch.cuda.Event() for _ in range(2)]

    def e2e_steps(nsteps, start):
        s_in.wait_event(start)
        for st_i in range(nsteps):
            bset = st_i % 2
            S = sets[bset]
            if st_i >= 2:
                s_in.wait_event(ev_used[bset])          # step st_i-2 has finished reading these inputs
            with torch.cuda.stream(s_in):
                for i in range(len(prob)):
                    S[i][0].copy_(hA[i], non_blocking=True)
                    S[i][1].copy_(hB[i], non_blocking=True)
                    ev_in[bset][i].record(s_in)
            for i, q in enumerate(prob):
                stream.wait_event(ev_in[bset][i])
                if st_i >= 2:
                    stream.wait_event(ev_out[bset][i])  # step st_i-2's result has been read back
                fp.fp_matmul(ctx, q["p"], q["n"], q["n"], q["n"], S[i][0], q["n"], S[i][1], q["n"], S[i][2], q["n"],
                             algo, stream=stream)
                ev_c[bset][i].record(stream)
            ev_used[bset].record(stream)
            with torch.cuda.stream(s_out):
                for i in range(len(prob)):
                    s_out.wait_event(ev_c[bset][i])
                    hC[i].copy_(S[i][2], non_blocking=True)
                    ev_out[bset][i].record(s_out)
        stream.wait_stream(s_in)
        stream.wait_stream(s_out)

    w0 = torch.cuda.Event()
    w0.record(stream)
    e2e_steps(2, w0)
    torch.cuda.synchronize()
    e_ms = []
    n_e2e = max(8, args.steps)
    for _ in range(2):
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        e2e_steps(n_e2e, a0)
        a1.record(stream)
        torch.cuda.synchronize()
        e_ms.append(a0.elapsed_time(a1) / n_e2e)
    fp.fp_ctx_status(ctx)
    for i, q in enumerate(prob):
        rows = np.array([1, q["n"] - 2])
        assert np.array_equal(hC[i][rows].numpy(), field.matmul_mod_rows(q["a"], q["b"], q["p"], rows))
    e2e_val = ws * macs_per_step / (statistics.mean(e_ms) / 1e3)

    # packed vs plain on the same inputs (one timed repetition each, after the headline)
    compare = None
    if not args.no_compare and rank == 0:
        compare = {}
        fp64_peak = ktab["k_mm_dmma"][1]
        fp64_rows = {}
        for name in ["RIGHT_F32", "LEFT_F32", "PLAIN_F32", "RIGHT_F64", "SPLIT_F64", "FULL_F64", "LEFT_F64", "CMM_F64",
                     "PLAIN_F64", "PLAIN_I8", "PLAIN_TC", "RIGHT_TC", "PLAIN_F8"]:
            row = {}
            for q in prob:
                al = getattr(fp, "FP_MM_" + name)
                if name in ("PLAIN_F64", "LEFT_F64", "CMM_F64") and q["n"] > 1024:
                    continue
                try:
                    fn = (lambda q=q, al=al: fp.fp_matmul(ctx, q["p"], q["n"], q["n"], q["n"], q["A"], q["n"],
                                                          q["B"], q["n"], q["C"], q["n"], al))
                    fn()
                    torch.cuda.synchronize()
                    flush.zero_()
                    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a0.record(stream)
                    fn()
                    a1.record(stream)
                    torch.cuda.synchronize()
                    fp.fp_ctx_status(ctx)
                    ms = a0.elapsed_time(a1)
                    row[f"p{q['p']}_n{q['n']}"] = q["n"] ** 3 / (ms / 1e3)
                    if name in ("RIGHT_F64", "SPLIT_F64", "FULL_F64"):
                        # FP64 word products on DMMA: the word flops of the packing against the FP64 roof
                        n_ = q["n"]
                        if name == "FULL_F64":
                            b_, q1, t1, piece = fp.fp_mm_full_choose(q["p"], n_)
                            wf, pk = 2.0 * (-(-n_ // q1)) * (-(-n_ // t1)) * n_, f"{q1}x{t1} digits, pieces of {piece}"
                        else:
                            b_, e_, piece = fp.fp_mm_choose(q["p"], n_, al)
                            wf, pk = 2.0 * n_ * (-(-n_ // e_)) * n_, f"e={e_}, pieces of {piece}"
                        fp64_rows.setdefault(name, {})[f"p{q['p']}_n{n_}"] = {
                            "ms": ms, "F_p MAC/s": n_ ** 3 / (ms / 1e3), "packing": pk,
                            "word_tflops": wf / (ms / 1e3) / 1e12, "frac_fp64_roof": wf / (ms / 1e3) / 1e12 / fp64_peak}
                except fp.FpError as ex:
                    row[f"p{q['p']}_n{q['n']}"] = f"unavailable: {ex.args[0][:60]}"
            compare[name] = row
        # packed DQT+REDQ against the plain product on the same pipe, same inputs
        pairs = (("RIGHT_TC", "PLAIN_TC"), ("RIGHT_F32", "PLAIN_F32"), ("LEFT_F32", "PLAIN_F32"),
                 ("RIGHT_F64", "PLAIN_F64"), ("LEFT_F64", "PLAIN_F64"), ("CMM_F64", "PLAIN_F64"))
        pvp = {}
        for packed, plain in pairs:
            for key, v in compare.get(packed, {}).items():
                w = compare.get(plain, {}).get(key)
                if isinstance(v, float) and isinstance(w, float):
                    pvp.setdefault(key, {})[f"{packed}/{plain}"] = v / w
        compare["packed_over_plain_same_pipe"] = pvp
        compare["fp64_words_on_dmma"] = {"roof_tflops": fp64_peak, "roof_source": ktab["k_mm_dmma"][2],
                                         "note": "one timed call each, includes any packing launch", "rows": fp64_rows}

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline("matmul", "F_p MAC/s", "16-row blocks of the four products in turn, numpy int64 matmul + % p")

    dt_of = {"RIGHT_F32": "f32", "PLAIN_F32": "f32", "RIGHT_F64": "f64", "PLAIN_F64": "f64",
             "PLAIN_I8": "u8", "PLAIN_TC": "bf16", "RIGHT_TC": "f16", "PLAIN_F8": "e4m3"}
    dtype = "/".join(sorted({dt_of[names[a]] for a in chosen.values()}))
    out = None
    if rank == 0:
        out = {
            "metric": METRIC,
            "value": value, "unit": "F_p MAC/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dtype, "data": "synthetic",
            "config": {"workload": WORKLOAD, "algo": args.algo,
                       "problems": {f"p={p} n={n}": names[chosen[(p, n)]] for p, n in PROBLEMS},
                       "macs_per_step": macs_per_step, "l2": "flushed between steps (512 MiB write)",
                       "parallelism": "replicas" if ws > 1 else "single GPU"},
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_val, "unit": "F_p MAC/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "timing": "CUDA graph replay of the step" if graph is not None else "plain launches",
            "value_plain_launches": whole_job_rate(macs_per_step, args.steps, ws, max_over_ranks(plain_ms, dev)),
            "clocks": clk.summary(),
            "compare_same_inputs": compare,
            "packed_dqt_redq": packed_res,
        }
    fp.fp_ctx_destroy(ctx)
    return out



def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="matmul", choices=["matmul", "batch", "serve", "polymul", "gf"],
                    help="matmul: the compressed-matmul configuration (default line); batch: 4096 uneven instances")
    ap.add_argument("--algo", default="AUTO")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the per-variant comparison block (batch: the per-instance arm)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--problems", default="", help="subset, e.g. 3:4096,7:1024 (default: all four)")
    ap.add_argument("--no-graph", action="store_true", help="time plain launches instead of CUDA-graph replays")
    ap.add_argument("--no-packed", action="store_true", help="skip the packed DQT+REDQ arm of the default line")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the nested polynomial, GF, uneven-batch and serving sub-results of the default line")
    ap.add_argument("--serve-window-us", type=int, default=100,
                    help="serving: how long a forming batch may wait to grow while the GPU is busy")
    ap.add_argument("--no-autotune", action="store_true",
                    help="AUTO uses the fixed rule instead of timing candidates (for runs under a profiler)")
    ap.add_argument("--min-warmup-s", type=float, default=1.0,
                    help="keep warming up at least this long (clock sampling under load)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    global PROBLEMS
    if args.problems:
        PROBLEMS = [tuple(int(x) for x in t.split(":")) for t in args.problems.split(",")]
    ws, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    if args.workload == "batch":
        run_batch(args, ws, rank, local)
        close_pool()
        return
    if args.workload == "serve":
        run_serve(args, ws, rank, local)
        close_pool()
        return
    if args.workload == "polymul":
        run_polymul(args, ws, rank, local)
        close_pool()
        return
    if args.workload == "gf":
        run_gf(args, ws, rank, local)
        close_pool()
        return

    import torch
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    out = run_matmul(args, ws, rank, local)
    if ws == 1 and not args.no_configs:
        # the other configurations of the metric, nested in the same line (one GPU; replicas
        # would repeat them unchanged)
        out["configs"] = {
            "polymul_2^20_F3_degree2": run_polymul(args, ws, rank, local, emit=False),
            "gf_mul_2^24_pairs_x3_fields": run_gf(args, ws, rank, local, emit=False),
            "uneven_batch_4096": run_batch(args, ws, rank, local, emit=False),
            "serving_poisson_20k": run_serve(args, ws, rank, local, emit=False),
        }
    close_pool()
    if rank == 0:
        print(json.dumps(out))
    if ws > 1:
        torch.distributed.destroy_process_group()

if __name__ == "__main__":
    main()
