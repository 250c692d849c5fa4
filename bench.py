#!/usr/bin/env python3
"""Benchmark of the structured-sketch hot path on GB300.

One step = one full pass of the sparse sign embedding over the embedding-throughput workload
(A 2^22 x 256 BF16 with N(0,1) entries times logspaced column scales, d = 2048, zeta = 8):
draw S and build its inverted index, gather S*A, reduce -- every step with a fresh seed, so
nothing is cached between steps.  The metric is GB/s of A read.  A (2.1 GB) is larger than L2, so
no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 (launched by torch.distributed.run): the headline A is split into N row blocks, one per rank
(strong scaling); each rank sketches its block (rsk_sparse_sign_apply_rows, its columns of the one
S), the N partial d x k sketches are gathered over NCCL and summed in rank order on every rank
(rsk_sketch_sum_partials); rank 0 prints the line with the max step time over ranks.
--impl reference times the FP64 CPU oracle on a bounded sample of the same workload.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "SA GB/s of A read (% HBM peak); LSQ solves/sec at 1e-10 bwd err, mixed vs FP64"
N_ROWS, K_COLS, D_SKETCH, ZETA = 1 << 22, 256, 2048, 8
LSQ_N, LSQ_K, LSQ_D = 1 << 20, 500, 2000
BATCH_COUNT = 512
RSVD_M, RSVD_N, RSVD_R, RSVD_Q, RSVD_RANK = 262144, 8192, 300, 2, 400
RSVD_TWIN = (16384, 2048, 100, 75)  # m, n, spectrum rank, r of the reduced twin the oracle also runs
NYS_N, NYS_K, NYS_RANK = 32768, 300, 1000
GEN_N, GEN_D, GEN_K, GEN_RANK = 131072, 40000, 200, 400
OSI_R = (10 ** 5, 10 ** 6, 10 ** 7)
FALLBACK_HBM_GBS = 6800.0
APPLY_SOURCES = ["paper_2508_21189_gb300/csrc/sparse_sign.cu", "paper_2508_21189_gb300/csrc/common.cuh"]


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--rows", type=int, default=N_ROWS, help="rows of A (smaller only for profiling captures)")
    p.add_argument("--dtypes", default="bf16,fp32", help="A storage types to time; the first is the headline")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-srtt", action="store_true")
    p.add_argument("--no-lsq", action="store_true", help="skip the least-squares solves/sec measurements")
    p.add_argument("--no-rsvd", action="store_true")
    p.add_argument("--solve-reps", type=int, default=3, help="timed calls per least-squares / RSVD form")
    p.add_argument("--lsq-rows", type=int, default=LSQ_N, help="rows of the single least-squares A (smaller only "
                   "for profiling captures)")
    p.add_argument("--batch-count", type=int, default=BATCH_COUNT, help="problems in the batched least-squares "
                   "workload (smaller only for profiling captures)")
    p.add_argument("--rsvd-rows", type=int, default=RSVD_M, help="rows of the RSVD A (smaller only for profiling "
                   "captures)")
    p.add_argument("--profile-rsvd", action="store_true", help="open the CUDA profiler range around the timed RSVD "
                   "calls only (for ncu --profile-from-start off)")
    p.add_argument("--no-autotune", action="store_true", help="keep the default launch parameters for the headline "
                   "shape instead of timing candidates first")
    p.add_argument("--no-variants", action="store_true", help="skip the SparseStack / SparseRTT sketches")
    p.add_argument("--no-nystrom", action="store_true", help="skip the Nystrom approximations")
    p.add_argument("--no-osi", action="store_true", help="skip the injectivity/dilation estimator")
    p.add_argument("--nystrom-n", type=int, default=NYS_N, help="order of the psd Nystrom matrix")
    p.add_argument("--gen-rows", type=int, default=GEN_N, help="rows of the generalized Nystrom matrix")
    p.add_argument("--gen-cols", type=int, default=GEN_D, help="columns of the generalized Nystrom matrix")
    return p.parse_args()


# ------------------------------------------------------------------------------------------
# distributed plumbing
# ------------------------------------------------------------------------------------------
def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def dist_init(backend):
    import torch.distributed as dist
    rank, world, _ = dist_env()
    if world > 1 and not dist.is_initialized():
        dist.init_process_group(backend=backend)
    return rank, world


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def max_over_ranks(x, device="cpu"):
    """Max of a float over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------------------------------
# clocks, peaks, traffic
# ------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id=None):
        self.gpu_id = gpu_id
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100"]
            if self.gpu_id:
                cmd += ["-i", self.gpu_id]
            self.proc = subprocess.Popen(cmd, stdout=self.file, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.file.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.file.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def bf16_peak():
    """(TFLOP/s, kind): the measured cuBLAS BF16 burst peak, else the fallback figure."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            v = float(json.load(f)["bf16_tflops"])
        return v, "measured"
    except (OSError, ValueError, KeyError):
        return 1900.0, "fallback"


def alu_add_peak(torch, dev):
    """FP32 adds per second derived from the unit counts and the clock: SMs x 128 FP32 lanes x the
    maximum SM clock (one add per lane per cycle; MEASURED_PEAKS.json's sm_max_mhz, else 2070 MHz)."""
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz, kind = float(json.load(f)["sm_max_mhz"]), "derived: SMs x 128 lanes x measured max SM clock"
    except (OSError, ValueError, KeyError):
        mhz, kind = 2070.0, "derived: SMs x 128 lanes x 2070 MHz (nominal)"
    return sms * 128 * mhz * 1e6, kind


def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def source_hash(paths):
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(key, paths):
    """DRAM bytes per launch from the committed ncu summary, or None if the kernel changed since."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f).get(key)
    except (OSError, ValueError):
        return None
    if not rec or rec.get("source_hash") != source_hash(paths):
        return None
    return rec.get("dram_bytes_per_launch")


# ------------------------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline and the reference arm)
# ------------------------------------------------------------------------------------------
def oracle_sample(rows, seed):
    """Time the FP64 oracle's sparse sign apply on `rows` rows of the workload (S drawn too)."""
    import torch
    import synthetic
    from oracle import sparse_sign as osk
    A = synthetic.colscaled_gaussian(rows, K_COLS, seed=seed, device="cpu", dtype=torch.float32).double().numpy()
    t0 = time.perf_counter()
    osk.apply(A, D_SKETCH, ZETA, seed)
    return time.perf_counter() - t0


def _oracle_block(args):
    """One worker's share of the all-core CPU baseline: the oracle's sketch of its own row block (the
    sketch is additive over row blocks, so the blocks are independent work)."""
    row0, rows, seed = args
    import numpy as np
    sys.path.insert(0, ROOT)
    from oracle import sparse_sign as osk
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((rows, K_COLS)) * np.logspace(-3, 0, K_COLS)[None, :]
    t0 = time.perf_counter()
    osk.apply_block(A, row0, D_SKETCH, ZETA, seed)
    return time.perf_counter() - t0


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


def cpu_extras():
    """Oracle timings of the other workloads on a bounded sample (single thread)."""
    import numpy as np
    from oracle import srtt as osr
    from oracle import lsq as olsq
    out = {}
    rng = np.random.default_rng(5)
    n = 1 << 17
    A = rng.standard_normal((n, K_COLS))
    t0 = time.perf_counter()
    osr.apply(A, D_SKETCH, 3)
    t = time.perf_counter() - t0
    out["srtt"] = {"sample": f"{n} x {K_COLS} FP64 (of 2^22 rows), d={D_SKETCH}", "s": round(t, 3),
                   "gbs_bf16_equiv": round(n * K_COLS * 2 / t / 1e9, 4)}
    nl, kl = 1 << 15, 100
    Q, _ = np.linalg.qr(rng.standard_normal((nl, kl)))
    V, _ = np.linalg.qr(rng.standard_normal((kl, kl)))
    Al = (Q * np.logspace(0, -8, kl)) @ V.T
    bl = Al @ rng.standard_normal(kl) + 1e-6 * rng.standard_normal(nl)
    t0 = time.perf_counter()
    olsq.sketch_precond(Al, bl, 4 * kl, ZETA, 7)
    t = time.perf_counter() - t0
    out["lsq"] = {"sample": f"sketch-and-precondition (oracle: FP64 sketch, QR, LSQR refinement) on {nl} x {kl}, "
                            "kappa=1e8 (reduced from 2^20 x 500)", "s": round(t, 3), "solves_per_s": round(1 / t, 4)}
    import synthetic
    from oracle import rsvd as orsvd
    m_t, n_t, rank_t, r_t = RSVD_TWIN
    At = synthetic.lowrank_plus_noise(m_t, n_t, rank_t, seed=m_t + n_t, noise=1e-4, device="cpu").double().numpy()
    t0 = time.perf_counter()
    Q = orsvd.range_finder(At, r_t, RSVD_Q, ZETA, 5)
    t = time.perf_counter() - t0
    out["rsvd_twin"] = {"sample": f"range finder (Alg. 1 + {RSVD_Q} power iterations, FP64) on {m_t} x {n_t}, r={r_t}",
                        "s": round(t, 3), "oracle_spectral_error": orsvd.spectral_error(At, Q, iters=30, seed=1)}
    return out


def cpu_baseline(target_s=12.0, a_bytes=2):
    rows = 1 << 14
    t = oracle_sample(rows, 1)
    while t < target_s / 4 and rows < (1 << 20):
        rows *= 2
        t = oracle_sample(rows, 1)
    single = rows * K_COLS * a_bytes / t / 1e9
    cores = os.cpu_count() or 1
    # all cores: one spawned worker per core, each sketching its own block of `rows` rows
    import multiprocessing as mp
    per = max(1 << 12, rows // 2)
    try:
        with mp.get_context("spawn").Pool(cores) as pool:
            pool.map(_oracle_block, [(0, 1 << 10, 1)] * cores)  # start-up and imports outside the timing
            t0 = time.perf_counter()
            pool.map(_oracle_block, [(g * per, per, 100 + g) for g in range(cores)])
            tall = time.perf_counter() - t0
        allc = cores * per * K_COLS * a_bytes / tall / 1e9
    except (OSError, RuntimeError):
        allc, tall = None, None
    res = {"value": round(allc if allc else single, 4), "unit": "GB/s", "cores": cores if allc else 1, "kind": "oracle",
           "single_thread": round(single, 4), "cpu_model": cpu_model(), "nproc": cores,
           "sample": f"single thread: {rows} of {N_ROWS} rows x {K_COLS} cols in {t:.2f} s; all cores: {cores} spawned "
                     f"workers x {per} rows in {tall:.2f} s (FP64 oracle: Philox+Floyd draw of S, scipy CSR product); "
                     "GB/s counted in BF16 bytes of A" if tall else f"{rows} rows single thread"}
    try:
        res["other_workloads"] = cpu_extras()
    except Exception as e:  # the extras are context only
        res["other_workloads"] = {"error": str(e)[:200]}
    return res


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    budget = 150.0
    rows = 1 << 14
    t = oracle_sample(rows, 0)
    per_step = budget / max(1, args.steps + args.warmup)
    rows = int(max(1 << 12, min(1 << 21, rows * per_step / max(t, 1e-3))))
    for w in range(args.warmup):
        oracle_sample(rows, 100 + w)
    times = [oracle_sample(rows, 1000 + s) for s in range(args.steps)]
    ms = 1000.0 * sum(times) / len(times)
    gbs = rows * K_COLS * 2 / (ms / 1e3) / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": round(gbs, 4), "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(),
            "cpu_baseline": {"value": round(gbs, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
                             "sample": f"{rows} of {N_ROWS} rows per step, FP64 oracle"},
            "e2e": {"value": round(gbs, 4), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def workload_config(world=1):
    cfg = {"workload": "sparse sign embedding S*A: A 2^22 x 256 BF16 (N(0,1) x logspace(-3,0) column scales), "
                       "S SparseUniform d=2048, zeta=8, fresh seed per step",
           "n": N_ROWS, "k": K_COLS, "d": D_SKETCH, "zeta": ZETA, "a_dtype": "bf16", "accumulate": "f32",
           "l2": "inputs larger than L2 (A is 2.1 GB), no flush"}
    if world > 1:
        cfg["parallelism"] = (f"A split into {world} row blocks (one per GPU); partial sketches gathered over "
                              "NCCL and summed in rank order")
    return cfg


# ------------------------------------------------------------------------------------------
# our arm
# ------------------------------------------------------------------------------------------
def sketch_step(rsk, A, out, seed, row0, world):
    """One headline step: S*A on one GPU, or this rank's row block plus the rank-ordered sum."""
    if world == 1:
        return rsk.rsk_sparse_sign_apply(A, D_SKETCH, ZETA, seed, out=out)
    from paper_2508_21189_gb300 import sharded
    return sharded.sparse_sign_apply(A, row0, D_SKETCH, ZETA, seed)


def srtt_step(rsk, A, out, seed, row0, n_total, world):
    if world == 1:
        return rsk.rsk_srtt_apply(A, D_SKETCH, seed, out=out)
    from paper_2508_21189_gb300 import sharded
    return sharded.srtt_apply(A, row0, n_total, D_SKETCH, seed)


def time_steps(rsk, A, out, steps, seed0, torch, row0=0, world=1):
    """Device time per step (ms) of `steps` sketch steps bracketed by barrier + synchronize."""
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    ev0.record()
    for s in range(steps):
        sketch_step(rsk, A, out, seed0 + s, row0, world)
    ev1.record()
    torch.cuda.synchronize()
    barrier()
    return ev0.elapsed_time(ev1) / steps


def timed_calls(fn, reps, torch, dev, after_warmup=None):
    """Median device time (ms, max over ranks) of `reps` calls, one warm-up call first."""
    out = fn()
    if after_warmup:
        after_warmup()
    times = []
    for _ in range(reps):
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        barrier()
        ev0.record()
        out = fn()
        ev1.record()
        torch.cuda.synchronize()
        times.append(max_over_ranks(ev0.elapsed_time(ev1), device=dev))
    return statistics.median(times), out


def bench_lsq(rsk, synthetic, torch, dev, rank, world, reps, rows=LSQ_N):
    """Single least-squares workload (A = Q_U diag(logspace(0,-8)) V^T, 2^20 x 500 FP64, b = A x* +
    1e-6 noise, d = 2000, zeta = 8): the mixed form (A split once into FP32 pairs; double-float sketch
    and CG operator on FP32 units; FP64 residual refinement) against the plain FP64 form (FP64 sketch,
    FP64 CG), each to eta <= 1e-10."""
    A, b, _ = synthetic.lsq_problem(rows, LSQ_K, seed=31 + rank, cond_exp=8.0, noise=1e-6, device=dev)
    forms = {"mixed": ("f32x2", "f32x2"), "fp64": (torch.float64, torch.float64)}
    res = {}
    for name, (sk, inner) in forms.items():
        ms, (x, info) = timed_calls(lambda: rsk.rsk_lstsq_sketch_precond(A, b, LSQ_D, zeta=ZETA, seed=7,
                                                                           sketch_dtype=sk, inner_dtype=inner),
                                    reps, torch, dev)
        res[name] = {"solves_per_s": round(world * 1e3 / ms, 3), "ms_per_solve": round(ms, 3),
                     "backward_err": info["backward_err"], "refine_steps": info["refine_steps"],
                     "inner_iters": info["inner_iters"],
                     "sketch": str(sk).replace("torch.", ""), "inner": str(inner).replace("torch.", "")}
    del A, b
    torch.cuda.empty_cache()
    return {"workload": f"least squares A = Q_U diag(logspace(0,-8)) V^T {rows} x 500 FP64, b = A x* + 1e-6 N(0,1), "
                        "sparse sign d=2000 zeta=8, to eta <= 1e-10",
            "value": res["mixed"]["solves_per_s"], "unit": "solves/s",
            "speedup_vs_fp64": round(res["mixed"]["solves_per_s"] / res["fp64"]["solves_per_s"], 3),
            "mixed": res["mixed"], "fp64": res["fp64"]}


def bench_lsq_batched(rsk, synthetic, torch, dev, rank, world, reps, count=BATCH_COUNT):
    """512 uneven problems (n_i log-uniform [4096, 262144], k_i uniform [16, 256], Gaussian A_i x
    logspace(-6, 0) column scales, Gaussian b_i, d_i = 4 k_i, zeta = 8) in one batched call: FP32
    storage with FP32 sketch and inner CG against FP64 storage with FP64 sketch and inner CG, both
    with the FP64 QR of the sketch; `mixed_qr_f32` is the mixed form with the QR in FP32 (an option
    of the library, not the configured workload)."""
    ns, ks = synthetic.batched_sizes(count, seed=404 + rank)
    As32, As64, bs = [], [], []
    for i, (n, k) in enumerate(zip(ns, ks)):
        A, b = synthetic.batched_problem(n, k, seed=10_000 * (rank + 1) + i, device=dev, dtype=torch.float64)
        As64.append(A)
        As32.append(A.float())
        bs.append(b)
    res = {}
    forms = {"mixed": (As32, torch.float32, torch.float64), "fp64": (As64, torch.float64, torch.float64),
             "mixed_qr_f32": (As32, torch.float32, torch.float32)}
    for name, (As, dt, qdt) in forms.items():
        ms, (xs, infos) = timed_calls(lambda: rsk.rsk_lstsq_sketch_precond_batched(As, bs, zeta=ZETA, seed=9,
                                                                                     sketch_dtype=dt, inner_dtype=dt,
                                                                                     qr_dtype=qdt),
                                      reps, torch, dev, after_warmup=lambda: rsk.rsk_profile_enable(True))
        phases = {k: rsk.rsk_profile_read("batch_" + k)[0] / reps for k in ("sketch", "qr", "resid", "cg")}
        rsk.rsk_profile_enable(False)
        res[name] = {"solves_per_s": round(world * count * 1e3 / ms, 3), "ms_per_batch": round(ms, 3),
                     "phases_ms": {k: round(v, 3) for k, v in phases.items()},
                     "max_backward_err": max(f["backward_err"] for f in infos),
                     "max_refine_steps": max(f["refine_steps"] for f in infos)}
    rows = sum(ns)
    elems = sum(n * k for n, k in zip(ns, ks))
    del As32, As64, bs
    torch.cuda.empty_cache()
    return {"workload": f"{count} uneven least-squares problems, n_i log-uniform [4096, 262144], k_i uniform "
                        "[16, 256], A_i Gaussian x logspace(-6,0) column scales, d_i = 4 k_i, zeta=8, eta <= 1e-10",
            "total_rows": rows, "total_elements": elems,
            "value": res["mixed"]["solves_per_s"], "unit": "solves/s",
            "speedup_vs_fp64": round(res["mixed"]["solves_per_s"] / res["fp64"]["solves_per_s"], 3),
            "mixed": res["mixed"], "fp64": res["fp64"], "mixed_qr_f32": res["mixed_qr_f32"]}


def spectral_error_gpu(torch, A, U, iters=20, seed=3):
    """||A - U U^T A||_2 by the power method in FP64 on the GPU (plain torch: a measurement, not the
    library's path)."""
    g = torch.Generator(device=A.device)
    g.manual_seed(seed)
    Ad, Ud = A.double(), U.double()
    v = torch.randn(A.shape[1], generator=g, device=A.device, dtype=torch.float64)
    v /= v.norm()
    est = 0.0
    for _ in range(iters):
        y = Ad @ v
        y = y - Ud @ (Ud.T @ y)
        est = y.norm().item()
        v = Ad.T @ y
        v /= v.norm()
    del Ad, Ud
    return est


def bench_rsvd(rsk, synthetic, torch, dev, rank, world, reps, rows=RSVD_M, profiler_range=False):
    """RSVD of A 262144 x 8192 FP32 (rank-400 spectrum j^-2 plus 1e-4 noise), r = 300, q = 2, on this
    library's kernels: time per call, per-phase device time, the big BF16 products against the BF16
    and HBM rooflines, and the spectral error ||A - U U^T A||_2 at full size (FP64 power method) and on
    the reduced twin that the FP64 oracle also runs (its error is filled in from the CPU leg).
    profiler_range: open the CUDA profiler range (cudaProfilerStart/Stop) around the timed calls only."""
    A = synthetic.lowrank_plus_noise(rows, RSVD_N, RSVD_RANK, seed=2025 + rank, noise=1e-4, device=dev)

    def after_warmup():
        rsk.rsk_profile_enable(True)
        if profiler_range:
            torch.cuda.synchronize()
            torch.cuda.profiler.start()

    ms, (U, s, Vt) = timed_calls(lambda: rsk.rsk_rsvd(A, RSVD_R, power_iters=RSVD_Q, zeta=ZETA, seed=0),
                                 reps, torch, dev, after_warmup=after_warmup)
    if profiler_range:
        torch.cuda.profiler.stop()
    phases = {k: rsk.rsk_profile_read(k) for k in ("gemm", "gemm_split", "factor", "small_svd", "convert",
                                                   "sketch_generate")}
    rsk.rsk_profile_enable(False)
    calls = reps + 0  # the profile covers the timed calls only
    big = 2 + 2 * RSVD_Q                    # Y = A Omega, q x (Z = A^T Q, Y = A Z), Z = A^T Q
    flops = big * 2 * rows * RSVD_N * RSVD_R
    gemm_ms = phases["gemm"][0] / calls
    bf16, bf16_kind = bf16_peak()
    sustained = bf16_sustained()
    hbm, hbm_kind = hbm_peak()
    a_bf16_bytes = rows * RSVD_N * 2        # each big product streams the BF16 copy of A once
    err = spectral_error_gpu(torch, A, U)
    floor = 1e-4 * (math.sqrt(rows) + math.sqrt(RSVD_N))
    sg = s.cpu()
    del A, U, s, Vt
    torch.cuda.empty_cache()
    m_t, n_t, rank_t, r_t = RSVD_TWIN
    At = synthetic.lowrank_plus_noise(m_t, n_t, rank_t, seed=m_t + n_t, noise=1e-4, device="cpu").to(dev)
    Ut, _, _ = rsk.rsk_rsvd(At, r_t, power_iters=RSVD_Q, zeta=ZETA, seed=5)
    err_t = spectral_error_gpu(torch, At, Ut)
    del At, Ut
    torch.cuda.empty_cache()
    gemm_tf = flops / (gemm_ms / 1e3) / 1e12 if gemm_ms > 0 else None
    return {"workload": f"RSVD A {rows} x {RSVD_N} FP32 (rank-400 spectrum j^-2 + 1e-4 noise), r=300, q=2, "
                        "sparse sign Omega zeta=8",
            "value": round(world * 1e3 / ms, 3), "unit": "calls/s", "ms_per_call": round(ms, 3),
            "phases_ms_per_call": {k: round(v[0] / calls, 3) for k, v in phases.items()},
            "launches_per_call": {k: v[1] // max(1, calls) for k, v in phases.items()},
            "gemm_big_products": {"count": big, "flops_per_call": flops, "ms_per_call": round(gemm_ms, 3),
                                  "tflops": round(gemm_tf, 1) if gemm_tf else None,
                                  "frac_of_bf16_burst": round(gemm_tf / bf16, 4) if gemm_tf else None,
                                  "frac_of_bf16_sustained": round(gemm_tf / sustained, 4) if gemm_tf else None,
                                  "peak_kind": bf16_kind,
                                  "a_stream_gbs": round(big * a_bf16_bytes / (gemm_ms / 1e3) / 1e9, 1) if gemm_ms else None,
                                  "frac_of_hbm": round(big * a_bf16_bytes / (gemm_ms / 1e3) / 1e9 / hbm, 4)
                                  if gemm_ms else None, "hbm_kind": hbm_kind},
            "spectral_error": {"value": err, "method": "FP64 power method, 20 iterations, on the GPU",
                               "noise_floor": floor, "best_rank_r_noise_free": (RSVD_R + 1) ** -2.0,
                               "sigma_1": float(sg[0])},
            "twin": {"workload": f"A {m_t} x {n_t} (rank-{rank_t} j^-2 + 1e-4 noise), r={r_t}, q={RSVD_Q}, "
                                 "Omega seed 5 (the FP64 oracle's reduced twin)",
                     "spectral_error": err_t}}


def bf16_sustained():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops_sustained"])
    except (OSError, ValueError, KeyError):
        return 1700.0


def time_variants(rsk, A, out, steps, torch, dev):
    """SparseStack (Def. SparseStack) and SparseRTT (Def. SparseRTT, xi = ceil(1.5 ln d)) on the headline A."""
    a_bytes = A.numel() * A.element_size()
    res = {}
    for name, fn in (("sparse_stack", lambda s: rsk.rsk_sparse_stack_apply(A, D_SKETCH, ZETA, s, out=out)),
                     ("sparse_rtt", lambda s: rsk.rsk_sparse_rtt_apply(A, D_SKETCH, s, out=out))):
        for w in range(3):
            fn(w)
        rsk.rsk_profile_enable(True)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record()
        for st in range(steps):
            fn(50_000 + st)
        ev1.record()
        torch.cuda.synchronize()
        kid = "sketch_apply" if name == "sparse_stack" else "srtt_apply"
        ap = rsk.rsk_profile_read(kid)
        rsk.rsk_profile_enable(False)
        rsk.rsk_sync_status()
        ms = max_over_ranks(ev0.elapsed_time(ev1) / steps, device=dev)
        apply_ms = ap[0] / max(1, ap[1])
        res[name] = {"value": round(a_bytes / (ms / 1e3) / 1e9, 3), "unit": "GB/s", "ms_per_step": round(ms, 4),
                     "apply_ms": round(apply_ms, 4),
                     "apply_hbm_frac": round(a_bytes / (apply_ms / 1e3) / 1e9 / hbm_peak()[0], 4)}
    res["sparse_rtt"]["xi"] = rsk.rsk_sparse_rtt_default_xi(D_SKETCH)
    res["sparse_stack"]["workload"] = f"SparseStack d={D_SKETCH} zeta={ZETA} on A 2^22 x 256 BF16"
    res["sparse_rtt"]["workload"] = f"SparseRTT d={D_SKETCH} (WHT, xi=ceil(1.5 ln d)) on A 2^22 x 256 BF16"
    return res


def spectral_norm(apply, n, torch, dev, iters=30, seed=9):
    """||M||_2 of the operator x -> M x (M^T M by power iteration from a seeded start)."""
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    x = torch.randn(n, 1, generator=g, device=dev, dtype=torch.float64)
    lam = 0.0
    for _ in range(iters):
        y = apply(x)
        lam = float(torch.linalg.norm(y))
        x = y / max(lam, 1e-300)
    return math.sqrt(lam)


def bench_nystrom(rsk, torch, dev, reps, n=NYS_N):
    """Alg. 2 on a psd A = U diag(j^-1, j <= 1000) U^T + 1e-6 I (n x n FP32), k = 300, SparseStack zeta = 4."""
    g = torch.Generator(device=dev)
    g.manual_seed(77)
    U, _ = torch.linalg.qr(torch.randn(n, NYS_RANK, generator=g, device=dev, dtype=torch.float32))
    lam = 1.0 / torch.arange(1, NYS_RANK + 1, device=dev, dtype=torch.float32)
    A = (U * lam) @ U.T
    A.diagonal().add_(1e-6)
    A = 0.5 * (A + A.T)
    del U
    ms, (Un, ln) = timed_calls(lambda: rsk.rsk_nystrom_psd(A, NYS_K, zeta=4, seed=1), reps, torch, dev)
    A64 = None
    # ||A - U diag(l) U^T||_2 against the best rank-k error lambda_{k+1}
    Ud, ld = Un.double(), ln.double()

    def err_op(x):
        y = (A.double() @ x) - Ud @ (ld[:, None] * (Ud.T @ x))
        return (A.double() @ y) - Ud @ (ld[:, None] * (Ud.T @ y))
    err = spectral_norm(err_op, n, torch, dev, iters=20)
    best = 1.0 / (NYS_K + 1) + 1e-6
    del A, Un, ln, Ud, ld, A64
    torch.cuda.empty_cache()
    return {"workload": f"psd Nystrom (Alg. 2): A = U diag(j^-1, j<=1000) U^T + 1e-6 I, {n} x {n} FP32, k={NYS_K}, "
                        "SparseStack zeta=4",
            "value": round(1e3 / ms, 3), "unit": "calls/s", "ms_per_call": round(ms, 3),
            "spectral_error": err, "best_rank_k_error": best, "error_over_best": round(err / best, 4)}


def bench_gen_nystrom(rsk, torch, dev, reps, n=GEN_N, d=GEN_D):
    """Algs. 4 and 5 on A = U diag(0.95^j, j < 400) V^T + 1e-6 noise (n x d FP32), k = 200, p = 300,
    SparseStack zeta = 4 (a stand-in for the paper's 131072 x 40000 simulation snapshots, whose
    singular values decay fast; with a slow decay the Frobenius tail dominates every sketch's error)."""
    g = torch.Generator(device=dev)
    g.manual_seed(88)
    U = torch.randn(n, GEN_RANK, generator=g, device=dev) / math.sqrt(n)
    V = torch.randn(d, GEN_RANK, generator=g, device=dev) / math.sqrt(d)
    s = 0.95 ** torch.arange(GEN_RANK, device=dev, dtype=torch.float32)
    A = (U * s) @ V.T
    del U, V
    A.add_(torch.randn(n, d, generator=g, device=dev), alpha=1e-6 / math.sqrt(max(n, d)))
    k, p = GEN_K, 300
    res = {"workload": f"generalized Nystrom (Algs. 4, 5): A {n} x {d} FP32 = rank-{GEN_RANK} (0.95^j) + 1e-6 noise, "
                       f"k={k}, p={p}, SparseStack zeta=4",
           "a_bytes": A.numel() * 4}
    nA = spectral_norm(lambda x: A.T.double() @ (A.double() @ x), d, torch, dev, iters=15)
    for form in ("outer", "svd"):
        ms, out = timed_calls(lambda: rsk.rsk_gen_nystrom(A, k, p=p, zeta=4, seed=2, form=form), reps, torch, dev)
        if form == "outer":
            F, G, r = out
            L, R = F.double(), G.double()
        else:
            Uo, so, Vo, r = out
            L, R = Uo.double() * so.double(), Vo.double()

        def op(x):
            y = A.double() @ x - L @ (R.T @ x)
            return A.T.double() @ y - R @ (L.T @ y)
        err = spectral_norm(op, d, torch, dev, iters=15)
        res[form] = {"ms_per_call": round(ms, 3), "calls_per_s": round(1e3 / ms, 3), "numerical_rank": r,
                     "relative_spectral_error": err / nA,
                     "sketch_pass_gbs": round(2 * res["a_bytes"] / (ms / 1e3) / 1e9, 1)}
        del out, L, R
    res["value"] = res["svd"]["calls_per_s"]
    res["unit"] = "calls/s"
    res["best_rank_k_relative_error"] = 0.95 ** k
    del A
    torch.cuda.empty_cache()
    return res


def bench_osi(rsk, torch, rs=OSI_R):
    """Fig. 2's estimates for SparseStack zeta = 8, k = 2r, Q = [e_1 ... e_r] (300 Lanczos steps)."""
    out = []
    for r in rs:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        a, b = rsk.rsk_osi_estimate(r, zeta=8, seed=1, kind="stack", iters=300)
        torch.cuda.synchronize()
        out.append({"r": r, "alpha": round(a, 5), "beta": round(b, 5), "s": round(time.perf_counter() - t0, 3)})
    return {"workload": "injectivity alpha / dilation beta of SparseStack zeta=8, k=2r, Q=[e_1..e_r], 300 Lanczos "
                        "steps", "gaussian_asymptotes": [round((1 - 2 ** -0.5) ** 2, 5), round((1 + 2 ** -0.5) ** 2, 5)],
            "estimates": out}


def run_ours(args):
    import torch
    rank, world = dist_init("nccl")
    _, _, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_2508_21189_gb300 as rsk
    import synthetic

    props = torch.cuda.get_device_properties(dev)
    uuid = getattr(props, "uuid", None)
    sampler = ClockSampler(f"GPU-{uuid}" if uuid else None)

    result = {}
    names = [x for x in args.dtypes.split(",") if x]
    dts = {"bf16": torch.bfloat16, "fp32": torch.float32, "fp64": torch.float64}
    head = names[0]
    sampler.start()
    from paper_2508_21189_gb300.sharded import row_partition
    # rows of this rank: the whole A on one GPU; a row block of it (2048-row aligned, so the SRTT
    # can use the same blocks) on several
    row0, n_local = row_partition(args.rows, world, 2048)[rank]
    tuned = {}
    for name in names:
        dt = dts[name]
        A = synthetic.colscaled_gaussian(n_local, K_COLS, seed=2022 + rank, device=dev, dtype=dt)
        out = torch.empty(D_SKETCH, K_COLS, device=dev, dtype=torch.float32)
        a_bytes = args.rows * K_COLS * A.element_size()  # the whole A, over all ranks
        if not args.no_autotune:
            # launch parameters of this shape chosen by timing candidates (outside the timed region)
            tuned[name] = {"sketch_row_ranges": rsk.rsk_autotune_sketch(0, A.dtype, n_local, K_COLS, D_SKETCH, ZETA),
                           "srtt_bands": (rsk.rsk_autotune_sketch(1, A.dtype, n_local, K_COLS, D_SKETCH, ZETA)
                                          if not args.no_srtt else None)}
        for w in range(args.warmup):
            sketch_step(rsk, A, out, w, row0, world)
        rsk.rsk_sync_status()
        rsk.rsk_profile_enable(True)
        ms_local = time_steps(rsk, A, out, args.steps, 10_000, torch, row0, world)
        prof = {k: rsk.rsk_profile_read(k) for k in ("sketch_index", "sketch_apply", "sketch_reduce")}
        rsk.rsk_profile_enable(False)
        rsk.rsk_sync_status()
        ms = max_over_ranks(ms_local, device=dev)
        apply_ms = prof["sketch_apply"][0] / max(1, prof["sketch_apply"][1])
        launches = sum(c for _, c in prof.values())
        r = {"ms_per_step": ms, "value": a_bytes / (ms / 1e3) / 1e9, "a_bytes": a_bytes,
             "local_bytes": A.numel() * A.element_size(),
             "apply_ms": apply_ms, "index_ms": prof["sketch_index"][0] / max(1, prof["sketch_index"][1]),
             "reduce_ms": prof["sketch_reduce"][0] / max(1, prof["sketch_reduce"][1]), "launches": launches}
        if not args.no_srtt:
            for w in range(args.warmup):
                srtt_step(rsk, A, out, w, row0, args.rows, world)
            rsk.rsk_profile_enable(True)
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            barrier()
            ev0.record()
            for st in range(args.steps):
                srtt_step(rsk, A, out, 30_000 + st, row0, args.rows, world)
            ev1.record()
            torch.cuda.synchronize()
            sp = {k: rsk.rsk_profile_read(k) for k in ("srtt_apply", "srtt_reduce", "dense")}
            rsk.rsk_profile_enable(False)
            rsk.rsk_sync_status()
            sms = max_over_ranks(ev0.elapsed_time(ev1) / args.steps, device=dev)
            r["srtt"] = {"ms_per_step": sms, "value": a_bytes / (sms / 1e3) / 1e9,
                         "apply_ms": sp["srtt_apply"][0] / max(1, sp["srtt_apply"][1]),
                         "draw_ms": sp["dense"][0] / max(1, sp["dense"][1]),
                         "launches": sum(c for _, c in sp.values())}
        if name == head and not args.no_e2e and world > 1:
            # end to end at N GPUs: every rank copies its row block from pinned host memory, the
            # sharded sketch runs, and the result is read back to the host
            A_host = A.cpu().pin_memory()
            out_host = torch.empty(D_SKETCH, K_COLS, dtype=torch.float32).pin_memory()
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            barrier()
            ev0.record()
            for s in range(args.steps):
                A.copy_(A_host, non_blocking=True)
                out_host.copy_(sketch_step(rsk, A, out, 20_000 + s, row0, world), non_blocking=True)
            ev1.record()
            torch.cuda.synchronize()
            e2e_ms = max_over_ranks(ev0.elapsed_time(ev1) / args.steps, device=dev)
            r["e2e"] = {"value": round(a_bytes / (e2e_ms / 1e3) / 1e9, 3), "unit": "GB/s",
                        "h2d_bytes_per_step": r["local_bytes"], "d2h_bytes_per_step": out.numel() * 4,
                        "ms_per_step": round(e2e_ms, 4)}
            del A_host
        elif name == head and not args.no_e2e:
            # end to end through the public host-input call: A in pinned host memory streams to the
            # device in row blocks while earlier blocks are sketched; SA is read back to the host
            A_host = A.cpu().pin_memory()
            out_host = torch.empty(D_SKETCH, K_COLS, dtype=torch.float32).pin_memory()
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            rsk.rsk_sparse_sign_apply_host(A_host, D_SKETCH, ZETA, 1, out=out)
            out_host.copy_(out, non_blocking=True)
            torch.cuda.synchronize()
            barrier()
            ev0.record()
            for s in range(args.steps):
                rsk.rsk_sparse_sign_apply_host(A_host, D_SKETCH, ZETA, 20_000 + s, out=out)
                out_host.copy_(out, non_blocking=True)
            ev1.record()
            torch.cuda.synchronize()
            e2e_ms = max_over_ranks(ev0.elapsed_time(ev1) / args.steps, device=dev)
            # the floor: a plain copy of the same pinned bytes to the device (no sketch)
            copies = 3
            ev0.record()
            for _ in range(copies):
                A.copy_(A_host, non_blocking=True)
            ev1.record()
            torch.cuda.synchronize()
            copy_ms = ev0.elapsed_time(ev1) / copies
            r["e2e"] = {"value": round(a_bytes / (e2e_ms / 1e3) / 1e9, 3), "unit": "GB/s",
                        "h2d_bytes_per_step": a_bytes, "d2h_bytes_per_step": out.numel() * 4,
                        "ms_per_step": round(e2e_ms, 4),
                        "h2d_copy_gbs": round(a_bytes / (copy_ms / 1e3) / 1e9, 3)}
            del A_host
        if name == head and not args.no_variants and world == 1:
            r["variants"] = time_variants(rsk, A, out, args.steps, torch, dev)
        result[name] = r
        del A
        torch.cuda.empty_cache()
    clocks = sampler.stop()
    extra = {}
    if tuned:
        extra["autotune"] = {"chosen": tuned, "note": "0 = the default rule was fastest"}
    if not args.no_nystrom and world == 1:
        extra["nystrom_psd"] = bench_nystrom(rsk, torch, dev, args.solve_reps, n=args.nystrom_n)
        extra["gen_nystrom"] = bench_gen_nystrom(rsk, torch, dev, args.solve_reps, n=args.gen_rows, d=args.gen_cols)
    if not args.no_osi and world == 1:
        extra["osi"] = bench_osi(rsk, torch)
    if not args.no_lsq:
        extra["lsq"] = bench_lsq(rsk, synthetic, torch, dev, rank, world, args.solve_reps, args.lsq_rows)
        extra["lsq_batched"] = bench_lsq_batched(rsk, synthetic, torch, dev, rank, world, args.solve_reps,
                                                 args.batch_count)
    if not args.no_rsvd:
        extra["rsvd"] = bench_rsvd(rsk, synthetic, torch, dev, rank, world, args.solve_reps, rows=args.rsvd_rows,
                                   profiler_range=args.profile_rsvd)

    if rank != 0:
        return
    peak, peak_kind = hbm_peak()
    main = result[head]
    alg_bytes = main["local_bytes"] + D_SKETCH * K_COLS * 4  # one launch reads this rank's rows
    achieved = alg_bytes / (main["apply_ms"] / 1e3) / 1e9
    line = {
        "metric": METRIC, "value": round(main["value"], 3), "unit": "GB/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(main["ms_per_step"], 4),
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "config": workload_config(world),
        "hbm_frac_of_step": round(main["value"] / world / peak, 4),
        "roofline": {"kernel": "k_apply (sparse sign gather)", "bound": "hbm", "achieved": round(achieved, 2),
                     "peak": peak, "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
                     "traffic": recorded_traffic("k_apply|bf16|n=4194304,k=256,d=2048,zeta=8", APPLY_SOURCES),
                     "algorithmic_bytes_per_launch": alg_bytes, "avg_launch_ms": round(main["apply_ms"], 4)},
        "e2e": main.get("e2e"),
        "gpu_launches": main["launches"],
        "kernel_ms": {"index": round(main["index_ms"], 4), "apply": round(main["apply_ms"], 4),
                      "reduce": round(main["reduce_ms"], 4)},
        "clocks": clocks,
    }
    alu_peak, alu_kind = alu_add_peak(torch, dev)
    for name in names:
        r = result[name]
        if "srtt" in r:
            sr = r["srtt"]
            key = "srtt" if name == head else f"srtt_{name}"
            # ~12 FP32 adds per element: 11 butterfly stages of the 2048-point transform + the gather
            adds = 12.0 * r["local_bytes"] / (2 if name == "bf16" else 4)
            line[key] = {"value": round(sr["value"], 3), "unit": "GB/s", "ms_per_step": round(sr["ms_per_step"], 4),
                         "apply_ms": round(sr["apply_ms"], 4), "draw_ms": round(sr["draw_ms"], 4),
                         "apply_hbm_frac": round(r["local_bytes"] / (sr["apply_ms"] / 1e3) / 1e9 / peak, 4),
                         "alu": {"adds_per_launch": adds, "achieved_tadds_per_s": round(adds / (sr["apply_ms"] / 1e3) / 1e12, 3),
                                 "peak_tadds_per_s": round(alu_peak / 1e12, 2), "peak_kind": alu_kind,
                                 "frac": round(adds / (sr["apply_ms"] / 1e3) / alu_peak, 4)},
                         "workload": f"SRTT d={D_SKETCH} (WHT, n=2^22), A {name}"}
    for name in names[1:]:
        r = result[name]
        line[name] = {"value": round(r["value"], 3), "unit": "GB/s", "ms_per_step": round(r["ms_per_step"], 4),
                      "apply_ms": round(r["apply_ms"], 4),
                      "apply_frac": round((r["local_bytes"] + D_SKETCH * K_COLS * 4) / (r["apply_ms"] / 1e3) / 1e9
                                          / peak, 4)}
    if "variants" in main:
        line.update(main["variants"])
    line.update(extra)
    if args.rows != N_ROWS:
        line["config"]["n"] = args.rows
        line["config"]["workload"] += f" (reduced to {args.rows} rows for profiling)"
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
        twin = line["cpu_baseline"].get("other_workloads", {}).get("rsvd_twin")
        if twin and "rsvd" in line:
            e_o = twin["oracle_spectral_error"]
            line["rsvd"]["twin"]["oracle_spectral_error"] = e_o
            line["rsvd"]["twin"]["ratio_to_oracle"] = round(line["rsvd"]["twin"]["spectral_error"] / e_o, 4)
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
