#!/usr/bin/env python3
"""Benchmark: randomized H^1 compression with graph-coloured test matrices.

Workload: 200,000 points uniform in parameter space on a torus (R = 1,
rho = 0.3), kernel 1/(4 pi |x - y|) with zero diagonal evaluated on the fly,
adaptive octree with leaves of at most 64 points, relative truncation
tolerance 1e-6 (r = 32 columns per colour, oversampling 10), black-box
contraction in split-BF16 on the tensor cores; peel products in double-float
with the subtraction in FP64; pivoted QR, Gram products and core solves in
FP64 (the default precision; --precision mixed-f32 and fp64 select the others).

One step = the whole hot path on resident inputs: cluster tree and lists,
colouring of every level, test matrices, black-box products, peeling, bases,
cores, leaf blocks, and one apply of the compressed operator to a vector.
value = jobs/s over all GPUs (each GPU compresses its own replica: weak
scaling, no collective in the data path).  The e2e number adds the host->device
copy of the points and of the apply vector and the device->host read of the
result, from pinned host memory.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time-to-compress (s) and jobs/s at stated rel. error; p50/p99 latency"

# precision modes: (hm_precision value, description, dtype key of the JSON line)
FORMATS = {"h1": 0, "uniform_h1": 1, "h2": 2}
PRECISIONS = {
    "mixed": (1, "split-BF16x6 tensor-core black box; double-float (2 x FP32) peel products with the "
                 "subtraction in FP64; FP64 pivoted QR, Gram products and core solves", "bf16x6-f32acc+df64+f64"),
    "mixed-f32": (2, "split-BF16x6 tensor-core black box; FP32 peel products, QR and core solves; "
                     "FP64 samples, factors and subtractions", "bf16x6-f32acc+f32+f64"),
    "fp64": (0, "FP64 throughout", "f64"),
}
# FP32 pipe of the GB300 (152 SMs x 128 lanes at the 2070 MHz maximum SM clock),
# and the FP32 instructions of one double-float multiply-add (csrc/df.cuh)
FP32_INSTR_PER_S = 152 * 128 * 2070e6
DF_INSTR_PER_MAC = 12
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}

# dram bytes (read + write) of the tensor-core contraction kernel per evaluated
# kernel entry, from the ncu capture summarised in profiles/ (scaled by the
# entries a step evaluates); valid only for the source whose sha256 prefix
# (full-line comments excluded, see source_sha) is recorded here
TRAFFIC = {"file": "paper_2205_03406_gb300/csrc/sample_tc.cu", "sha256": "599b47112ea36534", "bytes_per_eval": 0.5954}
# DRAM bytes per double-float multiply-add of k_peel_gemm_df from one ncu capture
# (profiles/), valid while the kernel's source is unchanged
TRAFFIC_DF = {"file": "paper_2205_03406_gb300/csrc/peel_mixed.cu", "sha256": "4b23cb547b30be69", "bytes_per_mac": 0.1502}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=200_000)
    ap.add_argument("--precision", choices=list(PRECISIONS), default="mixed")
    ap.add_argument("--peaks", action="store_true",
                    help="only measure cuBLAS DGEMM and SGEMM (no TF32) rates on this GPU and print them")
    ap.add_argument("--no-modes", action="store_true",
                    help="skip timing the other two precision modes beside the main line")
    ap.add_argument("--format", choices=list(FORMATS), default="h1",
                    help="format of the main line's operator (Algorithm 4.1, Section 4.2 or Section 4.3)")
    ap.add_argument("--r", type=int, default=0, help="sample columns of the main line (0: the workload's, 32)")
    ap.add_argument("--no-formats", action="store_true",
                    help="skip timing the uniform H^1 and H^2 formats of the same job")
    ap.add_argument("--formats-r", type=int, default=48, help="r of the uniform H^1 and H^2 measurements")
    ap.add_argument("--relerr-iters", type=int, default=20)
    ap.add_argument("--no-relerr", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--serving-jobs", type=int, default=48,
                    help="jobs of the serving measurement (the streamed-jobs configuration has 256)")
    ap.add_argument("--serving-matvecs", type=int, default=100,
                    help="matvecs per job in the serving measurement (the configuration has 1000)")
    ap.add_argument("--serving-slots", type=int, default=4)
    ap.add_argument("--sweep", action="store_true",
                    help="only the large precision sweep: a jittered Fibonacci sphere of --sweep-n points, "
                         "K = 1/|x-y|, leaf 64, tol --sweep-tol, r --sweep-r, in the three precision modes; "
                         "one JSON line")
    ap.add_argument("--sweep-n", type=int, default=1 << 20)  # 2^19 fits every mode's peel tables
    ap.add_argument("--sweep-tol", type=float, default=1e-4)
    ap.add_argument("--sweep-r", type=int, default=32)
    ap.add_argument("--sweep-modes", type=str, default="fp64,mixed,mixed-f32",
                    help="comma-separated precision modes of the sweep, in order (fp64 first: the reference)")
    ap.add_argument("--oracle-series", type=str, default=None,
                    help="comma-separated torus sizes: time the full CPU oracle compression at each (and the "
                         "2048-point 1D dense configuration, best of 3), print one JSON line, exit")
    return ap.parse_args()


def workload(n):
    import hm_workloads as W
    return W.torus_laplace(n=n, tol=1e-6, r=32)


def config_of(args, w):
    return {"workload": f"torus_laplace_{w.n}", "n": w.n, "geometry": "torus R=1 rho=0.3, uniform (u,v)",
            "kernel": "1/(4 pi |x-y|), zero diagonal, on the fly", "leaf_size": w.leaf_size, "tol": w.tol,
            "r": w.r, "oversample": w.oversample, "format": getattr(args, "format", "h1"),
            "precision": PRECISIONS[args.precision][1],
            "l2": "working set larger than L2 (samples ~5 GB per level); no flush", "seed": w.seed}


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------

class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        sms, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sms.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for name, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.f.name)
        sms.sort()
        med = sms[len(sms) // 2] if sms else None
        return {"sm_mhz": med, "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sms)}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p, "measured"
    except (OSError, ValueError):
        return PEAKS_FALLBACK, "fallback"


def source_sha(path: str) -> str:
    """sha256 prefix of a source file without its full-line // comments (a
    comment edit does not change the compiled kernel the counters describe)."""
    with open(path, "rb") as f:
        lines = [ln for ln in f.read().decode().splitlines() if not ln.strip().startswith("//")]
    return hashlib.sha256("\n".join(ln.rstrip() for ln in lines).encode()).hexdigest()[:16]


def roofline_tc(info, r: int):
    """Tensor-core contraction: every evaluated kernel entry (a row of a colour's
    sample tiles x one of its active rows) feeds r Y and r Z outputs, 4 r useful
    flops, executed as 6 BF16 products each."""
    useful = 4.0 * r * info.tc_kernel_evals
    t = info.seconds_phase[7]
    launches = sum(1 for l in range(2, info.L + 1) if info.colors[l] > 0)  # one k_sample_tc per level
    pk, src = peaks()
    bf16_flops = 6.0 * useful
    achieved = bf16_flops / t / 1e12 if t > 0 else 0.0
    peak = float(pk["bf16_tflops_sustained"])
    traffic = None
    try:
        src_path = os.path.join(ROOT, TRAFFIC["file"])
        sha = source_sha(src_path)
        if TRAFFIC["sha256"] == sha and TRAFFIC["bytes_per_eval"]:
            traffic = round(TRAFFIC["bytes_per_eval"] * info.tc_kernel_evals / max(launches, 1))
    except OSError:
        pass
    return {"kernel": "k_sample_tc (split-BF16 kernel-matrix x Omega contraction)", "bound": "tensor",
            "achieved": round(achieved, 2), "peak": peak, "unit": "TFLOP/s",
            "frac": round(achieved / peak, 4), "peak_source": f"{src} bf16_tflops_sustained",
            "traffic": traffic, "traffic_unit": "dram bytes per launch (ncu, scaled by evaluated entries)",
            "launches_per_step": launches, "seconds": round(t, 4), "bf16_flops": bf16_flops,
            "useful_fp64_equiv_flops": useful}


def roofline_df(info):
    """Double-float peel update: every multiply-add is 12 FP32 instructions, so
    the kernel is bound by the FP32 pipe's issue rate; achieved and peak are in
    FP64-equivalent flops (2 per multiply-add)."""
    t = info.seconds_peel_update
    flops = 2.0 * info.peel_update_macs
    launches = int(sum(1 for l in range(3, info.L + 1) if info.colors[l] > 0) * 2 +
                   (1 if info.colors[info.L + 1] > 0 else 0))
    traffic = None
    try:
        if TRAFFIC_DF["bytes_per_mac"] and TRAFFIC_DF["sha256"] == source_sha(os.path.join(ROOT, TRAFFIC_DF["file"])):
            traffic = round(TRAFFIC_DF["bytes_per_mac"] * info.peel_update_macs / max(launches, 1))
    except OSError:
        traffic = None
    peak = 2.0 * FP32_INSTR_PER_S / DF_INSTR_PER_MAC / 1e12
    achieved = flops / t / 1e12 if t > 0 else 0.0
    return {"kernel": "k_peel_gemm_df (double-float peel update)", "bound": "alu",
            "achieved": round(achieved, 3), "peak": round(peak, 3), "unit": "TFLOP/s (FP64-equivalent)",
            "frac": round(achieved / peak, 4),
            "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2070 MHz / 12 instructions per double-float "
                           "multiply-add x 2 flops",
            "traffic": traffic, "traffic_unit": "dram bytes per launch (ncu, scaled by multiply-adds)",
            "seconds": round(t, 4), "macs": int(info.peel_update_macs), "launches_per_step": launches}


def measure_peaks():
    """cuBLAS DGEMM (float64) and SGEMM (float32, TF32 off) rates on this GPU,
    best of 3 after a warm-up, by CUDA events."""
    import torch
    torch.backends.cuda.matmul.allow_tf32 = False
    out = {}
    for name, dt, n in (("fp64_dgemm_tflops", torch.float64, 4096), ("fp32_sgemm_tflops", torch.float32, 8192)):
        a = torch.randn(n, n, dtype=dt, device="cuda")
        b = torch.randn(n, n, dtype=dt, device="cuda")
        a @ b
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            a @ b
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1) / 1e3)
        out[name] = round(2.0 * n ** 3 / best / 1e12, 3)
    return out


def max_over_ranks(x: float, dist, device) -> float:
    """The job's time: the slowest rank's (all-reduce MAX); x itself on one rank."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, steps: int, tmax: float) -> float:
    """Whole-job jobs/s: every rank compresses its own job each step (weak scaling)."""
    return world * steps / tmax


def rank_seed(base: int, rank: int) -> int:
    """Each rank's job is an independent replica with its own test matrices."""
    return base + rank


def time_mode(hm, w, pts, op, precision: int, rank: int, steps: int, relerr_iters, fmt: int = 0, warm: bool = True):
    """Time-to-compress (CUDA events, after one warm-up job), relative error and
    storage of the same job in another precision mode or format."""
    import torch
    s = hm.Settings(d=3, leaf_size=w.leaf_size, r=w.r, oversample=w.oversample, tol=w.tol, precision=precision,
                    seed=rank_seed(w.seed, rank), format=fmt)
    comp = hm.Compressor(s, torch.cuda.current_stream())
    if warm:
        comp.tree_build(pts)
        comp.compress(op)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        comp.tree_build(pts)
        comp.compress(op)
    e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3 / steps
    info = comp.info()
    out = {"time_to_compress_s": round(t, 4), "steps": steps,
           "rel_error": None if relerr_iters is None else comp.relerr(op, relerr_iters),
           "floats_per_dof": round(info.factor_floats / w.n, 1), "max_rank": info.max_rank,
           "matvec_cols": info.matvec_cols,
           "phases_s": {n: round(info.seconds_phase[i], 4) for i, n in enumerate(hm.PHASES)}}
    comp.close()
    return out


def run_serving(hm, args):
    """A stream of compression jobs (N log-uniform in [4k, 64k]; 2D curves with
    log|x-y|, the torus with 1/|x-y| and exp(-|x-y|); tol 1e-6, spec precision)
    through hm_server: Poisson arrivals at 1.2 times the single-stream capacity
    (measured first on three jobs compressed one at a time), admission by
    device-memory footprint, and a client thread that serves matvecs on every
    job as soon as it is ready, while later jobs still compress."""
    import threading

    import numpy as np
    import torch

    import hm_workloads as W
    jobs = W.serving_jobs(args.serving_jobs, n_min=4096, n_max=65536)
    prec = PRECISIONS["mixed"][0]

    def settings(w):
        return hm.Settings(d=w.d, leaf_size=w.leaf_size, r=w.r, oversample=w.oversample, tol=w.tol,
                           precision=prec, seed=w.seed)

    one = hm.Server(slots=1)
    t_single = []
    for w in jobs[:3]:
        st = one.wait(one.submit(w.points, settings(w), hm.kernel_op(w.kernel)), 600.0)
        t_single.append(st.t_done - st.t_start)
    one.close()
    rate = 1.2 / (sum(t_single) / len(t_single))
    gaps = np.random.default_rng(7).exponential(1.0 / rate, len(jobs))
    srv = hm.Server(slots=args.serving_slots)
    ids = [None] * len(jobs)
    ready = threading.Semaphore(0)
    errors = []

    def client():
        try:
            for k, w in enumerate(jobs):
                ready.acquire()
                srv.wait(ids[k], 600.0)
                xs = [torch.from_numpy(np.random.default_rng(k * 10 + i).standard_normal(w.n)).cuda()
                      for i in range(2)]
                for i in range(args.serving_matvecs):
                    srv.apply(ids[k], xs[i % 2])
                srv.release(ids[k])
        except Exception as e:  # reported in the line
            errors.append(repr(e))

    th = threading.Thread(target=client)
    t0 = time.perf_counter()
    th.start()
    nxt = t0
    for k, w in enumerate(jobs):
        nxt += gaps[k]
        dt = nxt - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        ids[k] = srv.submit(w.points, settings(w), hm.kernel_op(w.kernel))
        ready.release()
    th.join()
    wall = time.perf_counter() - t0
    info = srv.info()
    srv.close()
    return {"jobs": len(jobs), "matvecs_per_job": args.serving_matvecs, "slots": args.serving_slots,
            "arrival_rate_jobs_per_s": round(rate, 3), "single_stream_s_per_job": round(sum(t_single) / 3, 4),
            "jobs_per_s": round(info.jobs_per_s, 3), "job_p50_s": round(info.job_p50_s, 4),
            "job_p99_s": round(info.job_p99_s, 4), "apply_p50_s": round(info.apply_p50_s, 6),
            "apply_p99_s": round(info.apply_p99_s, 6), "applies": int(info.applies),
            "max_running": int(info.max_running), "max_reserved_bytes": int(info.max_reserved),
            "budget_bytes": int(info.budget), "completed": int(info.completed), "failed": int(info.failed),
            "wall_s": round(wall, 2), "errors": errors,
            "workload": "N log-uniform in [4096, 65536]; 2D curve r=1+0.3cos(5t) with log|x-y|, torus with "
                        "1/|x-y| and exp(-|x-y|); tol 1e-6, r 32; Poisson arrivals"}


def run_ours(args):
    import numpy as np
    import torch

    import paper_2205_03406_gb300 as hm

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    w = workload(args.n)
    if args.r:
        import dataclasses
        w = dataclasses.replace(w, r=args.r)
    prec = PRECISIONS[args.precision][0]
    s = hm.Settings(d=3, leaf_size=w.leaf_size, r=w.r, oversample=w.oversample, tol=w.tol, precision=prec,
                    seed=rank_seed(w.seed, rank), format=FORMATS[args.format])
    stream = torch.cuda.current_stream()
    comp = hm.Compressor(s, stream)
    op = hm.kernel_op(w.kernel)
    pts = torch.from_numpy(w.points).cuda()
    x = torch.from_numpy(np.random.default_rng(rank).standard_normal(w.n)).cuda()

    def step():
        comp.tree_build(pts)
        comp.compress(op)
        return comp.apply(x)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier()
    launches0 = comp.info().launches_total
    clocks = Clocks(local)
    clocks.start()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    evs[0].record(stream)
    infos = []
    for k in range(args.steps):
        step()
        evs[k + 1].record(stream)
        infos.append(comp.info())
    torch.cuda.synchronize()
    elapsed_host = time.perf_counter() - t0
    barrier()
    clk = clocks.stop()
    launches = comp.info().launches_total - launches0
    per_step = [evs[k].elapsed_time(evs[k + 1]) / 1e3 for k in range(args.steps)]
    elapsed = evs[0].elapsed_time(evs[-1]) / 1e3
    tmax = max_over_ranks(elapsed, dist, "cuda")
    info = infos[-1]

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        hp = torch.from_numpy(w.points).pin_memory()
        hx = torch.from_numpy(np.random.default_rng(rank).standard_normal(w.n)).pin_memory()
        hy = torch.empty(w.n, dtype=torch.float64).pin_memory()
        dp = torch.empty_like(hp, device="cuda")
        dx = torch.empty_like(hx, device="cuda")
        torch.cuda.synchronize()
        barrier()
        t1 = time.perf_counter()
        for _ in range(args.steps):
            dp.copy_(hp, non_blocking=True)
            comp.tree_build(dp)
            comp.compress(op)
            dx.copy_(hx, non_blocking=True)
            y = comp.apply(dx)
            hy.copy_(y, non_blocking=True)
            torch.cuda.synchronize()
        te = max_over_ranks(time.perf_counter() - t1, dist, "cuda")
        e2e = {"value": round(job_throughput(world, args.steps, te), 4), "unit": "jobs/s",
               "h2d_bytes_per_step": int(hp.numel() * 8 + hx.numel() * 8),
               "d2h_bytes_per_step": int(hy.numel() * 8), "time_to_compress_s": round(te / args.steps, 4)}

    # the apply of the compressed operator alone (one right-hand side): every
    # stored factor entry (U, V, B and the leaf blocks) is read once
    apply_line = None
    if rank == 0:
        xs = [torch.from_numpy(np.random.default_rng(100 + k).standard_normal(w.n)).cuda() for k in range(2)]
        for k in range(3):
            comp.apply(xs[k % 2])
        torch.cuda.synchronize()
        reps = 20
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for k in range(reps):
            comp.apply(xs[k % 2])
        a1.record(stream)
        torch.cuda.synchronize()
        ta = a0.elapsed_time(a1) / 1e3 / reps
        pk, src = peaks()
        nbytes = 8 * int(info.factor_floats) + 4 * 8 * w.n  # factors + x, y and their permuted copies
        gbs = nbytes / ta / 1e9
        apply_line = {"seconds": round(ta, 6), "bytes": nbytes, "achieved": round(gbs, 1),
                      "peak": float(pk["hbm_gbs"]), "unit": "GB/s", "frac": round(gbs / float(pk["hbm_gbs"]), 4),
                      "bound": "hbm", "peak_source": f"{src} hbm_gbs", "nrhs": 1,
                      "l2": "factors (several GB) far larger than L2"}

    relerr = None
    if not args.no_relerr and rank == 0:
        relerr = comp.relerr(hm.kernel_op(w.kernel), args.relerr_iters)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, rows_per_level=100)

    serving = None
    if rank == 0 and world == 1 and not args.no_serving:
        serving = run_serving(hm, args)

    # the other precision modes on the same job, for the error / time trade-off
    # (one GPU only: under torchrun every GPU would be held meanwhile)
    modes = None
    if rank == 0 and world == 1 and not args.no_modes:
        modes = {}
        for name, (pv, desc, _) in PRECISIONS.items():
            if name == args.precision:
                continue
            modes[name] = time_mode(hm, w, pts, op, pv, rank, steps=1 if pv == 0 else 3,
                                    relerr_iters=None if args.no_relerr else args.relerr_iters)
            modes[name]["precision"] = desc

    # the same points, kernel and tolerance compressed to the uniform H^1 (Section
    # 4.2) and H^2 (Section 4.3) formats in the bench's precision mode, with
    # r = --formats-r: one basis per box holds the box's whole far field, which
    # needs more sample columns than a per-block basis
    formats = None
    if rank == 0 and world == 1 and not args.no_formats:
        import dataclasses
        wf = dataclasses.replace(w, r=args.formats_r)
        formats = {"r": wf.r}
        for name, fv in (("uniform_h1", hm.HM_FORMAT_UNIFORM_H1), ("h2", hm.HM_FORMAT_H2)):
            formats[name] = time_mode(hm, wf, pts, op, PRECISIONS[args.precision][0], rank, steps=3,
                                      relerr_iters=None if args.no_relerr else args.relerr_iters, fmt=fv)

    if rank != 0:
        comp.close()
        if dist is not None:
            dist.destroy_process_group()
        return
    # the roofline of the kernel with the most device time in a step, the other beside it
    roof_tc = roofline_tc(info, w.r)
    roof_df = roofline_df(info) if info.seconds_peel_update > 0 else None
    if roof_df is not None and roof_df["seconds"] > roof_tc["seconds"]:
        roof_main, roof_second = roof_df, roof_tc
    else:
        roof_main, roof_second = roof_tc, roof_df
    per_step.sort()
    p50 = per_step[len(per_step) // 2]
    p99 = per_step[min(len(per_step) - 1, int(math.ceil(0.99 * len(per_step))) - 1)]
    phases = {n: round(info.seconds_phase[i], 4) for i, n in enumerate(hm.PHASES)}
    out = {
        "metric": METRIC, "value": round(job_throughput(world, args.steps, tmax), 4), "unit": "jobs/s",
        "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * tmax / args.steps, 2),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": PRECISIONS[args.precision][2],
        "data": "synthetic (seeded torus point cloud)",
        "config": dict(config_of(args, w), parallelism=f"replicas x{world}"),
        "time_to_compress_s": round(tmax / args.steps, 4),
        "p50_s": round(p50, 4), "p99_s": round(p99, 4),
        "rel_error": relerr, "rel_error_iters": None if relerr is None else args.relerr_iters,
        "matvec_cols": int(info.matvec_cols), "floats_per_dof": round(info.factor_floats / w.n, 1),
        "colors": [int(info.colors[l]) for l in range(2, info.L + 2)], "max_rank": int(info.max_rank),
        "phases_s": phases, "host_elapsed_s": round(elapsed_host, 3),
        "roofline": roof_main, "roofline_second": roof_second, "apply": apply_line,
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches), "clocks": clk, "serving": serving,
        "modes": modes,
        "formats": formats,
    }
    print(json.dumps(out), flush=True)
    comp.close()
    if dist is not None:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# CPU oracle: bounded sample of the same workload
# ---------------------------------------------------------------------------

class OracleSample:
    """The CPU oracle on a bounded sample of the 200k-point job.

    Setup times the oracle's full cluster tree and every colouring once.  A
    sample then times the oracle's black-box product A(rows, :) Omega_l and
    A(rows, :) Psi_l (same shape and zero pattern as Omega_l, so Omega_l stands
    for both) for `rows_per_level` random rows of every level and
    extrapolates to all rows.  Peel, QR, cores and leaf extraction are not
    timed, so the estimate is a lower bound on the oracle's time-to-compress."""

    def __init__(self, w):
        from oracle import graph as og
        from oracle import h1 as oh1
        from oracle import tree as ot
        self.w = w
        t0 = time.perf_counter()
        self.t = ot.build_tree(w.points, w.leaf_size)
        self.cols = {l: og.color_level(self.t, l) for l in range(2, self.t.L + 1)}
        og.color_leaf(self.t)
        self.t_struct = time.perf_counter() - t0
        self.op = oh1.KernelOp(w.points[self.t.perm], w.kernel)
        # Omega_l of every level; Psi_l has the same shape and zero pattern, so
        # the product with Omega_l is timed twice to stand for both sides
        self.mats = {}
        for l, col in self.cols.items():
            if col.n_vertices == 0:
                continue
            GO = oh1.gaussians(self.t, l, 0, w.r, w.seed)
            self.mats[l] = oh1.test_matrix(self.t, l, col, GO, w.r)

    def sample(self, rows_per_level: int, seed: int = 0):
        import numpy as np
        rng = np.random.default_rng(seed)
        n = self.w.n
        t_bb = 0.0
        for l, Om in self.mats.items():
            for side in range(2):
                rows = np.sort(rng.choice(n, rows_per_level, replace=False))
                t1 = time.perf_counter()
                self.op.rows(rows, Om)
                t_bb += (time.perf_counter() - t1) * (n / rows_per_level)
        est = self.t_struct + t_bb
        cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
        return {"value": float(f"{1.0 / est:.4g}"), "unit": "jobs/s", "cores": cores, "kind": "oracle",
                "sample": f"oracle tree + all colourings timed in full ({self.t_struct:.1f} s); black-box "
                          f"product for {rows_per_level} random rows of each level ({len(self.mats)} levels), "
                          f"extrapolated to all {n} rows ({t_bb:.1f} s); peel/QR/cores/leaf not timed, so "
                          f"{est:.1f} s is a lower bound on the oracle's time-to-compress",
                "seconds_estimate": round(est, 2)}


def run_sweep(args):
    """The large precision configuration: time-to-compress, ranks and storage of
    one job per precision mode.  The FP64 operator is compressed first and kept;
    every other mode's error is measured against it, ||A_mode - A_fp64|| /
    ||A_fp64|| by 20 power iterations on the two compressed operators.  (An
    exact error against A would need N^2 FP64 kernel evaluations per product:
    about 25 s each at 2^20 points, 80 products for 20 iterations.)  One JSON
    line per finished mode, then a summary line."""
    import torch
    import hm_workloads as W
    import paper_2205_03406_gb300 as hm
    w = W.sphere_invr(n=args.sweep_n, tol=args.sweep_tol, r=args.sweep_r)
    pts = torch.from_numpy(w.points).cuda()
    op = hm.kernel_op(w.kernel)
    out = {"workload": f"sphere_invr_{w.n}", "n": w.n, "kernel": "1/|x-y|", "leaf_size": w.leaf_size,
           "tol": w.tol, "r": w.r, "oversample": w.oversample, "data": "synthetic (seeded jittered Fibonacci sphere)",
           "error_metric": "||A_mode - A_fp64|| / ||A_fp64||, 20 power iterations on the compressed operators",
           "modes": {}}
    stream = torch.cuda.current_stream()

    def compress(pv, warm):
        s = hm.Settings(d=3, leaf_size=w.leaf_size, r=w.r, oversample=w.oversample, tol=w.tol, precision=pv,
                        seed=w.seed)
        comp = hm.Compressor(s, stream)
        if warm:
            comp.tree_build(pts)
            comp.compress(op)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        comp.tree_build(pts)
        comp.compress(op)
        e1.record(stream)
        torch.cuda.synchronize()
        info = comp.info()
        return comp, {"time_to_compress_s": round(e0.elapsed_time(e1) / 1e3, 3), "warm_up_job": warm,
                      "floats_per_dof": round(info.factor_floats / w.n, 1), "max_rank": info.max_rank,
                      "matvec_cols": info.matvec_cols, "bb_tc_levels": info.bb_tc_levels,
                      "phases_s": {nm: round(info.seconds_phase[i], 3) for i, nm in enumerate(hm.PHASES)}}

    def norm_est(apply, apply_t, iters=20):
        g = torch.Generator(device="cuda").manual_seed(7)
        v = torch.randn(w.n, dtype=torch.float64, device="cuda", generator=g)
        v /= torch.linalg.norm(v)
        lam = 0.0
        for _ in range(iters):
            u = apply_t(apply(v))
            lam = float(torch.linalg.norm(u))
            if lam == 0.0:
                return 0.0
            v = u / lam
        return lam ** 0.5

    # exact A x on a random sample of rows, in FP64 from the point differences
    # (N kernel evaluations per row): the error of every mode against A itself
    gen = torch.Generator(device="cuda").manual_seed(11)
    xv = torch.randn(w.n, dtype=torch.float64, device="cuda", generator=gen)
    rows = torch.randperm(w.n, device="cuda", generator=gen)[:4096]
    xr = pts[rows]
    exact = torch.zeros(rows.numel(), dtype=torch.float64, device="cuda")
    for c0 in range(0, w.n, 8192):
        d = xr[:, None, :] - pts[None, c0:c0 + 8192, :]
        dist = torch.sqrt((d * d).sum(-1))
        kij = torch.where(dist > 0, 1.0 / torch.where(dist > 0, dist, torch.ones_like(dist)), torch.zeros_like(dist))
        exact += kij @ xv[c0:c0 + 8192]
    out["sampled_rows"] = int(rows.numel())
    out["error_metric_rows"] = "||(A x - A~ x)(S)|| / ||(A x)(S)||, x Gaussian, S 4096 random rows, A x exact in FP64"

    ref = None
    for name in args.sweep_modes.split(","):
        pv, desc, _ = PRECISIONS[name]
        try:
            comp, res = compress(pv, warm=name != "fp64")  # FP64 once, without a warm-up job (minutes)
            ya = comp.apply(xv)[rows]
            res["rel_error_rows"] = float(torch.linalg.norm(ya - exact) / torch.linalg.norm(exact))
            if name == "fp64":
                ref = comp
            elif ref is not None:
                num = norm_est(lambda x: comp.apply(x) - ref.apply(x),
                               lambda y: comp.apply(y, trans=1) - ref.apply(y, trans=1))
                den = norm_est(lambda x: ref.apply(x), lambda y: ref.apply(y, trans=1))
                res["rel_error_vs_fp64"] = num / den if den > 0 else None
                comp.close()
        except hm.HMError as e:  # a mode that does not fit on the device says so
            res = {"error": f"{e}"}
        res["precision"] = desc
        out["modes"][name] = res
        # one line per finished mode, so that a limit on the whole run keeps the finished ones
        print(json.dumps({"sweep_mode": name, "workload": out["workload"], "result": res}), flush=True)
    if ref is not None:
        ref.close()
    print(json.dumps(out), flush=True)


def oracle_series(sizes):
    """The full CPU oracle (tree, colourings, samples, peel, bases, cores, leaf
    blocks) timed end to end on the torus job at the given sizes, and on the
    2048-point 1D dense log-kernel configuration (best of 3)."""
    import hm_workloads as W
    from oracle import h1 as oh1
    from oracle import tree as ot
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    out = {"kind": "oracle", "cores": cores, "torus": [], "line1d_dense_2048": None}
    w = W.line1d_dense()
    best = float("inf")
    for _ in range(3):
        t0 = time.perf_counter()
        t = ot.build_tree(w.points, w.leaf_size, w.uniform_depth)
        oh1.compress(t, oh1.DenseOp(w.dense[t.perm][:, t.perm]), w.r, rank=w.rank, seed=w.seed)
        best = min(best, time.perf_counter() - t0)
    out["line1d_dense_2048"] = {"seconds_best_of_3": round(best, 3)}
    for n in sizes:
        w = W.torus_laplace(n=n, tol=1e-6, r=32)
        t0 = time.perf_counter()
        t = ot.build_tree(w.points, w.leaf_size)
        H = oh1.compress(t, oh1.KernelOp(w.points[t.perm], w.kernel), w.r, tol=w.tol, seed=w.seed,
                         oversample=w.oversample)
        out["torus"].append({"n": n, "levels": t.L, "seconds": round(time.perf_counter() - t0, 2),
                             "matvec_cols": H.matvec_cols, "floats_per_dof": round(H.floats() / n, 1)})
        print(json.dumps(out), flush=True)
    return out


def cpu_baseline(w, rows_per_level: int = 100):
    return OracleSample(w).sample(rows_per_level)


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = workload(args.n)
    orc = OracleSample(w)
    for k in range(args.warmup):
        orc.sample(40, seed=k)
    ests = []
    t0 = time.perf_counter()
    for k in range(args.steps):
        ests.append(orc.sample(40, seed=100 + k))
    wall = time.perf_counter() - t0
    est = sum(e["seconds_estimate"] for e in ests) / len(ests)
    value = float(f"{1.0 / est:.4g}")
    out = {"metric": METRIC, "value": value, "unit": "jobs/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(1e3 * est, 1), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded torus point cloud)",
           "impl": "reference",
           "config": dict(config_of(args, w), precision="FP64 CPU oracle (plain loops, numpy)", parallelism="cpu oracle"),
           "cpu_baseline": {"value": value, "unit": "jobs/s", "cores": ests[-1]["cores"], "kind": "oracle",
                            "sample": ests[-1]["sample"]},
           "e2e": {"value": value, "unit": "jobs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
           "host_wall_s": round(wall, 2)}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.peaks:
        print(json.dumps(measure_peaks()), flush=True)
        return
    if args.sweep:
        run_sweep(args)
        return
    if args.oracle_series:
        print(json.dumps(oracle_series([int(v) for v in args.oracle_series.split(",")])), flush=True)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
