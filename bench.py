#!/usr/bin/env python
"""Benchmark of the deflated Schur-complement solve (Algorithm 3 of Joshi &
Diamessis) on GB300.

Workload (default): the 2-D Poisson-Neumann problem on [0,1]^2, 16 x 16 SMPM
elements with n = 16 GLL points per direction (r = 65,536 nodes, k = 15,360
interface slots), FP64, one seeded Fourier right-hand side, GMRES(50) to a
relative residual of 1e-10.  A step is one complete schur_solve: right-hand
side projection, b_S, the deflated block-Jacobi GMRES, assembly, recovery and
zero-mean normalisation.  The factor step is timed once, separately.

Reported: solves/s (whole job, all ranks), the same metric end to end through
the host-pointer C ABI entry (host->device copy of f, device->host copy of u
inside the timed region), the roofline of the dominant kernel pair (the fused
S M^-1 apply) measured with CUDA events on the launching stream, SM clocks
sampled during the timed region, and the CPU oracle timed on a bounded sample.

--impl reference times the oracle (the plain FP64 CPU implementation written
from the paper) on the same workload, one oracle solve per step.
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GMRES solves/s to 1e-10 residual (mixed vs FP64); Schur-apply HBM GB/s"
WORKLOAD = {"mx": 16, "my": 16, "n": 16, "nrhs": 1, "tol": 1e-10, "restart": 50, "seed": 1000}
WORKLOAD_NAME = "SMPM Poisson-Neumann, 16x16 elements, n=16 (r=65536), FP64, 1 Fourier RHS, GMRES(50) to 1e-10"
L2_FLUSH_BYTES = 512 << 20          # written between timed steps: 3.9x the 135.5 MB L2 of a GB300
CONFIG = {"workload": WORKLOAD_NAME, **WORKLOAD, "precision": "fp64", "precond": "block-Jacobi + deflation"}
GMRES_PROFILE = os.path.join(ROOT, "profiles", "k_gmres_16x16_n16_fp64.md")
GMRES_SOURCES = [os.path.join(ROOT, "paper_1601_03432_gb300", "csrc", f) for f in ("smpm_gmres.cuh", "smpm_kernels.cuh")]


def kernel_traffic():
    """DRAM bytes (read + write) per k_gmres launch of the bench workload from
    the kept ncu summary, or None when the kernel's sources changed since that
    capture (the summary records their SHA-256)."""
    import hashlib
    import re
    try:
        text = open(GMRES_PROFILE).read()
    except OSError:
        return None, "no profile summary"
    h = hashlib.sha256()
    for f in GMRES_SOURCES:
        h.update(open(f, "rb").read())
    m_sha = re.search(r"sources sha256: ([0-9a-f]{16})", text)
    m_tr = re.search(r"traffic per launch \(read \+ write\): ([\d,]+) bytes", text)
    if not m_sha or not m_tr:
        return None, "profile summary without traffic or source hash"
    if m_sha.group(1) != h.hexdigest()[:16]:
        return None, "kernel changed since the ncu capture"
    return float(m_tr.group(1).replace(",", "")), "ncu capture " + os.path.basename(GMRES_PROFILE)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--batch", type=int, default=512,
                   help="grids of the uneven batch section (0 skips it; 512 is the full seeded batch)")
    p.add_argument("--headline-only", action="store_true",
                   help="only the headline, mixed-precision and end-to-end solves (for an ncu launch list)")
    p.add_argument("--profile", choices=["gmres", "apply", "apply96", "bapply", "batch"], default=None,
                   help="run only a small fixed case for an ncu capture and exit (prints no bench line)")
    return p.parse_args()


# ----------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------- ranks
def job_rate(local_ms, steps, world, dist=None, device="cpu"):
    """Whole-job rate of a weak-scaling run: each rank times its own steps,
    the job's time is the MAX over ranks, and the job processed world x
    steps units in it.  Returns (max ms, units per second)."""
    import torch
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms = float(t.item())
    return ms, world * steps / (ms / 1e3)


def rank_seed(seed, rank):
    """Right-hand-side seed of a rank: every replica solves its own problem."""
    return seed + rank


# ----------------------------------------------------------- CPU oracle
def oracle_solve_seconds(steps, warmup, seed, threads=1):
    """Time the oracle's Algorithm 3 on the bench workload in a fresh process
    with `threads` BLAS/OpenMP threads; returns (per-solve seconds list,
    iterations)."""
    code = r"""
import json, os, sys, time
sys.path.insert(0, %r)
from oracle.smpm import SMPMGrid
from oracle.schur import SchurSystem
from oracle import methods
from paper_1601_03432_gb300 import inputs
W = %r
g = SMPMGrid(W["mx"], W["my"], W["n"])
s = SchurSystem(g)
x, y = g.coords()
f, _ = inputs.fourier_rhs(x, y, seed=W["seed"])
times, its = [], None
for i in range(%d + %d):
    t = time.perf_counter()
    u, info = methods.algorithm3(s, g.rhs(f), tol=W["tol"], restart=W["restart"])
    dt = time.perf_counter() - t
    if i >= %d:
        times.append(dt)
    its = info["iterations"]
print(json.dumps({"times": times, "iterations": its}))
""" % (ROOT, WORKLOAD, warmup, steps, warmup)
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = str(threads)
    env["CUDA_VISIBLE_DEVICES"] = ""
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    out = json.loads(r.stdout.strip().splitlines()[-1])
    return out["times"], out["iterations"]


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    times, its = oracle_solve_seconds(args.steps, args.warmup, WORKLOAD["seed"])
    total = sum(times)
    value = len(times) / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(CONFIG), "l2": "n/a (CPU)",
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": 1, "kind": "oracle",
                         "sample": "%d oracle Algorithm-3 solves of the bench workload (setup excluded), "
                                   "%d GMRES iterations each" % (len(times), its)},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------- ours
def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_1601_03432_gb300 import Grid, inputs
    from paper_1601_03432_gb300.build import build

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0:
        build()
    if world > 1:
        dist.barrier()

    W = WORKLOAD
    g = Grid(W["mx"], W["my"], W["n"])
    t0 = time.perf_counter()
    g.factor(tol=W["tol"], restart=W["restart"])
    factor_s = time.perf_counter() - t0
    x, y = g.node_coords()
    f, _ = inputs.fourier_rhs(x, y, seed=rank_seed(W["seed"], rank))
    fd = torch.as_tensor(f, dtype=torch.float64, device="cuda")
    ud = torch.zeros_like(fd)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    rep = None
    for _ in range(args.warmup):
        rep = g.solve(fd, ud)[0]
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- device-resident timed region
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    iters = []
    reps_timed = []
    launches = 0
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(float(i))                   # evict L2 between steps (not timed)
        evs[i][0].record(stream)
        rep = g.solve(fd, ud)[0]
        evs[i][1].record(stream)
        iters.append(rep["iterations"])
        reps_timed.append(rep)
        launches += rep["launches"]
    barrier()
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    dev_ms, value = job_rate(sum(a.elapsed_time(b) for a, b in evs), args.steps, world, dist, "cuda")

    # ---- end to end through the host-pointer entry point
    fh = torch.empty(g.r, dtype=torch.float64).pin_memory()
    uh = torch.empty(g.r, dtype=torch.float64).pin_memory()
    fh.copy_(torch.as_tensor(f))
    fnp, unp = fh.numpy(), uh.numpy()
    g.solve_host(fnp, unp)
    barrier()
    e2e_ms = 0.0
    for i in range(args.steps):
        flush.fill_(float(i))
        torch.cuda.synchronize()
        a = time.perf_counter()
        g.solve_host(fnp, unp)
        e2e_ms += (time.perf_counter() - a) * 1e3
    _, e2e_value = job_rate(e2e_ms, args.steps, world, dist, "cuda")
    err_e2e = float(np.abs(unp - ud.cpu().numpy()).max())

    # ---- roofline of the dominant kernel: the persistent GMRES kernel
    # (k_gmres), timed by the library with CUDA events on the solve stream in
    # every timed step; algorithmic FLOPs/bytes from the iterations it ran.
    n, nel, M, kp, d = W["n"], W["mx"] * W["my"], 4 * W["n"], g.kp, g.d
    nblack = g.nblack
    per_step_fixed_flops = 2 * (M * M * (nel + nblack) + 4 * n * n * nblack + d * d)
    per_step_fixed_bytes = 8 * (M * M * (nel + nblack) + 4 * n * n * nblack + d * d + 10 * kp)
    tot_flops = tot_bytes = tot_ms = 0.0
    pre_ms = sum(r_["pre_ms"] for r_ in reps_timed) / len(reps_timed)
    post_ms = sum(r_["post_ms"] for r_ in reps_timed) / len(reps_timed)
    for r_ in reps_timed:
        J, m = r_["iterations"], W["restart"]
        cyc = [m] * (J // m) + ([J % m] if J % m else [])
        sj = sum(c * (c + 1) // 2 for c in cyc)          # sum over steps of (j + 1)
        tot_flops += J * per_step_fixed_flops + 2 * 4 * sj * kp
        tot_bytes += J * per_step_fixed_bytes + 8 * 3 * sj * kp
        tot_ms += r_["gmres_ms"]
    achieved_tf = tot_flops / (tot_ms * 1e-3) / 1e12
    achieved_gbs = tot_bytes / (tot_ms * 1e-3) / 1e9
    fp64_peak_tf = 152 * 2070e6 * 4 / 1e12    # 152 SMs x 2 FP64 FMA (4 flop) per clock at the 2.07 GHz max clock
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    gm_share = tot_ms / dev_ms

    # ---- mixed precision (FP32 inner GMRES + FP64 refinement), same workload
    g.factor(tol=W["tol"], restart=W["restart"], precision=1)
    for _ in range(args.warmup):
        g.solve(fd, ud)
    barrier()
    mix_ms = 0.0
    mix_rep = None
    for i in range(args.steps):
        flush.fill_(float(i))
        a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a_.record(stream)
        mix_rep = g.solve(fd, ud)[0]
        b_.record(stream)
        torch.cuda.synchronize()
        mix_ms += a_.elapsed_time(b_)
    mix_max, mix_rate = job_rate(mix_ms, args.steps, world, dist, "cuda")
    mixed = {"value": mix_rate, "unit": "solves/s",
             "ms_per_step": mix_max / args.steps, "inner_iterations": mix_rep["iterations"],
             "refinements": mix_rep["refinements"], "schur_relres": mix_rep["schur_relres"],
             "precision": "FP32 inner GMRES (FP32 operator; FP32 coarse product, or the FP64 fused coarse update on small grids; FP64 Givens and dot accumulation) + FP64 refinement"}

    # ---- Schur apply y = S v on single grids of growing size (operator-only
    # factor step: T_e only), L2 flushed before each launch (write + read
    # pass, so that no dirty line is written back inside the launch)
    from paper_1601_03432_gb300 import _binding as _B
    curve = []
    for (amx, amy, an) in (() if args.headline_only else ((32, 32, 24), (64, 64, 24), (96, 96, 24), (128, 128, 16))):
        ga = Grid(amx, amy, an)
        ga.factor(precision=1, flags=_B.FLAG_OPERATOR_ONLY)
        Ma, nela = 4 * an, amx * amy
        pt = {"grid": "%dx%d, n=%d" % (amx, amy, an)}
        for name, dt, fn, sz in (("fp64", torch.float64, ga.apply_schur, 8),
                                 ("fp32", torch.float32, ga.apply_schur32, 4)):
            va = torch.randn(ga.kp, dtype=dt, device="cuda")
            ya = torch.empty_like(va)
            for _ in range(3):
                fn(va, ya)
            times = []
            for i in range(15):
                flush.fill_(float(i))
                flush.sum()
                a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a_.record(stream)
                fn(va, ya)
                b_.record(stream)
                torch.cuda.synchronize()
                times.append(a_.elapsed_time(b_))
            us = 1e3 * sorted(times)[len(times) // 2]
            byts = nela * (Ma * Ma + 3 * Ma) * sz
            pt[name] = {"us": round(us, 2), "MB": round(byts / 1e6, 1), "gbs": round(byts / (us * 1e-6) / 1e9, 1),
                        "hbm_frac": round(byts / (us * 1e-6) / 1e9 / hbm_peak, 3),
                        "tflops": round(2.0 * nela * Ma * Ma / (us * 1e-6) / 1e12, 3)}
        # the element-class-shared path on the same grid: only the vectors
        # (and the <= 9 class matrices, once) stream from HBM
        ncls = len({(ix > 0, ix < amx - 1, iy > 0, iy < amy - 1) for ix in range(amx) for iy in range(amy)})
        for name, dt, fn, sz in (("fp64_class", torch.float64, ga.apply_schur_class, 8),
                                 ("fp32_class", torch.float32, ga.apply_schur_class32, 4)):
            va = torch.randn(ga.kp, dtype=dt, device="cuda")
            ya = torch.empty_like(va)
            for _ in range(3):
                fn(va, ya)
            times = []
            for i in range(15):
                flush.fill_(float(i))
                flush.sum()
                a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a_.record(stream)
                fn(va, ya)
                b_.record(stream)
                torch.cuda.synchronize()
                times.append(a_.elapsed_time(b_))
            us = 1e3 * sorted(times)[len(times) // 2]
            byts = (nela * 3 * Ma + ncls * Ma * Ma) * sz
            pt[name] = {"us": round(us, 2), "MB": round(byts / 1e6, 2), "gbs": round(byts / (us * 1e-6) / 1e9, 1),
                        "hbm_frac": round(byts / (us * 1e-6) / 1e9 / hbm_peak, 3),
                        "tflops": round(2.0 * nela * Ma * Ma / (us * 1e-6) / 1e12, 3),
                        "speedup_vs_per_element": round(pt[name.split("_")[0]]["us"] / us, 2)}
        # the autotuner's choice among the available apply kernels (its own
        # CUDA-event medians, 512 MiB written between launches)
        kind_names = {1: "warp", 2: "warp2", 3: "warp4", 4: "stream", 5: "class"}
        for precision, name in ((0, "fp64"), (1, "fp32")):
            chosen, ms = ga.autotune_apply(precision=precision, reps=5, flush=True)
            pt["autotune_" + name] = {"chosen": kind_names[chosen],
                                      "us": {kind_names[k]: round(1e3 * v, 2) for k, v in ms.items()}}
        curve.append(pt)
        ga.close()
    schur_apply = {"workload": "y = S v on one grid, operator-only factor step, L2 flushed before each launch "
                               "(512 MiB write, then a read pass); median of 15",
                   "algorithmic_bytes": "per element: nel (M^2 + 3M) s (T_e once, v read twice, y once); class-shared: "
                                        "3 M nel s + (classes) M^2 s",
                   "curve": curve,
                   "note": "FP64 at 0.25 flop/byte is bound by the FP64 pipe (1.26 TFLOP/s) near 5 TB/s; "
                           "FP32 is HBM-bound; the smallest grids are launch and first-load latency"}

    # the batch and precision-config sections run on single-GPU runs only: a
    # multi-GPU run measures the replicated headline solve and holds every GPU
    # for as short a time as that takes
    full = world == 1 and not args.headline_only
    batch = run_batch(args, stream, hbm_peak) if args.batch > 0 and full else None
    config3 = run_config3(args, stream) if full else None
    config1 = run_config1(stream) if full else None
    config5 = run_config5(stream) if full else None
    graded = run_graded(stream) if full else None
    sweeps = run_sweeps() if full else None

    traffic, traffic_src = kernel_traffic()
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle runs in fresh processes after the GPU timing, with one
        # BLAS thread and with all of the host's cores
        cpu = {}
        try:
            cpu["times"], cpu["its"] = oracle_solve_seconds(2, 0, WORKLOAD["seed"], 1)
            cpu["ncores"] = os.cpu_count() or 1
            cpu["times_all"], _ = oracle_solve_seconds(2, 0, WORKLOAD["seed"], cpu["ncores"])
        except Exception as ex:  # reported, not fatal
            cpu["error"] = str(ex)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dev_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(CONFIG),
            "l2": "flushed between steps (512 MiB write, not timed)",
            "run": {"factor_s": round(factor_s, 3), "gmres_iterations": iters[-1], "wall_s": round(wall, 3),
                    "device_ms": {"pre": round(pre_ms, 4), "gmres": round(tot_ms / len(reps_timed), 4),
                                  "post": round(post_ms, 4)}},
            "mixed": mixed,
            "schur_apply": schur_apply,
            "batch": batch,
            "config3": config3,
            "config1": config1,
            "config5": config5,
            "graded": graded,
            "paper_sweeps": sweeps,
            "clocks": clk,
            "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": 8 * g.r,
                    "d2h_bytes_per_step": 8 * g.r, "max_abs_diff_vs_device": err_e2e},
            "gpu_launches": launches,
            # traffic: dram bytes read + written per k_gmres launch of this
            # workload (L2 flushed before the step), from the kept ncu
            # capture of the current kernel (null once the kernel changed)
            "roofline": {"kernel": "k_gmres (persistent GMRES, FP64)", "bound": "alu",
                         "achieved": achieved_tf, "peak": fp64_peak_tf, "unit": "TFLOP/s",
                         "frac": achieved_tf / fp64_peak_tf, "traffic": traffic, "traffic_source": traffic_src,
                         "achieved_gbs": achieved_gbs, "hbm_peak_gbs": hbm_peak,
                         "hbm_frac": achieved_gbs / hbm_peak, "share_of_step": gm_share,
                         "ms_per_launch": tot_ms / len(reps_timed),
                         "note": "FP64 peak derived from SM count, FP64 FMA units and max clock; "
                                 "working set L2-resident after the first iteration"},
        }
        if cpu is not None:
            if "times_all" in cpu:
                cv = len(cpu["times"]) / sum(cpu["times"])
                ca = len(cpu["times_all"]) / sum(cpu["times_all"])
                best, cores = (ca, cpu["ncores"]) if ca > cv else (cv, 1)
                line["cpu_baseline"] = {"value": best, "unit": "solves/s", "cores": cores, "kind": "oracle",
                                        "sample": "%d oracle Algorithm-3 solves of the bench workload (setup "
                                                  "excluded), %d GMRES iterations; the faster of 1 BLAS thread and "
                                                  "%d" % (len(cpu["times"]), cpu["its"], cpu["ncores"]),
                                        "one_thread": cv, "all_cores": {"value": ca, "threads": cpu["ncores"]}}
            else:
                line["cpu_baseline"] = {"value": None, "unit": "solves/s", "cores": 1, "kind": "oracle",
                                        "sample": "failed: " + cpu.get("error", "")[:200]}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ------------------------------------------------------ precision config
def run_config3(args, stream):
    """32x32 elements, n = 24, 8 seeded Fourier right-hand sides, tol 1e-10:
    mixed precision (FP32 inner GMRES, FP64 refinement) against FP64, as
    8 consecutive solves on the handle and as one batched launch (the 8
    right-hand sides of the one grid, all SMs as one team)."""
    import numpy as np
    import torch
    from paper_1601_03432_gb300 import Batch, Grid, inputs
    W = WORKLOAD
    out = {"workload": "32x32 elements, n=24 (r=589824), 8 Fourier right-hand sides (seeds 1000-1007), tol 1e-10"}
    grids = {}
    for name, prec in (("mixed", 1), ("fp64", 0)):
        g = Grid(32, 32, 24)
        g.factor(tol=W["tol"], restart=W["restart"], precision=prec)
        grids[name] = g
    f = fourier_packed([grids["fp64"]], [8], torch, np, inputs)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    sols = {}
    for name, g in grids.items():
        u = torch.zeros_like(f)
        g.solve(f, u, nrhs=8)  # warm-up
        a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a_.record(stream)
        reps = g.solve(f, u, nrhs=8)
        b_.record(stream)
        torch.cuda.synchronize()
        ms = a_.elapsed_time(b_)
        b = Batch([g], [8], team_size=sms)
        ub = torch.zeros_like(f)
        b.solve(f, ub)
        rb = b.solve(f, ub)
        out[name] = {"solves_per_s": 8 / (ms / 1e3), "ms_for_8": ms,
                     "iterations": [r["iterations"] for r in reps],
                     "refinements_max": max(r["refinements"] for r in reps),
                     "all_converged": all(r["converged"] == 1 for r in reps),
                     "batched_one_launch": {"solves_per_s": 8 / (b.info()["last_ms"] / 1e3),
                                            "ms_for_8": b.info()["last_ms"],
                                            "all_converged": all(r["converged"] == 1 for r in rb)}}
        sols[name] = u.cpu().numpy().reshape(8, -1)
        b.close()
    out["mixed_vs_fp64_rel_l2_max"] = float(max(np.linalg.norm(sols["mixed"][k] - sols["fp64"][k]) /
                                                np.linalg.norm(sols["fp64"][k]) for k in range(8)))
    out["mixed_over_fp64"] = out["mixed"]["solves_per_s"] / out["fp64"]["solves_per_s"]
    for g in grids.values():
        g.close()
    return out


# ------------------------------------------------- differentiation config
def run_config1(stream):
    """2x2 elements, n = 8, the manufactured cos(pi x) cos(pi y) problem, FP64,
    tol 1e-12: solves per second (median of 20 CUDA-event timings) and the
    error against the exact solution."""
    import numpy as np
    import torch
    from paper_1601_03432_gb300 import Grid, inputs
    g = Grid(2, 2, 8)
    g.factor(tol=1e-12)
    x, y = g.node_coords()
    f, uex = inputs.cos_problem(x, y)
    fd = torch.as_tensor(f, dtype=torch.float64, device="cuda")
    u = torch.zeros_like(fd)
    rep = g.solve(fd, u)[0]
    ts = []
    for _ in range(20):
        a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a_.record(stream)
        rep = g.solve(fd, u)[0]
        b_.record(stream)
        torch.cuda.synchronize()
        ts.append(a_.elapsed_time(b_))
    ms = sorted(ts)[len(ts) // 2]
    w = g.node_mass()
    ue = uex - (w @ uex) / w.sum()
    err = float(np.abs(u.cpu().numpy() - ue).max())
    g.close()
    return {"workload": "2x2 elements, n=8, cos(pi x) cos(pi y), FP64, tol 1e-12", "solves_per_s": 1e3 / ms,
            "ms": round(ms, 4), "iterations": rep["iterations"], "max_error_vs_exact": err}


def run_config5(stream):
    """48x48 elements, n = 16, FP64, tol 1e-11: the forward solve of a seeded
    Fourier right-hand side and the adjoint solve (S^T, dl/df and dl/dg) of
    the loss ||u - u_t||^2, each timed with CUDA events (median of 5)."""
    import torch
    from paper_1601_03432_gb300 import Grid, inputs
    from paper_1601_03432_gb300 import _binding as _B
    g = Grid(48, 48, 16)
    t0 = time.perf_counter()
    g.factor(tol=1e-11, flags=_B.FLAG_ADJOINT)
    factor_s = time.perf_counter() - t0
    x, y = g.node_coords()
    f = torch.as_tensor(inputs.fourier_rhs(x, y, seed=6)[0], dtype=torch.float64, device="cuda")
    ut = torch.as_tensor(inputs.fourier_rhs(x, y, seed=5)[0], dtype=torch.float64, device="cuda")
    u = torch.zeros_like(f)
    gf = torch.zeros_like(f)
    gg = torch.zeros(g.kp, dtype=torch.float64, device="cuda")
    out = {"workload": "48x48 elements, n=16 (r=589824, d=4512), FP64, tol 1e-11, Fourier f (seed 6), "
                       "u_t Fourier (seed 5)", "factor_s": round(factor_s, 2)}
    for name, call in (("forward", lambda: g.solve(f, u)[0]),
                       ("adjoint", lambda: g.solve_adjoint(2.0 * (u - ut), gf, gg)[0])):
        rep = call()
        ts = []
        for _ in range(5):
            a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a_.record(stream)
            rep = call()
            b_.record(stream)
            torch.cuda.synchronize()
            ts.append(a_.elapsed_time(b_))
        ms = sorted(ts)[len(ts) // 2]
        out[name] = {"solves_per_s": 1e3 / ms, "ms": round(ms, 3), "iterations": rep["iterations"],
                     "gmres_us_per_step": round(1e3 * rep["gmres_ms"] / max(rep["iterations"], 1), 1),
                     "converged": rep["converged"]}
    out["coarse_bytes_per_step"] = 8 * g.d * g.d
    # the same forward solve in mixed precision (FP32 inner GMRES with the
    # FP32 copy of the coarse inverse, FP64 refinement)
    u64 = u.clone()
    g.factor(tol=1e-11, precision=1)
    rep = g.solve(f, u)[0]
    ts = []
    for _ in range(5):
        a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a_.record(stream)
        rep = g.solve(f, u)[0]
        b_.record(stream)
        torch.cuda.synchronize()
        ts.append(a_.elapsed_time(b_))
    ms = sorted(ts)[len(ts) // 2]
    out["forward_mixed"] = {"solves_per_s": 1e3 / ms, "ms": round(ms, 3), "inner_iterations": rep["iterations"],
                            "refinements": rep["refinements"], "converged": rep["converged"],
                            "rel_l2_vs_fp64": float(torch.linalg.norm(u - u64) / torch.linalg.norm(u64))}
    g.close()
    return out


def run_graded(stream):
    """32x32 elements, n = 16, both directions tanh-clustered toward the walls
    (element sizes spanning a factor of about 11), FP64, tol 1e-10, Fourier f:
    Algorithm 3 (deflation vectors weighted by B 1) and Algorithm 2, each timed
    with CUDA events (median of 5)."""
    import numpy as np
    import torch
    from paper_1601_03432_gb300 import Grid, inputs
    xs = inputs.clustered_edges(32, 1.0, 2.0)
    g = Grid(32, 32, 16, xs=xs, ys=xs)
    x, y = g.node_coords()
    f = torch.as_tensor(inputs.fourier_rhs(x, y, seed=7)[0], dtype=torch.float64, device="cuda")
    u = torch.zeros_like(f)
    h = np.diff(xs)
    out = {"workload": "32x32 elements, n=16, tanh-clustered edges (stretch 2, size ratio %.1f), FP64, tol 1e-10, "
                       "Fourier f (seed 7)" % (h.max() / h.min())}
    for precond, name in ((2, "algorithm3"), (1, "algorithm2")):
        g.factor(tol=1e-10, precond=precond)
        rep = g.solve(f, u)[0]
        ts = []
        for _ in range(5):
            a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a_.record(stream)
            rep = g.solve(f, u)[0]
            b_.record(stream)
            torch.cuda.synchronize()
            ts.append(a_.elapsed_time(b_))
        ms = sorted(ts)[len(ts) // 2]
        out[name] = {"solves_per_s": 1e3 / ms, "ms": round(ms, 3), "iterations": rep["iterations"],
                     "converged": rep["converged"], "schur_relres": rep["schur_relres"]}
    g.close()
    return out


# ------------------------------------------------------ paper's studies
def run_sweeps():
    """The paper's h- and p-refinement studies (Sec. 3.2, 3.3) through the GPU
    path: GMRES iterations of Algorithms 1, 2, 3 on the lambda = 7 cosine
    problem (unit square, homogeneous Neumann, tol 1e-10, GMRES(200)) for
    m_x = m_y = 4..32 at n = 5 and n = 5..15 at m = 4, and for a nodal white
    noise right-hand side in the p-study; the paper's own figures beside them."""
    import torch
    from paper_1601_03432_gb300 import Grid, inputs

    def iters(m, n, f_of):
        g = Grid(m, m, n)
        x, y = g.node_coords()
        f = torch.as_tensor(f_of(x, y, g.r), dtype=torch.float64, device="cuda")
        out = []
        for p in (0, 1, 2):
            g.factor(tol=1e-10, restart=200, precond=p)
            u = torch.zeros_like(f)
            out.append(g.solve(f, u)[0]["iterations"])
        g.close()
        return out

    cos = lambda x, y, r: inputs.paper_problem(x, y)[0]
    noise = lambda x, y, r: inputs.white_noise(r, 77)
    return {"algorithms": ["1 (S)", "2 (S M^-1)", "3 (P S M^-1)"],
            "h_refinement_n5": {str(m): iters(m, 5, cos) for m in (4, 8, 16, 32)},
            "p_refinement_m4": {str(n): iters(4, n, cos) for n in (5, 7, 9, 11, 13, 15)},
            "p_refinement_m4_white_noise": {str(n): iters(4, n, noise) for n in (5, 9, 15)},
            "paper": {"m32_n5": "Alg. 1 nearly 110, deflated just over 30 (Sec. 3.2)",
                      "m4_p4_14": "all < 40, preconditioned/deflated < 15 (Sec. 3.3)"}}


# ------------------------------------------------------------- batch
def fourier_packed(grids, nrhs, torch, np, inputs):
    """Packed right-hand sides of a batch: right-hand side j of every grid is
    the seeded Fourier field of seed 1000 + j, evaluated on the device from
    the seeded modes (input generation only)."""
    total = sum(g.r * k for g, k in zip(grids, nrhs))
    f = torch.empty(total, dtype=torch.float64, device="cuda")
    o = 0
    for g, k in zip(grids, nrhs):
        x, y = g.node_coords()
        xd = torch.as_tensor(x, device="cuda")
        yd = torch.as_tensor(y, device="cuda")
        for j in range(k):
            acc = torch.zeros_like(xd)
            for kx, ky, a in inputs.fourier_modes(1000 + j):
                acc += a * torch.cos(kx * np.pi * xd) * torch.cos(ky * np.pi * yd)
            f[o:o + g.r] = acc
            o += g.r
    return f


def run_batch(args, stream, hbm_peak):
    """The seeded uneven batch (512 grids, m_x, m_y ~ U{4..32}, n ~ U{8..24},
    1-16 Fourier right-hand sides each): every right-hand side of every grid
    in ONE persistent launch per solve (graph replay), mixed precision against
    FP64 on the same factored handles, tol 1e-10; then the batched Schur apply
    y_p = S_p v_p over all grids (inputs far larger than L2)."""
    import numpy as np
    import torch
    from paper_1601_03432_gb300 import Batch, Grid, factor_many, inputs
    probs = inputs.uneven_batch(512, seed=7)[:args.batch]
    grids = [Grid(mx, my, n) for (mx, my, n, k) in probs]
    nrhs = [p[3] for p in probs]
    t0 = time.perf_counter()
    factor_many(grids, tol=WORKLOAD["tol"], restart=WORKLOAD["restart"], precision=1)
    factor_s = time.perf_counter() - t0
    f = fourier_packed(grids, nrhs, torch, np, inputs)
    out = {"workload": "%d grids (seed 7), %d right-hand sides, r_total = %d, tol 1e-10, restart 50"
                       % (len(grids), sum(nrhs), int(f.numel())),
           "factor_s": round(factor_s, 2)}
    sols = {}
    for name, prec, steps in (("mixed", 1, 2), ("fp64", 0, 1)):
        b = Batch(grids, nrhs, precision=prec)
        u = torch.zeros_like(f)
        b.solve(f, u, allow_notconv=True)  # warm-up (captures the graph)
        ms = []
        for _ in range(steps):
            reps = b.solve(f, u, allow_notconv=True)
            ms.append(b.info()["last_ms"])
        its = [r["iterations"] for r in reps]
        out[name] = {"solves_per_s": len(reps) / (np.median(ms) / 1e3), "ms_per_batch": float(np.median(ms)),
                     "team_size": b.info()["team_size"], "launches_per_batch": 1,
                     "iterations_mean": float(np.mean(its)), "iterations_max": int(max(its)),
                     "refinements_max": int(max(r["refinements"] for r in reps)),
                     "not_converged": int(sum(r["converged"] != 1 for r in reps)),
                     "schur_relres_max": float(max(r["schur_relres"] for r in reps))}
        sols[name] = u
        b.close()
    # mixed against FP64, per right-hand side
    uo, um = sols["fp64"].cpu().numpy(), sols["mixed"].cpu().numpy()
    worst, o = 0.0, 0
    for g, k in zip(grids, nrhs):
        for _ in range(k):
            a, c = um[o:o + g.r], uo[o:o + g.r]
            worst = max(worst, float(np.linalg.norm(a - c) / max(np.linalg.norm(c), 1e-300)))
            o += g.r
    out["mixed_vs_fp64_rel_l2_max"] = worst
    out["mixed_over_fp64"] = out["mixed"]["solves_per_s"] / out["fp64"]["solves_per_s"]
    # batched Schur apply over all grids, FP32 and FP64
    b = Batch(grids, [1] * len(grids))
    ent = sum(mx * my * 16 * n * n for (mx, my, n, k) in probs)
    vlen = b.v_len()
    apply = {}
    for name, dt, fn, sz in (("fp32", torch.float32, b.apply_schur32, 4), ("fp64", torch.float64, b.apply_schur, 8)):
        v = torch.randn(vlen, dtype=dt, device="cuda")
        y = torch.empty_like(v)
        for _ in range(3):
            fn(v, y)
        ts = []
        for _ in range(10):
            a_, c_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a_.record(stream)
            fn(v, y)
            c_.record(stream)
            torch.cuda.synchronize()
            ts.append(a_.elapsed_time(c_))
        msa = float(np.median(ts))
        byts = (ent + 3 * vlen) * sz
        apply[name] = {"ms_per_launch": msa, "bytes_per_launch": byts, "gbs": byts / (msa * 1e-3) / 1e9,
                       "hbm_frac": byts / (msa * 1e-3) / 1e9 / hbm_peak}
    # DRAM traffic per launch: ncu (dram bytes read + written) on the same
    # kernel over the first 40 grids of this batch measured 1.0028 x the
    # algorithmic bytes; traffic grows with the elements streamed, so the
    # full launch is scaled by that ratio
    traffic_ratio = 1.0028
    apply["roofline"] = {"kernel": "k_schur_warp_batch<float> (batched y = S v, FP32)", "bound": "hbm",
                         "achieved": apply["fp32"]["gbs"], "peak": hbm_peak, "unit": "GB/s",
                         "frac": apply["fp32"]["hbm_frac"],
                         "traffic": traffic_ratio * apply["fp32"]["bytes_per_launch"],
                         "note": "operator %.2f GB FP32 / %.2f GB FP64, far above L2: no flush needed; traffic "
                                 "scaled from an ncu capture on 40 grids of the batch" % (ent * 4 / 1e9, ent * 8 / 1e9)}
    out["apply"] = apply
    b.close()
    for g in grids:
        g.close()
    return out


# ------------------------------------------------------------ ncu cases
def run_profile(which):
    """Small fixed cases for ncu captures: `gmres` runs three solves of the
    bench workload (FP64), `apply` three y = S v launches each in FP32 and
    FP64 on 32x32 elements, n = 24, `bapply` three batched FP32 applies over
    the first 40 grids of the uneven batch.  Prints "ok" and no bench line."""
    import torch
    from paper_1601_03432_gb300 import Grid, inputs
    from paper_1601_03432_gb300.build import build
    build()
    W = WORKLOAD
    if which == "gmres":
        g = Grid(W["mx"], W["my"], W["n"])
        g.factor(tol=W["tol"], restart=W["restart"])
        x, y = g.node_coords()
        f, _ = inputs.fourier_rhs(x, y, seed=W["seed"])
        fd = torch.as_tensor(f, dtype=torch.float64, device="cuda")
        ud = torch.zeros_like(fd)
        for _ in range(3):
            g.solve(fd, ud)
    elif which == "batch":
        # four grids of the uneven batch (large to small), two right-hand
        # sides each, mixed precision, teams of 8: three batched solves
        from paper_1601_03432_gb300 import Batch, factor_many
        probs = [(30, 27, 23, 2), (17, 25, 24, 2), (30, 17, 11, 2), (11, 13, 10, 2)]
        grids = [Grid(mx, my, n) for (mx, my, n, k) in probs]
        factor_many(grids, tol=W["tol"], restart=W["restart"], precision=1)
        import numpy as np
        f = fourier_packed(grids, [p[3] for p in probs], torch, np, inputs)
        b = Batch(grids, [p[3] for p in probs], team_size=8, use_graph=False)
        u = torch.zeros_like(f)
        for _ in range(3):
            b.solve(f, u)
        torch.cuda.synchronize()
        team, t0, t1 = b.task_times()
        print("ok", b.info()["last_ms"], [round(x, 2) for x in (t1 - t0)])
        b.close()
        return
    elif which == "bapply":
        # the first 40 grids of the seeded uneven batch (0.25 GB FP32 operator)
        from paper_1601_03432_gb300 import Batch, factor_many
        probs = inputs.uneven_batch(512, seed=7)[:40]
        grids = [Grid(mx, my, n) for (mx, my, n, k) in probs]
        factor_many(grids, tol=W["tol"], restart=W["restart"], precision=1)
        b = Batch(grids, [1] * len(grids))
        gen = torch.Generator(device="cuda").manual_seed(7)
        v = torch.randn(b.v_len(), dtype=torch.float32, device="cuda", generator=gen)
        yv = torch.empty_like(v)
        for _ in range(3):
            b.apply_schur32(v, yv)
        torch.cuda.synchronize()
        b.close()
        print("ok")
        return
    elif which == "apply96":
        # one grid of 96 x 96 elements, n = 24 (operator-only factor step):
        # three FP32 and three FP64 y = S v launches (0.35 / 0.70 GB of T_e)
        from paper_1601_03432_gb300 import _binding as _B
        g = Grid(96, 96, 24)
        g.factor(precision=1, flags=_B.FLAG_OPERATOR_ONLY)
        gen = torch.Generator(device="cuda").manual_seed(7)
        for dt, fn in ((torch.float32, g.apply_schur32), (torch.float64, g.apply_schur)):
            v = torch.randn(g.kp, dtype=dt, device="cuda", generator=gen)
            yv = torch.empty_like(v)
            for _ in range(3):
                fn(v, yv)
        torch.cuda.synchronize()
        print("ok")
        return
    else:
        g = Grid(32, 32, 24)
        g.factor(tol=W["tol"], restart=W["restart"], precision=1)
        gen = torch.Generator(device="cuda").manual_seed(7)
        for dt, fn in ((torch.float32, g.apply_schur32), (torch.float64, g.apply_schur)):
            v = torch.randn(g.kp, dtype=dt, device="cuda", generator=gen)
            yv = torch.empty_like(v)
            for _ in range(3):
                fn(v, yv)
    torch.cuda.synchronize()
    g.close()
    print("ok")


if __name__ == "__main__":
    a = parse()
    if a.profile:
        run_profile(a.profile)
    elif a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)
