#!/usr/bin/env python
"""Benchmark: time to ground state of the 2D non-rotating GPE (Fourier 256^2
on [-16,16]^2, V = (x^2+y^2)/2, beta = 1000, Gaussian initial guess, cascadic
multigrid 64^2 -> 128^2 -> 256^2) with the float32-bulk / float64-refined
regularized Newton solver, against the plain float64 GPU solver, plus the
H psi apply throughput of the operator kernels against the HBM roofline.

One step = one complete ground-state solve (Algorithm 3 around Algorithm 2,
every operator application, Cayley step, reduction and ratio test on the GPU)
from the initial guess resident in HBM.  Stopping rule: ||H psi - mu psi||_h
<= 1e-9, which puts |E - E_oracle| far below 1e-9 E (checked against the FP64
oracle's ground state in the CPU-baseline leg).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank solves its own replica (the solve does not shard).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = ("time-to-ground-state at ΔE≤1e-9, mixed vs FP64 on GB300; "
          "Hψ apply GB/s vs peak")
WORKLOAD = ("2D non-rotating GPE, Fourier 256^2 on [-16,16]^2, V=(x^2+y^2)/2, beta=1000, real psi, "
            "Gaussian init, cascade 64^2->128^2->256^2, float32 bulk + float64 regularized Newton "
            "until ||H psi - mu psi||_h <= 1e-9 or Eq. crit2 (accepted step <= 1e-8), whichever first; "
            "|dE|/E vs the float64 oracle reported")
RES_TOL = 1e-9
L2_FLUSH_BYTES = 256 << 20

# Algorithmic bytes per grid point of one operator application, by the kind of
# its final pass (read the operands the method needs once, write the result
# once): H psi apply (read X, write G); an Algorithm 1 iteration with the
# Cayley step formed in the first pass's load (read X_c, G_c, write G_new, plus
# the trial point Y); the ratio pass (read Z, X^k, G^k).  Per real number: 4 B
# (float32) or 8 B (float64); complex doubles it.
ALG_REALS_PER_POINT = {"grad": 2, "hess": 3, "F": 4, "W": 4, "ratio": 3, "WS": 5, "acc": 2}
# DRAM bytes (read + write) of one H psi apply of the happly workload come
# from an ncu capture recorded in profiles/happly_traffic.json together with a
# SHA-256 of the kernel sources it was taken with; once any of those sources
# changes the figure no longer describes the kernel and is reported as null.
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "happly_traffic.json")
# the sources that define each implementation's kernels
KERNEL_SOURCES = {"lines": ["lines2d.cuh", "linefft.cuh", "ops_impl.cuh", "ops_launch.cuh", "gpe_kernels.cuh"],
                  "fused2d": ["fused2d.cuh", "ops_impl.cuh", "ops_launch.cuh", "gpe_kernels.cuh"]}


def kernel_sources_sha256(impl="lines"):
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[impl]:
        with open(os.path.join(ROOT, "paper_1504_02891_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def measured_traffic(impl="lines"):
    """(bytes per apply, note) from the committed ncu record of implementation
    impl, or (None, why)."""
    try:
        rec = json.load(open(TRAFFIC_FILE))[impl]
    except Exception:
        return None, f"no ncu traffic record for {impl}"
    if rec.get("kernel_sources_sha256") != kernel_sources_sha256(impl):
        return None, f"{impl} kernel sources changed since the ncu traffic capture"
    return float(rec["dram_bytes_per_apply"]), rec.get("capture", "")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--only", choices=["happly", "solve"], default=None,
                    help="profiling aid: run only the H-apply loop (3 warm-up + 10 applies) or only two "
                         "mixed solves of the workload, print a one-line summary, no JSON contract line")
    ap.add_argument("--happly-n", type=int, choices=[64, 128, 256, 512, 1024], default=512,
                    help="with --only happly: the grid n x n of the 64-instance complex64 batch")
    ap.add_argument("--happly-path", type=int, choices=[0, 1, 2], default=0,
                    help="with --only happly: 0 = autotuned implementation, 1 = the fused kernel, 2 = the two "
                         "line kernels (1 and 2 skip the autotuning, so the launch sequence is fixed)")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def max_over_ranks(values, world):
    """Element-wise maximum of per-rank values (the slowest rank's step
    times); the identity at world = 1.  Works on any initialised process
    group (NCCL on the GPU machine, gloo in the CPU tests)."""
    if world <= 1:
        return [float(v) for v in values]
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


# --------------------------------------------------------------------------- oracle legs
ORACLE_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import oracle as O, workloads as W
p = W.config("c2")
psi0 = W.gaussian(p)
t_end = time.perf_counter() + {budget}
times, E = [], None
while True:
    t0 = time.perf_counter()
    g, psi, res = O.cascadic(p, psi0, levels=3, method="rn", res_tol_psi={res_tol})
    times.append(time.perf_counter() - t0)
    E = O.energy(g, psi)
    if len(times) >= {max_runs} or time.perf_counter() > t_end:
        break
print(json.dumps({{"times": times, "E": E, "mu": O.chem_potential(g, psi)}}))
"""


def run_oracle(budget_s, max_runs, threads=1):
    """The FP64 oracle's cascade solve of the same workload on the host cores,
    in a subprocess with BLAS pinned to `threads` threads."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        env[k] = str(threads)
    code = ORACLE_SNIPPET.format(root=ROOT, budget=budget_s, res_tol=RES_TOL, max_runs=max_runs)
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def reference_arm(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    per_step_budget = 60.0
    times = []
    E = None
    for i in range(args.warmup + args.steps):
        r = run_oracle(per_step_budget, 1)
        if i >= args.warmup:
            times.append(r["times"][0])
        E = r["E"]
    t = statistics.mean(times)
    line = {
        "impl": "reference", "metric": METRIC, "value": t, "unit": "s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "parallelism": "rank 0 only (host oracle)"},
        "cpu_baseline": {"value": t, "unit": "s", "cores": 1, "kind": "oracle",
                         "sample": "one full FP64 oracle cascade solve of the workload per step (numpy, dense DFT matrices, BLAS pinned to 1 thread)"},
        "e2e": {"value": t, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "E": E,
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self):
        self.proc = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self, gpu_index=0):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9 or f[0] != str(gpu_index):
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------- our arm
def roofline_from_profile(prof, peaks):
    """Dominant operator application of the profiled solve: group the pass
    kernels by (precision, complexity, grid size), take the group with the
    largest total time, count its applications by its final-pass launches."""
    groups = {}
    for name, (n, ms) in prof.items():
        if "@" not in name:
            continue
        kern, size = name.split("@")
        parts = kern.split("_")             # pass_f32_r_W
        if parts[0] not in ("pass", "fd", "step", "linesy", "linesx", "fused2d"):
            continue
        key = (parts[1], parts[2], int(size))
        g = groups.setdefault(key, {"ms": 0.0, "final": {}, "kernels": {}})
        g["ms"] += ms
        g["kernels"][kern] = (n, ms)
        if len(parts) > 3 and parts[3] != "acc":
            g["final"][parts[3]] = g["final"].get(parts[3], 0) + n
    if not groups:
        return None
    key = max(groups, key=lambda k: groups[k]["ms"])
    g = groups[key]
    prec, cplx, M = key
    napp = sum(g["final"].values())
    kind = max(g["final"], key=lambda k: g["final"][k]) if g["final"] else "grad"
    real_bytes = 4 if prec == "f32" else 8
    per_point = sum(ALG_REALS_PER_POINT.get(k, 2) * c for k, c in g["final"].items()) / max(napp, 1)
    per_point *= real_bytes * (2 if cplx == "c" else 1)
    t_app = g["ms"] / max(napp, 1) * 1e-3
    achieved = per_point * M / t_app / 1e9
    peak = peaks.get("hbm_gbs", 6800.0)
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": None, "kernel": f"operator application {prec}/{cplx}/M={M} ({kind} final pass)",
            "launches_per_application": sum(n for n, _ in g["kernels"].values()) / max(napp, 1),
            "us_per_application": t_app * 1e6, "alg_bytes_per_point": per_point,
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (burst copy)" if "hbm_gbs" in peaks else "fallback 6.8 TB/s"}


AUTOTUNE_ERRORS = []


def tune_or_note(G, plan, levels):
    """gpe_plan_autotune; a failure it can recover from (no memory for a
    candidate shape, a shape the plan rejects) is recorded in the JSON line and
    the run continues with the fixed launch rule (the choice never changes
    results).  Any other status -- a CUDA error, an expired device wait -- may
    leave the context unusable, so it stops the run."""
    try:
        plan.autotune(levels=levels)
    except G.GPEError as e:
        if getattr(e, "status", None) not in (G.ENOMEM, G.EINVAL):
            raise
        AUTOTUNE_ERRORS.append(str(e)[:200])


def happly_throughput(G, torch, W, peaks, reps=20):
    """H psi apply on inputs far above L2: 64 instances of the 512^2 rotating
    grid in complex64 (256 MiB read+write per apply)."""
    p = W.config("c4")
    nb = 64
    plan = G.Plan(p, nbatch=nb, prec=G.F32)
    tune_or_note(G, plan, 1)       # measured launch shapes (untimed)
    psi = plan.empty()
    psi.real.normal_()
    psi.imag.normal_()
    psi.mul_(1e-2)
    out = plan.empty()
    st = torch.cuda.current_stream()
    for _ in range(3):
        plan.grad(psi, out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(reps):
        plan.grad(psi, out)
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    # Hessian-vector product (Lemma 3.1) on the same batch: read psi and d, write the result
    d = plan.empty()
    d.real.normal_()
    d.imag.normal_()
    for _ in range(3):
        plan.hessvec(psi, d, 0.5, out)
    torch.cuda.synchronize()
    e0.record(st)
    for _ in range(reps):
        plan.hessvec(psi, d, 0.5, out)
    e1.record(st)
    torch.cuda.synchronize()
    ms_h = e0.elapsed_time(e1) / reps
    M = plan.M * nb
    alg = 16.0 * M                 # read psi (8 B) + write H psi (8 B) per point, complex64
    achieved = alg / (ms * 1e-3) / 1e9
    peak = peaks.get("hbm_gbs", 6800.0)
    alg_h = 24.0 * M               # read psi, d (8 B each) + write (8 B) per point, complex64
    plan.close()
    hess = {"bound": "hbm", "achieved": alg_h / (ms_h * 1e-3) / 1e9, "peak": peak, "unit": "GB/s",
            "frac": alg_h / (ms_h * 1e-3) / 1e9 / peak, "traffic": None,
            "kernel": "",
            "us_per_apply": ms_h * 1e3, "alg_bytes_per_apply": alg_h}
    fused = "512x512 nbatch 64: fused kernel" in G.autotune_report()
    traffic, tnote = measured_traffic("fused2d" if fused else "lines")
    kern = ("k_fused2d (one persistent launch: warp-per-line FFTs, y- and x-tasks per instance)" if fused else
            "k_lines_y + k_lines_x (two register-FFT line kernels)")
    hess["kernel"] = f"Hessian-vector product (gpe_hessvec) = {kern}, same batch"
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "hessvec": hess,
            "traffic": traffic, "traffic_source": tnote,
            "kernel": f"H psi apply = {kern}, 64 x 512^2 complex64 rotating (Omega=0.9), float32, "
                      "implementation chosen by gpe_plan_autotune",
            "us_per_apply": ms * 1e3, "alg_bytes_per_apply": alg, "launches_per_apply": 1 if fused else 2,
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (burst copy)" if "hbm_gbs" in peaks else "fallback 6.8 TB/s"}


def config3_times(G, torch, W):
    """Config 3 (3D sine 128^3, depth-100 lattice, beta = 1600, cascade
    32^3 -> 64^3 -> 128^3): time to ||H psi - mu psi||_h <= 1e-9 (or Eq.
    crit2), mixed schedule against plain float64, one warm-up and one timed
    solve each (CUDA events on the caller's stream)."""
    p = W.config("c3")
    out = {"workload": "3D sine 128^3 (127^3 unknowns), V = |x|^2/2 + 100 sum sin^2(pi x/4), beta = 1600, "
                       "Gaussian init, cascade 32^3->64^3->128^3"}
    with G.Plan(p, prec=G.F64) as plan:
        init = G.to_device(W.gaussian(p))
        st = torch.cuda.current_stream()
        for name, mode in (("mixed", 1), ("fp64", 0)):
            work = init.clone()
            plan.solve(work, mode=mode, levels=3, res_tol=RES_TOL)
            work.copy_(init)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(st)
            r = plan.solve(work, mode=mode, levels=3, res_tol=RES_TOL)
            e1.record(st)
            torch.cuda.synchronize()
            out[name] = {"time_s": e0.elapsed_time(e1) / 1e3, "E": r["E"], "res": r["res"],
                         "outer_f64": r["outer_f64"]}
    out["speedup_mixed_vs_fp64"] = out["fp64"]["time_s"] / out["mixed"]["time_s"]
    out["delta_E_rel_mixed_vs_fp64"] = abs(out["mixed"]["E"] - out["fp64"]["E"]) / abs(out["fp64"]["E"])
    return out


SWEEP_FP64_SAMPLE = 16


def sweep_throughput(G, torch, W, np):
    """Config 5, the batched sweep: 256 independent 2D rotating problems
    (grids 64^2-256^2, beta, Omega, gamma_y drawn from the seeded sweep), one
    gpe_solve_batch call (float32 Algorithm 1, float64 sums, each instance to
    ||H psi - mu psi||_h <= 1e-7 or its float32 floor), against (a) the same
    256 problems one gpe_solve_batch call each and (b) plain float64
    gpe_rnewton_solve calls one problem at a time (Algorithm 2, float64
    throughout, the same tolerance), timed on the first SWEEP_FP64_SAMPLE
    problems and scaled to 256."""
    ps = W.batched_sweep(256)
    init_np = [W.sweep_initial(p, i) for i, p in enumerate(ps)]
    init = [torch.from_numpy(a.astype(np.complex64)).cuda() for a in init_np]
    opts = dict(max_iter=1000, res_tol=1e-7, mode=2)
    G.solve_batch(ps[:8], [t.clone() for t in init[:8]], **opts)
    x = [t.clone() for t in init]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    reps = G.solve_batch(ps, x, **opts)
    torch.cuda.synchronize()
    tb = time.perf_counter() - t0
    # the mixed schedule batched: float32 stage + float64 refinement (<= 30 outer steps each)
    x = [t.clone() for t in init]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    reps_m = G.solve_batch(ps, x, max_iter=1000, res_tol=1e-7, mode=1, max_outer=30)
    torch.cuda.synchronize()
    tm = time.perf_counter() - t0
    x = [t.clone() for t in init]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i, p in enumerate(ps):
        G.solve_batch([p], [x[i]], **opts)
    torch.cuda.synchronize()
    ts = time.perf_counter() - t0
    # plain float64 solves, one problem per call (plan creation untimed)
    t64, conv64 = 0.0, 0
    for i in range(SWEEP_FP64_SAMPLE):
        with G.Plan(ps[i], prec=G.F64) as plan:
            t = G.to_device(init_np[i], G.F64)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = plan.solve(t, mode=0, levels=1, res_tol=1e-7, max_outer=200)
            torch.cuda.synchronize()
            t64 += time.perf_counter() - t0
            conv64 += int(r["status"] == 0 and r["res"] <= 1e-7)
    its = [r["inner_f32"] for r in reps]
    return {"workload": "256 x 2D rotating (64^2/128^2/256^2 on [-12,12]^2, beta~U[100,1000], "
                        "Omega~U[0,0.9], gamma_y~U[1,1.2]), complex64 bulk, float64 sums",
            "batched_solves_per_s": 256 / tb, "sequential_solves_per_s": 256 / ts, "speedup": ts / tb,
            "sequential_fp64_solves_per_s": SWEEP_FP64_SAMPLE / t64,
            "speedup_vs_sequential_fp64": (t64 / SWEEP_FP64_SAMPLE * 256) / tb,
            "fp64_sample": f"first {SWEEP_FP64_SAMPLE} problems, plain float64 gpe_rnewton_solve each, "
                           f"scaled to 256; {conv64} of {SWEEP_FP64_SAMPLE} reached res 1e-7 within 200 outer steps",
            "batched_ms": tb * 1e3, "iterations_median": float(np.median(its)), "iterations_max": int(max(its)),
            "converged": int(sum(1 for r in reps if r["status"] == 0 and r["res"] <= 1e-7)),
            "stopped_at_float32_floor": int(sum(1 for r in reps if r["status"] == 5)),
            "mixed_batched": {"solves_per_s": 256 / tm, "ms": tm * 1e3,
                              "converged_res_1e-7": int(sum(1 for r in reps_m if r["status"] == 0)),
                              "outer_f64_median": float(np.median([r["outer_f64"] for r in reps_m])),
                              "speedup_vs_sequential_fp64": (t64 / SWEEP_FP64_SAMPLE * 256) / tm}}


def our_arm(args):
    import numpy as np
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import workloads as W
    import paper_1504_02891_gb300 as G
    G.load()
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    def phase(name):
        # cumulative libgpe launches at each phase boundary (stderr): where a
        # launch-count-limited ncu capture of this command ends
        print(f"[bench] libgpe launches after {name}: {G.kernel_launches()}", file=sys.stderr, flush=True)

    p = W.config("c2")
    psi0 = W.gaussian(p)
    plan = G.Plan(p, prec=G.F64)
    tune_or_note(G, plan, 3)       # measured launch shapes for the three cascade grids (untimed)
    phase("autotuning")
    init = G.to_device(psi0)
    work = torch.empty_like(init)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    st = torch.cuda.current_stream()
    opts_mixed = dict(mode=1, levels=3, res_tol=RES_TOL)
    opts_fp64 = dict(mode=0, levels=3, res_tol=RES_TOL)

    def step(opts):
        work.copy_(init)
        return plan.solve(work, **opts)

    def timed(opts, k):
        times, reps = [], []
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for _ in range(k):
            flush.fill_(1.0)                      # evict L2 between steps (untimed)
            torch.cuda.synchronize()
            e0.record(st)
            rep = step(opts)
            e1.record(st)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
            reps.append(rep)
        return times, reps

    for _ in range(args.warmup):
        step(opts_mixed)
        step(opts_fp64)
    torch.cuda.synchronize()
    phase("warm-up")

    clocks = ClockSampler()
    time.sleep(0.3)
    barrier()
    l0 = G.kernel_launches()
    t_mixed, reps_mixed = timed(opts_mixed, args.steps)
    l1 = G.kernel_launches()
    barrier()
    t_fp64, reps_fp64 = timed(opts_fp64, max(3, args.steps // 2))
    barrier()
    clk = clocks.stop(gpu_index=local)
    phase("the timed mixed and float64 solves")

    ms_mixed, ms_fp64 = max_over_ranks([statistics.mean(t_mixed), statistics.mean(t_fp64)], world)

    # end to end through the public API with host buffers (pinned)
    h_init = torch.from_numpy(np.ascontiguousarray(psi0)).pin_memory()
    h_out = torch.empty_like(h_init).pin_memory()
    e2e = []
    for _ in range(max(3, args.steps // 2)):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        work.copy_(h_init, non_blocking=True)
        plan.solve(work, **opts_mixed)
        h_out.copy_(work, non_blocking=True)
        torch.cuda.synchronize()
        e2e.append(time.perf_counter() - t0)
    nbytes = h_init.numel() * h_init.element_size()

    # profiled solve (CUDA events around every launch, graphs off) -> roofline
    G.profile_enable(True)
    step(opts_mixed)
    torch.cuda.synchronize()
    prof = G.profile_summary()
    G.profile_enable(False)
    roof = roofline_from_profile(prof, peaks)
    phase("the end-to-end and profiled solves")
    c3 = config3_times(G, torch, W)
    phase("the 3D sine solves")
    happly = happly_throughput(G, torch, W, peaks)
    phase("the H-apply loop")
    sweep = sweep_throughput(G, torch, W, np)
    phase("the batched sweep")

    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    cpu = None
    dE = dE64 = None
    if not args.no_cpu_baseline:
        try:
            r = run_oracle(args.cpu_seconds, 50, threads=1)
            tcpu = statistics.mean(r["times"])
            cpu = {"value": tcpu, "unit": "s", "cores": 1, "kind": "oracle",
                   "sample": f"{len(r['times'])} complete FP64 oracle cascade solves of the same workload "
                             "(numpy, dense DFT matrices, BLAS pinned to 1 thread)"}
            dE = abs(reps_mixed[-1]["E"] - r["E"]) / abs(r["E"])
            dE64 = abs(reps_fp64[-1]["E"] - r["E"]) / abs(r["E"])
        except Exception as e:  # reported, never fatal
            cpu = {"value": None, "unit": "s", "cores": 1, "kind": "oracle", "sample": f"failed: {e}"[:300]}
    rep = reps_mixed[-1]
    line = {
        "metric": METRIC, "value": ms_mixed / 1e3, "unit": "s",
        "fp64_time_s": ms_fp64 / 1e3, "speedup_mixed_vs_fp64": ms_fp64 / ms_mixed,
        "delta_E_rel_vs_oracle": dE, "delta_E_rel_vs_oracle_fp64": dE64,
        "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_mixed, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": [256, 256], "levels": 3, "beta": 1000.0,
                   "l2": "flushed between steps (256 MiB write, untimed); each step timed with CUDA events",
                   "parallelism": f"replicas x{world} (no data-path collective)"},
        "throughput": {"value": world * 1e3 / ms_mixed, "unit": "ground states/s"},
        "E": rep["E"], "mu": rep["mu"], "res": rep["res"],
        "E_fp64": reps_fp64[-1]["E"], "res_fp64": reps_fp64[-1]["res"],
        "c3": c3,
        "solver": {k: rep[k] for k in ("outer_f32", "outer_f64", "inner_f32", "inner_f64", "nfe", "ms_f32", "ms_f64")},
        "roofline": happly, "solve_operator_roofline": roof,
        "autotune": G.autotune_report() + ("".join(f" failed: {e};" for e in AUTOTUNE_ERRORS)),
        "sweep": sweep,
        "cpu_baseline": cpu,
        "e2e": {"value": statistics.mean(e2e), "unit": "s", "h2d_bytes_per_step": nbytes,
                "d2h_bytes_per_step": nbytes},
        "gpu_launches": int((l1 - l0) / max(args.steps, 1)) * args.steps,
        "clocks": clk,
        "profile": {k: [n, round(ms, 4)] for k, (n, ms) in sorted(prof.items(), key=lambda kv: -kv[1][1])[:12]},
    }
    print(json.dumps(line), flush=True)
    phase("the report")
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def profiling_run(args):
    """Small fixed runs for ncu captures (see profiles/)."""
    import torch
    import workloads as W
    import paper_1504_02891_gb300 as G
    G.load()
    if args.only == "happly":
        p = W.config("c4")
        p["n"] = (args.happly_n, args.happly_n)
        plan = G.Plan(p, nbatch=64, prec=G.F32)
        if args.happly_path == 0:
            plan.autotune()
        else:
            G.set_operator_path(args.happly_path)
        psi = plan.empty()
        psi.real.normal_()
        psi.imag.normal_()
        psi.mul_(1e-2)
        out = plan.empty()
        for _ in range(3):
            plan.grad(psi, out)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(10):
            plan.grad(psi, out)
        e1.record()
        torch.cuda.synchronize()
        print(f"happly us/apply {e0.elapsed_time(e1) / 10 * 1e3:.1f}")
    else:
        p = W.config("c2")
        plan = G.Plan(p)
        plan.autotune(levels=3)
        init = G.to_device(W.gaussian(p))
        for _ in range(2):
            t = init.clone()
            rep = plan.solve(t, mode=1, levels=3, res_tol=RES_TOL)
        torch.cuda.synchronize()
        print("solve", rep)


def main():
    args = parse()
    if args.only:
        profiling_run(args)
        return
    if args.impl == "reference":
        reference_arm(args)
    else:
        our_arm(args)


if __name__ == "__main__":
    main()
