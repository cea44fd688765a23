#!/usr/bin/env python
"""Throughput of the sweeping-preconditioned FGMRES solve on one GB300.

Metric: unknowns x RHS solved per second to a true relative residual of 1e-6
(the paper times only the GMRES phase, Section 6; the subdomain factors are
built once, outside the timed region, and their time is reported beside it).

Workload (the configuration the metric is quoted on): 1023 x 1023 grid,
8 x 8 checkerboard (128-node subdomains, the last row/column 127), three-layer
medium with a smooth +-10% random perturbation at 8 points per wavelength,
one Gaussian source; complex64 subdomain factors and preconditioner inside
FP64 flexible GMRES.  One step = one complete solve of that system.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 (torchrun) runs independent replicas, one per GPU (the path does not
exchange data between solves): weak scaling, value = all ranks' work / max time.
"""
from __future__ import annotations

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

METRIC = "unknowns×RHS solved/s to rel. residual 1e-6 (mixed vs FP64, 1 GB300); % of roofline"
UNIT = "unknowns*RHS/s"
WORKLOAD = "plain_mixed"
# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per launch measured by ncu,
# keyed by the kernel source files and the sha256 prefixes they had when it was measured:
# None once a source changes.  The interface stages of one RHS: mean over 36 consecutive
# interface-stage launches of the bench (32 sweep stages in iface_kernel, the residual and
# S stages in iface_sym_kernel), caches left warm (--cache-control none).
NCU_TRAFFIC = {(("k_iface.cu", "4eb8ed015935f074"), ("k_iface_sym.cu", "630bbaa666058470")): 9.716e6}
FP64_PEAK_TFLOPS = 1.25


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--prec", default="c64", choices=["c64", "c128"])
    ap.add_argument("--sched", default="BSP", choices=["BSP", "SP"])
    ap.add_argument("--restart", type=int, default=150)
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--no-fp64-form", action="store_true", help="skip the all-FP64 comparison solve")
    ap.add_argument("--no-habc-form", action="store_true", help="skip the Pade HABC transmission solve")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-iters", type=int, default=2, help="oracle FGMRES iterations per CPU sample")
    ap.add_argument("--cpu-pool", type=int, default=-1,
                    help="worker processes of the all-cores oracle sample (-1: every host core, 0: skip it)")
    ap.add_argument("--mode", default="solve", choices=["solve", "precond", "schedules"],
                    help="precond: factor once, then time --steps preconditioner applications only "
                         "(a small, fixed launch sequence for profilers); schedules: SP vs BSP on 5 x N2 "
                         "checkerboards, N2 = 5, 10, 15, 20 (the shape of Table 1)")
    ap.add_argument("--workload", default=None, choices=["plain_mixed", "batching", "large"],
                    help="the workload to factor (default: the 1023^2 one-source bench workload); solve mode "
                         "reports the oracle baseline for the default workload only")
    ap.add_argument("--nrhs", type=int, default=None,
                    help="right-hand sides (default: the workload's)")
    ap.add_argument("--tensor-cores", default="3xtf32", choices=["3xtf32", "tf32", "off"],
                    help="complex64 multi-RHS block solves (construction of K, batched RHS): tensor cores with "
                         "split TF32 operands, plain TF32, or FP32 on the CUDA cores")
    ap.add_argument("--inner-maxit", type=int, default=300,
                    help="> 0: each preconditioner application solves the interface problem (I - S) g = b by "
                         "FGMRES with the sweep as preconditioner (at most this many steps); 0: one sweep")
    ap.add_argument("--inner-restart", type=int, default=30)
    ap.add_argument("--inner-tol", type=float, default=1e-2)
    ap.add_argument("--sweep", default="stages", choices=["stages", "barrier", "dependency"],
                    help="the sweeps of the interface iterations: stage launches (default), one cooperative launch "
                         "with grid barriers between stages, or one dependency-driven cooperative launch")
    ap.add_argument("--inner-fp64", action="store_true",
                    help="FP64 interface Krylov vectors with complex64 factors (default: complex64 vectors)")
    ap.add_argument("--transmission", default="optimized", choices=["optimized", "habc"],
                    help="interface condition of --mode schedules / precond: the optimized Robin parameter, or the "
                         "Pade HABC (N_pade 8, phi pi/3; base factors with the optimized Robin parameter)")
    ap.add_argument("--tc-scale", type=float, default=0.5,
                    help="scale s of the optimized Robin parameter T_e = (i - 1) s sqrt(kappa_e pi / (2 h))")
    ap.add_argument("--graph", action="store_true",
                    help="replay every preconditioner application from a captured CUDA graph")
    ap.add_argument("--no-autotune", action="store_true",
                    help="fixed launch-shape rules for the interface stages (no autotuner)")
    ap.add_argument("--tc-iface-min-ctas", type=int, default=-1,
                    help="interface stages of fewer CTAs stay on the CUDA cores (-1: two per SM)")
    ap.add_argument("--no-tc-factor", action="store_true",
                    help="complex64 factorisation on the CUDA cores (default: trailing updates on the tensor cores)")
    ap.add_argument("--no-sym-k", action="store_true",
                    help="one-RHS interface stages apply the full K (default: the stages that apply every "
                         "subdomain's whole K stream its packed symmetric tiles)")
    ap.add_argument("--tc-min-rhs", type=int, default=16,
                    help="stages with at least this many RHS run on the tensor cores (1: all)")
    return ap.parse_args()


TC_MODES = {"3xtf32": "3xtf32", "tf32": "tf32", "off": False}


# the oracle's own solve (the CPU baseline and the reference arm): volume FGMRES(150)
# with one sweep per preconditioner application, to 1e-6 (oracle/reference_counts.json)
ORACLE_RESTART = 150


def inner_kw(args):
    """Interface-Krylov options of Problem.solve."""
    return dict(inner_maxit=args.inner_maxit, inner_restart=args.inner_restart, inner_tol=args.inner_tol,
                inner_fp64=args.inner_fp64, persistent={"stages": 0, "barrier": 1, "dependency": 2}[args.sweep])


def precond_only(args):
    """Factor a workload and apply the preconditioner --steps times."""
    import torch

    import workloads as W
    from paper_2209_10886_gb300 import Problem
    name = args.workload or WORKLOAD
    w = W.workload(name, nrhs=args.nrhs) if args.nrhs else W.workload(name)
    m2 = torch.as_tensor(w.m2, dtype=torch.float64, device="cuda")
    p = Problem(w.n, w.n, w.h, w.omega, m2, w.N1, w.N2, w.xcuts, w.ycuts, tensor_cores=TC_MODES[args.tensor_cores],
                tc_min_rhs=args.tc_min_rhs, tc_scale=args.tc_scale, tc_iface_min_ctas=args.tc_iface_min_ctas,
                autotune=not args.no_autotune, transmission=args.transmission, tc_factor=not args.no_tc_factor,
                sym_k=not args.no_sym_k)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    p.factor(args.prec)
    torch.cuda.synchronize()
    factor_ms = (time.perf_counter() - t0) * 1e3
    r = torch.as_tensor(w.f, dtype=torch.complex128, device="cuda")
    from paper_2209_10886_gb300 import helm
    for _ in range(args.warmup):
        p.precond_apply(r, sched=args.sched)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        p.precond_apply(r, sched=args.sched)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(args.steps, 1)
    # the same applications again with library-side events around every stage launch
    helm.profile(p, True)
    for _ in range(args.steps):
        p.precond_apply(r, sched=args.sched)
    torch.cuda.synchronize()
    kern = {}
    for k in ("stage", "trace"):
        n, kms, kb, kf = helm.profile_read(p, k)
        if n:
            kern[k] = {"launches_per_apply": n / args.steps, "ms_per_apply": kms / args.steps,
                       "GB_per_s": kb / (kms / 1e3) / 1e9 if kms else None,
                       "TFLOP_per_s": kf / (kms / 1e3) / 1e12 if kms else None}
    helm.profile(p, False)
    print(json.dumps({"mode": "precond", "workload": name, "nrhs": int(r.shape[0]), "prec": args.prec,
                      "sched": args.sched, "tensor_cores": args.tensor_cores, "factor_ms": factor_ms,
                      "factor_on_tensor_cores": p.factor_on_tensor_cores(),
                      "iface_symmetric": p.iface_symmetric(r.shape[0]),
                      "ms_per_apply": ms, "unknowns_rhs_per_s": w.N * r.shape[0] / (ms / 1e3),
                      "kernels": kern}))
    p.close()


def max_over_ranks(x, world, device):
    """The largest x over the ranks: the job ends when its slowest replica ends."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, world, ms):
    """Units of all replicas per second of the slowest one."""
    return units_per_rank * world / (ms / 1e3)


def schedules(args):
    """SP against BSP on 5 x N2 checkerboards (the shape of the paper's Table 1).

    The 639^2 domain (layered + random medium, 10 points per wavelength, one source
    at (0.5, 0.2)) is cut into 5 columns of 128 nodes (the last 127) and N2 = 5, 10,
    15, 20 rows.  Per schedule: Krylov steps to 1e-6 (ni: the interface FGMRES steps
    when the interface problem is solved iteratively, as in the paper, else the
    volume FGMRES steps), sweep steps per application of the sweep (ns: SP
    2(N1+N2-2), BSP 2 N1, as in Table 1; BSP with non-overlapping bands 2(N1-1))
    and the solve time (t), with t / (ni ns).  Per schedule also the residual
    history of the interface FGMRES (unrestarted, to 1e-6) in one preconditioner
    application (the paper's 'drop at the number of partial sweeps'): its first
    values and the step of the largest one-step decrease.
    """
    import torch

    import workloads as W
    from paper_2209_10886_gb300 import Problem, helm, schedule_info
    n = 639
    rows = []
    for N2 in (5, 10, 15, 20):
        w = W.workload("custom", n=n, N1=5, N2=N2, medium="layered", seed=0, ppw=10.0,
                       xcuts=W.even_cuts(n, 5, 128))
        h = w.h
        f = torch.as_tensor(W.gaussian_source(n, h, (0.5, 0.2), 2 * h)[None, :], dtype=torch.complex128,
                            device="cuda")
        m2 = torch.as_tensor(w.m2, dtype=torch.float64, device="cuda")
        p = Problem(w.n, w.n, w.h, w.omega, m2, w.N1, w.N2, w.xcuts, w.ycuts, transmission=args.transmission,
                    tensor_cores=TC_MODES[args.tensor_cores], tc_scale=args.tc_scale).factor(args.prec)
        row = {"N1xN2": f"5x{N2}"}
        for sched in ("SP", "BSP", "BSP_NONOVERLAP"):
            kw = dict(restart=args.restart, maxit=2000, tol=args.tol, sched=sched, use_graph=args.graph,
                      raise_on_noconv=False, **inner_kw(args))
            p.solve(f, **kw)                                                    # warm-up
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0 = helm.inner_steps(p)
            e0.record()
            _, info, _ = p.solve(f, **kw)
            e1.record()
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1) / 1e3
            outer = info[0][0]
            ni = helm.inner_steps(p) - s0 if args.inner_maxit > 0 else outer
            ns = schedule_info(5, N2, sched)[0]          # SP 2(N1+N2-2), BSP 2 N1, non-overlapping 2(N1-1)
            row[sched] = {"ni": ni, "outer": outer, "ns": ns, "t_s": t, "relres": info[0][1],
                          "converged": info[0][1] <= args.tol, "t_per_ni_ns_ms": 1e3 * t / (max(ni, 1) * ns)}
            # the paper's observation (Section 6, its Fig. 3): in GMRES on the interface
            # problem the residual drops suddenly at the iteration equal to the number of
            # partial sweeps (bands); here the interface FGMRES of the first preconditioner
            # application, unrestarted, to 1e-6 (one outer step)
            p.solve(f, restart=args.restart, maxit=1, tol=args.tol, sched=sched, raise_on_noconv=False,
                    inner_maxit=300, inner_restart=300, inner_tol=1e-6, inner_history=True)
            hist = p.last_inner_history[0]
            ratios = [hist[k] / hist[k - 1] for k in range(1, len(hist)) if hist[k - 1] > 0]
            k_drop = 1 + min(range(len(ratios)), key=lambda k: ratios[k]) if ratios else None
            Ng = 5 + N2 - 1
            nb = -(-(Ng - 1) // 5) if sched == "BSP" else (-(-Ng // 5) if sched == "BSP_NONOVERLAP" else 1)
            row[sched]["interface_history"] = {
                "relres_first_16": [float(f"{v:.3e}") for v in hist[:16]], "steps_to_1e-6": len(hist),
                "largest_drop_at_step": (k_drop + 1) if k_drop is not None else None,
                "largest_drop_ratio": min(ratios) if ratios else None, "bands": nb}
        p.close()
        rows.append(row)
    print(json.dumps({"mode": "schedules", "workload": f"{n}^2 layered+random 10 ppw, 5 x N2, 1 source",
                      "prec": args.prec, "restart": args.restart, "tol": args.tol, "tc_scale": args.tc_scale,
                      "transmission": args.transmission,
                      "interface_krylov": inner_kw(args), "rows": rows}))


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_hash(name="k_stage.cu"):
    src = os.path.join(ROOT, "paper_2209_10886_gb300", "csrc", name)
    return (name, hashlib.sha256(open(src, "rb").read()).hexdigest()[:16])


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- CPU oracle
# The oracle's solve of the bench workload with the bench's own method (the paper's
# formulation: volume FGMRES whose preconditioner solves (I - S) g = b by FGMRES(30) to
# 1e-2 with the BSP sweep as its preconditioner, Robin scale 0.5).  A full oracle solve
# takes minutes, so a sample times one outer FGMRES step with the interface iteration
# capped at k1 and at k2 steps: their difference gives the time per interface step
# (one sweep + one S), the rest the fixed time per outer step (liftings,
# reconstruction, two volume matvecs); the solve time is the oracle's own counts
# (oracle/reference_counts.json) times these.  The single-sweep form (volume
# FGMRES(150), one sweep per application, scale 1.0) is timed per FGMRES iteration.
ORACLE_SAMPLE = r"""
import json, os, sys, time
sys.path.insert(0, {root!r})
import numpy as np
import workloads as W
from oracle import Decomposition, Sweeper, assemble_operator, fgmres
w = W.workload({workload!r})
A = assemble_operator(w.n, w.h, w.omega, w.m2)
scale = {scale}
dec = Decomposition(w.n, w.h, w.omega, w.m2, w.xcuts, w.ycuts, tc_scale=scale)
P = {pool}
t0 = time.perf_counter()
if P > 1:
    from oracle.parallel import PoolSweeper
    sw = PoolSweeper(dec, (w.n, w.h, w.omega, w.m2, w.xcuts, w.ycuts), dict(tc_scale=scale), processes=P)
else:
    sw = Sweeper(dec)
    for i in dec.subdomains:
        dec.local_solver(i)
t_factor = time.perf_counter() - t0
b = w.h ** 2 * w.f[0]
out = dict(t_factor=t_factor, samples=[])
for rep in range({reps}):
    if {method!r} == "interface":
        t = []
        for k in ({k1}, {k2}):
            t0 = time.perf_counter()
            fgmres(lambda v: A @ v, lambda v: sw.precondition_interface_krylov(v, {sched!r}, tol=1e-2, restart=30,
                                                                               maxit=k), b, tol=1e-300, restart=1,
                   maxit=1)
            t.append(time.perf_counter() - t0)
        step = (t[1] - t[0]) / ({k2} - {k1})
        out["samples"].append(dict(t_step=step, t_outer=t[0] - {k1} * step, t_k=t))
    else:
        t0 = time.perf_counter()
        x, it, rr = fgmres(lambda v: A @ v, lambda v: sw.precondition(v, {sched!r}), b, tol=1e-300,
                           restart={restart}, maxit={iters})
        out["samples"].append(dict(t_iter=(time.perf_counter() - t0) / it))
print(json.dumps(out))
if P > 1:
    sw.close()
"""
K1, K2 = 1, 3                    # interface steps of the two samples


def oracle_counts(sched, method):
    """The oracle's own iteration counts on the bench workload: (outer FGMRES steps,
    interface steps summed over the applications or None, source), or Nones."""
    p = os.path.join(ROOT, "oracle", "reference_counts.json")
    key = f"{sched}_interface_krylov_restart150" if method == "interface" else f"{sched}_restart{ORACLE_RESTART}"
    try:
        e = json.load(open(p))[WORKLOAD][key]
        return int(e["iterations"]), e.get("interface_steps"), f"oracle to 1e-6, oracle/reference_counts.json [{key}]"
    except Exception:
        return None, None, None


def run_oracle_sample(sched, method, reps=1, pool=1, iters=2, timeout=1800):
    """Time the oracle on the bench workload in a CPU-only child process: one thread
    (pool = 1), or its local solves spread over `pool` worker processes (oracle.parallel,
    one thread each).  method: "interface" (the bench's method) or "single"."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    env["CUDA_VISIBLE_DEVICES"] = ""
    code = ORACLE_SAMPLE.format(root=ROOT, workload=WORKLOAD, sched=sched, restart=max(ORACLE_RESTART, iters),
                                iters=iters, reps=reps, pool=int(pool), method=method, k1=K1, k2=K2,
                                scale=0.5 if method == "interface" else 1.0)
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=timeout)
    if r.returncode != 0:
        raise RuntimeError("oracle sample failed: " + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def oracle_solve_time(sched, sample):
    """Extrapolated oracle solve time (s) of the interface-Krylov method from one sample,
    and a description of the extrapolation."""
    outer, inner, src = oracle_counts(sched, "interface")
    if outer is None:
        return None, "no recorded oracle counts"
    t = outer * sample["t_outer"] + inner * sample["t_step"]
    return t, (f"{outer} outer steps x {sample['t_outer']:.3f} s + {inner} interface steps x "
               f"{sample['t_step']:.3f} s ({src})")


# ------------------------------------------------------------------- arms
def reference_arm(args):
    """The oracle, as it stands, on the bench's workload, method and metric (the paper has no
    code: the oracle is the reference).  Each step is one bounded sample (one outer step at
    two interface-iteration caps); the value extrapolates the oracle's own counts."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import workloads as W
    w = W.workload(WORKLOAD)
    res = run_oracle_sample(args.sched, "interface", reps=args.warmup + args.steps)
    timed = res["samples"][args.warmup:] or res["samples"]
    sample = {k: statistics.median(s[k] for s in timed) for k in ("t_step", "t_outer")}
    t_solve, how = oracle_solve_time(args.sched, sample)
    if t_solve is None:
        print(json.dumps({"impl": "reference", "unavailable": "no recorded oracle iteration counts"}))
        return
    value = w.N * w.nrhs / t_solve
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_solve * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
        "config": {"workload": w.description, "n": w.n, "N1": w.N1, "N2": w.N2, "nrhs": w.nrhs,
                   "sched": args.sched, "restart": 150, "tol": args.tol, "transmission": "optimized, scale 0.5",
                   "method": "oracle volume FGMRES(150) with the interface problem solved by FGMRES(30) to 1e-2 "
                             "with the sweep as preconditioner (the GPU arm's method)",
                   "extrapolation": how},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"per step one outer FGMRES step of the oracle with the interface iteration "
                                   f"capped at {K1} and at {K2} steps (scipy splu local solves, one thread; "
                                   f"{len(os.sched_getaffinity(0))} host cores available); solve time "
                                   f"extrapolated: {how}; factorisation {res['t_factor']:.1f} s excluded like on "
                                   f"the GPU"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def habc_form(args, w, m2, f, ms, st, err_vs_oracle):
    """The paper's transmission (Pade HABC, N_pade = 8, phi = pi/3, Sections 3 and 6) on the
    same workload and method: factors with the optimized Robin condition plus the HABC
    boundary maps; one warm solve, one timed.  Runs after the main problem is released."""
    import torch
    from paper_2209_10886_gb300 import Problem, helm
    qh = Problem(w.n, w.n, w.h, w.omega, m2, w.N1, w.N2, w.xcuts, w.ycuts, transmission="habc",
                 tc_scale=args.tc_scale, tensor_cores=TC_MODES[args.tensor_cores], tc_factor=not args.no_tc_factor)
    try:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        qh.factor(args.prec)
        torch.cuda.synchronize()
        hfac = (time.perf_counter() - t0) * 1e3
        hkw = dict(restart=args.restart, maxit=3000, tol=args.tol, sched=args.sched, use_graph=args.graph,
                   **inner_kw(args))
        qh.solve(f, **hkw)
        torch.cuda.synchronize()
        h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0 = helm.inner_steps(qh)
        h0.record(st)
        uh_, ih, _ = qh.solve(f, **hkw)
        h1.record(st)
        torch.cuda.synchronize()
        msh = h0.elapsed_time(h1)
        return {"value": w.N * w.nrhs / (msh / 1e3), "ms_per_step": msh, "iterations": ih[0][0],
                "interface_steps": helm.inner_steps(qh) - s0, "relres": max(i[1] for i in ih),
                "err_vs_oracle": err_vs_oracle(uh_.cpu().numpy()), "factor_ms": hfac,
                "transmission": "Pade HABC, N_pade 8, phi pi/3 (base factors: optimized Robin, scale "
                                f"{args.tc_scale:g})", "speedup_over_robin": ms / msh}
    except helm.HelmError as e:
        return {"error": str(e)[:300]}
    finally:
        qh.close()


def gpu_arm(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import workloads as W
    from paper_2209_10886_gb300 import Problem, helm

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    def barrier():
        if world > 1:
            dist.barrier()

    wname = args.workload or WORKLOAD
    w = W.workload(wname, nrhs=args.nrhs) if args.nrhs else W.workload(wname)
    m2 = torch.as_tensor(w.m2, dtype=torch.float64, device=dev)
    f = torch.as_tensor(w.f, dtype=torch.complex128, device=dev)
    p = Problem(w.n, w.n, w.h, w.omega, m2, w.N1, w.N2, w.xcuts, w.ycuts, tensor_cores=TC_MODES[args.tensor_cores],
                tc_min_rhs=args.tc_min_rhs, tc_scale=args.tc_scale, tc_iface_min_ctas=args.tc_iface_min_ctas,
                autotune=not args.no_autotune, tc_factor=not args.no_tc_factor, sym_k=not args.no_sym_k)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    p.factor(args.prec)
    torch.cuda.synchronize()
    factor_ms = (time.perf_counter() - t0) * 1e3
    st = torch.cuda.current_stream()
    u = torch.empty_like(f)

    def solve():
        _, info, _ = p.solve(f, u=u, restart=args.restart, maxit=3000, tol=args.tol, sched=args.sched, use_graph=args.graph, **inner_kw(args))
        return info[0]

    for _ in range(args.warmup):
        info = solve()
    # timed region: the solves as a user runs them (no per-launch profiling events, so the
    # interface Arnoldi steps run as device-driven graph loops)
    clocks = ClockSampler(local)
    clocks.start()
    l0 = helm.launch_count()
    s0 = helm.inner_steps(p)
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    iters = []
    for _ in range(args.steps):
        info = solve()
        iters.append(info)
    e1.record(st)
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1) / args.steps
    launches = helm.launch_count() - l0
    inner_per_solve = (helm.inner_steps(p) - s0) / args.steps
    clk = clocks.stop()
    # second timed pass of the same solves with CUDA events around every launch (the
    # host-driven interface loop): per-class kernel time and the live roofline
    helm.profile(p, True)
    torch.cuda.synchronize()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(st)
    for _ in range(args.steps):
        solve()
    p1.record(st)
    torch.cuda.synchronize()
    ms_prof = p0.elapsed_time(p1) / args.steps
    stage = helm.profile_read(p, "stage")
    trace = helm.profile_read(p, "trace")
    matv = helm.profile_read(p, "matvec")
    orth = helm.profile_read(p, "ortho")
    helm.profile(p, False)
    ms = max_over_ranks(ms, world, dev)
    relres = info[1]

    # true residual on the host with the oracle's sparse matrix (property check at full size),
    # and the error against the oracle's sparse direct solution of the global system (outside
    # the timed region; rank 0, the first RHS)
    check = None
    exact = None
    u_main = u.cpu().numpy()
    if rank == 0:
        from oracle import assemble_operator
        from oracle.discretization import GridDirectSolver
        A = assemble_operator(w.n, w.h, w.omega, w.m2)
        bh = w.h ** 2 * w.f[0]
        check = float(np.linalg.norm(bh - A @ u_main[0]) / np.linalg.norm(bh))
        if w.n <= 1600:
            exact = GridDirectSolver(A, w.n).solve(bh)

    def err_vs_oracle(uu):
        if exact is None:
            return None
        return float(np.linalg.norm(uu[0] - exact) / np.linalg.norm(exact))

    # end to end through the public API with host buffers
    fh = torch.empty(f.shape, dtype=f.dtype, pin_memory=True)
    fh.copy_(torch.as_tensor(w.f))
    uh_pinned = torch.empty_like(fh, pin_memory=True)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        fd = fh.to(dev, non_blocking=True)
        ud, info2, _ = p.solve(fd, restart=args.restart, maxit=3000, tol=args.tol, sched=args.sched, use_graph=args.graph, **inner_kw(args))
        uh_pinned.copy_(ud, non_blocking=True)
        torch.cuda.synchronize()
    e2e_ms = max_over_ranks((time.perf_counter() - t0) * 1e3 / args.steps, world, dev)

    # the paper's other schedule (symmetric Gauss-Seidel sweeps, Section 4) on the same factors
    sp_form = usp = None
    if args.sched == "BSP" and not args.no_fp64_form:
        _, isp, _ = p.solve(f, restart=args.restart, maxit=3000, tol=args.tol, sched="SP", use_graph=args.graph, **inner_kw(args))    # warm
        torch.cuda.synchronize()
        b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        b0.record(st)
        usp, isp, _ = p.solve(f, restart=args.restart, maxit=3000, tol=args.tol, sched="SP", use_graph=args.graph, **inner_kw(args))
        b1.record(st)
        torch.cuda.synchronize()
        mssp = b0.elapsed_time(b1)
        sp_form = {"value": w.N * w.nrhs / (mssp / 1e3), "ms_per_step": mssp, "iterations": isp[0][0],
                   "relres": isp[0][1], "err_vs_oracle": err_vs_oracle(usp.cpu().numpy()),
                   "sweep_steps_per_application": {"SP": 2 * (w.N1 + w.N2 - 2), "BSP": 2 * w.N1}}

    # the all-FP64 form on the same GPU (one solve), for the mixed-vs-FP64 speedup
    fp64 = q = u64 = None
    if not args.no_fp64_form and args.prec == "c64":
        q = Problem(w.n, w.n, w.h, w.omega, m2, w.N1, w.N2, w.xcuts, w.ycuts, tc_scale=args.tc_scale)
        try:
            q.factor("c128")
        except helm.HelmError as e:
            # the complex128 factors of the largest workloads do not fit beside the complex64 ones
            if e.status != 3:
                raise
            q.close()
            q = None
            fp64 = {"unavailable": "the complex128 factors do not fit in device memory beside the complex64 ones: "
                                   + str(e)[:200]}
    if fp64 is None and q is not None:
        _, i64, _ = q.solve(f, restart=args.restart, maxit=3000, tol=args.tol, sched=args.sched, use_graph=args.graph, **inner_kw(args))  # warm
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(st)
        u64, i64, _ = q.solve(f, restart=args.restart, maxit=3000, tol=args.tol, sched=args.sched, use_graph=args.graph, **inner_kw(args))
        a1.record(st)
        torch.cuda.synchronize()
        ms64 = a0.elapsed_time(a1)
        fp64 = {"value": w.N * w.nrhs / (ms64 / 1e3), "ms_per_step": ms64, "iterations": i64[0][0],
                "relres": i64[0][1], "err_vs_oracle": err_vs_oracle(u64.cpu().numpy()),
                "speedup_mixed_over_fp64": ms64 / ms}
        q.close()

    if rank != 0:
        return
    total_units = w.N * w.nrhs * world
    value = job_throughput(w.N * w.nrhs, world, ms)
    peak, peak_src = peaks()
    achieved = stage[2] / (stage[1] / 1e3) / 1e9 if stage[1] > 0 else 0.0
    traffic = NCU_TRAFFIC.get(kernel_hash())
    stage_roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                  "traffic": traffic, "kernel": "stage_kernel (block-tridiagonal solves + transmission)",
                  "launches": stage[0], "peak_source": f"hbm_gbs of {peak_src}"}
    # the dominant kernel class by live event time
    classes = {"stage": stage, "trace": trace, "matvec": matv, "ortho": orth}
    dom = max(classes, key=lambda k: classes[k][1])
    if dom == "ortho":
        tf = orth[3] / (orth[1] / 1e3) / 1e12
        roofline = {"bound": "alu", "achieved": tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": tf / FP64_PEAK_TFLOPS, "traffic": None,
                    "kernel": "mgs_kernel (FP64 modified Gram-Schmidt, one persistent launch per Arnoldi step)",
                    "launches": orth[0],
                    "peak_source": "FP64 1.25 TFLOP/s nominal (152 SMs x 2 FP64 FMA/clk x 2.07 GHz); "
                                   "cuBLAS DGEMM measured 1.10 TFLOP/s on GB300"}
    elif dom == "stage":
        roofline = stage_roof
    else:
        st_ = classes[dom]
        bw = st_[2] / (st_[1] / 1e3) / 1e9
        names = {"trace": "iface_kernel (boundary-operator GEMV + transmission)", "matvec": "matvec_kernel"}
        tc_form = helm.iface_shape(p, w.nrhs)["tensor_cores"] != 0
        if tc_form:
            names["trace"] = ("iface_kernel (CUDA-core GEMV, the smaller stages) + tc_iface_kernel "
                              "(tcgen05 GEMM, the stages that fill the GPU)")
        sym_form = p.iface_symmetric(w.nrhs)
        if sym_form:
            names["trace"] = ("iface_kernel (the sweep stages: boundary-operator GEMV + transmission) + "
                              "iface_sym_kernel (the stages over every subdomain's whole K: packed symmetric "
                              "tiles streamed by bulk copies, each counted once)")
        # the ncu traffic figure belongs to the 1-RHS default workload it was captured on
        same_capture = dom == "trace" and wname == WORKLOAD and w.nrhs == 1 and not tc_form and sym_form
        key = (kernel_hash("k_iface.cu"), kernel_hash("k_iface_sym.cu"))
        roofline = {"bound": "hbm", "achieved": bw, "peak": peak, "unit": "GB/s", "frac": bw / peak,
                    "traffic": NCU_TRAFFIC.get(key) if same_capture else None,
                    "algorithmic_bytes_per_launch": st_[2] / max(st_[0], 1),
                    "kernel": names.get(dom, dom), "launches": st_[0],
                    "peak_source": f"hbm_gbs of {peak_src}"}
    cpu = cpu_pool = cpu_single = None
    ncores = len(os.sched_getaffinity(0))
    npool = ncores if args.cpu_pool < 0 else args.cpu_pool
    if not args.no_cpu_baseline and world == 1 and wname == WORKLOAD and not args.nrhs and args.inner_maxit > 0:
        # the oracle with the GPU's method: one thread, then its local solves over npool processes
        for P in [1] + ([npool] if npool >= 2 else []):
            if P > 1 and (cpu is None or not cpu.get("value")):
                continue
            try:
                res = run_oracle_sample(args.sched, "interface", pool=P, timeout=600)
                t_solve, how = oracle_solve_time(args.sched, res["samples"][-1])
                where = ("one thread" if P == 1 else
                         f"local solves over {P} worker processes of one thread (oracle.parallel, subdomain i on "
                         f"worker i mod {P})")
                entry = {"value": w.N * w.nrhs / t_solve if t_solve else None, "unit": UNIT, "cores": P,
                         "kind": "oracle", "method": "interface-Krylov (the GPU line's method)",
                         "sample": f"one outer FGMRES step of the oracle with the interface iteration capped at "
                                   f"{K1} and at {K2} steps ({where}; {ncores} host cores available), "
                                   f"extrapolated: {how}"}
            except Exception as e:  # the baseline must not hide the GPU line
                entry = {"value": None, "unit": UNIT, "cores": P, "kind": "oracle", "sample": f"failed: {e}"[:300]}
            if P == 1:
                cpu = entry
            else:
                cpu_pool = entry
        # the single-sweep form of the oracle (volume FGMRES(150), one sweep per application), for reference
        try:
            res = run_oracle_sample(args.sched, "single", iters=args.cpu_iters)
            t_iter = res["samples"][-1]["t_iter"]
            ni, _, src = oracle_counts(args.sched, "single")
            cpu_single = {"value": w.N * w.nrhs / (t_iter * ni) if ni else None, "unit": UNIT, "cores": 1,
                          "kind": "oracle", "method": "volume FGMRES(150), one sweep per application, scale 1.0",
                          "sample": f"{args.cpu_iters} oracle FGMRES iterations (one thread): {t_iter:.3f} s per "
                                    f"iteration x {ni} iterations ({src})"}
        except Exception as e:
            cpu_single = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": f"failed: {e}"[:300]}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c64+f64" if args.prec == "c64" else "c128", "data": "synthetic",
        "config": {
            "workload": w.description, "n": w.n, "N1": w.N1, "N2": w.N2, "nrhs": w.nrhs, "unknowns": w.N,
            "prec": args.prec, "sched": args.sched, "restart": args.restart, "tol": args.tol,
            "transmission": f"optimized, scale {args.tc_scale:g}", "iterations": iters[-1][0], "relres": relres,
            "tensor_cores": args.tensor_cores, "tc_min_rhs": args.tc_min_rhs,
            "tc_iface_min_ctas": args.tc_iface_min_ctas, "cuda_graph": args.graph,
            "interface_krylov": ({"inner_maxit": args.inner_maxit, "inner_restart": args.inner_restart,
                                  "inner_tol": args.inner_tol, "inner_steps_per_solve": inner_per_solve,
                                  "vectors": "c128" if (args.inner_fp64 or args.prec == "c128") else "c64",
                                  "sweep": {"stages": "stage launches (programmatic dependencies)",
                                            "barrier": "one cooperative launch, grid barriers",
                                            "dependency": "one cooperative launch, per-item dependencies"}[args.sweep]}
                                 if args.inner_maxit > 0 else None),
            "relres_host_check": check,
            "factor_on_tensor_cores": p.factor_on_tensor_cores(),
            "iface_symmetric": p.iface_symmetric(w.nrhs),
            "err_vs_oracle": err_vs_oracle(u_main),
            "err_vs_oracle_note": ("rel. L2 of the first RHS's solution (tol above) against the oracle's sparse "
                                   "direct solution of the global system (nested-dissection LU + refinement)"),
            "factor_ms": factor_ms, "factor_bytes": p.info()["factor_bytes"],
            "l2": (f"inputs larger than L2: every timed solve streams the {p.info()['factor_bytes'] / 1e9:.2f} GB "
                   "of factors in each lifting and reconstruction, so no solve starts with a warm L2 (within a "
                   "solve the boundary operators are reused across the interface iterations)"),
            "parallelism": f"replicas x{world}",
            "iface_shape": helm.iface_shape(p, w.nrhs),
            "stage_shape": helm.stage_shape(p, w.nrhs),
            "profiled_pass": {"ms_per_step": ms_prof,
                              "note": "the same solves again with CUDA events around every launch (host-driven "
                                      "interface loop); kernel_time_ms_per_step and the roofline come from it"},
            "kernel_time_ms_per_step": {"stage": stage[1] / args.steps, "trace": trace[1] / args.steps,
                                        "matvec": matv[1] / args.steps, "ortho": orth[1] / args.steps},
            "launches_per_step": {"stage": stage[0] / args.steps, "trace": trace[0] / args.steps},
            "fp64_form": fp64,
            "sp_schedule": sp_form,
            "habc_form": None,
        },
        "roofline": roofline,
        "roofline_stage_kernel": stage_roof,
        "clocks": clk,
        "e2e": {"value": job_throughput(w.N * w.nrhs, world, e2e_ms), "unit": UNIT, "h2d_bytes_per_step": int(f.numel() * 16),
                "d2h_bytes_per_step": int(f.numel() * 16)},
        "gpu_launches": launches,
        "cpu_baseline": cpu,
        "cpu_baseline_all_cores": cpu_pool,
        "cpu_baseline_single_sweep": cpu_single,
    }
    p.close()
    # the HABC form sizes its RHS chunks by the free device memory: release the main solves' vectors
    u = fd = ud = usp = u64 = None
    torch.cuda.empty_cache()
    if not args.no_habc_form:
        line["config"]["habc_form"] = habc_form(args, w, m2, f, ms, st, err_vs_oracle)
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
    elif args.mode == "precond":
        precond_only(args)
    elif args.mode == "schedules":
        schedules(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
