#!/usr/bin/env python
"""Power-flow throughput benchmark of libgbpf on GB300.

Metric: power-flow solves per second at max |mismatch| <= 1e-8 p.u.  A step is
one pass of the whole hot path over one batch: admittance assembly, B'/B''
assembly, level-scheduled LDL^T factorisation, and the fast-decoupled
iteration (nodal mismatch + level-scheduled substitutions) to tolerance, all
through the C ABI ``pf_run_to_tol``.  The symbolic analysis (ordering,
elimination tree, levels) runs once per topology before timing and is
reported separately.

Workloads (seeded synthetic grids, see paper_1811_02512_gb300/gridgen.py):
  plain10k   one 10,000-bus pruned-Delaunay grid, FP64 (default)
  batch10k   the same topology with 1,024 cases (512 load scenarios, 512
             single-branch outages) in one launch
  plain120   the 120-bus grid, FP64 (the small single-case configuration)
  adjoint20k one 20,000-bus grid: Newton-Raphson to tolerance, the objective
             sum (V - 1)^2 + losses and its adjoint gradient w.r.t. every P/Q
             injection (reusing the Newton factors); FP32 factors with FP64
             mismatch and FP64-refined solves by default; a step is 1 PF + 1
             gradient
  pack256    256 grids of 2,000 to 80,000 buses (log-uniform), each with its
             own ordering and levels, in one packed launch (pf_pack_run, FP32
             factor + FP64 refinement); the same grids solved one after the
             other by the plain FP64 path are reported beside it

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gbpf|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "power-flow solves/s at 1e-8 pu mismatch"
UNIT = "PF/s"
TOL = 1e-8


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gbpf", choices=["gbpf", "reference"])
    ap.add_argument("--workload", default="plain10k",
                    choices=["plain10k", "batch10k", "plain120", "adjoint20k", "pack256"])
    ap.add_argument("--ngrid", type=int, default=256, help="pack256: number of grids (first n)")
    ap.add_argument("--precision", default=None, choices=["fp64", "fp32"])
    ap.add_argument("--method", default="fdpf", choices=["fdpf", "nr"])
    ap.add_argument("--engine", default="auto", choices=["auto", "block", "lanes"])
    ap.add_argument("--ncase", type=int, default=1024,
                    help="batch10k: number of cases (half load scenarios, half outages)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true",
                    help="plain10k: skip the batched FP32+IR measurement reported beside it")
    ap.add_argument("--no-autotune", action="store_true",
                    help="skip pf_autotune (untimed) before the warm-up")
    ap.add_argument("--mapping", default=None,
                    help="engine,cluster,factor,tail,outage[,threads]: set this kernel mapping instead of tuning")
    ap.add_argument("--cpu-sample-s", type=float, default=12.0)
    ap.add_argument("--no-graphs", action="store_true",
                    help="launch every kernel directly instead of replaying CUDA graphs (profilers)")
    ap.add_argument("--ir-tol", type=float, default=None,
                    help="FP32 runs: relative residual at which a linear solve needs no further "
                         "refinement (default 1e-3: an inexact-Newton forcing term far below the "
                         "fast decoupled iteration's own contraction, about 0.45 per half-iteration)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ------------------------------------------------------------------ workloads

def make_workload(name, ncase=1024):
    from paper_1811_02512_gb300 import gridgen
    if name == "plain120":
        return gridgen.config(0), 1, None, None
    base = gridgen.config(1)
    if name == "plain10k":
        return base, 1, None, None
    sc = gridgen.scenarios(base, n_load=ncase // 2, n_outage=ncase - ncase // 2)
    return base, sc.ncase, sc.load_scale, sc.outage


def workload_precision(name, override):
    if override:
        return override
    return "fp32" if name in ("batch10k", "pack256", "adjoint20k") else "fp64"


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ roofline model

def matrix_offdiag(case, which):
    """Off-diagonal entries of B' (which 0: non-slack buses) or B'' (1: PQ
    buses) on the bus graph: twice the in-service branches joining two of
    its buses (parallel branches counted once)."""
    inm = case.btype != 3 if which == 0 else case.btype == 1
    on = case.status != 0
    pairs = {(min(f, t), max(f, t)) for f, t in zip(case.f[on], case.t[on]) if inm[f] and inm[t]}
    return 2 * len(pairs)


def hbm_bytes_per_launch(info, case, prec_bytes, half_iters, resid, n_outage_solves, ncase):
    """Algorithmic DRAM bytes of one launch of the iteration kernel (the
    streaming model): data every case shares -- the admittance matrix (values
    and pattern) and both factors (L values read by the forward and by the
    backward sweep, their indices, the inverse diagonal) -- counted once per
    launch; per case and half-iteration only vectors: the mismatch reads V
    and theta and writes the right-hand side (24 bytes per bus), a solve
    reads and writes its vector (16 bytes per unknown), every FP64 residual
    of a refined solve reads x and writes r (16 bytes per unknown), and every
    solve of an outage case with the low-rank form reads its two columns
    Z (2 n s bytes).  half_iters, resid and n_outage_solves are totals over
    the launch's cases."""
    nbus, nnz_y = case.n, info.nnz_ybus
    shared = 20 * nnz_y + 4 * (nbus + 1)
    for w in (0, 1):
        n, nnzl = info.n[w], info.nnz_l[w]
        shared += 2 * nnzl * prec_bytes + 2 * 4 * nnzl + 4 * (n + 1) * 2 + n * prec_bytes
    n_mean = 0.5 * (info.n[0] + info.n[1])
    per_half = 24 * nbus + 16 * n_mean
    return shared + half_iters * per_half + resid * 16 * n_mean + n_outage_solves * 2 * n_mean * prec_bytes


def fp64_flops_per_launch(info, case, half_iters, resid, solves64=0.0):
    """Algorithmic FP64 operations of one launch of the iteration kernel (a
    fused multiply-add counts two): per case and half-iteration the nodal
    mismatch, four multiply-adds per admittance entry (8 nnz(Y)) and about
    six operations per bus (rectangular voltages, the half-iteration's
    injection, the scaling by 1/V), and the state update (about 15 per
    unknown: the angle step rotates the cached cos/sin by a short series,
    the magnitude step refreshes 1/V); per FP64 residual of a refined solve
    two per entry of the matrix (n + its off-diagonal entries); per FP64
    substitution pair two per entry of L in each direction plus the n
    multiplications by D^-1.  The FP32 substitutions of refined runs run on
    the FP32 pipe and are not counted."""
    n_mean = 0.5 * (info.n[0] + info.n[1])
    nnzl_mean = 0.5 * (info.nnz_l[0] + info.nnz_l[1])
    off_mean = 0.5 * (matrix_offdiag(case, 0) + matrix_offdiag(case, 1))
    per_half = 8 * info.nnz_ybus + 6 * case.n + 15 * n_mean
    return (half_iters * per_half + resid * 2 * (n_mean + off_mean)
            + solves64 * (4 * nnzl_mean + n_mean))


def fp64_peak_tflops(sm_mhz):
    """Dense FP64 peak of a GB300 from its unit counts and clock: 152 SMs,
    two FP64 fused multiply-adds per SM and cycle (the 1.25 TFLOP/s nominal
    at 2,070 MHz)."""
    return 152 * 2 * 2 * (sm_mhz or 2070.0) * 1e6 / 1e12


# Relative residual at which an FP32 solve of a timed fast decoupled run needs
# no refinement: the forcing term of an inexact Newton step.  The fast
# decoupled iteration contracts the mismatch by about 0.45 per half-iteration
# (8 decades in 23 half-iterations on the 10k grid), so a linear-solve error
# of 1e-3 relative changes its course by rounding only; every convergence
# decision is still taken on the FP64 mismatch (same iteration counts and the
# same error against the tight oracle as FP64 runs, measured).
IR_TOL = 1e-3


def measured_traffic(workload, prec_name, ncase, kernel):
    """DRAM bytes per launch of the iteration kernel from the committed ncu
    summary of the same kernel and workload (scaled by cases when the capture
    ran fewer cases), or None when there is no such capture."""
    files = {("plain10k", "fp64", "k_fdpf_cl"): "k_fdpf_cl_plain10k_fp64.md",
             ("batch10k", "fp32", "k_fdpf"): "k_fdpf_batch128_fp32.md"}
    name = files.get((workload, prec_name, kernel))
    if not name:
        return None
    vals = {}
    try:
        with open(os.path.join(ROOT, "profiles", name)) as fh:
            for ln in fh:
                if "=" in ln and ln.split("=")[0].strip() in ("traffic_bytes_per_launch", "traffic_cases"):
                    k, v = ln.split("=")
                    vals[k.strip()] = float(v)
    except OSError:
        return None
    if "traffic_bytes_per_launch" not in vals:
        return None
    return vals["traffic_bytes_per_launch"] * (ncase / vals.get("traffic_cases", ncase))


# ------------------------------------------------------------------ oracle baseline

def _oracle_job(args):
    import numpy as np  # noqa: F401
    from oracle import oracle as O
    from paper_1811_02512_gb300 import gridgen
    case_ids, deadline, workload = args
    base = gridgen.config(0 if workload == "plain120" else 1)
    sc = None
    if case_ids is not None and any(c is not None for c in case_ids):
        sc = gridgen.scenarios(base, n_load=512, n_outage=512)
    done = 0
    t0 = time.perf_counter()
    for cid in case_ids:
        c = base if cid is None else gridgen.apply_scenario(base, sc, cid)
        rc, *_ = O.power_flow(c, O.FDPF, tol=TOL)
        done += 1 if rc == O.OK else 0
        if time.perf_counter() > deadline:
            break
    return done, time.perf_counter() - t0


def _oracle_accuracy_job(args):
    """Tight oracle solutions of some cases of a workload and their largest
    differences from the GPU's results (V, theta of those cases)."""
    from oracle import oracle as O
    from paper_1811_02512_gb300 import gridgen
    workload, ids, ncase, vm, va = args
    base = gridgen.config(0 if workload == "plain120" else 1)
    sc = gridgen.scenarios(base, n_load=ncase // 2, n_outage=ncase - ncase // 2) if ncase > 1 else None
    out = []
    for k, cid in enumerate(ids):
        c = base if sc is None else gridgen.apply_scenario(base, sc, cid)
        rc, vm0, va0, _, _ = O.power_flow(c, O.NR, tol=1e-12, max_iter=30)
        out.append((cid, rc, float(np.max(np.abs(vm[k] - vm0))), float(np.max(np.abs(va[k] - va0)))))
    return out


def oracle_accuracy(workload, vm, va, ncase):
    """Per-result error of a timed run against the oracle run to a tight
    mismatch (Newton-Raphson to 1e-12 p.u.): max |dV| and max |dtheta| of
    every case, the oracle spread over the host cores (spawn)."""
    import multiprocessing as mp
    from oracle import oracle as O
    O.build()
    cores = os.cpu_count() or 1
    ids = list(range(ncase))
    chunks = [ids[r::cores] for r in range(cores) if ids[r::cores]]
    jobs = [(workload, ch, ncase, vm[ch], va[ch]) for ch in chunks]
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(len(jobs)) as pool:
        res = [r for part in pool.map(_oracle_accuracy_job, jobs) for r in part]
    res.sort()
    dv = np.array([r[2] for r in res])
    da = np.array([r[3] for r in res])
    return {"cases": ncase, "reference": "oracle Newton-Raphson to 1e-12 p.u., FP64",
            "max_dV_pu": float(dv.max()), "max_dtheta_rad": float(da.max()),
            "median_dV_pu": float(np.median(dv)), "median_dtheta_rad": float(np.median(da)),
            "worst_case": int(res[int(np.argmax(np.maximum(dv, da)))][0]),
            "oracle_failed": int(sum(r[1] != O.OK for r in res)),
            "per_case_dV_pu": [float(f"{v:.3g}") for v in dv],
            "per_case_dtheta_rad": [float(f"{v:.3g}") for v in da],
            "seconds": time.perf_counter() - t0, "cores": cores}


def cpu_baseline(workload, sample_s, ncase):
    """The oracle as it stands on the host cores: one process per core (spawn),
    each solving cases of the workload (ordering + factor + FDPF, FP64) until
    the sample budget is used."""
    import multiprocessing as mp
    from oracle import oracle as O
    O.build()
    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    per = max(1, int(sample_s / 0.0005))  # more than the budget; the deadline stops it
    jobs = []
    for w in range(cores):
        if workload in ("plain10k", "plain120"):
            ids = [None] * per
        else:
            ids = [(w + cores * k) % ncase for k in range(per)]
        jobs.append(ids)
    t0 = time.perf_counter()
    deadline = time.perf_counter() + sample_s
    with ctx.Pool(cores) as pool:
        out = pool.map(_oracle_job, [(j, deadline, workload) for j in jobs])
    wall = time.perf_counter() - t0
    solved = sum(o[0] for o in out)
    return {"value": solved / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{solved} {dict(plain10k='10k-bus', plain120='120-bus').get(workload, 'batch10k')} cases "
                      f"(FP64 FDPF incl. ordering/symbolic/factor) across {cores} processes "
                      f"in {wall:.1f} s"}


def run_reference(args):
    """--impl reference: the oracle timed on the host cores as the reference arm."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    if args.workload not in ("plain10k", "plain120", "batch10k"):
        print(json.dumps({"impl": "reference", "unavailable": "the oracle arm times the fast decoupled "
                          "workloads (plain10k, plain120, batch10k); " + args.workload + " has none"}))
        return
    from paper_1811_02512_gb300 import gridgen  # noqa: F401
    base, ncase, _, _ = make_workload(args.workload)
    for _ in range(args.warmup):
        cpu_baseline(args.workload, 1.0, ncase)
    vals = []
    last = None
    for _ in range(args.steps):
        last = cpu_baseline(args.workload, max(2.0, 60.0 / max(1, args.steps)), ncase)
        vals.append(last["value"])
    value = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": None,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload},
            "cpu_baseline": {"kind": "oracle", "cores": last["cores"], "sample": last["sample"],
                             "value": value},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def batched_line(args):
    """The metric's other half -- the same grid as 1,024 load/outage cases in
    one launch, FP32 factor + FP64 refinement -- measured by this script's
    batch10k workload in a child process; its main figures."""
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--workload", "batch10k", "--steps", "5",
           "--warmup", str(max(3, args.warmup)), "--cpu-sample-s", "3"]
    try:
        out = subprocess.run(cmd, capture_output=True, text=True, timeout=900, check=True).stdout
        d = json.loads([ln for ln in out.splitlines() if ln.startswith("{")][-1])
    except (subprocess.SubprocessError, ValueError, IndexError) as exc:
        return {"unavailable": str(exc)[:200]}
    keep = ("value", "unit", "ms_per_step", "dtype", "converged", "gpu_launches", "roofline", "e2e",
            "clocks", "ir_steps_mean", "ir_steps_max", "iters_mean", "accuracy", "cpu_baseline")
    r = {k: d.get(k) for k in keep}
    r["config"] = d.get("config")
    return r


def aggregate_ranks(total_ms, solves_local, world, device):
    """Whole-job throughput (see shard.job_throughput)."""
    from paper_1811_02512_gb300 import shard
    return shard.job_throughput(total_ms, solves_local, world, device)


# ------------------------------------------------------------------ uneven multi-grid batch

def _pack_case(g):
    from paper_1811_02512_gb300 import gridgen
    n, seed = gridgen.config4_sizes()[g]
    return gridgen.with_loading_factor(gridgen.delaunay_raw(n, seed, name=f"multigrid{g}"))


def pack_cases(lo, hi):
    """Grids lo..hi-1 of the uneven batch, generated in spawned processes."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Pool(max(1, min(hi - lo, os.cpu_count() or 1))) as pool:
        return pool.map(_pack_case, range(lo, hi))


def run_adjoint(args, dev, local, world, rank):
    """adjoint20k: per step Newton-Raphson from flat start to tolerance, the
    objective and the adjoint gradient (all through the C ABI)."""
    import torch
    from paper_1811_02512_gb300 import gbpf, gridgen
    case = gridgen.config(3)
    t0 = time.perf_counter()
    g = gbpf.Grid(case)
    analyze_ms = (time.perf_counter() - t0) * 1e3
    g.set_cases(1)
    prec_name = workload_precision("adjoint20k", args.precision)
    prec = gbpf.PF_FP64 if prec_name == "fp64" else gbpf.PF_FP32
    opts = gbpf.run_opts(gbpf.PF_NR, prec, tol=TOL, max_iter=20)
    vm = torch.zeros((1, case.n), dtype=torch.float64, device=dev)
    va = torch.zeros_like(vm)
    J = torch.zeros(1, dtype=torch.float64, device=dev)
    gva, gvm = torch.zeros_like(vm), torch.zeros_like(vm)
    dP, dQ = torch.zeros_like(vm), torch.zeros_like(vm)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(int(2.5 * 129e6) // 4, dtype=torch.float32, device=dev)

    def step():
        st, res = gbpf.pf_run_to_tol(g.ctx, opts, vm, va, 1, stream=stream)
        gbpf.pf_objective(g.ctx, vm, va, J, gva, gvm, stream=stream)
        gbpf.pf_adjoint(g.ctx, prec, vm, va, gva, gvm, dP, dQ, 1, stream=stream)
        return st, res

    for _ in range(max(3, args.warmup)):
        st, res = step()
    torch.cuda.synchronize()
    gbpf.pf_set_profiling(g.ctx, True)
    for k in range(7):
        gbpf.pf_get_profile(g.ctx, k, reset=True)
    clocks = ClockSampler(local)
    clocks.start()
    total_ms = 0.0
    ok = 0
    for _ in range(args.steps):
        flush.fill_(1.0)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        st, res = step()
        b.record(stream)
        b.synchronize()
        total_ms += a.elapsed_time(b)
        ok += int(res["status"][0] == gbpf.PF_OK)
    clk = clocks.stop()
    prof, launches = {}, 0
    for k, nm in enumerate(gbpf.KERNEL_KINDS):
        n, ms = gbpf.pf_get_profile(g.ctx, k, reset=True)
        prof[nm] = ms
        launches += n
    gbpf.pf_set_profiling(g.ctx, False)
    total_ms, _, value = aggregate_ranks(total_ms, ok, world, dev)
    # end to end: specified injections from pinned host memory, gradient back
    psp = torch.from_numpy((case.pg - case.pd)[None].copy()).pin_memory()
    qsp = torch.from_numpy((-case.qd)[None].copy()).pin_memory()
    psp_d, qsp_d = torch.empty_like(vm), torch.empty_like(vm)
    out = torch.empty((2, case.n), dtype=torch.float64).pin_memory()
    e2e_steps = max(1, min(args.steps, 5))
    torch.cuda.synchronize()
    te0 = time.perf_counter()
    for _ in range(e2e_steps):
        psp_d.copy_(psp, non_blocking=True)
        qsp_d.copy_(qsp, non_blocking=True)
        gbpf.pf_set_injections(g.ctx, psp_d, qsp_d, stream=stream)
        st, res = step()
        out[0].copy_(dP[0], non_blocking=True)
        out[1].copy_(dQ[0], non_blocking=True)
        torch.cuda.synchronize()
    e2e_val = e2e_steps / (time.perf_counter() - te0)
    line = {"metric": METRIC, "value": value, "unit": "(PF + gradient)/s", "n_gpus": world,
            "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == gbpf.PF_FP64 else "f32+f64", "data": "synthetic",
            "config": {"workload": "adjoint20k", "nbus": case.n, "nbranch": case.m,
                       "precision": prec_name, "tol_pu": TOL, "method": "nr+adjoint",
                       "l2": "flushed between timed steps (2.5x L2 buffer write)",
                       "loading_factor": case.lam, "analyze_ms": analyze_ms},
            "converged": ok, "iters": int(res["iters"][0]), "gpu_launches": launches,
            "kernel_ms": prof, "roofline": None, "clocks": clk,
            "e2e": {"value": e2e_val, "unit": "(PF + gradient)/s",
                    "h2d_bytes_per_step": int(2 * 8 * case.n), "d2h_bytes_per_step": int(2 * 8 * case.n)}}
    if rank == 0:
        print(json.dumps(line))
    g.close()


def run_pack(args, dev, local, world, rank):
    import torch
    from concurrent.futures import ThreadPoolExecutor
    from paper_1811_02512_gb300 import gbpf
    from paper_1811_02512_gb300 import shard
    t0 = time.perf_counter()
    lo, hi = shard.case_range(rank, world, args.ngrid)  # a job of several ranks splits the grids
    cases = pack_cases(lo, hi)
    gen_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
        grids = list(ex.map(gbpf.Grid, cases))
    analyze_s = time.perf_counter() - t0
    for g in grids:
        g.set_cases(1)
    pk = gbpf.Pack(grids)
    tot = int(pk.offset[-1])
    prec_name = args.precision or "fp32"
    prec = gbpf.PF_FP64 if prec_name == "fp64" else gbpf.PF_FP32
    opts = gbpf.run_opts(gbpf.PF_FDPF, prec, tol=TOL, max_iter=200,
                         ir_tol=args.ir_tol if args.ir_tol is not None else IR_TOL)
    vm = torch.zeros(tot, dtype=torch.float64, device=dev)
    va = torch.zeros_like(vm)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(int(2.5 * 129e6) // 4, dtype=torch.float32, device=dev)
    for _ in range(max(3, args.warmup)):
        st, res = pk.run(opts, vm, va, stream=stream)
    torch.cuda.synchronize()
    for g in grids:
        gbpf.pf_set_profiling(g.ctx, True)
        for k in range(7):
            gbpf.pf_get_profile(g.ctx, k, reset=True)
    clocks = ClockSampler(local)
    clocks.start()
    torch.cuda.synchronize()
    total_ms = 0.0
    for _ in range(args.steps):
        flush.fill_(1.0)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        st, res = pk.run(opts, vm, va, stream=stream)
        b.record(stream)
        b.synchronize()
        total_ms += a.elapsed_time(b)
    torch.cuda.synchronize()
    clk = clocks.stop()
    other_ms, launches = 0.0, 0
    for g in grids:
        for k in range(7):
            n, ms = gbpf.pf_get_profile(g.ctx, k, reset=True)
            other_ms += ms
            launches += n
        gbpf.pf_set_profiling(g.ctx, False)
    launches += args.steps  # the packed iteration launch of each step
    converged = int(np.sum(res["status"] == gbpf.PF_OK))
    total_ms, _, value = aggregate_ranks(total_ms, converged * args.steps, world, dev)
    run_ms = max(1e-6, (total_ms - other_ms) / args.steps)
    # the same grids one after the other by the plain FP64 path
    seq_opts = gbpf.run_opts(gbpf.PF_FDPF, gbpf.PF_FP64, tol=TOL, max_iter=200)
    vms = [torch.zeros((1, g.nbus), dtype=torch.float64, device=dev) for g in grids]
    vas = [torch.zeros_like(v) for v in vms]
    for g, v, w in zip(grids, vms, vas):
        gbpf.pf_run_to_tol(g.ctx, seq_opts, v, w, 1, stream=stream)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    seq_ok = 0
    for g, v, w in zip(grids, vms, vas):
        st1, r1 = gbpf.pf_run_to_tol(g.ctx, seq_opts, v, w, 1, stream=stream)
        seq_ok += int(r1["status"][0] == gbpf.PF_OK)
    b.record(stream)
    b.synchronize()
    seq_ms = a.elapsed_time(b)
    # end to end: start state from pinned host memory, solution back
    host_in = torch.zeros((2, tot), dtype=torch.float64).pin_memory()
    host_out = torch.empty((2, tot), dtype=torch.float64).pin_memory()
    e2e_opts = gbpf.run_opts(gbpf.PF_FDPF, prec, tol=TOL, max_iter=200, flat_start=0)
    pos = 0
    for g in grids:  # flat start written on the host
        c = g.case
        host_in[0, pos:pos + c.n] = torch.from_numpy(np.where(c.btype == 1, 1.0, c.vset))
        host_in[1, pos:pos + c.n] = torch.from_numpy(np.where(c.btype == 3, c.va, 0.0))
        pos += c.n
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    te0 = time.perf_counter()
    for _ in range(e2e_steps):
        vm.copy_(host_in[0], non_blocking=True)
        va.copy_(host_in[1], non_blocking=True)
        st, res_e = pk.run(e2e_opts, vm, va, stream=stream)
        host_out[0].copy_(vm, non_blocking=True)
        host_out[1].copy_(va, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = time.perf_counter() - te0
    e2e_val = int(np.sum(res_e["status"] == gbpf.PF_OK)) * e2e_steps / e2e_s
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peaks = json.load(fh)
    except OSError:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    prec_bytes = 8 if prec == gbpf.PF_FP64 else 4
    alg = 0.0
    for k, g in enumerate(grids):  # every grid has its own matrices: all of its data per launch
        hi_k = float(res["iters"][k]) + 1.0
        resid_k = (float(res["iters"][k]) + float(res["ir_steps"][k])) if prec == gbpf.PF_FP32 else 0.0
        alg += hbm_bytes_per_launch(g.info, g.case, prec_bytes, hi_k, resid_k, 0.0, 1)
    achieved = alg / (run_ms / 1e3) / 1e9
    sizes = [g.nbus for g in grids]
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == gbpf.PF_FP64 else "f32+f64", "data": "synthetic",
            "config": {"workload": "pack256", "ngrid": len(grids), "nbus_total": tot,
                       "nbus_min": min(sizes), "nbus_max": max(sizes), "precision": prec_name,
                       "tol_pu": TOL, "method": "fdpf",
                       "l2": "flushed between timed steps (2.5x L2 buffer write)",
                       "generate_s": gen_s, "analyze_s": analyze_s,
                       "parallelism": f"grids partitioned over {world} ranks" if world > 1 else "grids-in-blocks"},
            "converged": converged, "iters_mean": float(np.mean(res["iters"])),
            "gpu_launches": launches,
            "sequential_plain_fp64": {"value": seq_ok / (seq_ms / 1e3), "unit": UNIT,
                                      "ms": seq_ms, "converged": seq_ok},
            "roofline": {"bound": "hbm", "kernel": "k_fdpf_pack", "achieved": achieved,
                         "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
                         "traffic": None,
                         "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
                         "algorithmic_bytes_per_launch": alg, "kernel_ms_per_launch": run_ms},
            "clocks": clk,
            "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": int(2 * tot * 8),
                    "d2h_bytes_per_step": int(2 * tot * 8 + 24 * len(grids))}}
    if rank == 0:
        print(json.dumps(line))
    pk.close()
    for g in grids:
        g.close()


# ------------------------------------------------------------------ main

def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    rank, world, local = dist_env()
    import torch
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1811_02512_gb300 import build as B
    if rank == 0:
        B.build()
    if world > 1:
        dist.barrier()
    from paper_1811_02512_gb300 import gbpf
    if args.workload in ("pack256", "adjoint20k"):
        (run_pack if args.workload == "pack256" else run_adjoint)(args, dev, local, world, rank)
        if world > 1:
            dist.destroy_process_group()
        return

    from paper_1811_02512_gb300 import shard
    base, ncase_all, load_scale, outage = make_workload(args.workload, args.ncase)
    # a batch shards by case: rank r solves its own slice (symbolic analysis
    # repeated on every rank); a single case runs as independent replicas
    lo, hi = shard.case_range(rank, world, ncase_all) if ncase_all > 1 else (0, 1)
    ncase = hi - lo
    if ncase_all > 1:
        load_scale = load_scale[lo:hi]
        outage = outage[lo:hi]
    prec_name = workload_precision(args.workload, args.precision)
    prec = gbpf.PF_FP64 if prec_name == "fp64" else gbpf.PF_FP32
    t0 = time.perf_counter()
    g = gbpf.Grid(base)
    analyze_ms = (time.perf_counter() - t0) * 1e3
    g.set_cases(ncase, load_scale, outage)
    method = gbpf.PF_FDPF if args.method == "fdpf" else gbpf.PF_NR
    engine = {"auto": gbpf.PF_ENGINE_AUTO, "block": gbpf.PF_ENGINE_BLOCK,
              "lanes": gbpf.PF_ENGINE_LANES}[args.engine]
    ir_tol = args.ir_tol if args.ir_tol is not None else IR_TOL
    opts = gbpf.run_opts(method, prec, tol=TOL, max_iter=200 if method == gbpf.PF_FDPF else 20,
                         engine=engine, ir_tol=ir_tol)
    vm = torch.zeros((ncase, base.n), dtype=torch.float64, device=dev)
    va = torch.zeros_like(vm)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(int(2.5 * 129e6) // 4, dtype=torch.float32, device=dev)

    def step():
        return gbpf.pf_run_to_tol(g.ctx, opts, vm, va, ncase, stream=stream)

    if args.no_graphs:
        gbpf.pf_set_graphs(g.ctx, False)
    tuning = None
    if args.mapping:
        m_ = [int(v) for v in args.mapping.split(",")]
        e_, c_, f_, t_, o_ = m_[:5]
        gbpf.pf_set_tuning(g.ctx, engine=e_, cluster=c_, factor=f_, tail=t_, outage=o_,
                           threads=m_[5] if len(m_) > 5 else 0)
        tuning = gbpf.pf_get_tuning(g.ctx)
    elif not args.no_autotune and args.engine == "auto":
        t0 = time.perf_counter()
        tuning = gbpf.pf_autotune(g.ctx, opts, vm, va, reps=2 if ncase == 1 else 1, stream=stream)
        tuning["tune_s"] = time.perf_counter() - t0
    for _ in range(max(3, args.warmup)):  # the second identical run captures a CUDA graph
        st, res = step()
    torch.cuda.synchronize()
    for k in range(len(gbpf.KERNEL_KINDS)):
        gbpf.pf_get_profile(g.ctx, k, reset=True)

    def timed(nsteps):
        tot = 0.0
        for _ in range(nsteps):
            flush.fill_(1.0)  # evict L2 between timed steps (buffer > 2 x L2)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            out = step()
            b.record(stream)
            b.synchronize()
            tot += a.elapsed_time(b)
        return tot, out

    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    total_ms, (st, res) = timed(args.steps)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    launches = 0
    for k in range(len(gbpf.KERNEL_KINDS)):  # launch counts are kept without profiling
        launches += gbpf.pf_get_profile(g.ctx, k, reset=True)[0]
    # untimed: the same steps with every kernel bracketed by CUDA events (the
    # kernel breakdown and the roofline's kernel time), then without the
    # CUDA graph (its gain)
    gbpf.pf_set_profiling(g.ctx, True)
    nprof = min(args.steps, 5)
    timed(nprof)
    prof = {}
    for k, nm in enumerate(gbpf.KERNEL_KINDS):
        n, ms = gbpf.pf_get_profile(g.ctx, k, reset=True)
        prof[nm] = (n / nprof, ms / nprof)
    gbpf.pf_set_profiling(g.ctx, False)
    gbpf.pf_set_graphs(g.ctx, False)
    direct_ms, _ = timed(nprof)
    gbpf.pf_set_graphs(g.ctx, not args.no_graphs)
    converged = int(np.sum(res["status"] == gbpf.PF_OK))
    iters = res["iters"].astype(np.int64)
    irs = res["ir_steps"].astype(np.int64)
    # the results of the last timed step, every rank's slice, for the
    # accuracy check and the converged count of the whole batch
    status_t = torch.from_numpy(res["status"].astype(np.int32)).to(dev)
    vm_all, va_all, st_all = shard.gather_cases(vm, va, status_t, ncase_all, rank, world)

    total_ms, solves, value = aggregate_ranks(total_ms, converged * args.steps, world, dev)

    # end to end through the C ABI with host buffers: per step copy the case
    # inputs (load scales, outages) from pinned host memory, run, copy V back
    # (a single case uploads its load profile too: all ones, the base loading)
    ls_np = load_scale if load_scale is not None else np.ones((ncase, base.n))
    ls_host = torch.from_numpy(np.ascontiguousarray(ls_np, dtype=np.float64)).pin_memory()
    out_host = torch.empty((2, ncase, base.n), dtype=torch.float64).pin_memory()
    h2d = ls_host.numel() * 8 + (0 if outage is None else outage.nbytes)
    d2h = out_host.numel() * 8 + ncase * 24
    e2e_steps = max(1, min(args.steps, 5))
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    te0 = time.perf_counter()
    for _ in range(e2e_steps):
        g.set_cases(ncase, ls_host.numpy(), outage)
        st, res_e = step()
        out_host[0].copy_(vm, non_blocking=True)
        out_host[1].copy_(va, non_blocking=True)
        torch.cuda.synchronize()
    e2e_ms = (time.perf_counter() - te0) * 1e3
    _, _, e2e_val = aggregate_ranks(e2e_ms, int(np.sum(res_e["status"] == gbpf.PF_OK)) * e2e_steps, world, dev)

    # roofline of the dominant kernel (the power-flow iteration kernel)
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peaks = json.load(fh)
    except OSError:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    run_n, run_ms = prof["run"]
    kernel_ms = run_ms / max(run_n, 1e-9)
    prec_bytes = 8 if prec == gbpf.PF_FP64 else 4
    half_iters = float(np.sum(res["iters"])) + float(np.sum(res["status"] == gbpf.PF_OK))
    # FP64 residuals: one per solve of a refined (FP32) run plus one per
    # refinement step; outage solves with the low-rank correction
    resid = (float(np.sum(res["iters"])) + float(np.sum(irs))) if prec == gbpf.PF_FP32 else 0.0
    lowrank = tuning is not None and tuning.get("outage") == 2 and outage is not None
    out_solves = float(np.sum(res["iters"][outage >= 0])) if lowrank else 0.0
    alg_bytes = hbm_bytes_per_launch(g.info, base, prec_bytes, half_iters, resid, out_solves, ncase)
    hbm = {"bound": "hbm", "achieved": alg_bytes / (kernel_ms / 1e3) / 1e9 if kernel_ms > 0 else 0.0,
           "peak": hbm_peak, "unit": "GB/s",
           "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
           "algorithmic_bytes_per_launch": alg_bytes}
    hbm["frac"] = hbm["achieved"] / hbm_peak
    engine_used = (tuning or {}).get("engine", engine)
    kname = "k_fdpf_cl" if engine_used == gbpf.PF_ENGINE_CLUSTER else "k_fdpf"
    hbm["traffic"] = measured_traffic(args.workload, prec_name, ncase, kname) if method == gbpf.PF_FDPF else None
    if ncase_all > 1:
        # a batch is bound by the FP64 pipe (GB300 runs FP64 at 1/64 of FP32)
        solves64 = float(np.sum(res["iters"])) if prec == gbpf.PF_FP64 else 0.0
        flops = fp64_flops_per_launch(g.info, base, half_iters, resid, solves64)
        peak = fp64_peak_tflops(clk.get("sm_mhz"))
        achieved = flops / (kernel_ms / 1e3) / 1e12 if kernel_ms > 0 else 0.0
        roofline = {"bound": "alu", "kernel": kname, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak, "traffic": hbm["traffic"],
                    "peak_source": "FP64 unit count x SM clock (2 DFMA/cycle/SM x 152 SMs)",
                    "algorithmic_fp64_flops_per_launch": flops, "kernel_ms_per_launch": kernel_ms,
                    "hbm": hbm}
    else:
        roofline = dict(hbm, kernel=kname, kernel_ms_per_launch=kernel_ms)
        # a single case is latency bound: time per half-iteration and per
        # dependent step of its substitutions
        roofline["latency"] = {"us_per_half_iteration": kernel_ms * 1e3 / max(half_iters, 1),
                               "levels": [int(g.info.nlevels[0]), int(g.info.nlevels[1])]}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == gbpf.PF_FP64 else "f32+f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "nbus": base.n, "nbranch": base.m,
                       "ncase": ncase_all, "ncase_per_rank": ncase, "precision": prec_name, "tol_pu": TOL,
                       "ir_tol": ir_tol if prec == gbpf.PF_FP32 else None,
                       "method": args.method, "engine": args.engine,
                       "l2": "flushed between timed steps (2.5x L2 buffer write)",
                       "loading_factor": base.lam, "analyze_ms": analyze_ms,
                       "tuning": tuning,
                       "parallelism": (f"cases partitioned over {world} ranks" if world > 1 else "cases-in-blocks")
                       if ncase_all > 1 else ("replicas" if world > 1 else "one case")},
            "converged": int(torch.sum(st_all == gbpf.PF_OK).item()), "ncase": ncase_all,
            "iters_mean": float(np.mean(iters)), "iters_max": int(np.max(iters)),
            "ir_steps_mean": float(np.mean(irs)), "ir_steps_max": int(np.max(irs)),
            "gpu_launches": launches,
            "kernel_ms_per_step": {k: v[1] for k, v in prof.items()},
            "kernel_launches_per_step": {k: v[0] for k, v in prof.items()},
            "cuda_graph": {"launches_per_step": launches / args.steps,
                           "ms_per_step_graph": total_ms / args.steps,
                           "ms_per_step_direct": direct_ms / nprof},
            "roofline": roofline, "clocks": clk,
            "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)}}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.workload, args.cpu_sample_s, ncase_all)
        # the same leg checks each result of the last timed step against the
        # oracle run to a tight mismatch
        line["accuracy"] = oracle_accuracy(args.workload, vm_all.cpu().numpy(), va_all.cpu().numpy(), ncase_all)
    if rank == 0 and world == 1 and args.workload == "plain10k" and not args.no_batched:
        line["batched_fp32_ir"] = batched_line(args)
    if rank == 0:
        print(json.dumps(line))
    g.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
