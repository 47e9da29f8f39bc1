#!/usr/bin/env python
"""Benchmark of the multilevel ELM-FBPINN hot path on one GB300 (per rank).

One step = the whole path the paper times (basis construction, assembly of the
global system and iterative solution, §4.1 "Optimisation and solvers"), plus
the evaluation of u_hat and its error norms on the test points:

    elmfb_create -> elmfb_assemble -> elmfb_solve -> elmfb_eval -> elmfb_error_norms

by default on the large 2-D multilevel Poisson workload (levels 1,2,4,...,64
per dimension, K = 64, 2048^2 + 8192 collocation rows, 349,504 unknowns,
5.7e9 stored entries, a random 8-mode right-hand side), the largest of the
five workloads that fits one GPU.  The solve is LSQR with the block-Jacobi
preconditioner, stopped by its own criterion, with no knowledge of the exact
solution: the estimate of the preconditioned normal-equations residual
||(M P)^T r|| falls to 1e-4 of its start.  (The 1e-8 the workload states for
its CG comparison lies below what FP32 panels support: LSQR's estimate stalls
near 1e-7 of its start on both 2-D workloads.)  Inputs (points,
right-hand sides, test points, reference values) are resident in HBM when the
timed region starts; the e2e leg repeats the step from pinned host buffers
with the copies inside the timed region.  The panels (23 GB) exceed L2, so no
flush is needed between steps.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
instead (the paper's protocol, on a bounded sample of the same workload).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as WL  # noqa: E402

METRIC = "ELM-FBPINN time-to-solution (s) at oracle-matched L2 error; assembly HBM GB/s"
DOMINANT = "fused_Mt_MTu"   # the LSQR pass: the largest share of a step
# roofline.traffic is null: the fused pass has changed (the device-side stopping
# test, the CTAs-per-SM budget, the multi-instance variant) since its DRAM bytes
# were last captured with ncu
TRAFFIC_NOTE = ("null: the fused pass changed after its last ncu DRAM capture (then 1.022x the "
                "algorithmic bytes for FP32 panels on the 200x200 2-D case, 1.016x for FP32-pair "
                "panels on the DHO workload)")
# workload -> (problem, oracle golden name, panel precision)
WORKLOADS = {
    "poisson2d_large": (WL.config_poisson2d_large, "poisson2d_L1-64_K64_N2048_f0", "fp32"),
    "poisson2d_ml": (WL.config_poisson2d_ml, "poisson2d_L1-16_K128_N400", "fp32"),
    # FP64-accuracy workloads run FP32-pair (DF32) panels: FP32 storage is an
    # accuracy floor for them, and GB300's FP64 rate is 1/64 of FP32
    "dho_ml": (WL.config_dho_ml, "dho_L1-64_K96_N20000", "df32"),
    "poisson1d": (WL.config_poisson1d, "poisson1d_J16_K64_N2000", "df32"),
    # a quarter-size case of the 2-D workload (same levels and K; inputs still
    # larger than L2) for ncu captures that must stay small
    "poisson2d_ml_n200": (lambda: WL.poisson2d(levels=(1, 2, 4, 8, 16), features=128, n_side=200,
                                               n_boundary_side=200),
                          "poisson2d_L1-16_K128_N200", "fp32"),
}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x, device=None):
    """The largest x over the ranks of the process group (one rank: x).

    With N replicas (one per GPU, each solving the workload on its own) the
    job's time is the slowest replica's: every rank passes its own time and
    all receive the maximum."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def _golden(name):
    p = os.path.join(ROOT, "tests", "golden", "oracle_errors.json")
    if os.path.exists(p):
        return json.load(open(p)).get(name)
    return None


class Clocks:
    """nvidia-smi sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.path = None
        self.gpu = gpu_index

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _sets(P, device):
    import torch
    sets = []
    for rs in [P.interior] + list(P.boundary):
        pts = torch.as_tensor(np.ascontiguousarray(rs.points, dtype=np.float64))
        rhs = torch.as_tensor(np.ascontiguousarray(rs.rhs, dtype=np.float64))
        if device == "pinned":
            pts, rhs = pts.pin_memory(), rhs.pin_memory()
        elif device is not None:
            pts, rhs = pts.to(device), rhs.to(device)
        sets.append(dict(points=pts, rhs=rhs, c0=rs.c0, c1=rs.c1, c2=rs.c2, weight=rs.weight,
                         n=rs.points.shape[0]))
    return sets


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_2409_01949_gb300 as E

    ws, rank, local = _dist()
    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    make, golden_name, default_prec = WORKLOADS[args.workload]
    P = make()
    prec = {"fp64": E.FP64, "fp32": E.FP32, "df32": E.DF32}[args.precision or default_prec]
    if args.shift is None:
        # block-Jacobi Tikhonov shift (fraction of tr G_jj / K): FP64-accurate
        # panels take a smaller one than FP32 panels.  The Gram blocks of FP32
        # panels (products rounded to FP32) are indefinite near 1e-7: from 1e-10
        # every block of the 2-D workload retries twice (x100 each) and settles
        # at 1e-6, so the bench starts there (the same factors, two
        # factorisations fewer per block)
        args.shift = 1e-12 if prec in (E.FP64, E.DF32) else 1e-6
    stream = torch.cuda.current_stream()
    g = _golden(golden_name)
    target = None
    if args.target == "paper" and g and "lsqr" in g:
        target = 1.01 * g["lsqr"]["rel_l2"]
    elif args.target == "qr" and g and "qr" in g:
        target = 1.01 * g["qr"]["rel_l2"]

    sets_dev = _sets(P, dev)
    xs_dev = torch.as_tensor(P.test_points).to(dev)
    u_dev = torch.as_tensor(P.exact(P.test_points)).to(dev)
    uh_dev = torch.empty(xs_dev.shape[0], dtype=torch.float64, device=dev)
    kstats = {}   # dominant kernel, timed steps
    kall = {}     # every kernel, one extra untimed step
    launches = [0]
    last = {}

    def step(sets, xs, u, uh, profile, stats=None):
        # profile: "fused" times only the dominant kernel, every
        # --roofline-stride-th launch of it (events around every kernel would add
        # about 1000 event records to a step); "all" times every kernel, for the
        # breakdown taken on an extra untimed step
        s = E.Solver.from_problem(P, precision=prec, stream=stream.cuda_stream)
        if profile == "fused":
            s.set_profiling_only(DOMINANT)
            s.set_profiling_stride(args.roofline_stride)
        elif profile == "all":
            s.set_profiling(True)
        s.assemble(sets)
        info = s.solve(opts)
        s.eval(xs, out=uh)
        err = s.error_norms(uh, u)
        if profile:
            for k, (ms, n, by) in s.kernel_stats().items():
                t = stats.setdefault(k, [0.0, 0, by])
                t[0] += ms
                t[1] += n
                t[2] = by
        if profile == "fused":
            launches[0] += s.kernel_launches()
        last.update(info=info, err=err)
        if profile is None or (profile == "all" and "stages" not in last):
            # report-only queries (sizes() counts the Gram pairs on the host on
            # first use): taken on the untimed steps, preferably one without events
            last.update(sizes=s.sizes(), stages=s.stage_times())
        s.close()
        return err

    # the solver stops by its own criterion (no knowledge of u): the relative
    # preconditioned normal-equations residual reaches --ntol, or --max-iter
    budget = args.max_iter
    opts = E.default_solve_opts(max_iter=budget, atol=0.0, btol=0.0, ntol=args.ntol,
                                shift=args.shift, check_every=args.check_every)

    for _ in range(args.warmup):
        step(sets_dev, xs_dev, u_dev, uh_dev, None)
    # per-kernel breakdown: one more untimed step with every kernel timed
    step(sets_dev, xs_dev, u_dev, uh_dev, "all", kall)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clocks = Clocks(local)
    clocks.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record(stream)
    torch.cuda.nvtx.range_push("timed_steps")   # lets ncu filter the timed launches
    for _ in range(args.steps):
        step(sets_dev, xs_dev, u_dev, uh_dev, "fused", kstats)
    torch.cuda.nvtx.range_pop()
    t1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = max_over_ranks(t0.elapsed_time(t1) / args.steps, dev)
    if ws > 1:
        dist.barrier()

    # end-to-end through the public API from pinned host buffers
    sets_h = _sets(P, "pinned")
    xs_h = torch.as_tensor(P.test_points).pin_memory()
    u_h = torch.as_tensor(P.exact(P.test_points)).pin_memory()
    uh_h = torch.empty(xs_h.shape[0], dtype=torch.float64).pin_memory()
    a_h = torch.empty(P.n_columns, dtype=torch.float64).pin_memory()
    h2d = sum(s["points"].numel() * 8 + s["rhs"].numel() * 8 for s in sets_h) + \
        xs_h.numel() * 8 + u_h.numel() * 8
    d2h = uh_h.numel() * 8 + a_h.numel() * 8 + 3 * 8

    def step_e2e():
        s = E.Solver.from_problem(P, precision=prec, stream=stream.cuda_stream)
        s.assemble(sets_h)
        s.solve(opts)
        s.eval(xs_h, out=uh_h)
        s.error_norms(uh_h, u_h)
        E.lib().elmfb_get_coeffs(s.h, a_h.data_ptr())
        s.close()

    torch.cuda.synchronize()
    e0 = time.perf_counter()
    for _ in range(args.steps):
        step_e2e()
    torch.cuda.synchronize()
    e2e_s = max_over_ranks((time.perf_counter() - e0) / args.steps, dev)

    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return

    hbm, peak_kind = _peaks()
    # per-kernel breakdown from the extra untimed step with every kernel timed
    kern = {}
    for k, (tms, n, by) in kall.items():
        avg = tms / max(n, 1)
        kern[k] = {"launches_per_step": n, "avg_ms": round(avg, 5),
                   "share": None, "gbs": round(by / (avg * 1e-3) / 1e9, 1) if avg > 0 else None}
    tot = sum(v[0] for v in kall.values()) or 1.0
    for k in kern:
        kern[k]["share"] = round(kall[k][0] / tot, 4)
    # the roofline kernel: timed live in the timed steps (events around it only)
    dom = DOMINANT
    dms = kstats[dom][0] / kstats[dom][1]
    ach = kstats[dom][2] / (dms * 1e-3) / 1e9
    asm = kern.get("assemble_panels", {})
    info, err, sz = last["info"], last["err"], last["sizes"]
    line = {
        "metric": METRIC,
        "value": round(ms / 1000.0, 5),
        "unit": "s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms, 3),
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": {E.FP32: "f32+f64", E.DF32: "f32x2+f64"}.get(prec, "f64"),
        "data": "synthetic",
        "config": {"workload": golden_name, "levels": list(P.levels), "features": P.features,
                   "rows": P.n_rows, "columns": P.n_columns, "nnz_stored": int(sz.nnz),
                   "solver": f"LSQR + block-Jacobi (shift {args.shift}), stopped at "
                             f"||(MP)^T r|| <= {args.ntol:g} ||(MP)^T h|| (cap {budget})",
                   "parallelism": f"replicas x{ws}", "l2_flush": "inputs larger than L2 (panels "
                   f"{sz.panel_rows * P.features * (4 if prec == E.FP32 else 8) / 1e9:.2f} GB)"},
        "solution": {"rel_l2": float(err["rel_l2"]), "e_l1": float(err["e_l1"]),
                     "iterations": info.iterations,
                     "precond_retries": info.precond_retries,
                     "stop": {E.OK: "ntol", E.ERR_NOT_CONVERGED: "iteration cap"}.get(
                         info.status, str(info.status)),
                     "kappa_MP_lower_bound": (info.sigma_max / info.sigma_min
                                              if info.sigma_min > 0 else None),
                     "target": target, "target_kind": args.target,
                     "matched": bool(err["rel_l2"] <= target) if target is not None else None,
                     "target_note": None if target is not None else
                     "no oracle error exists for this workload: the oracle's LSQR-15000 on "
                     "its 5.7e9 stored entries (46 GB in FP64) does not fit the host",
                     "oracle_lsqr15000_rel_l2": (g or {}).get("lsqr", {}).get("rel_l2"),
                     "oracle_qr_rel_l2": (g or {}).get("qr", {}).get("rel_l2")},
        "roofline": {"kernel": dom, "bound": "hbm", "achieved": round(ach, 1), "peak": hbm,
                     "unit": "GB/s", "frac": round(ach / hbm, 4),
                     "traffic": None,
                     "traffic_note": TRAFFIC_NOTE,
                     "peak_kind": peak_kind,
                     "timed_launches": int(kstats[dom][1]),
                     "timed_every": args.roofline_stride},
        "assembly": {"kernel": "assemble_panels", "achieved_gbs": asm.get("gbs"),
                     "frac": round(asm["gbs"] / hbm, 4) if asm.get("gbs") else None,
                     "avg_ms": asm.get("avg_ms")},
        "kernels": kern,
        "kernels_note": "per-kernel times from one extra untimed step with every kernel "
                        "timed; in the timed steps only the roofline kernel carries events, "
                        "on every roofline.timed_every-th launch",
        "stages_ms": {k: round(v, 3) for k, v in last["stages"].items()},
        "gpu_launches": int(launches[0]),
        "e2e": {"value": round(e2e_s, 5), "unit": "s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "clocks": clk,
    }
    if not args.no_gram:
        line["gram_tc"] = gram_measure(P, stream)
    if not args.no_compare_fp64 and prec != E.FP64:
        line["precision_comparison"] = compare_fp64(P, stream, opts, ms, float(err["rel_l2"]),
                                                    info.iterations, args)
    if not args.no_cpu_baseline and ws == 1:
        line["cpu_baseline"] = cpu_baseline(P, args)
    print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def compare_fp64(P, stream, opts32, ms32, err32, its32, args, reps=2):
    """The same step with FP64 panels (the plain FP64 GPU form: FP64 entries,
    FP64 products and sums) under the same stopping rule, timed the same way
    (CUDA events around whole steps, after one warm-up step): its error and
    time beside the FP32-panel form's (FP32 storage and products, FP64
    accumulation of the scalars and vectors)."""
    import torch

    import paper_2409_01949_gb300 as E
    opts = E.default_solve_opts(max_iter=opts32.max_iter, atol=0.0, btol=0.0, ntol=opts32.ntol,
                                shift=1e-12, check_every=opts32.check_every)
    dev = torch.device("cuda", torch.cuda.current_device())
    sets = _sets(P, dev)
    xs = torch.as_tensor(P.test_points).to(dev)
    u = torch.as_tensor(P.exact(P.test_points)).to(dev)
    uh = torch.empty(xs.shape[0], dtype=torch.float64, device=dev)
    res = {}

    def step():
        s = E.Solver.from_problem(P, precision=E.FP64, stream=stream.cuda_stream)
        s.assemble(sets)
        info = s.solve(opts)
        s.eval(xs, out=uh)
        e = s.error_norms(uh, u)
        s.close()
        res.update(info=info, err=e)

    step()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record(stream)
    for _ in range(reps):
        step()
    t1.record(stream)
    torch.cuda.synchronize()
    ms64 = t0.elapsed_time(t1) / reps
    e64 = float(res["err"]["rel_l2"])
    return {"fp64_form": {"ms_per_step": round(ms64, 3), "rel_l2": e64,
                          "iterations": res["info"].iterations, "shift": 1e-12},
            "fp32_form": {"ms_per_step": round(ms32, 3), "rel_l2": err32, "iterations": its32},
            "speedup_fp32_over_fp64": round(ms64 / ms32, 2),
            "error_ratio_fp32_over_fp64": round(err32 / e64, 3),
            "note": "same workload and stopping rule (||(MP)^T r|| <= ntol ||(MP)^T h||); the "
                    "learned preconditioner applies to FCG only and is not part of either form"}


def gram_measure(P, stream, reps=3):
    """The tensor-core Gram blocks (tcgen05, BF16 products, FP32 accumulation
    in TMEM) of every subdomain pair sharing rows, on the same workload in
    mixed precision: CUDA events around each launch (untimed for the step),
    TFLOP/s of the algorithmic 2 K^2 flops per shared row and pair against the
    measured dense BF16 peak."""
    import paper_2409_01949_gb300 as E
    s = E.Solver.from_problem(P, precision=E.MIXED, stream=stream.cuda_stream)
    try:
        s.assemble_problem(P)
        flops = float(s.sizes().gram_flops)
        s.compute_gram()                       # warm-up (pair lists, TMEM, descriptors)
        s.set_profiling_only("gram_tc")
        for _ in range(reps):
            s.compute_gram()
        ms, n, by = s.kernel_stats()["gram_tc"]
    finally:
        s.close()
    avg = ms / n
    tf = flops / (avg * 1e-3) / 1e12
    peak = None
    pp = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pp):
        peak = json.load(open(pp)).get("bf16_tflops")
    return {"kernel": "gram_tc", "flops_per_launch": flops, "avg_ms": round(avg, 4),
            "tflops": round(tf, 1), "peak_bf16_tflops": peak,
            "frac": round(tf / peak, 4) if peak else None, "launches": n,
            "note": "BF16 panels, FP32 accumulation; 2 K^2 flops per shared row and subdomain "
                    "pair (i <= j); measured after the timed steps"}


def run_batch(args):
    """All instances of the uneven batched workload through elmfb_batch_solve."""
    import torch

    import paper_2409_01949_gb300 as E
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    specs = WL.batch_specs(args.batch_n, 0)
    probs = [WL.batch_instance(sp, i, 0) for i, sp in enumerate(specs)]
    opts = E.default_solve_opts(max_iter=args.batch_iters, atol=0.0, btol=0.0, ntol=args.ntol,
                                shift=1e-6, check_every=10, graph=0,
                                batch_shared=0 if args.no_shared else 1, autotune=1)
    # under-resolved instances (fewer than 4 support points per feature: their
    # Gram blocks are singular up to rounding, and block-Jacobi LSQR leaves
    # their null directions to rounding noise) take the paper's unpreconditioned
    # LSQR
    plain = E.default_solve_opts(max_iter=args.batch_iters, atol=0.0, btol=0.0, ntol=args.ntol,
                                 check_every=10, preconditioner=E.PREC_NONE)
    item_opts = [plain if WL.support_points_per_feature(P) < 4.0 else None for P in probs]
    # autotuning, one worker (each shape class timed alone on the GPU): one
    # instance per (K, log2 rows), the largest of its group; the timed batch
    # looks the choices up
    reps = {}
    for P, o in zip(probs, item_opts):
        if o is None:
            key = (P.features, int(np.log2(P.n_rows)))
            if key not in reps or P.n_rows > reps[key].n_rows:
                reps[key] = P
    tune = E.default_solve_opts(max_iter=10, atol=0.0, btol=0.0, shift=1e-6, check_every=10,
                                autotune=1)
    E.batch_solve(list(reps.values()), precision=E.FP32, n_workers=1, opts=tune)
    for _ in range(args.warmup):
        E.batch_solve(probs[:16], precision=E.FP32, n_workers=args.batch_workers, opts=opts,
                      item_opts=item_opts[:16])
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        res, _, _ = E.batch_solve(probs, precision=E.FP32, n_workers=args.batch_workers, opts=opts,
                                  item_opts=item_opts)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / args.steps
    clk = clocks.stop()
    errs = np.array([r.rel_l2 for r in res])
    line = {"metric": "batched time-to-solution (s) for all instances", "value": round(dt, 4),
            "unit": "s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": False, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": f"batch{args.batch_n}_uneven_poisson2d",
                       "instances": len(probs), "rows": int(sum(P.n_rows for P in probs)),
                       "columns": int(sum(P.n_columns for P in probs)),
                       "solver": f"LSQR + block-Jacobi (unpreconditioned on the "
                                 f"{sum(o is not None for o in item_opts)} instances with < 4 "
                                 f"support points per feature), stopped at ||(MP)^T r|| <= "
                                 f"{args.ntol:g} ||(MP)^T h|| (cap {args.batch_iters})",
                       "workers": args.batch_workers,
                       "launches": "per instance" if args.no_shared else "shared multi-instance"},
            "instances_per_s": round(len(probs) / dt, 2),
            "rel_l2": {"median": float(np.median(errs)), "p90": float(np.percentile(errs, 90)),
                       "max": float(errs.max())},
            "iterations": {"median": float(np.median([r.iterations for r in res])),
                           "max": int(max(r.iterations for r in res)),
                           "capped": int(sum(r.iterations >= args.batch_iters for r in res))},
            "gpu_launches": int(sum(r.launches for r in res)),
            "autotuner": E.tuning_table(),
            "clocks": clk}
    print(json.dumps(line), flush=True)


def cpu_baseline(P, args, n_samples=1):
    """The FP64 oracle as it stands on a bounded sample, projected to the full paper protocol.

    One sample assembles about 30,000 rows (about 30 s of the host's time on the large 2-D
    workload); a run of n_samples of them (the reference arm's warm-up and timed steps) takes
    proportionally smaller samples, at least 3,000 rows, so that the whole run stays near two
    minutes."""
    from oracle import lstsq as OL
    from oracle import system as OS
    target = max(3000, int(30000 * min(1.0, 4.0 / max(1, n_samples))))
    frac = args.cpu_row_stride or max(1, P.n_rows // target)
    its = args.cpu_lsqr_its
    rows = np.arange(0, P.n_rows, frac)
    c0 = time.process_time()
    w0 = time.perf_counter()
    out = OS.assemble(P, rows=rows, fmt="csr")
    t_as = time.perf_counter() - w0
    w1 = time.perf_counter()
    OL.lstsq_lsqr(out["M"], out["h"], iter_lim=its)
    t_ls = time.perf_counter() - w1
    wall = time.perf_counter() - w0
    cpu = time.process_time() - c0
    projected = t_as * frac + t_ls * frac * (15000.0 / its)
    return {"value": round(projected, 2), "unit": "s", "cores": max(1, round(cpu / wall)),
            "kind": "oracle",
            "sample": f"every {frac}th row assembled ({t_as:.2f} s) and {its} LSQR iterations on "
                      f"that sample ({t_ls:.2f} s); projected x{frac} rows and x{15000 // its} "
                      f"iterations to the paper protocol (15000 LSQR iterations); host "
                      f"{os.cpu_count()} cores"}


def run_reference(args):
    ws, rank, local = _dist()
    if rank != 0:
        return
    make, golden_name, _ = WORKLOADS[args.workload]
    P = make()
    vals = []
    for i in range(args.warmup + args.steps):
        cb = cpu_baseline(P, args, args.warmup + args.steps)
        if i >= args.warmup:
            vals.append(cb)
    v = statistics.mean(c["value"] for c in vals)
    cb = dict(vals[-1])
    cb["value"] = round(v, 2)
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 2), "unit": "s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(v * 1000.0, 1), "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": golden_name, "levels": list(P.levels), "features": P.features,
                       "rows": P.n_rows, "columns": P.n_columns,
                       "solver": "oracle: SciPy LSQR, 15000 iterations (paper protocol)"},
            "cpu_baseline": cb,
            "e2e": {"value": round(v, 2), "unit": "s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="poisson2d_large",
                    choices=list(WORKLOADS) + ["batch"])
    ap.add_argument("--precision", default=None, choices=["fp32", "fp64", "df32"])
    ap.add_argument("--target", default="paper", choices=["paper", "qr", "none"])
    ap.add_argument("--max-iter", type=int, default=5000)
    ap.add_argument("--ntol", type=float, default=1e-4,
                    help="stop when ||(MP)^T r|| <= ntol ||(MP)^T h|| (LSQR's estimate)")
    ap.add_argument("--shift", type=float, default=None)
    ap.add_argument("--check-every", type=int, default=10)
    ap.add_argument("--cpu-row-stride", type=int, default=None,
                    help="oracle sample: every n-th row (default: about 40k rows)")
    ap.add_argument("--cpu-lsqr-its", type=int, default=60)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-gram", action="store_true",
                    help="skip the tensor-core Gram measurement after the timed steps")
    ap.add_argument("--no-compare-fp64", action="store_true",
                    help="skip timing the same step with FP64 panels (the plain FP64 form)")
    ap.add_argument("--roofline-stride", type=int, default=8,
                    help="time every n-th launch of the roofline kernel in the timed steps")
    ap.add_argument("--batch-n", type=int, default=512)
    ap.add_argument("--batch-iters", type=int, default=5000)
    ap.add_argument("--batch-workers", type=int, default=32)
    ap.add_argument("--no-shared", action="store_true",
                    help="batched workload: launch each instance's LSQR kernels alone instead of "
                         "in shared multi-instance launches")
    args = ap.parse_args()
    if args.workload == "batch":
        run_batch(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
