#!/usr/bin/env python
"""Benchmark of the MCS Stokes hot path on GB300: Stokes solves per second.

One step = static condensation (mcs_condense) + the ASP-preconditioned MinRes solve (mcs_solve) of
the workload c3: the unit cube with 32^3 cubes x 6 = 196,608 tetrahedra, k = 2, nu = 1, manufactured
solution, 4-level geometric multigrid (4^3 coarsest) for the conforming space; 6,610,944 condensed
dofs.  A solve ends when the relative preconditioned residual is <= 1e-8 and the a-posteriori error
estimate of the solution (mcs_options.etol) is <= the form's accuracy bar: 1e-8 relative L2 error of
u and of p for the mixed form (FP32 preconditioner, FP64 outer Krylov), 1e-10 for the FP64 form.
`value` is the mixed form; the FP64 form, the same forms on c2 (2D, 256^2 x 2 triangles, k = 3,
nu = 1e-2) and the residual-only stopping rule are reported beside it.  `err_vs_oracle` states the
error of both forms against the CPU FP64 oracle's direct solve on cases of the same element types
the oracle finishes in seconds (the oracle runs only in the cpu_baseline leg).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]
  python bench.py --profile-case c3s [--form mixed|fp64]     (one condense + apply + precond, for ncu)

Under torchrun each rank solves its own copy of the workload (independent problems, "replicas":
the path has no exchange between problems), value = total solves / max time over ranks.
--impl reference times the CPU FP64 oracle (the test oracle of this repository) on bounded samples
of the same workload and extrapolates with the cost exponent fitted over three sample sizes.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Stokes solves/s to rel. res 1e-8, mixed vs FP64 form; HBM roofline %; p50/p99"
WORKLOADS = {
    "c3": dict(dim=3, N=32, k=2, nu=1.0, levels=4,
               name="c3: 3D unit cube, 32^3 cubes x 6 = 196,608 tetrahedra (3 refinements of 4^3 for the "
                    "multigrid), MCS k=2, nu=1, manufactured solution"),
    "c2": dict(dim=2, N=256, k=3, nu=1e-2, levels=5,
               name="c2: 2D unit square, 256x256 cells split into 131,072 triangles (4 refinements of 16x16 "
                    "for the multigrid), MCS k=3, nu=1e-2, manufactured solution"),
}
HEADLINE = "c3"
# The timed forms: rel. preconditioned residual 1e-8 and the error estimate at the form's accuracy bar.
ERR_BAR = {"mixed": 1e-8, "fp64": 1e-10}
FORMS = {
    "mixed": dict(precision=1, rtol=1e-8, etol=1e-8),
    "fp64": dict(precision=0, rtol=1e-8, etol=1e-10),
}
# Cases of the two element types small enough for the oracle's direct solve (err_vs_oracle).
ORACLE_CASES = {
    "c3": dict(dim=3, N=4, k=2, nu=1.0, levels=2),
    "c2": dict(dim=2, N=32, k=3, nu=1e-2, levels=2),
}
PROFILE_CASES = {"c2": dict(dim=2, N=256, k=3, nu=1e-2, levels=5), "c3": dict(dim=3, N=32, k=2, nu=1.0, levels=4),
                 "c3s": dict(dim=3, N=16, k=2, nu=1.0, levels=3)}


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                     timeout=5).stdout.strip()
                if out:
                    self.samples.append([c.strip() for c in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = sorted(float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit())
        mx = max(float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit())
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for s in self.samples:
            for i, n in enumerate(names):
                if len(s) > 5 + i and s[5 + i].lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(self.samples)}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p.get("hbm_gbs", 6800.0), "measured"
    except Exception:
        return 6800.0, "fallback"


def _traffic(kernel: str, workload: str):
    """Per-launch DRAM bytes of `kernel` from the committed ncu summary of this workload, if any."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.txt")
    try:
        for line in open(path):
            if line.startswith("dram_bytes_per_launch:"):
                return float(line.split(":")[1])
    except OSError:
        pass
    return None


def _over_ranks(values, dist, device, op="max"):
    """Element-wise max (or sum) of a list of floats over all ranks; identity without dist."""
    if dist is None:
        return [float(v) for v in values]
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return [float(v) for v in t.tolist()]


def _make_handle(mcs, w, form, **extra):
    o = dict(FORMS[form])
    o.update(extra)
    return mcs.Handle.structured(w["dim"], w["N"], w["k"], w["nu"], gmg_levels=w["levels"], **o)


def _rhs(h, torch, workloads, w):
    s = h.sizes
    xq = torch.zeros((s.ne * s.nq_load, w["dim"]), dtype=torch.float64, device="cuda")
    h.load_points(xq)
    F = torch.zeros(s.ndof, dtype=torch.float64, device="cuda")
    h.load_vector(workloads.manufactured_f(w["dim"], w["nu"], xq), F)
    del xq
    return F


def _s8d_bytes_per_colour_launch(s, ncol):
    """Algorithmic bytes of one facet-block Gauss-Seidel colour launch by the packed-triangle count: one
    A^d pass = s*E*n_d(n_d+1)/2 (each element's Schur complement read once as a packed triangle) plus
    the block solves s*F_int*m_F^2, divided over the colours of a sweep (s = 4 in the mixed form)."""
    return 4.0 * (s.ne * s.n_c * (s.n_c + 1) / 2 + s.nint * s.mF * s.mF) / ncol


def _roofline(stats, sizes, peak, peak_kind):
    """The roofline object of the bench line for the dominant kernel class of a profiled step.  stats:
    per class {launches, ms, bytes, flops} from the library's CUDA-event timers; sizes: the handle's
    mcs_sizes (ne, nint, n_c, mF, ncolours); peak: HBM GB/s."""
    # the facet-block Gauss-Seidel sweep runs as two kernels (maintained-residual forward colours and
    # row-product backward colours, the same bytes per facet): one class for the choice of the dominant one
    rstats = dict(stats)
    sweep_parts = {}
    if stats.get("facet_push", {}).get("launches"):
        a_, b_ = stats["facet_gs_step"], stats["facet_push"]
        rstats["facet_gs_step"] = {k: a_[k] + b_[k] for k in ("launches", "ms", "bytes", "flops")}
        del rstats["facet_push"]
        for label, key in (("row_products", "facet_gs_step"), ("push", "facet_push")):
            v = stats[key]
            if v["launches"]:
                us = 1e3 * v["ms"] / v["launches"]
                sweep_parts[label] = {"launches": v["launches"], "avg_launch_us": round(us, 2),
                                      "frac": round(v["bytes"] / v["launches"] / (us * 1e-6) / 1e9 / peak, 4),
                                      "traffic": _traffic(key, HEADLINE)}
    name, st = max(rstats.items(), key=lambda kv: kv[1]["ms"])
    nl = max(st["launches"], 1)
    per_launch_ms = st["ms"] / nl
    if name in ("condense",):
        achieved = st["flops"] / nl / (per_launch_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "kernel": name, "achieved": achieved, "peak": 1.20, "unit": "TFLOP/s",
                "frac": achieved / 1.20, "traffic": None, "peak_kind": "measured FP64 FMA probe"}
    else:
        achieved = st["bytes"] / nl / (per_launch_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "kernel": name, "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": _traffic(name, HEADLINE),
                "algorithmic_bytes_per_launch": st["bytes"] / nl,
                "avg_launch_us": round(per_launch_ms * 1e3, 2), "peak_kind": peak_kind,
                "measured": "CUDA events around each launch on the handle's stream, one profiled step after "
                            "the timed loop"}
        if name == "facet_gs_step" and sweep_parts:
            roof["kernel"] = "facet_gs_step (push forward colours + row-product backward colours)"
            roof["parts"] = sweep_parts
            tr = [(p_["traffic"], p_["launches"]) for p_ in sweep_parts.values()]
            roof["traffic"] = (sum(t * n for t, n in tr) / sum(n for _, n in tr)
                               if all(t is not None for t, _ in tr) else None)
        if name in ("facet_gs_step", "facet_push"):
            s8 = _s8d_bytes_per_colour_launch(sizes, sizes.ncolours)
            roof["s8d_bytes_per_launch"] = s8
            roof["frac_s8d"] = round(s8 / (per_launch_ms * 1e-3) / 1e9 / peak, 4)
            roof["layout_over_s8d"] = round(st["bytes"] / nl / s8, 3)
    return roof


def run_gpu(args):
    import torch

    import workloads
    from paper_2207_08481_gb300 import build
    rank, world, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    # one rank compiles; the others wait for the library
    if rank == 0:
        build.build()
    if world > 1:
        dist.barrier()
    import paper_2207_08481_gb300.mcs as mcs
    dd = dist if world > 1 else None

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    launches = [0]      # library kernels launched in the last timed region (its own counter)

    def timed(h, F, x, steps, warmup, profile=False):
        def step():
            h.condense()
            x.zero_()
            return h.solve(F, x)
        info = None
        for _ in range(warmup):
            info = step()
        if profile:
            h.profile(True)
        barrier()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n0 = mcs.launch_count()
        ev0.record()
        its = []
        for _ in range(steps):
            info = step()
            its.append(info.iterations)
        ev1.record()
        launches[0] = mcs.launch_count() - n0
        barrier()
        ms = _over_ranks([ev0.elapsed_time(ev1)], dd, "cuda")[0]
        stats = h.profile_read() if profile else None
        if profile:
            h.profile(False)
        return ms, its, info, stats

    def info_dict(info):
        return {"iterations": info.iterations, "cycles": info.refinements,
                "rel_res": {"precond": info.rel_res_precond, "true": info.rel_res_true},
                "err_est": info.err_est}

    w = WORKLOADS[HEADLINE]
    # ---------------- mixed form (headline)
    hm = _make_handle(mcs, w, "mixed")
    F = _rhs(hm, torch, workloads, w)
    x = torch.zeros_like(F)
    ndof = hm.sizes.ndof
    with ClockSampler(local) as clk:
        ms_mixed, its_mixed, info_m, _ = timed(hm, F, x, args.steps, args.warmup)
    gpu_launches = launches[0]
    value = args.steps * world / (ms_mixed / 1e3)
    # per-kernel CUDA-event timers: one further step of the same workload with the library's timers
    # on (the timed loop runs the captured-graph path without per-launch events)
    _, _, _, stats = timed(hm, F, x, 1, 0, profile=True)
    sizes = hm.sizes

    # ---------------- end to end through the host-buffer entry point
    import numpy as np
    Fh = F.cpu().numpy().copy()
    xh = np.zeros_like(Fh)
    for _ in range(args.warmup):
        hm.condense()
        xh[:] = 0.0
        hm.solve_host(Fh, xh)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        hm.condense()
        xh[:] = 0.0
        hm.solve_host(Fh, xh)
    barrier()
    e2e_s = _over_ranks([time.perf_counter() - t0], dd, "cuda")[0]
    e2e_value = args.steps * world / e2e_s
    x_mixed = x.clone()
    hm.close()

    # ---------------- FP64 form
    hd = _make_handle(mcs, w, "fp64")
    xd = torch.zeros_like(F)
    fp64_steps = max(1, args.steps // 4)
    ms_fp64, its_fp64, info_d, _ = timed(hd, F, xd, fp64_steps, min(args.warmup, 1))
    value_fp64 = fp64_steps * world / (ms_fp64 / 1e3)
    hd.close()
    # the two forms' solutions agree within the mixed form's bar (a property at full size)
    n_p = sizes.off_p
    agree = {"u": float(torch.linalg.norm(x_mixed[:n_p] - xd[:n_p]) / torch.linalg.norm(xd[:n_p])),
             "p": float(torch.linalg.norm(x_mixed[n_p:] - xd[n_p:]) / torch.linalg.norm(xd[n_p:]))}
    del x_mixed

    # ---------------- the residual-only stopping rule (rel. res 1e-8 alone), for context
    resid_only = {}
    for form in ("mixed", "fp64"):
        h = _make_handle(mcs, w, form, etol=0.0)
        xr = torch.zeros_like(F)
        ms_r, _, info_r, _ = timed(h, F, xr, 2, 1)
        resid_only[form] = {"value": round(2 * world / (ms_r / 1e3), 4), "unit": "solves/s",
                            "ms_per_step": round(ms_r / 2, 2), **info_dict(info_r)}
        h.close()
        del xr
    del F, x, xd

    # ---------------- c2: the same forms on the 2D workload
    c2 = _c2(args, torch, mcs, workloads, timed, info_dict) if not args.quick else None

    # ---------------- iteration counts under h-refinement, several degrees in one launch, ASP forms
    h_series = _h_series(torch, mcs, workloads) if (rank == 0 and not args.quick) else None
    multi = _multi_degree(args, torch, mcs) if (rank == 0 and not args.quick) else None
    smoothing = _smoothing(args, torch, mcs) if (rank == 0 and not args.quick) else None

    # ---------------- serving: Poisson traces of mixed requests through the continuous-batching loop
    serving = None
    if args.serve_requests > 0 and not args.quick:
        serving = {"at_trace_rate": _serving(args, rank, world, torch, dd, args.serve_requests, args.serve_rate)}
        if args.serve_rate2 > 0:
            serving["at_sustainable_rate"] = _serving(args, rank, world, torch, dd, args.serve_requests2,
                                                      args.serve_rate2)

    # ---------------- error against the oracle (cpu_baseline leg: the only place the oracle runs)
    cpu, err_vs_oracle = (None, None)
    if rank == 0 and not args.no_cpu_baseline:
        cpu, err_vs_oracle = _cpu_baseline(args, torch, mcs, workloads)

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    # ---------------- roofline of the dominant kernel class
    peak, peak_kind = _peaks()
    roof = _roofline(stats, sizes, peak, peak_kind)
    share = {k: round(v["ms"] / sum(u["ms"] for u in stats.values()), 4) for k, v in stats.items() if v["launches"]}
    # per class of the profiled step: launches, device ms, algorithmic GB/s (or TFLOP/s for the condensation)
    kstats = {k: {"launches": v["launches"], "ms": round(v["ms"], 3),
                  "us_per_launch": round(1e3 * v["ms"] / v["launches"], 2),
                  "alg_gb_per_s": round(v["bytes"] / (v["ms"] * 1e-3) / 1e9, 1) if v["bytes"] else None,
                  "tflop_per_s": round(v["flops"] / (v["ms"] * 1e-3) / 1e12, 3) if v["flops"] else None}
              for k, v in stats.items() if v["launches"]}

    out = {
        "metric": METRIC, "value": round(value, 4), "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_mixed / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64 outer Krylov + K, f32 preconditioner",
        "data": "synthetic (manufactured solution on a structured Kuhn mesh)",
        "config": {"workload": w["name"], "step": "mcs_condense + mcs_solve (MinRes with refinement cycles: rel. "
                   "preconditioned residual <= 1e-8 and estimated relative L2 error of u and p <= 1e-8)",
                   "ndof": ndof, "form": "mixed", "options": FORMS["mixed"], "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 (resident operators ~4.4 GB per problem)"},
        **info_dict(info_m),
        "condensed_dofs_per_s": round(value * ndof, 1),
        "fp64_form": {"value": round(value_fp64, 4), "unit": "solves/s",
                      "ms_per_step": round(ms_fp64 / fp64_steps, 3), "steps": fp64_steps,
                      "options": FORMS["fp64"], **info_dict(info_d)},
        "forms_agree_full_size": agree,
        "residual_only_stopping": resid_only,
        "err_vs_oracle": err_vs_oracle,
        "e2e": {"value": round(e2e_value, 4), "unit": "solves/s", "h2d_bytes_per_step": 2 * ndof * 8,
                "d2h_bytes_per_step": ndof * 8},
        "roofline": roof, "kernel_time_share": share, "kernel_stats": kstats,
        "gpu_launches": gpu_launches,
        "clocks": clk.summary(),
        "cpu_baseline": cpu,
        "c2": c2,
        "h_series": h_series,
        "serving": serving,
        "multi_degree": multi,
        "asp_smoothing": smoothing,
    }
    print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


def _c2(args, torch, mcs, workloads, timed, info_dict):
    w = WORKLOADS["c2"]
    out = {"workload": w["name"]}
    F = None
    for form in ("mixed", "fp64"):
        h = _make_handle(mcs, w, form)
        if F is None:
            F = _rhs(h, torch, workloads, w)
        x = torch.zeros_like(F)
        steps = 5 if form == "mixed" else 2
        ms, _, info, _ = timed(h, F, x, steps, 1)
        out[form] = {"value": round(steps / (ms / 1e3), 4), "unit": "solves/s", "ms_per_step": round(ms / steps, 2),
                     **info_dict(info)}
        h.close()
    return out


def _random_solve(h, torch, seed, warm=True, keep_x=False):
    """One warm-up (optional) and one timed mcs_solve for F = M_u c, c ~ N(0, 1) on the velocity dofs
    (seeded); keep_x: also the solution (host copy)."""
    s = h.sizes
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    c = torch.zeros(s.ndof, dtype=torch.float64, device="cuda")
    c[:s.off_h] = torch.randn(s.off_h, dtype=torch.float64, device="cuda", generator=g)
    F = torch.zeros_like(c)
    h.mass_velocity(c, F)
    x = torch.zeros_like(F)
    if warm:
        h.solve(F, x)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    x.zero_()
    e0.record()
    info = h.solve(F, x)
    e1.record()
    torch.cuda.synchronize()
    if keep_x:
        return round(e0.elapsed_time(e1), 2), info, x.cpu()
    return round(e0.elapsed_time(e1), 2), info


def _h_series(torch, mcs, workloads):
    """MinRes iterations of the mixed form (headline stopping rule) under uniform refinement of both
    workload types (Theorem aux_pc_schur: bounded in h), manufactured right-hand side."""
    out = {"stopping": FORMS["mixed"]}
    for key, Ns in (("c3_type", (8, 16, 32)), ("c2_type", (32, 64, 128, 256))):
        base = WORKLOADS["c3" if key == "c3_type" else "c2"]
        rows = []
        for N in Ns:
            w = dict(base, N=N, levels=-1)
            h = _make_handle(mcs, w, "mixed")
            h.condense()
            F = _rhs(h, torch, workloads, w)
            x = torch.zeros_like(F)
            h.solve(F, x)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            x.zero_()
            e0.record()
            info = h.solve(F, x)
            e1.record()
            torch.cuda.synchronize()
            rows.append({"N": N, "ne": int(h.sizes.ne), "ndof": int(h.sizes.ndof), "levels": int(h.sizes.gmg_levels),
                         "iterations": info.iterations, "cycles": info.refinements,
                         "solve_ms": round(e0.elapsed_time(e1), 2)})
            h.close()
        out[key] = rows
    return out


def _smoothing(args, torch, mcs):
    """Multiplicative against additive ASP (Table ST_smoothing re-run on the c3 mesh: 3D 32^3 x 6
    tetrahedra, k = 2, nu = 1, mixed form, random F = M_u c, seeded): iterations and solve time."""
    out = {"config": "3D unit cube, 32^3 cells x 6 = 196,608 tetrahedra, k = 2, nu = 1, mixed form, "
                     "random F = M_u c (c ~ N(0,1)), rel. preconditioned residual 1e-8"}
    for name, asp in (("multiplicative", 0), ("additive", 1)):
        h = mcs.Handle.structured(3, 32, 2, 1.0, precision=mcs.MCS_MIXED, asp=asp, maxit=4000)
        h.condense()
        ms, info = _random_solve(h, torch, 7)
        out[name] = {"ms": ms, "iterations": info.iterations, "rel_res": info.rel_res_precond,
                     "ms_per_iteration": round(ms / max(info.iterations, 1), 3)}
        h.close()
    return out


def _multi_degree(args, torch, mcs):
    """The batched degree sweep: six problems on 3D 16^3 x 6 tetrahedra, the lowest-order variant k = 1 and
    k = 2..6, condensed in one persistent launch (against one launch per problem), then solved one by one
    (mixed form with the headline's stopping rule, random F = M_u c, c ~ N(0, 1), seeded)."""
    ks = (1, 2, 3, 4, 5, 6)
    # k = 1: the ASP condition number grows under refinement (stabilisation weight nu), hence more
    # MinRes iterations
    hs = [mcs.Handle.structured(3, 16, k, 1.0, maxit=8000 if k == 1 else 2000, **FORMS["mixed"]) for k in ks]
    ev = lambda: torch.cuda.Event(enable_timing=True)

    def timed(fn, warm):
        if warm:
            fn()
        torch.cuda.synchronize()
        e0, e1 = ev(), ev()
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    # one launch per problem (the first of each kernel instantiation warmed up on the cheap degrees), then
    # the batched launch once: the separate launches have loaded every kernel it runs
    t_sep = {}
    for k, h in zip(ks, hs):
        t_sep[f"k={k}"] = round(timed(h.condense, warm=k <= 4), 2)
    t_batch = timed(lambda: mcs.condense_batch(hs), warm=False)
    solves = {}
    x_seq = []
    for k, h in zip(ks, hs):
        ms, info, x = _random_solve(h, torch, 100 + k, warm=k <= 4, keep_x=True)
        x_seq.append(x)
        solves[f"k={k}"] = {"ndof": int(h.sizes.ndof), "ms": ms, "iterations": info.iterations,
                            "cycles": info.refinements, "rel_res": info.rel_res_precond, "err_est": info.err_est,
                            "resident_gb": round(h.sizes.bytes_resident / 1e9, 2)}
    for h in hs:
        h.close()
    concurrent = _concurrent_solves(ks, torch, mcs, x_seq, sum(v["ms"] for v in solves.values()))
    # k = 1 with the stabilisation weight nu h_T^2 (lo_stab = 1) instead of nu: same right-hand side
    h1 = mcs.Handle.structured(3, 16, 1, 1.0, maxit=8000, lo_stab=1, **FORMS["mixed"])
    h1.condense()
    ms, info = _random_solve(h1, torch, 101)
    solves["k=1, weight nu h_T^2"] = {"ndof": int(h1.sizes.ndof), "ms": ms, "iterations": info.iterations,
                                      "cycles": info.refinements, "rel_res": info.rel_res_precond}
    h1.close()
    return {"config": "3D unit cube, 16^3 cells x 6 = 24,576 tetrahedra each, k = 1 (lowest-order variant), 2, 3, 4, 5, 6, "
                      "nu = 1, mixed form (rel. residual 1e-8, error estimate <= 1e-8), random F = M_u c (c ~ N(0,1))",
            "condense_batched_ms": round(t_batch, 2), "condense_separate_ms": round(sum(t_sep.values()), 2),
            "condense_separate_by_k_ms": t_sep, "solves": solves, "solves_concurrent": concurrent}


def _concurrent_solves(ks, torch, mcs, x_seq, sequential_ms):
    """The six problems again, each handle on a stream of its own: condensed in one batched launch, then
    the six solves issued at once from one host thread each, so their kernels overlap on the device.  Same
    right-hand sides as the solves one by one; the solutions must agree with those bit for bit."""
    hs = [mcs.Handle.structured(3, 16, k, 1.0, stream=torch.cuda.Stream(), maxit=8000 if k == 1 else 2000,
                                **FORMS["mixed"]) for k in ks]
    mcs.condense_batch(hs)
    Fs, xs = [], []
    for k, h in zip(ks, hs):
        with torch.cuda.stream(h.stream):
            s = h.sizes
            g = torch.Generator(device="cuda")
            g.manual_seed(100 + k)
            c = torch.zeros(s.ndof, dtype=torch.float64, device="cuda")
            c[:s.off_h] = torch.randn(s.off_h, dtype=torch.float64, device="cuda", generator=g)
            F = torch.zeros_like(c)
            h.mass_velocity(c, F)
            Fs.append(F)
            xs.append(torch.zeros_like(F))
    torch.cuda.synchronize()
    infos = [None] * len(hs)

    def run(i):
        infos[i] = hs[i].solve(Fs[i], xs[i])

    threads = [threading.Thread(target=run, args=(i,)) for i in range(len(hs))]
    t0 = time.perf_counter()
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    torch.cuda.synchronize()
    wall = (time.perf_counter() - t0) * 1e3
    same = all(torch.equal(xs[i].cpu(), x_seq[i]) for i in range(len(hs)))
    out = {"wall_ms": round(wall, 2), "sum_of_solves_one_by_one_ms": round(sequential_ms, 2),
           "iterations": {f"k={k}": infos[i].iterations for i, k in enumerate(ks)},
           "identical_to_solves_one_by_one": bool(same),
           "how": "one stream per handle, one host thread per solve, after one batched condensation"}
    for h in hs:
        h.close()
    return out


def _serving(args, rank, world, torch, dist, n, rate):
    """Replays a seeded trace (each rank its own replica) through serve.SolveServer from a cold
    operator cache.  Latency = completion - arrival; throughput = requests / wall time."""
    from paper_2207_08481_gb300 import serve
    reqs = serve.make_trace(n, rate, seed=2207 + rank)
    srv = serve.SolveServer(serve.GpuBackend(), slots=args.serve_slots, budget_bytes=120e9)
    t0 = time.perf_counter()
    res = srv.run(reqs, realtime=True)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    srv.close()
    summ = serve.summarize(res, wall)
    import numpy as np
    for label, sel in (("cache_hit", [r for r in res if r.cache_hit]), ("cache_miss", [r for r in res if not r.cache_hit])):
        if sel:
            lat = [r.latency * 1e3 for r in sel]
            summ[f"p50_ms_{label}"] = round(float(np.percentile(lat, 50)), 3)
            summ[f"p99_ms_{label}"] = round(float(np.percentile(lat, 99)), 3)
    by_size = {}
    for r in res:
        rq = reqs[r.rid]
        cls = "small (< 2^10 elements)" if rq.e < 10 else ("medium (2^10..2^13)" if rq.e < 14 else "large (>= 2^14)")
        by_size.setdefault(cls, []).append(r.latency * 1e3)
    summ["by_size"] = {c: {"requests": len(v), "p50_ms": round(float(np.percentile(v, 50)), 3),
                           "p99_ms": round(float(np.percentile(v, 99)), 3)} for c, v in sorted(by_size.items())}
    if dist is not None:
        total = _over_ranks([summ["requests"]], dist, "cuda", op="sum")[0]
        wall_max = _over_ranks([wall], dist, "cuda")[0]
        summ["throughput_solves_per_s"] = total / wall_max
    summ.update({"rate_per_s": rate, "slots": args.serve_slots, "budget_gb": 120,
                 "peak_resident_gb": round(srv.peak_bytes / 1e9, 3), "evictions": srv.evictions,
                 "trace": f"{n} requests, Poisson {rate}/s, dim in {{2,3}}, 2^3..2^17 elements, k in {{2,3,4}}, "
                          f"nu log-uniform [1e-3,1], N(0,1) body force; cold operator cache; mixed form, rtol 1e-8, "
                          f"error estimate <= 1e-8"})
    for key in ("p50_ms", "p99_ms", "mean_ms", "max_ms", "throughput_solves_per_s"):
        summ[key] = round(summ[key], 3)
    return summ


# ------------------------------------------------------------------ CPU legs (the oracle)
def _oracle_sample(case: dict, F=None):
    """The oracle (CPU, FP64) on one case: discretize, condense, load, direct solve of the condensed
    system, mean-zero pressure.  F: a given right-hand side (else the oracle's own load vector).
    Returns (seconds, solution)."""
    from oracle import manufactured, mesh, system
    t0 = time.perf_counter()
    c0 = time.process_time()
    D = system.discretize(mesh.structured(case["dim"], case["N"]), case["k"], case["nu"])
    AT = system.condense(D)
    if F is None:
        F = system.load(D, manufactured.Manufactured(case["dim"], case["nu"]).f)
    x = system.mean_zero_pressure(D, system.solve_condensed(D, F, AT))
    wall = time.perf_counter() - t0
    _oracle_sample.threads = (time.process_time() - c0) / max(wall, 1e-9)   # CPU time / wall time
    return wall, x, D.off_p


def _fit(samples):
    """Least-squares fit t = a * ne^b over (ne, t) samples; returns (a, b)."""
    import numpy as np
    X = np.log([s[0] for s in samples])
    Y = np.log([s[1] for s in samples])
    b, loga = np.polyfit(X, Y, 1)
    return math.exp(loga), b


def _cpu_baseline(args, torch, mcs, workloads):
    """The oracle timed on the machine's host cores at three sizes of the headline's element type, its cost
    fitted as a power of the element count and extrapolated to the headline mesh; and the error of both
    GPU forms (the timed options) against the oracle's direct solve on the ORACLE_CASES."""
    w = WORKLOADS[HEADLINE]
    samples = []
    for N in (2, 3, 4):
        case = dict(w, N=N)
        secs, _, _ = _oracle_sample(case)
        ne = 6 * N ** 3 if w["dim"] == 3 else 2 * N * N
        samples.append((ne, secs))
    a, b = _fit(samples)
    ne_full = 6 * w["N"] ** 3 if w["dim"] == 3 else 2 * w["N"] ** 2
    est = a * ne_full ** b
    thr = getattr(_oracle_sample, "threads", 1.0)
    cpu = {"value": round(1.0 / est, 8), "unit": "solves/s", "cores": max(1, round(thr)), "kind": "fitted",
           "exponent": round(b, 3),
           "sample": f"oracle (discretize + condense + load + sparse direct solve of the condensed system, CPU FP64) on "
                     f"the headline's element type at N = 2, 3, 4 ({', '.join(f'{ne} tets: {t:.2f} s' for ne, t in samples)}); "
                     f"time fitted as a*ne^b (b = {b:.2f}) and evaluated at {ne_full} tets; cores = CPU time / wall "
                     f"time ({thr:.2f}) of {os.cpu_count()} available"}
    err = {}
    import numpy as np
    for key, case in ORACLE_CASES.items():
        entry = {"case": f"{case['dim']}D N={case['N']} k={case['k']} nu={case['nu']} ({'x6 tets' if case['dim'] == 3 else 'x2 triangles'}), "
                         f"{case['levels']} GMG levels, manufactured f; both sides take the library's load vector"}
        F = None
        for form in ("mixed", "fp64"):
            h = _make_handle(mcs, case, form)
            h.condense()
            if F is None:
                F = _rhs(h, torch, workloads, case)
                _, xo, n_p = _oracle_sample(case, F.cpu().numpy())
            x = torch.zeros_like(F)
            info = h.solve(F, x)
            xg = x.cpu().numpy()
            eu = float(np.linalg.norm(xg[:n_p] - xo[:n_p]) / np.linalg.norm(xo[:n_p]))
            ep = float(np.linalg.norm(xg[n_p:] - xo[n_p:]) / np.linalg.norm(xo[n_p:]))
            entry[form] = {"rel_l2_u": eu, "rel_l2_p": ep, "bar": ERR_BAR[form],
                           "meets_bar": eu <= ERR_BAR[form] and ep <= ERR_BAR[form],
                           "iterations": info.iterations, "err_est": info.err_est}
            h.close()
        if not all(entry[f]["meets_bar"] for f in ("mixed", "fp64")):
            # the FP64 rounding floor of the discrete problem: the oracle's condensed against its full solve
            from oracle import mesh, system
            D = system.discretize(mesh.structured(case["dim"], case["N"]), case["k"], case["nu"])
            xf, _, _ = system.solve_full(D, F.cpu().numpy())
            xf = system.mean_zero_pressure(D, xf)
            entry["oracle_condensed_vs_full"] = {
                "rel_l2_u": float(np.linalg.norm(xo[:n_p] - xf[:n_p]) / np.linalg.norm(xf[:n_p])),
                "rel_l2_p": float(np.linalg.norm(xo[n_p:] - xf[n_p:]) / np.linalg.norm(xf[n_p:]))}
        err[key] = entry
    return cpu, err


def run_reference(args):
    """The oracle as the reference arm: each step one bounded sample (N = 3 of the headline's element
    type), extrapolated to the headline mesh with the exponent fitted over N = 2, 3, 4 in the warm-up."""
    rank, world, local = _dist()
    if rank != 0:
        return
    w = WORKLOADS[HEADLINE]
    ne_of = lambda N: 6 * N ** 3 if w["dim"] == 3 else 2 * N * N
    fit_samples = []
    for i in range(max(args.warmup, 3)):
        N = (2, 3, 4)[i % 3]
        secs, _, _ = _oracle_sample(dict(w, N=N))
        fit_samples.append((ne_of(N), secs))
    _, b = _fit(fit_samples)
    times = []
    for _ in range(args.steps):
        secs, _, _ = _oracle_sample(dict(w, N=3))
        times.append(secs)
    ne_full = ne_of(w["N"])
    per = sum(times) / len(times) * (ne_full / ne_of(3)) ** b
    value = 1.0 / per
    thr = getattr(_oracle_sample, "threads", 1.0)
    cpu = {"value": round(value, 8), "unit": "solves/s", "cores": max(1, round(thr)), "kind": "fitted",
           "exponent": round(b, 3),
           "sample": f"each step: oracle (direct solve of the condensed system) on N = 3 ({ne_of(3)} tets), "
                     f"extrapolated by (ne ratio)^{b:.2f} to {ne_full} tets, exponent fitted over N = 2, 3, 4 in the "
                     f"warm-up; cores = CPU time / wall time ({thr:.2f}) of {os.cpu_count()} available"}
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 8), "unit": "solves/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(per * 1e3, 1), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": w["name"], "form": "oracle: direct solve of the condensed system"},
           "cpu_baseline": cpu,
           "e2e": {"value": round(value, 8), "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_profile_case(args):
    """One condense, one K apply and one preconditioner application of a case, for ncu to capture
    (c3s: the c3 element type on 16^3 x 6 cells, small enough for full captures)."""
    import torch

    import paper_2207_08481_gb300.mcs as mcs
    import workloads
    from paper_2207_08481_gb300 import build
    build.build()
    w = PROFILE_CASES[args.profile_case]
    torch.cuda.set_device(0)
    opts = dict(FORMS[args.form])
    opts.pop("etol", None)
    h = mcs.Handle.structured(w["dim"], w["N"], w["k"], w["nu"], gmg_levels=w["levels"], **opts)
    h.condense()
    F = _rhs(h, torch, workloads, w)
    y = torch.zeros_like(F)
    h.apply(F, y)
    h.precond(F, y)
    torch.cuda.synchronize()
    h.close()
    print("profile case done", flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--quick", action="store_true", help="headline only (no c2, series, serving, batch)")
    ap.add_argument("--serve-requests", type=int, default=200,
                    help="requests of the serving trace at --serve-rate (2000 = the full trace; 0 = skip)")
    ap.add_argument("--serve-rate", type=float, default=50.0)
    ap.add_argument("--serve-requests2", type=int, default=150)
    ap.add_argument("--serve-rate2", type=float, default=5.0,
                    help="second trace at an arrival rate the GPU sustains (0 = skip)")
    ap.add_argument("--serve-slots", type=int, default=4)
    ap.add_argument("--serve-only", action="store_true",
                    help="run only the serving traces (--serve-requests at --serve-rate, then --serve-requests2 at "
                         "--serve-rate2) and print their summaries")
    ap.add_argument("--c4-only", action="store_true",
                    help="the batched six-degree sweep alone (condensation batched and one by one, solves one by "
                         "one and concurrently)")
    ap.add_argument("--profile-case", choices=sorted(PROFILE_CASES), default=None)
    ap.add_argument("--form", choices=["mixed", "fp64"], default="mixed")
    args = ap.parse_args()
    if args.profile_case:
        run_profile_case(args)
    elif args.c4_only:
        import torch
        from paper_2207_08481_gb300 import build
        build.build()
        import paper_2207_08481_gb300.mcs as mcs
        print(json.dumps({"multi_degree": _multi_degree(args, torch, mcs)}), flush=True)
    elif args.serve_only:
        import torch
        from paper_2207_08481_gb300 import build
        build.build()
        out = {"at_trace_rate": _serving(args, 0, 1, torch, None, args.serve_requests, args.serve_rate)}
        if args.serve_rate2 > 0 and args.serve_requests2 > 0:
            out["at_sustainable_rate"] = _serving(args, 0, 1, torch, None, args.serve_requests2, args.serve_rate2)
        print(json.dumps({"serving": out}), flush=True)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
