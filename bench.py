#!/usr/bin/env python
"""Benchmark of the MCS Stokes hot path on GB300: solves per second.

One step = static condensation (mcs_condense) + the ASP-preconditioned MinRes solve
(mcs_solve) to relative preconditioned residual 1e-8, on the workload c2: the unit
square with 256x256 cells (131,072 triangles), k = 3, nu = 1e-2, manufactured
solution, 5-level geometric multigrid (16^2 coarsest) for the conforming space.
`value` is the mixed form (FP32 preconditioner, FP64 outer Krylov and operator);
the FP64 form is reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]

Under torchrun each rank solves its own copy of the workload (independent problems,
"replicas": the path has no exchange between problems), value = total solves / max time.
--impl reference times the CPU FP64 oracle (the test oracle of this repository) on a
bounded sample of the same workload and scales it to the full problem size.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Stokes solves/s to rel. res 1e-8, mixed vs FP64 form; HBM roofline %; p50/p99"
WORKLOAD = dict(dim=2, N=256, k=3, nu=1e-2, levels=5, rtol=1e-8)
WORKLOAD_NAME = ("c2: 2D unit square, 256x256 cells split into 131,072 triangles (4 uniform refinements of "
                 "16x16 for the multigrid), MCS k=3, nu=1e-2, manufactured solution")


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


def _traffic(kernel: str):
    """Per-launch DRAM bytes of `kernel` from the committed ncu summary, if it is current."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_c2.txt")
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


def _make_handle(mcs, precision):
    w = WORKLOAD
    return mcs.Handle.structured(w["dim"], w["N"], w["k"], w["nu"], precision=precision, gmg_levels=w["levels"],
                                 rtol=w["rtol"])


def _rhs(h, torch, workloads):
    w = WORKLOAD
    s = h.sizes
    xq = torch.zeros((s.ne * s.nq_load, w["dim"]), dtype=torch.float64, device="cuda")
    h.load_points(xq)
    F = torch.zeros(s.ndof, dtype=torch.float64, device="cuda")
    h.load_vector(workloads.manufactured_f(w["dim"], w["nu"], xq), F)
    del xq
    return F


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

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    launches = [0]      # library kernels launched in the last timed region (its own counter)

    def timed(h, F, x, steps, profile=False):
        def step():
            h.condense()
            x.zero_()
            return h.solve(F, x)
        for _ in range(0 if profile else args.warmup):
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
        ms = _over_ranks([ev0.elapsed_time(ev1)], dist if world > 1 else None, "cuda")[0]
        stats = h.profile_read() if profile else None
        if profile:
            h.profile(False)
        return ms, its, info, stats

    # ---------------- mixed form (headline)
    hm = _make_handle(mcs, mcs.MCS_MIXED)
    F = _rhs(hm, torch, workloads)
    x = torch.zeros_like(F)
    ndof = hm.sizes.ndof
    with ClockSampler(local) as clk:
        ms_mixed, its_mixed, info_m, _ = timed(hm, F, x, args.steps)
    gpu_launches = launches[0]
    value = args.steps * world / (ms_mixed / 1e3)
    # per-kernel CUDA-event timers: one further step of the same workload with the library's
    # timers on (the timed loop above runs the captured-graph path without per-launch events)
    _, _, _, stats = timed(hm, F, x, 1, profile=True)
    # error of the solution against the exact one is not part of the metric; residuals are
    resid_m = dict(precond=info_m.rel_res_precond, true=info_m.rel_res_true)

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
    e2e_s = _over_ranks([time.perf_counter() - t0], dist if world > 1 else None, "cuda")[0]
    e2e_value = args.steps * world / e2e_s

    hm.close()

    # ---------------- FP64 form
    hd = _make_handle(mcs, mcs.MCS_FP64)
    xd = torch.zeros_like(F)
    fp64_steps = max(1, args.steps // 2)
    ms_fp64, its_fp64, info_d, _ = timed(hd, F, xd, fp64_steps)
    value_fp64 = fp64_steps * world / (ms_fp64 / 1e3)
    hd.close()

    # ---------------- several degrees in one condensation launch (3D, 16^3 x 6 tets, k = 2, 3, 4)
    multi = _multi_degree(args, torch, mcs) if (rank == 0 and not args.no_multi) else None
    smoothing = _smoothing(args, torch, mcs) if (rank == 0 and not args.no_multi) else None

    # ---------------- serving: Poisson trace of mixed requests through the continuous-batching loop
    serving = None
    if args.serve_requests > 0:
        serving = _serving(args, rank, world, torch, dist if world > 1 else None)

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    # ---------------- roofline of the dominant kernel class
    peak, peak_kind = _peaks()
    dom = max(stats.items(), key=lambda kv: kv[1]["ms"])
    name, st = dom
    per_launch_ms = st["ms"] / max(st["launches"], 1)
    if name in ("condense", "apply_K"):
        achieved = st["flops"] / max(st["launches"], 1) / (per_launch_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "kernel": name, "achieved": achieved, "peak": 1.20, "unit": "TFLOP/s",
                "frac": achieved / 1.20, "traffic": None, "peak_kind": "measured FP64 FMA probe"}
    else:
        achieved = st["bytes"] / max(st["launches"], 1) / (per_launch_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "kernel": name, "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": _traffic(name),
                "algorithmic_bytes_per_launch": st["bytes"] / max(st["launches"], 1),
                "avg_launch_us": round(per_launch_ms * 1e3, 2), "peak_kind": peak_kind,
                "measured": "CUDA events around each launch, one profiled step after the timed loop"}
    share = {k: round(v["ms"] / sum(u["ms"] for u in stats.values()), 4) for k, v in stats.items() if v["launches"]}

    cpu = _cpu_baseline(args) if not args.no_cpu_baseline else None
    out = {
        "metric": METRIC, "value": round(value, 4), "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_mixed / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64 outer Krylov + K, f32 preconditioner",
        "data": "synthetic (manufactured solution on a structured Kuhn mesh)",
        "config": {"workload": WORKLOAD_NAME, "step": "mcs_condense + mcs_solve (MinRes, rel. preconditioned "
                   "residual 1e-8)", "ndof": ndof, "form": "mixed", "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 (resident operators ~1.7 GB per problem)"},
        "iterations": its_mixed[-1], "rel_res": resid_m,
        "condensed_dofs_per_s": round(value * ndof, 1),
        "fp64_form": {"value": round(value_fp64, 4), "unit": "solves/s", "ms_per_step": round(ms_fp64 / fp64_steps, 3),
                      "steps": fp64_steps, "iterations": its_fp64[-1],
                      "rel_res": dict(precond=info_d.rel_res_precond, true=info_d.rel_res_true)},
        "e2e": {"value": round(e2e_value, 4), "unit": "solves/s", "h2d_bytes_per_step": 2 * ndof * 8,
                "d2h_bytes_per_step": ndof * 8},
        "roofline": roof, "kernel_time_share": share,
        "gpu_launches": gpu_launches,
        "clocks": clk.summary(),
        "cpu_baseline": cpu,
        "serving": serving,
        "multi_degree": multi,
        "asp_smoothing": smoothing,
    }
    print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


def _random_solve(h, torch, seed):
    """One warm-up and one timed mcs_solve for F = M_u c, c ~ N(0, 1) on the velocity dofs (seeded)."""
    s = h.sizes
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    c = torch.zeros(s.ndof, dtype=torch.float64, device="cuda")
    c[:s.off_h] = torch.randn(s.off_h, dtype=torch.float64, device="cuda", generator=g)
    F = torch.zeros_like(c)
    h.mass_velocity(c, F)
    x = torch.zeros_like(F)
    h.solve(F, x)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    x.zero_()
    e0.record()
    info = h.solve(F, x)
    e1.record()
    torch.cuda.synchronize()
    return round(e0.elapsed_time(e1), 2), info


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
    """Mixed-degree batch: one persistent condensation launch for four problems (the lowest-order
    variant k = 1 and k = 2, 3, 4) against one launch per problem, then the four solves (random
    F = M_u c, seeded)."""
    ks = (1, 2, 3, 4)
    # k = 1: the ASP condition number grows under refinement (stabilisation weight nu), hence more
    # MinRes iterations
    hs = [mcs.Handle.structured(3, 16, k, 1.0, precision=mcs.MCS_MIXED, maxit=8000 if k == 1 else 1000)
          for k in ks]
    ev = lambda: torch.cuda.Event(enable_timing=True)

    def timed(fn, reps=2):
        fn()
        torch.cuda.synchronize()
        e0, e1 = ev(), ev()
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    t_batch = timed(lambda: mcs.condense_batch(hs))
    t_sep = timed(lambda: [h.condense() for h in hs])
    mcs.condense_batch(hs)
    solves = {}
    for k, h in zip(ks, hs):
        ms, info = _random_solve(h, torch, 100 + k)
        solves[f"k={k}"] = {"ndof": int(h.sizes.ndof), "ms": ms, "iterations": info.iterations,
                            "rel_res": info.rel_res_precond}
    # k = 1 with the stabilisation weight nu h_T^2 (lo_stab = 1) instead of nu: same right-hand side
    h1 = mcs.Handle.structured(3, 16, 1, 1.0, precision=mcs.MCS_MIXED, maxit=8000, lo_stab=1)
    h1.condense()
    ms, info = _random_solve(h1, torch, 101)
    solves["k=1, weight nu h_T^2"] = {"ndof": int(h1.sizes.ndof), "ms": ms, "iterations": info.iterations,
                                      "rel_res": info.rel_res_precond}
    h1.close()
    for h in hs:
        h.close()
    return {"config": "3D unit cube, 16^3 cells x 6 = 24,576 tetrahedra each, k = 1 (lowest-order variant), 2, 3, 4, "
                      "nu = 1, mixed form, random F = M_u c (c ~ N(0,1)); k = 5, 6 of the six-problem batch are "
                      "not supported",
            "condense_batched_ms": round(t_batch, 2), "condense_separate_ms": round(t_sep, 2), "solves": solves}


def _serving(args, rank, world, torch, dist):
    """Replays a seeded trace (each rank its own replica) through serve.SolveServer from a cold
    operator cache.  Latency = completion - arrival; throughput = requests / wall time."""
    from paper_2207_08481_gb300 import serve
    reqs = serve.make_trace(args.serve_requests, args.serve_rate, seed=2207 + rank)
    srv = serve.SolveServer(serve.GpuBackend(), slots=args.serve_slots, budget_bytes=120e9)
    t0 = time.perf_counter()
    res = srv.run(reqs, realtime=True)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    srv.close()
    summ = serve.summarize(res, wall)
    hits = [r for r in res if r.cache_hit]
    if hits:
        lat = [r.latency * 1e3 for r in hits]
        import numpy as np
        summ["p50_ms_cache_hit"] = float(np.percentile(lat, 50))
        summ["p99_ms_cache_hit"] = float(np.percentile(lat, 99))
    if dist is not None:
        total = _over_ranks([summ["requests"]], dist, "cuda", op="sum")[0]
        wall_max = _over_ranks([wall], dist, "cuda")[0]
        summ["throughput_solves_per_s"] = total / wall_max
    summ.update({"rate_per_s": args.serve_rate, "slots": args.serve_slots, "budget_gb": 120,
                 "peak_resident_gb": round(srv.peak_bytes / 1e9, 3), "evictions": srv.evictions,
                 "trace": f"{args.serve_requests} requests, Poisson {args.serve_rate}/s, dim in {{2,3}}, "
                          f"2^3..2^17 elements, k in {{2,3,4}}, nu log-uniform [1e-3,1], N(0,1) body force; "
                          f"cold operator cache; mixed form, rtol 1e-8"})
    for key in ("p50_ms", "p99_ms", "mean_ms", "max_ms", "throughput_solves_per_s"):
        summ[key] = round(summ[key], 3)
    return summ


def _oracle_sample(N: int):
    """Oracle (CPU, FP64) on the c2 workload type at N cells per direction: discretize,
    condense, load and direct solve.  Returns seconds."""
    from oracle import manufactured, mesh, system
    w = WORKLOAD
    t0 = time.perf_counter()
    c0 = time.process_time()
    D = system.discretize(mesh.structured(w["dim"], N), w["k"], w["nu"])
    AT = system.condense(D)
    F = system.load(D, manufactured.Manufactured(w["dim"], w["nu"]).f)
    x = system.solve_condensed(D, F, AT)
    system.mean_zero_pressure(D, x)
    wall = time.perf_counter() - t0
    _oracle_sample.threads = (time.process_time() - c0) / max(wall, 1e-9)   # CPU time / wall time
    return wall


def _cpu_baseline(args, N=48):
    secs = _oracle_sample(N)
    w = WORKLOAD
    scale = (w["N"] / N) ** w["dim"]
    est = secs * scale
    thr = getattr(_oracle_sample, "threads", 1.0)
    return {"value": round(1.0 / est, 6), "unit": "solves/s", "cores": max(1, round(thr)), "kind": "oracle",
            "sample": f"oracle (discretize + condense + sparse direct solve) on the c2 workload type at "
                      f"{N}x{N} cells ({2 * N * N} triangles) took {secs:.1f} s; scaled linearly by elements "
                      f"(x{scale:.1f}) to 256x256; cores = CPU time / wall time of the sample ({thr:.2f}) "
                      f"of {os.cpu_count()} available (NumPy/SciPy, sparse LU single-threaded)"}


def run_reference(args):
    rank, world, local = _dist()
    if rank != 0:
        return
    times = []
    for _ in range(args.warmup):
        _oracle_sample(args.ref_N)
    for _ in range(args.steps):
        times.append(_oracle_sample(args.ref_N))
    w = WORKLOAD
    scale = (w["N"] / args.ref_N) ** w["dim"]
    per = sum(times) / len(times) * scale
    value = 1.0 / per
    thr = getattr(_oracle_sample, "threads", 1.0)
    cpu = {"value": round(value, 6), "unit": "solves/s", "cores": max(1, round(thr)), "kind": "oracle",
           "sample": f"each step: oracle on {args.ref_N}x{args.ref_N} cells, scaled linearly by elements "
                     f"(x{scale:.0f}); cores = CPU time / wall time ({thr:.2f}) of {os.cpu_count()} available"}
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": "solves/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(per * 1e3, 1), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD_NAME, "form": "oracle: direct solve of the condensed system"},
           "cpu_baseline": cpu,
           "e2e": {"value": round(value, 6), "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--ref-N", type=int, default=24)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=300,
                    help="requests of the serving trace (2000 = the full trace; 0 = skip)")
    ap.add_argument("--serve-rate", type=float, default=50.0)
    ap.add_argument("--serve-slots", type=int, default=4)
    ap.add_argument("--no-multi", action="store_true", help="skip the mixed-degree batch and the ASP comparison")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
