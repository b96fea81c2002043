#!/usr/bin/env python3
"""Benchmark: time to residual 1e-8 of the additive (solve) phase of the
self-learning AMG triplet method, mixed precision (float32 V-cycle, float64
residual/Ritz) vs plain float64, on one GB300.

Workload (default): 8 minimal singular triplets of the 256 x 256
forward-difference gradient (m = 131,584, n = 65,536, nnz = 262,144), seeded
synthetic input (--workload 3 selects the 1024 x 1024 member of the family).
One step = one solve from the same post-setup boot triplets (already resident
in HBM) to max_j rho_j <= 1e-8: every outer iteration runs the whole hot path
(V-cycle with Kaczmarz block Gauss-Seidel, residual + restriction, coarsest
pseudo-inverse, interpolation, Ritz step, residual norms).  value = seconds
per solve (lower is better), mixed precision.  The plain float64 path is
timed from the same boot triplets with max(1, W // 3) warm-up and
max(1, K // 3) timed solves (it is the slower comparison arm).

Beside the line ("other_workloads"), the default run also times the 32 x 32
Laplacian's 4 minimal eigenpairs to residual 1e-8 in both precisions, and
("variants") the main workload with two guard triplets (n_b = 10, the first
8 converged); --no-small skips both.

--impl reference runs the FP64 CPU oracle on a bounded sample of the same
workload instead (rank 0 only).
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

PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")


def _peaks():
    try:
        with open(PEAKS) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def log(msg):
    sys.stderr.write("[bench] %s\n" % msg)
    sys.stderr.flush()


def _env_rank():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def max_over_ranks(x: float, device) -> float:
    """The largest of every rank's x (the replicas' timing rule); x itself
    when no process group is up.  Collective on `device` (cuda under NCCL,
    cpu under gloo)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# --------------------------------------------------------------- clocks
class Clocks:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        # the raw samples (SAMG_CLOCKS_CSV, else a temporary file)
        self.path = os.environ.get("SAMG_CLOCKS_CSV") or os.path.join(
            tempfile.gettempdir(), "samg_clocks_%d.csv" % os.getpid())

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except OSError:
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
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax = float(p[2])
            except ValueError:
                continue
            for k, name in enumerate(names):
                if p[5 + k].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------- workload
def workload(i):
    import workloads as W

    wl = W.workload(i)
    return wl, dict(wl.params, seed=W.problem_seed(i))


# --------------------------------------------------------------- CPU oracle sample
def oracle_sample(i: int, gpu_iters: int | None):
    """Oracle per-outer-iteration time on the 256 x 256 member of the same
    gradient family (the oracle's setup of the full workload takes tens of
    minutes), scaled linearly in m + n (the paper's cost model, Sec. 6.1) to
    the benchmarked size and multiplied by the iteration count."""
    import numpy as np

    import oracle
    import workloads as W

    wl, prm = workload(i)
    full = wl.build()
    if wl.kind == "svd" and wl.target == "minimal" and i in (2, 3):
        small = W.gradient(256)
    else:
        small = full
    A = small.to_scipy()
    t0 = time.perf_counter()
    H, s, U, V = oracle.setup(A, wl.nb, wl.target, wl.kind, dict(prm, n_mult=1))
    t_setup = time.perf_counter() - t0
    iters = 2
    XY = oracle.dense_XY(H.levels[-1], H.spd)
    t0 = time.perf_counter()
    for _ in range(iters):
        oracle.vcycle(H, 0, s, U, V, np.zeros_like(U), None if H.spd else np.zeros_like(V), XY)
        s, U, V = oracle.ritz(H.levels[0].A, H.spd, H.target, U, V)
        oracle.residual_norms(H.levels[0].A, H.spd, s, U, V)
    per_it = (time.perf_counter() - t0) / iters
    scale = (full.m + full.n) / float(A.shape[0] + A.shape[1])
    # without a GPU count (the reference arm): the outer iterations the GPU
    # solve needs on the 256 x 256 gradient from its 20-cycle setup (103;
    # the oracle's own 1-cycle hierarchy does not reach 1e-8), else 30
    n_it = gpu_iters if gpu_iters else (103 if i == 2 else 30)
    return {
        "value": per_it * scale * n_it, "unit": "s", "cores": 1, "kind": "oracle",
        "sample": ("%d oracle outer iterations (V-cycle + Ritz + residual norms, float64, one "
                   "thread) on the %dx%d gradient of the same family with a 1-cycle oracle "
                   "hierarchy (setup %.1f s, untimed): %.3f s/iteration, scaled by (m+n) x%.1f "
                   "to the benchmarked size and by %d iterations" %
                   (iters, A.shape[0], A.shape[1], t_setup, per_it, scale, n_it)),
    }


def run_reference(args):
    rank, _, world = _env_rank()
    if rank != 0:
        return 0
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    wl, _ = workload(args.workload)
    vals = []
    cb = None
    for _ in range(args.warmup + args.steps):
        cb = oracle_sample(args.workload, None)
        vals.append(cb["value"])
    v = statistics.median(vals[args.warmup:])
    line = {
        "impl": "reference", "metric": "time to residual 1e-8 (s)", "value": v, "unit": "s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": wl.name},
        "cpu_baseline": dict(cb, value=v),
        "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# --------------------------------------------------------------- GPU arm
def run_gpu(args):
    import numpy as np
    import torch

    rank, local, world = _env_rank()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    import paper_1102_0919_gb300 as samg

    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    wl, prm = workload(args.workload)
    A = wl.build()
    m, n = A.m, A.n
    mu = n if wl.kind == "spd" else m
    t0 = time.perf_counter()
    s = samg.Solver.setup(A, wl.nb, wl.target, wl.kind, stream=stream, prec="fp32", **prm)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    levels = s.levels()
    log("setup %.1f s, levels %s" % (t_setup, levels))
    sig0, U0, V0, res0 = s.triplets()
    # initial boot triplets resident in HBM (torch owns the memory)
    dsig = torch.tensor(sig0, device=dev, dtype=torch.float64)
    dU = torch.tensor(U0, device=dev, dtype=torch.float64).contiguous()
    dV = None if V0 is None else torch.tensor(V0, device=dev, dtype=torch.float64).contiguous()

    def reset():
        s.set_triplets_device(dsig.data_ptr(), dU.data_ptr(),
                              None if dV is None else dV.data_ptr())

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    results = {}
    log("launches after setup: %d" % samg.samg_launch_count())
    for prec in args.arms.split(","):
        s.set_precision(prec)
        warm = args.warmup if prec == "fp32" else max(1, args.warmup // 3)
        steps = args.steps if prec == "fp32" else max(1, args.steps // 3)
        for _ in range(warm):
            reset()
            tw = time.perf_counter()
            ok, it = s.solve(args.tol, args.max_outer)
            log("%s warm-up solve: %d iterations, converged %s, %.2f s" %
                (prec, it, ok, time.perf_counter() - tw))
        iters = []
        barrier()
        launches0 = samg.samg_launch_count()
        log("%s: launches before the timed region: %d" % (prec, launches0))
        rng = args.ncu_range and prec == "fp32"
        if rng:
            torch.cuda.profiler.start()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        prof = prec == "fp32"
        if prof:
            s.profile(True)
        with Clocks(local) as clk:
            ev0.record(stream)
            for _ in range(steps):
                reset()
                ok, it = s.solve(args.tol, args.max_outer)
                iters.append((ok, it))
            ev1.record(stream)
            barrier()
        if rng:
            torch.cuda.profiler.stop()
        ms = ev0.elapsed_time(ev1) / steps
        if prof:
            s.profile(False)
            pr = s.profile_read()
        launches = samg.samg_launch_count() - launches0
        results[prec] = dict(ms=max_over_ranks(ms, dev), iters=iters, launches=launches, steps=steps,
                             clocks=clk.summary(), prof=pr if prof else None)
        log("%s: %.1f ms/solve, iterations %s" % (prec, ms, iters))
        if prof:
            log("kernels: %s" % json.dumps(pr))
        _, _, _, rf = s.triplets()
        results[prec]["resid"] = float(rf.max())
    # end to end through the C ABI with host buffers (mixed precision)
    s.set_precision("fp32")
    e2e = []
    for k in range(max(args.steps, 1) + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.set_triplets(sig0, U0, V0)
        ok, it = s.solve(args.tol, args.max_outer)
        sg, Uh, Vh, rh = s.triplets()
        t1 = time.perf_counter()
        if k:
            e2e.append(t1 - t0)
    h2d = 8 * (wl.nb + mu * wl.nb + (0 if V0 is None else n * wl.nb))
    d2h = h2d + 8 * wl.nb
    s.close()
    if rank != 0:
        return 0
    peaks, how = _peaks()
    mixed = results["fp32"]
    f64 = results.get("fp64", {"ms": float("nan"), "steps": 0, "iters": [(False, 0)], "resid": float("nan")})
    kz = mixed["prof"]["kaczmarz_sweep"]
    achieved = kz["bytes"] / (kz["ms"] * 1e-3) / 1e9 if kz["ms"] > 0 else 0.0
    cpu = oracle_sample(args.workload, mixed["iters"][-1][1]) if world == 1 and not args.no_cpu else None
    value = mixed["ms"] / 1e3
    line = {
        "metric": "time to residual 1e-8 (s)",
        "value": value,
        "unit": "s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": mixed["ms"],
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": wl.name, "m": m, "n": n, "nnz": A.nnz, "n_b": wl.nb,
                   "tol": args.tol, "levels": [[a, b] for a, b, _ in levels],
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "inputs larger than L2 (vectors + operators > 129 MB); no flush",
                   "setup_s": round(t_setup, 3)},
        "fp64": {"value": f64["ms"] / 1e3, "unit": "s", "steps": f64["steps"],
                 "outer_iterations": f64["iters"][-1][1],
                 "converged": all(o for o, _ in f64["iters"]), "resid": f64["resid"]},
        "mixed": {"outer_iterations": mixed["iters"][-1][1],
                  "converged": all(o for o, _ in mixed["iters"]), "resid": mixed["resid"]},
        "speedup_mixed_vs_fp64": f64["ms"] / mixed["ms"] if mixed["ms"] else None,
        "e2e": {"value": statistics.median(e2e), "unit": "s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": mixed["launches"],
        "clocks": mixed["clocks"],
        "roofline": {"bound": "hbm", "kernel": "kaczmarz_sweep (float32)",
                     "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / peaks["hbm_gbs"], "traffic": None,
                     "peak_source": how, "launches": kz["launches"],
                     "avg_launch_us": 1e3 * kz["ms"] / max(kz["launches"], 1),
                     "alg_bytes_per_launch": kz["bytes"] / max(kz["launches"], 1)},
        "kernel_time_ms_per_solve": {k: v["ms"] / mixed["steps"] for k, v in mixed["prof"].items()},
        # the V-cycle's sparse products (residual, restriction, interpolation,
        # right-hand sides): algorithmic GB/s over their CUDA-event time
        "spmm_gbs": (mixed["prof"]["block_spmm"]["bytes"] / (mixed["prof"]["block_spmm"]["ms"] * 1e-3) / 1e9
                     if mixed["prof"]["block_spmm"]["ms"] > 0 else None),
        "cpu_baseline": cpu,
    }
    if world == 1 and args.workload == 2 and not args.no_small:
        line["other_workloads"] = {"laplacian5_N32_nb4_minimal": small_workload(1, dev, stream)}
        line["variants"] = {"guard_nb10_nconv8": guard_variant(args, dev, stream)}
    print(json.dumps(line))
    return 0


def guard_variant(args, dev, stream):
    """The main workload with two guard triplets (n_b = 10, of which the
    first 8 must reach the tolerance; not the paper's form): setup, then one
    warm-up and one timed solve per precision.  Errors are reported, not
    raised."""
    try:
        import torch

        import paper_1102_0919_gb300 as samg

        wl, prm = workload(args.workload)
        A = wl.build()
        t0 = time.perf_counter()
        s = samg.Solver.setup(A, 10, wl.target, wl.kind, stream=stream, prec="fp32", n_conv=8, **prm)
        torch.cuda.synchronize()
        out = {"setup_s": round(time.perf_counter() - t0, 3), "unit": "s",
               "levels": [[a, b] for a, b, _ in s.levels()]}
        sig0, U0, V0, _ = s.triplets()
        dsig = torch.tensor(sig0, device=dev, dtype=torch.float64)
        dU = torch.tensor(U0, device=dev, dtype=torch.float64).contiguous()
        dV = torch.tensor(V0, device=dev, dtype=torch.float64).contiguous()
        for prec in ("fp64", "fp32"):
            s.set_precision(prec)
            s.set_triplets_device(dsig.data_ptr(), dU.data_ptr(), dV.data_ptr())
            s.solve(args.tol, args.max_outer)
            torch.cuda.synchronize()
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            s.set_triplets_device(dsig.data_ptr(), dU.data_ptr(), dV.data_ptr())
            ev0.record(stream)
            ok, it = s.solve(args.tol, args.max_outer)
            ev1.record(stream)
            torch.cuda.synchronize()
            _, _, _, rf = s.triplets()
            out[prec] = {"value": ev0.elapsed_time(ev1) / 1e3, "outer_iterations": it,
                         "converged": ok, "resid_first8": float(rf[:8].max())}
        s.close()
        return out
    except Exception as e:  # noqa: BLE001 -- the main line must still print
        return {"error": "%s: %s" % (type(e).__name__, e)}


def small_workload(i, dev, stream, warm=3, steps=5):
    """Time to residual 1e-8 of a small workload (the 32 x 32 Laplacian's 4
    minimal eigenpairs), float64 and mixed precision, from the same setup
    output, with CUDA events on the library's stream; sigma against the
    closed form.  Reported beside the main line; errors are reported, not
    raised."""
    try:
        import numpy as np
        import torch

        import paper_1102_0919_gb300 as samg
        sys.path.insert(0, os.path.join(ROOT, "tests"))
        from closed_forms import laplacian5_eigs

        wl, prm = workload(i)
        A = wl.build()
        s = samg.Solver.setup(A, wl.nb, wl.target, wl.kind, stream=stream, prec="fp32", **prm)
        sig0, U0, V0, _ = s.triplets()
        dsig = torch.tensor(sig0, device=dev, dtype=torch.float64)
        dU = torch.tensor(U0, device=dev, dtype=torch.float64).contiguous()
        exact = laplacian5_eigs(32)[:wl.nb]
        out = {"levels": [[a, b] for a, b, _ in s.levels()], "unit": "s", "steps": steps}
        for prec in ("fp64", "fp32"):
            s.set_precision(prec)
            for _ in range(warm):
                s.set_triplets_device(dsig.data_ptr(), dU.data_ptr(), None)
                s.solve(1e-8, 300)
            torch.cuda.synchronize()
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            res = []
            for _ in range(steps):
                s.set_triplets_device(dsig.data_ptr(), dU.data_ptr(), None)
                res.append(s.solve(1e-8, 300))
            ev1.record(stream)
            torch.cuda.synchronize()
            sg, _, _, rf = s.triplets()
            out[prec] = {"value": ev0.elapsed_time(ev1) / steps / 1e3,
                         "outer_iterations": res[-1][1], "converged": all(o for o, _ in res),
                         "resid": float(rf.max()),
                         "sigma_relerr_max": float(np.max(np.abs(sg - exact) / exact))}
        s.close()
        return out
    except Exception as e:  # noqa: BLE001 -- the main line must still print
        return {"error": "%s: %s" % (type(e).__name__, e)}


def run_sweep_roofline(args):
    """Roofline of the relaxation at the workload's full size: block
    Gauss-Seidel relaxations (Kaczmarz sweeps over the rows of A and A^t,
    with their right-hand sides) on level 0 of a two-level aggregation
    hierarchy (no setup phase).  Prints one JSON line with the algorithmic
    GB/s of the sweep and sparse-product kernels per precision (CUDA events
    on the library's stream)."""
    import numpy as np
    import scipy.sparse as sp
    import torch

    import paper_1102_0919_gb300 as samg

    torch.cuda.set_device(0)
    wl, prm = workload(args.workload)
    A = wl.build().to_scipy()
    m, n = A.shape
    nb = wl.nb
    rng = np.random.default_rng(11)
    P = sp.csr_matrix((np.ones(m), (np.arange(m), np.minimum(np.arange(m) * 100 // m, 99))),
                      shape=(m, 100))
    Q = sp.csr_matrix((np.ones(n), (np.arange(n), np.minimum(np.arange(n) * 90 // n, 89))),
                      shape=(n, 90))
    sig = np.linspace(4.0, 12.0, nb)
    U = rng.standard_normal((m, nb))
    V = rng.standard_normal((n, nb))
    K = rng.standard_normal((m, nb))
    T = rng.standard_normal((n, nb))
    g = samg.Solver.from_hierarchy(A, [P], [Q], nb, sig, U, V, wl.target, wl.kind, prec="fp64",
                                   mu_b=1)
    peaks, how = _peaks()
    line = {"mode": "sweep_roofline", "workload": wl.name, "m": m, "n": n, "nnz": int(A.nnz),
            "n_b": nb, "steps": args.steps, "warmup": args.warmup, "peak_gbs": peaks["hbm_gbs"],
            "peak_source": how}
    for prec in args.arms.split(","):
        g.set_precision(prec)
        for _ in range(args.warmup):
            g.relax(0, sig, U, V, K, T, count=1)
        g.profile(True)
        g.profile_read(reset=True)
        if args.ncu_range and prec == "fp32":
            torch.cuda.profiler.start()
        for _ in range(args.steps):
            g.relax(0, sig, U, V, K, T, count=1)
        if args.ncu_range and prec == "fp32":
            torch.cuda.profiler.stop()
        pr = g.profile_read()
        g.profile(False)
        kz, spm = pr["kaczmarz_sweep"], pr["block_spmm"]
        line[prec] = {
            "kaczmarz_gbs": kz["bytes"] / (kz["ms"] * 1e-3) / 1e9,
            "kaczmarz_us_per_launch": 1e3 * kz["ms"] / max(kz["launches"], 1),
            "kaczmarz_bytes_per_launch": kz["bytes"] / max(kz["launches"], 1),
            "kaczmarz_frac": kz["bytes"] / (kz["ms"] * 1e-3) / 1e9 / peaks["hbm_gbs"],
            "spmm_gbs": spm["bytes"] / (spm["ms"] * 1e-3) / 1e9 if spm["ms"] > 0 else None,
        }
    g.close()
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="samg", choices=["samg", "reference"])
    ap.add_argument("--workload", type=int, default=2)
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--max-outer", type=int, default=300)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-small", action="store_true",
                    help="skip the small 32 x 32 Laplacian measurement reported beside the line")
    ap.add_argument("--arms", default="fp64,fp32",
                    help="precision arms to time, in order (the JSON line needs both)")
    ap.add_argument("--ncu-range", action="store_true",
                    help="bracket the timed mixed-precision solves with cudaProfilerStart/Stop "
                         "(for ncu --profile-from-start off)")
    ap.add_argument("--sweep-roofline", action="store_true",
                    help="time only level-0 relaxations at full size on a two-level "
                         "aggregation hierarchy and print their algorithmic GB/s")
    args = ap.parse_args()
    if args.sweep_roofline:
        return run_sweep_roofline(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
