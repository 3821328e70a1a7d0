"""Benchmark: space-time unknowns solved per second to a true relative residual of 1e-8.

Workload: 2D heat equation on the unit square, a = 1, 255 x 255 interior nodes, Crank-Nicolson
(theta = 1/2), n = 256 time steps, T = 1; right-hand side from the manufactured solution
u = sin(pi x) sin(pi y) e^t plus seeded N(0, 1e-3) noise on f_H (16,646,400 unknowns).
One step = assemble f_H on the device + one full preconditioned MINRES solve to ||r||/||b|| <=
1e-8 (mixed precision: float32 preconditioner inside float64 refinement).  The float64 path is
timed too and reported under "fp64".  Every vector (133 MB) is larger than L2.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun) every rank solves its own replica on its own GPU: the single-instance
solve has no data-parallel split without exchanges, so the multi-GPU form is replicas.
--impl reference times the CPU oracle (test infrastructure) on the host: each step is a bounded
sample of oracle MINRES iterations on the same workload, scaled by the oracle's iteration count.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "space-time unknowns solved/s to rel-res 1e-8 (FP64 vs mixed), % HBM roofline"
UNIT = "unknowns/s"
TOL = 1e-8
WORKLOAD = "2d_heat_cn_255x255_n256_a1_manufactured_noise1e-3"

# algorithmic bytes per unknown per launch for each kernel class (reads + writes of length-N
# vectors each launch must make), float64 / mixed
# Algorithmic bytes per unknown, per launch of each kernel class (each vector read or written
# once).  The Lanczos step is fused into the first x-DST of every preconditioner pass, so the
# two x-DST launches of an iteration move 36 + 8 (mixed) or 40 + 16 (FP64) bytes per unknown.
ALG_BYTES = {
    "fp64": {"stencil": 16, "lanczos": 32, "dst_x": 28, "dst_y": 16, "time_dst_scale": 16,
             "update": 48, "residual": 24},
    "mixed": {"stencil": 12, "lanczos": 32, "dst_x": 22, "dst_y": 8, "time_dst_scale": 8,
              "update": 44, "residual": 24},
}
# per MINRES iteration (2D): stencil + 2 x-DST + 2 y-DST + time kernel + update
ITER_BYTES = {"fp64": 16 + 56 + 32 + 16 + 48, "mixed": 12 + 44 + 16 + 8 + 44}
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum from one ncu capture of the
# mixed 2D Crank-Nicolson solve, 255^2 x 256), per kernel class, for the classes captured with the
# current kernels: profiles/k_dst_space_traffic_cn2d_255x255_n256.md
NCU_TRAFFIC = {("mixed", 255, 256, "dst_x"): 313.9e6}


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return {"hbm_gbs": float(d["hbm_gbs"]), "src": "measured", "sm_max_mhz": d.get("sm_max_mhz")}
    return {"hbm_gbs": 6800.0, "src": "fallback", "sm_max_mhz": 2070.0}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        rows = []
        for line in (self.out or "").strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, fl in rows for i, v in enumerate(fl)
                          if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def dist_setup():
    world = _env_int("WORLD_SIZE", 1)
    rank = _env_int("RANK", 0)
    local = _env_int("LOCAL_RANK", 0)
    if world > 1:
        import torch.distributed as dist

        backend = "nccl"
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(x, world):
    """The largest per-rank value (the slowest rank's time) on every rank: an NCCL all-reduce on a
    device scalar, or a host scalar under the gloo backend."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, units_per_rank, seconds):
    """Whole-job unknowns/s of N independent replicas (weak scaling): every rank solves its own
    copy, and the job takes as long as the slowest rank."""
    return world * units_per_rank / seconds


# ------------------------------------------------------------------------------ oracle legs
class OracleLeg:
    """The CPU oracle (test infrastructure) on the bench workload, timed in bounded samples."""

    def __init__(self):
        from oracle import heat as H
        from workloads import synthetic as W

        with open(os.path.join(ROOT, "tests", "golden", "oracle_counts.json")) as fh:
            self.iters = int(json.load(fh)["iterations"])
        self.H = H
        w = W.config_2d_sine_cn()
        self.p = p = H.Problem.from_workload(w)
        fH = H.rhs(p, w.f, w.u0) + w.noise
        K = H.stiffness(p)
        A = H.time_blocks(p, K)
        self.b = H.flip(fH, p.n)
        self.Minv = H._prec_apply(p, K)
        self.Aop = lambda v: H.apply_op(p, v, A)  # noqa: E731
        self.Aop(self.b)  # warm-up
        self.Minv(self.b)

    def sample(self, seconds_budget):
        """Seconds per oracle MINRES iteration, from a run stopped once the budget is spent (the
        run's initial preconditioner application is included: a small over-estimate)."""
        t0 = time.time()
        cnt = [0]

        def stop(k, x, est):
            cnt[0] = k
            return time.time() - t0 >= seconds_budget

        self.H.minres(self.Aop, self.Minv, self.b, 0.0, 400, stop=stop)
        elapsed = time.time() - t0
        done = max(cnt[0], 1)
        return elapsed / done, done, elapsed


def oracle_sample(seconds_budget=12.0):
    leg = OracleLeg()
    per_iter, done, elapsed = leg.sample(seconds_budget)
    t_solve = per_iter * leg.iters
    return {
        "value": leg.p.N / t_solve,
        "unit": UNIT,
        "cores": 1,
        "kind": "oracle",
        "sample": (f"{done} oracle MINRES iterations on the full {WORKLOAD} system "
                   f"({elapsed:.1f} s), scaled to the oracle's {leg.iters} iterations to 1e-8 "
                   f"(tests/golden/oracle_counts.json); numpy/scipy, single-threaded FFTs"),
        "seconds_per_iteration": per_iter,
    }


def run_reference(args, world, rank):
    if rank != 0:
        return
    steps, warm = args.steps, args.warmup
    leg = OracleLeg()
    times = []
    for i in range(warm + steps):
        per_iter, done, _ = leg.sample(1.0)
        if i >= warm:
            times.append(per_iter)
    per_iter = statistics.median(times)
    N = leg.p.N
    value = N / (per_iter * leg.iters)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": steps, "warmup": warm, "ms_per_step": per_iter * leg.iters * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "tol": TOL},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"each step: oracle MINRES iterations on the full system for "
                                   f"about 1 s (at least one), scaled to the oracle's "
                                   f"{leg.iters} iterations to 1e-8"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------ our arm
def run_ours(args, world, rank, local):
    import numpy as np
    import torch

    import __graft_entry__ as ge

    torch.cuda.set_device(local)
    if rank == 0 or world > 1:
        ge.build()
    import paper_2201_10062_gb300 as P
    from workloads import synthetic as W

    w = W.config_2d_sine_cn()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    f = torch.tensor(w.f, device=dev)
    u0 = torch.tensor(w.u0, device=dev)
    noise = torch.tensor(w.noise, device=dev)
    N = w.N
    peaks = load_peaks()

    def make(precision):
        spec = P.ProblemSpec(w.dim, w.mx, w.my, w.n, w.T, w.scheme, w.theta, None, "PH", precision)
        s = P.Solver(spec, stream)
        s.st_autotune()  # launch shapes for this size (part of the public API; timed outside)
        fH = s.empty(w.n, w.m)
        u = s.empty(w.n, w.m)
        return s, fH, u

    def step(s, fH, u):
        s.st_assemble_rhs(f, u0, extra=noise, out=fH)
        _, st = s.st_solve(fH, tol=TOL, maxit=400, out=u)
        return st

    results = {}
    for precision, steps in (("mixed", args.steps), ("fp64", max(2, args.steps // 4))):
        s, fH, u = make(precision)
        for _ in range(args.warmup):
            st = step(s, fH, u)
        torch.cuda.synchronize()
        barrier(world)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        prof = None
        with ClockSampler(local) as clk:
            if precision == "mixed":
                s.st_profile_begin(1 << 17)
            e0.record(stream)
            for _ in range(steps):
                st = step(s, fH, u)
            e1.record(stream)
            torch.cuda.synchronize()
            if precision == "mixed":
                prof = s.st_profile_end()
        barrier(world)
        ms = e0.elapsed_time(e1) / steps
        ms = max_over_ranks(ms, world)
        results[precision] = {"ms": ms, "stats": st, "clocks": clk.summary(), "prof": prof,
                              "steps": steps}
        if precision == "mixed":
            # end to end through the public API with host buffers: H2D of f_H, solve, D2H of u
            fH_host = torch.empty(N, dtype=torch.float64, pin_memory=True)
            fH_host.copy_(fH.reshape(-1))
            u_host = torch.empty(N, dtype=torch.float64, pin_memory=True)
            s.st_solve_host(fH_host, u_host, tol=TOL, maxit=400)
            torch.cuda.synchronize()
            barrier(world)
            t0 = time.perf_counter()
            e2e_steps = max(2, steps // 2)
            for _ in range(e2e_steps):
                s.st_solve_host(fH_host, u_host, tol=TOL, maxit=400)
            t_e2e = (time.perf_counter() - t0) / e2e_steps
            t_e2e = max_over_ranks(t_e2e, world)
            results["e2e"] = {"value": job_throughput(world, N, t_e2e), "unit": UNIT,
                              "h2d_bytes_per_step": N * 8, "d2h_bytes_per_step": N * 8,
                              "ms_per_step": t_e2e * 1e3}
        s.close()

    extra = {} if args.no_extra else run_extra_workloads(P, W, stream, dev, world)

    if rank != 0:
        return
    mixed = results["mixed"]
    prof = mixed["prof"]
    steps = mixed["steps"]
    # dominant kernel class and its live roofline
    classes = {k: v for k, v in prof.items() if k != "aux" and v["timed"] > 0}
    total_ms = sum(v["ms"] for v in prof.values())
    dom = max(classes, key=lambda k: classes[k]["ms"])
    d = classes[dom]
    avg_ms = d["ms"] / d["timed"]
    alg_bytes = ALG_BYTES["mixed"][dom] * N
    achieved = alg_bytes / (avg_ms * 1e-3) / 1e9
    launches = sum(v["launches"] for v in prof.values())
    roofline = {
        "bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peaks["hbm_gbs"],
        "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
        "traffic": NCU_TRAFFIC.get(("mixed", w.mx, w.n, dom)),
        "peak_source": peaks["src"], "alg_bytes_per_launch": alg_bytes,
        "avg_launch_ms": avg_ms,
        "share_of_kernel_time": d["ms"] / total_ms if total_ms else None,
    }
    iters = mixed["stats"]["iterations"]
    # whole-solve roofline: algorithmic bytes per iteration x iterations at the measured HBM
    # bandwidth, over the solve time
    solve_frac = (ITER_BYTES["mixed"] * N * iters / (peaks["hbm_gbs"] * 1e9)) / (mixed["ms"] * 1e-3)
    per_class = {k: {"ms_per_step": v["ms"] / steps, "launches_per_step": v["launches"] / steps,
                     "share": (v["ms"] / total_ms if total_ms else None)}
                 for k, v in prof.items()}
    fp = results["fp64"]
    # the oracle baseline runs at N = 1 only (under torchrun the other ranks have already left)
    cpu = oracle_sample(seconds_budget=12.0) if world == 1 else None
    value = job_throughput(world, N, mixed["ms"] * 1e-3)
    line = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": steps,
        "warmup": args.warmup,
        "ms_per_step": mixed["ms"],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64+f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "mx": 255, "my": 255, "n": 256, "theta": 0.5,
                   "unknowns": N, "tol": TOL, "precision": "mixed", "parallelism":
                   ("replicas" if world > 1 else "single"),
                   "l2": "no flush: every vector (133 MB) and the ~1.1 GB working set exceed L2"},
        "iterations": iters,
        "outer_steps": mixed["stats"]["outer_steps"],
        "true_rel_res": mixed["stats"]["true_rel_res"],
        "clocks": mixed["clocks"],
        "e2e": {k: v for k, v in results["e2e"].items()},
        "gpu_launches": launches // steps * steps,
        "gpu_launches_per_step": launches / steps,
        "roofline": roofline,
        "solve_hbm_frac": solve_frac,
        "kernels": per_class,
        "fp64": {"value": job_throughput(world, N, fp["ms"] * 1e-3), "ms_per_step": fp["ms"],
                 "iterations": fp["stats"]["iterations"], "true_rel_res": fp["stats"]["true_rel_res"],
                 "steps": fp["steps"], "clocks": fp["clocks"], "dtype": "f64",
                 "solve_hbm_frac": (ITER_BYTES["fp64"] * N * fp["stats"]["iterations"]
                                    / (peaks["hbm_gbs"] * 1e9)) / (fp["ms"] * 1e-3)},
        "cpu_baseline": ({k: cpu[k] for k in ("value", "unit", "cores", "kind", "sample")}
                         if cpu is not None else None),
    }
    line.update(extra)
    print(json.dumps(line), flush=True)


def _timed(stream, fn, reps):
    import torch

    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    out = None
    for _ in range(reps):
        out = fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps, out


def _solve_leg(P, w, spec, stream, dev, world, reps):
    """Time `reps` solves of workload w with spec after one warm-up (CUDA events)."""
    import torch

    s = P.Solver(spec, stream)
    s.st_autotune()
    up = torch.tensor(w.u_prev, device=dev) if w.u_prev is not None else None
    fH = s.st_assemble_rhs(torch.tensor(w.f, device=dev), torch.tensor(w.u0, device=dev), up)
    u = s.empty(w.n, w.m)
    s.st_solve(fH, tol=TOL, maxit=600, out=u)  # warm-up
    ms, (_, st) = _timed(stream, lambda: s.st_solve(fH, tol=TOL, maxit=600, out=u), reps)
    ms = max_over_ranks(ms, world)
    s.close()
    return {"value": job_throughput(world, w.N, ms * 1e-3), "ms_per_step": ms, "iterations": st["iterations"],
            "true_rel_res": st["true_rel_res"], "steps": reps}


def run_extra_workloads(P, W, stream, dev, world):
    """The other solve workloads, one line object each: 2D variable-coefficient BDF2 at
    511^2 x 128 (mixed and FP64); 2D variable a with the theta-method at 255^2 x 256 under P_H and
    under P_theta with its Chebyshev inner map; the paper's 3D Example 3 at 63^3 x 64; and the
    64-instance uneven batch (one captured graph, mixed) against the same 64 instances solved one
    by one in mixed and in FP64."""
    import torch

    out = {}
    # ---- 2D variable a, BDF2, 511^2 x 128
    w = W.config_2d_varcoef_bdf2()
    f = torch.tensor(w.f, device=dev)
    u0 = torch.tensor(w.u0, device=dev)
    up = torch.tensor(w.u_prev, device=dev)
    res = {}
    for precision, reps in (("mixed", 3), ("fp64", 1)):
        s = P.Solver(P.ProblemSpec(2, w.mx, w.my, w.n, w.T, "bdf2", 1.0, w.a_nodal, "PH", precision),
                     stream)
        s.st_autotune()
        fH = s.st_assemble_rhs(f, u0, up)
        u = s.empty(w.n, w.m)
        s.st_solve(fH, tol=TOL, maxit=600, out=u)  # warm-up
        ms, (_, st) = _timed(stream, lambda: s.st_solve(fH, tol=TOL, maxit=600, out=u), reps)
        ms = max_over_ranks(ms, world)
        res[precision] = {"value": job_throughput(world, w.N, ms * 1e-3), "ms_per_step": ms,
                          "iterations": st["iterations"], "true_rel_res": st["true_rel_res"],
                          "steps": reps}
        s.close()
    del f, u0, up
    out["bdf2_var_511x511_n128"] = {"unit": UNIT, "unknowns": w.N, "tol": TOL, **res}
    # ---- 2D variable a, theta = 1, 255^2 x 256: P_H against P_theta (Chebyshev inner map)
    w = W.config_2d_varcoef_theta(255, 256, 1.0, seed=5)

    def spec2(prec, precision):
        return P.ProblemSpec(2, w.mx, w.my, w.n, w.T, "theta", 1.0, w.a_nodal, prec, precision)

    out["ptheta_var_255x255_n256"] = {
        "unit": UNIT, "unknowns": w.N, "tol": TOL,
        "inner_degree": P.ST_PTHETA_DEFAULT_DEGREE,
        "PH_mixed": _solve_leg(P, w, spec2("PH", "mixed"), stream, dev, world, 3),
        "Ptheta_mixed": _solve_leg(P, w, spec2("Ptheta", "mixed"), stream, dev, world, 3),
        "Ptheta_fp64": _solve_leg(P, w, spec2("Ptheta", "fp64"), stream, dev, world, 1),
    }
    # ---- 3D, Sec. 5 Example 3 (a = 1e-3, f = 0), 63^3 x 64 = 16,003,008 unknowns
    w = W.paper_example3(63, 64, 1.0)

    def spec3(prec, precision):
        return P.ProblemSpec(3, w.mx, w.my, w.n, w.T, "theta", 1.0, w.a_nodal, prec, precision,
                             0, w.mz)

    out["example3_3d_63x63x63_n64"] = {
        "unit": UNIT, "unknowns": w.N, "tol": TOL,
        "PH_mixed": _solve_leg(P, w, spec3("PH", "mixed"), stream, dev, world, 3),
        "Ptheta_mixed": _solve_leg(P, w, spec3("Ptheta", "mixed"), stream, dev, world, 3),
        "PH_fp64": _solve_leg(P, w, spec3("PH", "fp64"), stream, dev, world, 1),
    }
    # ---- 64 uneven instances
    draws = W.batch_draws(64, seed=4)
    ws = [W.config_2d_varcoef_theta(d["mx"], d["n"], d["theta"], d["seed"]) for d in draws]
    total = sum(x.N for x in ws)
    specs = [P.ProblemSpec(2, x.mx, x.my, x.n, x.T, "theta", x.theta, x.a_nodal, "PH", "mixed")
             for x in ws]
    B = P.BatchSolver(specs, stream)
    fHs = [B.instance(i).st_assemble_rhs(torch.tensor(x.f, device=dev), torch.tensor(x.u0, device=dev))
           for i, x in enumerate(ws)]
    outs = [torch.empty_like(x) for x in fHs]
    B.st_solve_batch(fHs, tol=TOL, maxit=800, outs=outs)  # capture + warm-up
    ms_b, (_, stats) = _timed(stream, lambda: B.st_solve_batch(fHs, tol=TOL, maxit=800, outs=outs), 2)
    ms_b = max_over_ranks(ms_b, world)
    ok = all(q["status"] == 0 and q["true_rel_res"] <= TOL for q in stats)
    B.close()
    seq = {}
    for precision in ("mixed", "fp64"):
        solvers = [P.Solver(sp if precision == "mixed" else
                            P.ProblemSpec(2, x.mx, x.my, x.n, x.T, "theta", x.theta, x.a_nodal, "PH",
                                          "fp64"), stream) for sp, x in zip(specs, ws)]
        for sv in solvers:  # same launch shapes as the batch (per-shape cache)
            sv.st_autotune()

        def one_by_one():
            return [sv.st_solve(fh, tol=TOL, maxit=800, out=o)[1] for sv, fh, o in zip(solvers, fHs, outs)]

        ms, st = _timed(stream, one_by_one, 1)
        ms = max_over_ranks(ms, world)
        seq[precision] = {"value": job_throughput(world, total, ms * 1e-3), "ms_per_step": ms,
                          "iterations_total": sum(q["iterations"] for q in st)}
        for sv in solvers:
            sv.close()
    del fHs, outs
    out["batch_64_uneven"] = {
        "unit": UNIT, "instances": 64, "unknowns": total, "tol": TOL,
        "graph": {"value": job_throughput(world, total, ms_b * 1e-3), "ms_per_step": ms_b, "steps": 2,
                  "all_converged": ok, "iterations_total": sum(q["iterations"] for q in stats)},
        "one_by_one_mixed": seq["mixed"], "one_by_one_fp64": seq["fp64"],
    }
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=8)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extra", action="store_true",
                    help="time only the 2D Crank-Nicolson 255^2 x 256 workload")
    args = ap.parse_args()
    if args.impl == "reference":
        world = _env_int("WORLD_SIZE", 1)
        rank = _env_int("RANK", 0)
        run_reference(args, world, rank)
        return
    world, rank, local = dist_setup()
    run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
