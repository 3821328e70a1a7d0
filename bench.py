"""Benchmark: space-time unknowns solved per second to a true relative residual of 1e-8.

Workload (the line's `value`): 2D heat equation on the unit square, a = 1, 255 x 255 interior
nodes, Crank-Nicolson (theta = 1/2), n = 256 time steps, T = 1; right-hand side from the
manufactured solution u = sin(pi x) sin(pi y) e^t plus seeded N(0, 1e-3) noise on f_H
(16,646,400 unknowns).  One step = assemble f_H on the device + one full preconditioned MINRES
solve to ||r||/||b|| <= 1e-8 (mixed precision: float32 preconditioner inside float64
refinement).  The float64 path is timed too ("fp64").  Every vector (133 MB) exceeds L2.

Other legs (one object each): the 1D sine workload 63 x 64 (microseconds per solve), 2D BDF2 with
a variable coefficient at 511^2 x 128, 2D variable a under P_H and P_theta at 255^2 x 256, the 3D
Example 3 at 63^3 x 64, the adjoint workload (forward solve, transposed solve and gradients) at
255^2 x 256, and the 64-instance uneven batch.  Each solution is compared with the oracle's direct
solve (tests/golden/oracle_digest.json, sampled at seeded indices).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--no-extra]

With N > 1 (torchrun) every rank solves its own replica of the single-instance workloads (their
solve has no data-parallel split without exchanges), and the batch's instances are partitioned
over the ranks (paper_2201_10062_gb300.shard): no collective on the data path.
--impl reference times the CPU oracle on the host: each step is a bounded sample of oracle
MINRES iterations on the same workload, extrapolated to the oracle's iteration count.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import platform
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
CONFIG = {"workload": WORKLOAD, "mx": 255, "my": 255, "n": 256, "theta": 0.5, "unknowns": 16646400,
          "tol": TOL}
DIGEST = os.path.join(ROOT, "tests", "golden", "oracle_digest.json")

# Algorithmic bytes per unknown per MINRES iteration (Sec. 8(d) of the scope: every length-N
# vector of the minimal MINRES dataflow read or written once: 8 reads + 4 writes), float64 words
# except the preconditioned vector z, float32 in mixed precision; plus, per refinement step of the
# mixed solve, one residual (x and f_H read, r written).
ITER_BYTES = {"fp64": 96, "mixed": 84}
OUTER_BYTES = 24
# Bytes per unknown each launch of a kernel class moves (its own reads and writes of length-N
# vectors; the implementation's launches, not the algorithm's floor), mixed / float64.
# The mixed single solve's update applies G iterations per launch (grouped update): its bytes
# are counted per step by update_bytes_per_step instead.
CLASS_BYTES = {
    "mixed": {"stencil": 12, "lanczos_dst_x": 36, "dst_x": 8, "dst_y": 8, "time_dst_scale": 8,
              "residual": 24},
    "fp64": {"stencil": 16, "lanczos_dst_x": 40, "dst_x": 16, "dst_y": 16, "time_dst_scale": 16,
             "update": 48, "residual": 24},
}
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum, one ncu capture of every
# launch of one mixed 2D Crank-Nicolson solve at 255^2 x 256), per kernel class, for the kernels
# whose code is unchanged since: profiles/dram_traffic_mixed_cn2d_255x255_n256.md
# (the last x pass, now on the tensor cores, and the grouped update, now two elements per
# thread, have changed since, so they report none)
NCU_TRAFFIC = {("mixed", "stencil"): 136.0e6, ("mixed", "lanczos_dst_x"): 539.6e6,
               ("mixed", "residual"): 373.3e6}
NCU_TRAFFIC_STEP = {}
# the same capture summed over the solve's iteration kernels, per unknown and iteration: none
# while two of those kernels differ from the captured ones
NCU_ITER_TRAFFIC = {"mixed": None}
# steps of the per-kernel-class profile, run after each timed region
PROF_STEPS = 3


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


def load_digest():
    with open(DIGEST) as fh:
        return json.load(fh)["workloads"]


def sampled_rel_err(u, d):
    """||u[idx] - x*[idx]|| / ||x*[idx]|| at the digest's seeded indices (x* the oracle's direct
    solve): a sampled estimate of the relative 2-norm error against the oracle."""
    import numpy as np
    import torch

    idx = np.asarray(d["idx"])
    ref = np.asarray(d["val"])
    got = u.reshape(-1)[torch.as_tensor(idx, device=u.device)].double().cpu().numpy()
    return float(np.linalg.norm(got - ref) / np.linalg.norm(ref))


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return platform.processor() or platform.machine()


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

        dist.init_process_group(backend="nccl")
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


def batch_shard(draws, unknowns, world, rank):
    """The batch instances rank `rank` solves: greedy largest-first partition of the instances by
    cost (unknowns x estimated iterations) over the ranks; every rank computes the same split."""
    from paper_2201_10062_gb300 import shard

    costs = [shard.instance_cost(u, d["theta"]) for d, u in zip(draws, unknowns)]
    return shard.partition(costs, world)[rank]


def roofline_iter(precision, unknowns, iterations, outer, seconds, peak):
    """Sec. 8(d): algorithmic bytes of the whole solve (per-iteration bytes x iterations plus one
    residual per refinement step) over the solve time, against the measured HBM bandwidth."""
    alg = ITER_BYTES[precision] * unknowns * iterations + OUTER_BYTES * unknowns * outer
    achieved = alg / seconds / 1e9
    return {"bound": "hbm", "unit": "GB/s", "achieved": achieved, "peak": peak["hbm_gbs"],
            "frac": achieved / peak["hbm_gbs"], "peak_source": peak["src"],
            "alg_bytes_per_iteration": ITER_BYTES[precision] * unknowns,
            "alg_bytes_per_outer_step": OUTER_BYTES * unknowns, "iterations": iterations,
            "outer_steps": outer}


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

    def sample(self, seconds_budget, workers=1):
        """Seconds per oracle MINRES iteration from a run stopped once the budget is spent (the
        run's initial preconditioner application is included: a small over-estimate).  `workers`
        threads serve the oracle's FFTs (scipy.fft); its sparse products stay single-threaded."""
        import scipy.fft

        t0 = time.time()
        cnt = [0]

        def stop(k, x, est):
            cnt[0] = k
            return time.time() - t0 >= seconds_budget

        with scipy.fft.set_workers(workers):
            self.H.minres(self.Aop, self.Minv, self.b, 0.0, 400, stop=stop)
        elapsed = time.time() - t0
        done = max(cnt[0], 1)
        return elapsed / done, done, elapsed


def oracle_sample(seconds_budget=10.0):
    """The oracle's MINRES on the full bench system, one thread and all host cores."""
    leg = OracleLeg()
    cores = os.cpu_count() or 1
    model = cpu_model()
    res = {}
    for name, workers in (("single_thread", 1), ("all_cores", cores)):
        per_iter, done, elapsed = leg.sample(seconds_budget, workers)
        res[name] = {"value": leg.p.N / (per_iter * leg.iters), "unit": UNIT, "cores": workers,
                     "iterations_sampled": done, "seconds": elapsed,
                     "seconds_per_iteration": per_iter}
    best = res["all_cores"]
    return {
        "value": best["value"], "unit": UNIT, "cores": cores, "kind": "oracle",
        "cpu_model": model,
        "sample": (f"{best['iterations_sampled']} oracle MINRES iterations on the full {WORKLOAD} "
                   f"system ({best['seconds']:.1f} s, FFTs on {cores} threads), extrapolated to the "
                   f"oracle's {leg.iters} iterations to 1e-8 (tests/golden/oracle_counts.json)"),
        "single_thread": res["single_thread"], "all_cores": res["all_cores"],
    }


def run_reference(args, world, rank):
    if rank != 0:
        return
    steps, warm = args.steps, args.warmup
    leg = OracleLeg()
    cores = os.cpu_count() or 1
    times, sampled, wall = [], [], 0.0
    for i in range(warm + steps):
        per_iter, done, elapsed = leg.sample(1.0, cores)
        if i >= warm:
            times.append(per_iter)
            sampled.append(done)
            wall += elapsed
    per_iter = statistics.median(times)
    N = leg.p.N
    value = N / (per_iter * leg.iters)
    ext = {"iterations_sampled_per_step": sampled, "iterations_to_tol": leg.iters,
           "scale": leg.iters / statistics.median(sampled),
           "measured_seconds_per_step": wall / max(steps, 1),
           "note": "each step times oracle MINRES iterations on the full system for about 1 s and "
                   "extrapolates to the oracle's iteration count to 1e-8; ms_per_step is that "
                   "extrapolated full solve"}
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": steps, "warmup": warm, "ms_per_step": per_iter * leg.iters * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": dict(CONFIG, precision="fp64", parallelism="single"),
        "extrapolation": ext,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "cpu_model": cpu_model(),
                         "sample": f"each step: oracle MINRES iterations on the full system for "
                                   f"about 1 s (FFTs on {cores} threads), extrapolated to the "
                                   f"oracle's {leg.iters} iterations to 1e-8"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------ our arm
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


def update_bytes_per_step(unknowns, iterations, group):
    """Bytes the grouped update moves in one solve of `iterations` MINRES iterations: each launch
    reads its pending z_j (4 B each) and, once, the two latest directions and x (24 B), and
    writes the directions and x (24 B).  ceil(iterations / group) launches is the fewest that
    apply every update; a solve with several refinement steps may take one more per step, so the
    GB/s derived from this count is a lower bound."""
    return (4 * iterations + 48 * math.ceil(iterations / group)) * unknowns


def kernel_table(prof, precision, unknowns, steps, peak, iterations=None, group=None):
    """Per kernel class: time and launches per step, and for the classes with a fixed byte count
    per launch, that count, the achieved GB/s over the average launch and its fraction of HBM.
    The mixed path's grouped update gets bytes and GB/s per step (iterations and group given)."""
    total_ms = sum(v["ms"] for v in prof.values())
    out = {}
    for k, v in prof.items():
        row = {"ms_per_step": v["ms"] / steps, "launches_per_step": v["launches"] / steps,
               "share": (v["ms"] / total_ms if total_ms else None)}
        b = CLASS_BYTES[precision].get(k)
        if b is not None and v["timed"] > 0:
            avg_ms = v["ms"] / v["timed"]
            gbs = b * unknowns / (avg_ms * 1e-3) / 1e9
            row.update({"avg_launch_us": avg_ms * 1e3, "bytes_per_launch": b * unknowns,
                        "achieved_gbs": gbs, "frac_hbm": gbs / peak["hbm_gbs"],
                        "traffic": NCU_TRAFFIC.get((precision, k))})
        elif (precision, k) == ("mixed", "update") and iterations and v["ms"] > 0:
            bstep = update_bytes_per_step(unknowns, iterations, group)
            gbs = bstep / (v["ms"] / steps * 1e-3) / 1e9
            row.update({"avg_launch_us": v["ms"] / max(v["timed"], 1) * 1e3,
                        "iterations_per_launch": group, "bytes_per_step": bstep,
                        "achieved_gbs": gbs, "frac_hbm": gbs / peak["hbm_gbs"],
                        "traffic_per_step": NCU_TRAFFIC_STEP.get((precision, k))})
        out[k] = row
    return out


def run_ours(args, world, rank, local):
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
    digest = load_digest()

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
        with ClockSampler(local) as clk:
            e0.record(stream)
            for _ in range(steps):
                st = step(s, fH, u)
            e1.record(stream)
            torch.cuda.synchronize()
        barrier(world)
        ms = e0.elapsed_time(e1) / steps
        ms = max_over_ranks(ms, world)
        # per-kernel-class CUDA events (two per launch) on a further PROF_STEPS steps after the
        # timed region: recording them costs about 1 ms per solve of host enqueue time, so the
        # headline time is taken without them
        s.st_profile_begin(1 << 17)
        for _ in range(PROF_STEPS):
            step(s, fH, u)
        torch.cuda.synchronize()
        prof = s.st_profile_end()
        results[precision] = {"ms": ms, "stats": st, "clocks": clk.summary(), "prof": prof,
                              "steps": steps, "err": sampled_rel_err(u, digest["2d_cn_255_n256"]["u"])}
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

    extra = {} if args.no_extra else run_extra_workloads(P, W, stream, dev, world, rank, digest,
                                                         peaks)

    if rank != 0:
        return
    mixed = results["mixed"]
    steps = mixed["steps"]
    iters = mixed["stats"]["iterations"]
    outer = mixed["stats"]["outer_steps"]
    roof = roofline_iter("mixed", N, iters, outer, mixed["ms"] * 1e-3, peaks)
    roof["scope"] = ("whole solve: every kernel of every MINRES iteration plus the refinement "
                     "residuals, algorithmic bytes of Sec. 8(d)")
    # DRAM bytes of one iteration's launches from ncu, per iteration like alg_bytes_per_iteration
    it_traffic = NCU_ITER_TRAFFIC["mixed"]
    roof["traffic"] = it_traffic * N if it_traffic and (w.mx, w.n) == (255, 256) else None
    roof["traffic_unit"] = "bytes per MINRES iteration"
    kern = kernel_table(mixed["prof"], "mixed", N, PROF_STEPS, peaks, iterations=iters,
                        group=P.update_group())
    # kernels launched per step (the same solve every step), counted by the profiled steps
    launches = sum(v["launches"] for v in mixed["prof"].values()) / PROF_STEPS
    fp = results["fp64"]
    fp_roof = roofline_iter("fp64", N, fp["stats"]["iterations"], 1, fp["ms"] * 1e-3, peaks)
    # the oracle baseline runs at N = 1 only (under torchrun the other ranks have already left)
    cpu = oracle_sample() if world == 1 else None
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
        "config": dict(CONFIG, precision="mixed",
                       parallelism=("replicas" if world > 1 else "single"),
                       l2="no flush: every vector (133 MB) and the ~1.6 GB working set exceed L2"),
        "iterations": iters,
        "outer_steps": outer,
        "true_rel_res": mixed["stats"]["true_rel_res"],
        "error_vs_oracle": {"rel_err": mixed["err"], "estimate": "sampled at 2048 seeded indices",
                            "reference": "oracle direct solve (tests/golden/oracle_digest.json)"},
        "clocks": mixed["clocks"],
        "e2e": {k: v for k, v in results["e2e"].items()},
        "gpu_launches": int(round(launches * steps)),
        "gpu_launches_per_step": launches,
        "roofline": roof,
        "kernels": kern,
        "fp64": {"value": job_throughput(world, N, fp["ms"] * 1e-3), "ms_per_step": fp["ms"],
                 "iterations": fp["stats"]["iterations"], "true_rel_res": fp["stats"]["true_rel_res"],
                 "error_vs_oracle": fp["err"], "steps": fp["steps"], "clocks": fp["clocks"],
                 "dtype": "f64", "roofline": fp_roof,
                 "kernels": kernel_table(fp["prof"], "fp64", N, PROF_STEPS, peaks)},
        "cpu_baseline": cpu,
    }
    line.update(extra)
    print(json.dumps(line), flush=True)


def _solve_leg(P, w, spec, stream, dev, world, reps, digest_u=None, extra=None):
    """Time `reps` solves of workload w with spec after one warm-up (CUDA events); the error of the
    last solution against the oracle's direct solve when its digest is given."""
    import torch

    s = P.Solver(spec, stream)
    s.st_autotune()
    up = torch.tensor(w.u_prev, device=dev) if w.u_prev is not None else None
    ex = torch.tensor(extra, device=dev) if extra is not None else None
    fH = s.st_assemble_rhs(torch.tensor(w.f, device=dev), torch.tensor(w.u0, device=dev), up, ex)
    u = s.empty(w.n, w.m)
    s.st_solve(fH, tol=TOL, maxit=600, out=u)  # warm-up
    ms, (_, st) = _timed(stream, lambda: s.st_solve(fH, tol=TOL, maxit=600, out=u), reps)
    ms = max_over_ranks(ms, world)
    out = {"value": job_throughput(world, w.N, ms * 1e-3), "ms_per_step": ms,
           "iterations": st["iterations"], "outer_steps": st["outer_steps"],
           "true_rel_res": st["true_rel_res"], "steps": reps}
    if digest_u is not None:
        out["error_vs_oracle"] = sampled_rel_err(u, digest_u)
    s.close()
    return out


def adjoint_leg(P, W, stream, dev, world, digest, precision, reps):
    """Forward solve, transposed solve and the f, u0, a gradients of L = 1/2 ||u - u_obs||^2 on the
    adjoint workload (2D 255^2 x 256, backward Euler, gradients at a = (a_true + 1)/2), both solves
    to 1e-8.  u_obs = the solution at the seeded true a plus 1% seeded Gaussian noise; the digest
    takes that solution from the oracle's direct solve, this leg from a float64 solve on the
    device to 1e-11 (outside the timed region), which agree far below the errors reported."""
    import torch

    w = W.config_adjoint()
    a_true = w.a_nodal
    a_eval = 0.5 * (a_true + 1.0)
    f = torch.tensor(w.f, device=dev)
    u0 = torch.tensor(w.u0, device=dev)
    # observations: the float64 solution at the true coefficient (to 1e-11, near the attainable
    # relative residual of this system, condition ~1e5) plus 1% noise
    st_true = P.Solver(P.ProblemSpec(2, w.mx, w.my, w.n, w.T, "theta", 1.0, a_true, "PH", "fp64"),
                       stream)
    u_true, _ = st_true.st_solve(st_true.st_assemble_rhs(f, u0), tol=1e-11, maxit=800,
                                 allow_not_converged=True)
    st_true.close()
    noise = torch.tensor(w.extra["obs_normal"], device=dev).reshape(-1)
    u_true = u_true.reshape(-1)
    u_obs = u_true + 0.01 * torch.sqrt(torch.mean(u_true ** 2)) * noise
    del noise
    s = P.Solver(P.ProblemSpec(2, w.mx, w.my, w.n, w.T, "theta", 1.0, a_eval, "PH", precision), stream)
    s.st_autotune()
    fH = s.empty(w.n, w.m)
    u = s.empty(w.n, w.m)
    lam = s.empty(w.n * w.m)

    def run():
        s.st_assemble_rhs(f, u0, out=fH)
        _, st1 = s.st_solve(fH, tol=TOL, maxit=800, out=u)
        _, st2 = s.st_solve_transpose(u.reshape(-1) - u_obs, tol=TOL, maxit=800, out=lam)
        gf, gu0, _ = s.st_grad_rhs(lam)
        ga = s.st_grad_a(lam, u, u0)
        return st1, st2, gf, gu0, ga

    run()  # warm-up
    ms, (st1, st2, gf, gu0, ga) = _timed(stream, run, reps)
    ms = max_over_ranks(ms, world)
    d = digest["adjoint_255_n256"]
    errs = {"u": sampled_rel_err(u, d["u"]), "lam": sampled_rel_err(lam, d["lam"]),
            "grad_f": sampled_rel_err(gf, d["grad_f"]), "grad_u0": sampled_rel_err(gu0, d["grad_u0"]),
            "grad_a": sampled_rel_err(ga, d["grad_a"])}
    s.close()
    return {"value": job_throughput(world, w.N, ms * 1e-3), "ms_per_step": ms, "steps": reps,
            "forward_iterations": st1["iterations"], "adjoint_iterations": st2["iterations"],
            "true_rel_res": [st1["true_rel_res"], st2["true_rel_res"]],
            "error_vs_oracle": errs}


def run_extra_workloads(P, W, stream, dev, world, rank, digest, peaks):
    """The other workloads, one line object each (see the module docstring)."""
    import torch

    out = {}
    # ---- 1D sine, 63 x 64, backward Euler: latency-bound (4,032 unknowns), microseconds per solve
    w = W.config_1d_sine()
    res = {}
    for precision, reps in (("fp64", 50), ("mixed", 50)):
        spec = P.ProblemSpec(1, w.mx, 1, w.n, w.T, "theta", w.theta, None, "PH", precision)
        r = _solve_leg(P, w, spec, stream, dev, world, reps, digest["1d_sine_63_n64"]["u"])
        r["us_per_solve"] = r["ms_per_step"] * 1e3
        res[precision] = r
    out["sine1d_63_n64"] = {"unit": UNIT, "unknowns": w.N, "tol": TOL,
                            "note": "latency-bound: no roofline claim", **res}
    # ---- 2D variable a, BDF2, 511^2 x 128
    w = W.config_2d_varcoef_bdf2()
    res = {}
    for precision, reps in (("mixed", 3), ("fp64", 1)):
        spec = P.ProblemSpec(2, w.mx, w.my, w.n, w.T, "bdf2", 1.0, w.a_nodal, "PH", precision)
        r = _solve_leg(P, w, spec, stream, dev, world, reps, digest["2d_bdf2var_511_n128"]["u"])
        r["roofline"] = roofline_iter(precision, w.N, r["iterations"], r["outer_steps"],
                                      r["ms_per_step"] * 1e-3, peaks)
        res[precision] = r
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
    # ---- adjoint: forward + transposed solve + gradients, 255^2 x 256
    out["adjoint_255x255_n256"] = {
        "unit": UNIT, "unknowns": 16646400, "tol": TOL,
        "note": "value = unknowns / (forward solve + transposed solve + gradient kernels)",
        "mixed": adjoint_leg(P, W, stream, dev, world, digest, "mixed", 3),
        "fp64": adjoint_leg(P, W, stream, dev, world, digest, "fp64", 1),
    }
    torch.cuda.empty_cache()
    out["batch_64_uneven"] = batch_leg(P, W, stream, dev, world, rank)
    return out


def batch_leg(P, W, stream, dev, world, rank):
    """The 64-instance uneven batch, mixed precision, one batched solve (CUDA graph); with N > 1
    ranks the instances are partitioned over the ranks (no collective).  Also the same instances
    solved one by one in mixed and in float64 on each rank."""
    import torch

    draws = W.batch_draws(64, seed=4)
    ws_all = [W.config_2d_varcoef_theta(d["mx"], d["n"], d["theta"], d["seed"]) for d in draws]
    total = sum(x.N for x in ws_all)
    mine = batch_shard(draws, [x.N for x in ws_all], world, rank)
    ws = [ws_all[i] for i in mine]
    my_unknowns = sum(x.N for x in ws)
    specs = [P.ProblemSpec(2, x.mx, x.my, x.n, x.T, "theta", x.theta, x.a_nodal, "PH", "mixed")
             for x in ws]
    B = P.BatchSolver(specs, stream)
    fHs = [B.instance(i).st_assemble_rhs(torch.tensor(x.f, device=dev), torch.tensor(x.u0, device=dev))
           for i, x in enumerate(ws)]
    outs = [torch.empty_like(x) for x in fHs]
    B.st_solve_batch(fHs, tol=TOL, maxit=800, outs=outs)  # capture + warm-up
    barrier(world)
    ms_b, (_, stats) = _timed(stream, lambda: B.st_solve_batch(fHs, tol=TOL, maxit=800, outs=outs), 2)
    ms_b = max_over_ranks(ms_b, world)
    ok = all(q["status"] == 0 and q["true_rel_res"] <= TOL for q in stats)
    ok = max_over_ranks(0.0 if ok else 1.0, world) == 0.0
    iters = [q["iterations"] for q in stats]
    unknown_iters = sum(x.N * q["iterations"] for x, q in zip(ws, stats))
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

        barrier(world)
        ms, st = _timed(stream, one_by_one, 1)
        ms = max_over_ranks(ms, world)
        seq[precision] = {"value": total / (ms * 1e-3), "ms_per_step": ms,
                          "iterations_total": sum(q["iterations"] for q in st)}
        for sv in solvers:
            sv.close()
    del fHs, outs
    return {
        "unit": UNIT, "instances": 64, "unknowns": total, "tol": TOL,
        "ranks": world, "scaling": "strong (the 64 instances are split over the ranks)",
        "instances_this_rank": len(ws), "unknowns_this_rank": my_unknowns,
        "graph": {"value": total / (ms_b * 1e-3), "ms_per_step": ms_b, "steps": 2,
                  "all_converged": ok, "iterations_total": sum(iters),
                  "iterations_per_instance": iters,
                  "unknown_iterations_per_s": unknown_iters / (ms_b * 1e-3)},
        "one_by_one_mixed": seq["mixed"], "one_by_one_fp64": seq["fp64"],
    }


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
