"""Write oracle_digest.json: exact solutions of the measured workloads, sampled.

For each workload the all-at-once system T u = f_H is solved directly by the oracle's block
forward substitution (T is block lower triangular, Sec. 1), which is exact up to the rounding of
the sparse LU solves; the transposed system of the adjoint workload goes through T^T = Y T Y.
The file keeps, per vector, its 2-norm and its values at seeded indices, so that a test or a
bench leg can state the relative error of a GPU solution against the oracle without holding the
oracle's full vector (133-267 MB at these sizes):

    err = ||u[idx] - x*[idx]||_2 / ||x*[idx]||_2     (a sampled estimate of ||u - x*|| / ||x*||)

Workloads (seeded inputs from workloads.synthetic):
  1d_sine_63_n64        1D, 63 points, backward Euler, n = 64 (4,032 unknowns)
  2d_cn_255_n256        2D 255^2, Crank-Nicolson, n = 256, a = 1, manufactured rhs + N(0, 1e-3)
  2d_bdf2var_511_n128   2D 511^2, BDF2, n = 128, seeded variable a
  adjoint_255_n256      2D 255^2, backward Euler, n = 256: forward solution u at the evaluation
                        coefficient, adjoint lam = T^-T (u - u_obs) and the gradients of
                        L = 1/2 ||u - u_obs||^2 (u_obs = solution at the true coefficient plus 1%
                        Gaussian noise)
For 2d_cn_255_n256 it also records the error of the oracle's own MINRES solve stopped at the
bench tolerance (true relative residual 1e-8), i.e. what an exact-arithmetic solve at that
tolerance attains.

Calls only oracle/ (and the seeded inputs).  Takes several minutes.
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import heat as H  # noqa: E402
from workloads import synthetic as W  # noqa: E402

SAMPLES = 2048


def sample(vec, seed, count=SAMPLES):
    v = np.asarray(vec, dtype=np.float64).reshape(-1)
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(v.size, size=min(count, v.size), replace=False))
    return {"size": int(v.size), "norm2": float(np.linalg.norm(v)), "idx": [int(i) for i in idx],
            "val": [float(x) for x in v[idx]]}


def sampled_rel(u, d):
    idx = np.asarray(d["idx"])
    ref = np.asarray(d["val"])
    return float(np.linalg.norm(np.asarray(u).reshape(-1)[idx] - ref) / np.linalg.norm(ref))


def main():
    out = {"written_by": "tests/golden/make_oracle_digest.py (oracle only)",
           "method": "oracle forward_substitution (direct block solve of T u = f_H)",
           "samples": SAMPLES, "workloads": {}}
    t0 = time.time()

    w = W.config_1d_sine()
    p = H.Problem.from_workload(w)
    u = H.forward_substitution(p, H.rhs(p, w.f, w.u0))
    out["workloads"]["1d_sine_63_n64"] = {"N": p.N, "u": sample(u, 101, count=p.N)}
    print("1d done", time.time() - t0, flush=True)

    w = W.config_2d_sine_cn()
    p = H.Problem.from_workload(w)
    fH = H.rhs(p, w.f, w.u0) + w.noise
    u = H.forward_substitution(p, fH)
    ent = {"N": p.N, "u": sample(u, 102)}
    # the oracle's own MINRES at the bench tolerance, against the exact solution
    x8, info = H.solve(p, fH, tol=1e-8, maxit=400)
    ent["oracle_minres_tol1e-8"] = {
        "iterations": info["iterations"], "true_rel_res": info["true_rel_res"],
        "rel_err": float(np.linalg.norm(x8 - u) / np.linalg.norm(u)),
        "sampled_rel_err": sampled_rel(x8, ent["u"])}
    out["workloads"]["2d_cn_255_n256"] = ent
    del x8, fH, u
    print("2d cn done", time.time() - t0, flush=True)

    w = W.config_2d_varcoef_bdf2()
    p = H.Problem.from_workload(w)
    u = H.forward_substitution(p, H.rhs(p, w.f, w.u0, w.u_prev))
    out["workloads"]["2d_bdf2var_511_n128"] = {"N": p.N, "u": sample(u, 103)}
    del u
    print("bdf2 done", time.time() - t0, flush=True)

    w = W.config_adjoint()
    p_true = H.Problem.from_workload(w)
    u_true = H.march(p_true, w.f, w.u0)
    u_obs = u_true + 0.01 * np.sqrt(np.mean(u_true ** 2)) * w.extra["obs_normal"]
    a_eval = 0.5 * (w.a_nodal + 1.0)
    w.a_nodal = a_eval
    p = H.Problem.from_workload(w)
    u = H.march(p, w.f, w.u0)
    g = u - u_obs
    lam = H.flip(H.forward_substitution(p, H.flip(g, p.n)), p.n)
    gf, gu0, ga = H.adjoint_gradients(p, u, lam, w.u0)
    out["workloads"]["adjoint_255_n256"] = {
        "N": p.N, "loss": float(0.5 * np.sum(g ** 2)),
        "u": sample(u, 104), "lam": sample(lam, 105), "grad_f": sample(gf, 106, count=1024),
        "grad_u0": sample(gu0, 107, count=1024), "grad_a": sample(ga, 108, count=1024)}
    print("adjoint done", time.time() - t0, flush=True)

    out["seconds_here"] = time.time() - t0
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_digest.json")
    with open(path, "w") as fh:
        json.dump(out, fh, separators=(",", ":"))
    print(json.dumps({k: (v if k != "workloads" else list(v)) for k, v in out.items()}))


if __name__ == "__main__":
    main()
