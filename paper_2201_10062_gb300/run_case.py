"""Run solves of one synthetic workload from the command line (also the command the ncu profiles run).

  python -m paper_2201_10062_gb300.run_case --workload cn2d --mx 255 --n 256 --precision mixed \
      --repeat 3

Workloads (seeded, from ``workloads.synthetic``): ``cn2d`` (a = 1, Crank-Nicolson, manufactured
rhs + N(0, 1e-3) noise), ``bdf2var`` (random a field, BDF2), ``thetavar`` (random a field,
theta-method with --theta; with --prec Ptheta the Chebyshev inner map of --degree steps),
``sine1d`` (1D, backward Euler), ``sine3d`` (3D, a = 1, manufactured, --theta) and ``ex3``
(the paper's Example 3: 3D, a = 1e-3, f = 0, --theta; mx + 1 = m + 1 of Tables 6-7).
Prints one JSON line per solve with the iteration count, residuals and the time.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="cn2d", choices=["cn2d", "bdf2var", "thetavar", "sine1d", "sine3d", "ex3"])
    ap.add_argument("--mx", type=int, default=255)
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--prec", default="PH", choices=["PH", "Ptheta"])
    ap.add_argument("--theta", type=float, default=1.0, help="thetavar: theta of the time scheme")
    ap.add_argument("--degree", type=int, default=0, help="Ptheta, 2D varying a: Chebyshev steps")
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--maxit", type=int, default=400)
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--autotune", action="store_true", help="tune launch shapes before solving")
    args = ap.parse_args(argv)

    import torch

    import paper_2201_10062_gb300 as P
    from paper_2201_10062_gb300 import build
    from workloads import synthetic as W

    build.build()
    if args.workload == "cn2d":
        w = W.config_2d_sine_cn(mx=args.mx, n=args.n)
    elif args.workload == "bdf2var":
        w = W.config_2d_varcoef_bdf2(mx=args.mx, n=args.n)
    elif args.workload == "thetavar":
        w = W.config_2d_varcoef_theta(args.mx, args.n, args.theta, seed=5)
    elif args.workload == "sine3d":
        w = W.config_3d_sine(args.mx, args.n, theta=args.theta)
    elif args.workload == "ex3":
        w = W.paper_example3(args.mx, args.n, args.theta)
    else:
        w = W.config_1d_sine(mx=args.mx, n=args.n)
    spec = P.ProblemSpec(w.dim, w.mx, w.my, w.n, w.T, w.scheme, w.theta, w.a_nodal, args.prec,
                         args.precision, args.degree, w.mz)
    s = P.Solver(spec)
    if args.autotune:
        s.st_autotune()
    dev = s.device
    f = torch.tensor(w.f, device=dev)
    u0 = torch.tensor(w.u0, device=dev)
    up = torch.tensor(w.u_prev, device=dev) if w.u_prev is not None else None
    ex = torch.tensor(w.noise, device=dev) if w.noise is not None else None
    fH = s.st_assemble_rhs(f, u0, up, ex)
    for r in range(args.repeat):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        u, st = s.st_solve(fH, tol=args.tol, maxit=args.maxit)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        print(json.dumps({"workload": w.name, "unknowns": w.N, "precision": args.precision,
                          "prec": args.prec, "degree": args.degree,
                          "repeat": r, "seconds": dt, "unknowns_per_s": w.N / dt, **st}),
              flush=True)
    s.close()


if __name__ == "__main__":
    main()
