"""Write oracle_counts.json: the oracle's MINRES iteration count to a true relative residual of
1e-8 on the 2D Crank-Nicolson workload (255^2 interior nodes, n = 256, a = 1, manufactured rhs
plus seeded N(0, 1e-3) noise), and the time of one oracle iteration on this machine.

Calls only oracle/ (and the seeded inputs).  The bench's CPU baseline scales its timed sample
of oracle iterations by this count.  Takes a few minutes.
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import heat as H  # noqa: E402
from workloads import synthetic as W  # noqa: E402


def main():
    w = W.config_2d_sine_cn()
    p = H.Problem.from_workload(w)
    fH = H.rhs(p, w.f, w.u0) + w.noise
    t0 = time.time()
    x, info = H.solve(p, fH, tol=1e-8, maxit=400)
    dt = time.time() - t0
    out = {
        "workload": "2d_cn_255x255_n256_a1_noise1e-3",
        "tol": 1e-8,
        "iterations": info["iterations"],
        "true_rel_res": info["true_rel_res"],
        "true_checks": info["true_checks"],
        "solve_seconds_here": dt,
        "written_by": "tests/golden/make_oracle_counts.py (oracle only)",
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_counts.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
