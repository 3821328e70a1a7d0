"""The paper's 2D examples at their largest sizes on the GPU (Sec. 5): Example 1 (a = 1e-5) and
Example 2 (a = 1e-5 sin(pi x y)) with n = 256, m + 1 = 256 (16,646,400 unknowns), solved in float64
to the paper's tolerance 1e-6.  The MINRES iteration counts of Tables 1-4 are reproduced within
two for P_H (both examples) and P_theta (Example 1); every solution's relative residual, checked
with the oracle's operator, is below the tolerance.

P_theta with Example 2's field converges faster here than the tables print (15 against 19 at the
largest size).  The oracle, with exact per-frequency solves, agrees with the GPU: it also needs 11
iterations at n = 32, m + 1 = 256 where Table 3 prints 16.  The paper does not say how its shifted
systems were solved.  Those rows check that the GPU needs no more iterations than printed, and a
separate test compares the GPU with the oracle on Example 2's P_theta."""
import numpy as np
import pytest

from oracle import heat as H
from workloads import synthetic as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2201_10062_gb300 as P
    from paper_2201_10062_gb300 import build

    build.build()
    P.load_library()
    return P


def _d(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


# (table, example, theta, prec, iterations printed for n = 2^8, m + 1 = 2^8)
ROWS = [
    ("Table 1", 1, 1.0, "PH", 14), ("Table 1", 1, 1.0, "Ptheta", 15),
    ("Table 2", 1, 0.5, "PH", 14), ("Table 2", 1, 0.5, "Ptheta", 15),
    ("Table 3", 2, 1.0, "PH", 15), ("Table 3", 2, 1.0, "Ptheta", 19),
    ("Table 4", 2, 0.5, "PH", 15), ("Table 4", 2, 0.5, "Ptheta", 19),
]


@pytest.mark.parametrize("table,example,theta,prec,iters", ROWS,
                         ids=[f"{r[0].replace(' ', '')}-{r[3]}" for r in ROWS])
def test_largest_2d_rows(pkg, table, example, theta, prec, iters):
    w = (W.paper_example1 if example == 1 else W.paper_example2)(255, 256, theta)
    # P_theta: the paper solves the shifted systems exactly; a constant a (Example 1) makes the
    # inner map exact in one step, and for Example 2's field (interval ratio at most 2.68) degree 8
    # keeps it within the Chebyshev bound 1/T_8 = 2.3e-5 of exact
    degree = 8 if prec == "Ptheta" else 0
    spec = pkg.ProblemSpec(2, w.mx, w.my, w.n, w.T, "theta", theta, w.a_nodal, prec, "fp64",
                           degree)
    s = pkg.Solver(spec)
    fH = s.st_assemble_rhs(_d(w.f), _d(w.u0))
    u, st = s.st_solve(fH, tol=1e-6, maxit=200)
    if example == 2 and prec == "Ptheta":
        assert st["iterations"] <= iters + 2, (table, prec, st)
    else:
        assert abs(st["iterations"] - iters) <= 2, (table, prec, st)
    p = H.Problem.from_workload(w)
    fH_or = H.rhs(p, w.f, w.u0)
    r = H.flip(fH_or, p.n) - H.apply_op(p, u.cpu().numpy().reshape(p.n, p.m))
    assert np.linalg.norm(r) / np.linalg.norm(fH_or) <= 1e-6 * (1 + 1e-6)
    s.close()


@pytest.mark.parametrize("theta", [1.0, 0.5])
def test_example2_ptheta_against_oracle(pkg, theta):
    """Example 2 with P_theta (Chebyshev inner map of degree 8) at n = 32, m + 1 = 128: the GPU's
    float64 iteration count equals the oracle's within one, at the paper's tolerance 1e-6."""
    w = W.paper_example2(127, 32, theta)
    p = H.Problem.from_workload(w, prec="Ptheta", inner_degree=8)
    fH = H.rhs(p, w.f, w.u0)
    _, info = H.solve(p, fH, tol=1e-6, maxit=100)
    spec = pkg.ProblemSpec(2, w.mx, w.my, w.n, w.T, "theta", theta, w.a_nodal, "Ptheta", "fp64", 8)
    s = pkg.Solver(spec)
    _, st = s.st_solve(_d(fH), tol=1e-6, maxit=100)
    assert abs(st["iterations"] - info["iterations"]) <= 1, (st, info["iterations"])
    s.close()


def test_table5_errors_on_gpu(pkg):
    """Example 2's backward-Euler errors printed in Table 5 (m + 1 = 32, three digits), from the
    GPU's float64 P_H solves at the paper's tolerance."""
    import json
    import os

    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                    "table5_backward_euler.json")))
    for n, ref in zip(g["n"], g["error"]):
        w = W.paper_example2(g["m_plus_1"] - 1, n, 1.0)
        s = pkg.Solver(pkg.ProblemSpec(2, w.mx, w.my, w.n, w.T, "theta", 1.0, w.a_nodal, "PH",
                                       "fp64"))
        fH = s.st_assemble_rhs(_d(w.f), _d(w.u0))
        u, _ = s.st_solve(fH, tol=1e-6, maxit=100)
        err = np.abs(u.cpu().numpy().reshape(w.n, w.m) - w.u_exact).max()
        assert float(f"{err:.2e}") == ref, (n, err, ref)
        s.close()
