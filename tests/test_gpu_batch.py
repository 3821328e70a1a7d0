"""Batched mixed-precision solves (one CUDA graph over many uneven instances) against the oracle."""
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


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


SMALL = [  # (mx, n, scheme, theta): uneven spatial sizes, n on and off the tensor-core path
    (15, 32, "theta", 0.5),
    (31, 64, "theta", 1.0),
    (63, 40, "theta", 0.5),
    (15, 17, "theta", 1.0),
    (31, 96, "bdf2", 1.0),
    (63, 128, "theta", 0.7),
]


def _instances(cases, seed0=60):
    ws = []
    for i, (mx, n, scheme, theta) in enumerate(cases):
        w = W.small_case(2, mx, mx, n, scheme=scheme, theta=theta, varcoef=True, seed=seed0 + i)
        ws.append(w)
    return ws


def test_batch_matches_oracle_and_single_solves(pkg):
    ws = _instances(SMALL)
    specs = [pkg.ProblemSpec(2, w.mx, w.my, w.n, w.T, w.scheme, w.theta, w.a_nodal, "PH", "mixed")
             for w in ws]
    B = pkg.BatchSolver(specs)
    fHs = []
    for i, w in enumerate(ws):
        s = B.instance(i)
        up = _d(w.u_prev) if w.u_prev is not None else None
        fHs.append(s.st_assemble_rhs(_d(w.f), _d(w.u0), up))
    outs, stats = B.st_solve_batch(fHs, tol=1e-10, maxit=600)
    for i, w in enumerate(ws):
        p = H.Problem.from_workload(w)
        fH = H.rhs(p, w.f, w.u0, w.u_prev)
        x_ref, _ = H.solve(p, fH, tol=1e-13, maxit=600)
        u = outs[i].cpu().numpy().reshape(p.n, p.m)
        assert stats[i]["status"] == 0 and stats[i]["true_rel_res"] <= 1e-10, stats[i]
        assert _rel(u, x_ref) <= 1e-8, (i, _rel(u, x_ref))
        # same refinement rules as the single-instance mixed solve
        single = pkg.Solver(specs[i])
        u1, st1 = single.st_solve(fHs[i], tol=1e-10, maxit=600)
        assert abs(st1["iterations"] - stats[i]["iterations"]) <= 2, (st1, stats[i])
        single.close()
    # a second solve reuses the captured graph and gives the same answers
    outs2, stats2 = B.st_solve_batch(fHs, tol=1e-10, maxit=600)
    for a, b in zip(outs, outs2):
        assert torch.equal(a, b)
    B.close()


def test_batch_of_64_uneven_instances(pkg):
    """64 instances drawn like the batched workload (mx+1 in {64,128,256}, n in {32..512},
    theta in {1/2, 1}, own coefficient field each), solved to 1e-8 in one graph; three sampled
    instances re-checked with the oracle's operator."""
    draws = W.batch_draws(64, seed=4)
    ws = [W.config_2d_varcoef_theta(d["mx"], d["n"], d["theta"], d["seed"]) for d in draws]
    specs = [pkg.ProblemSpec(2, w.mx, w.my, w.n, w.T, "theta", w.theta, w.a_nodal, "PH", "mixed")
             for w in ws]
    B = pkg.BatchSolver(specs)
    fHs = [B.instance(i).st_assemble_rhs(_d(w.f), _d(w.u0)) for i, w in enumerate(ws)]
    outs, stats = B.st_solve_batch(fHs, tol=1e-8, maxit=800)
    assert all(s["status"] == 0 and s["true_rel_res"] <= 1e-8 for s in stats)
    for i in (0, 17, 63):
        w = ws[i]
        p = H.Problem.from_workload(w)
        fH = H.rhs(p, w.f, w.u0)
        r = H.flip(fH, p.n) - H.apply_op(p, outs[i].cpu().numpy().reshape(p.n, p.m))
        assert np.linalg.norm(r) / np.linalg.norm(fH) <= 1e-8 * (1 + 1e-6)
    B.close()


def test_batch_mixes_preconditioners_and_dimensions(pkg):
    """One graph over instances with different preconditioner paths and grids: 2D P_H, 2D P_theta
    (Chebyshev inner map), 1D P_theta (PCR), 3D P_H and 3D P_theta.  Each instance against the
    oracle's converged solution and against its own single solve."""
    cases = [  # (dim, mx, my, mz, n, theta, prec, degree)
        (2, 31, 15, 1, 24, 0.5, "PH", 0),
        (2, 15, 31, 1, 32, 1.0, "Ptheta", 2),
        (1, 127, 1, 1, 40, 0.5, "Ptheta", 0),
        (3, 7, 15, 7, 16, 1.0, "PH", 0),
        (3, 15, 7, 7, 12, 0.5, "Ptheta", 3),
    ]
    ws, specs, probs = [], [], []
    for i, (dim, mx, my, mz, n, th, prec, deg) in enumerate(cases):
        w = W.small_case(dim, mx, my, n, scheme="theta", theta=th, varcoef=True, seed=90 + i, mz=mz)
        ws.append(w)
        specs.append(pkg.ProblemSpec(dim, mx, my, n, w.T, "theta", th, w.a_nodal, prec, "mixed",
                                     deg, mz))
        probs.append(H.Problem.from_workload(
            w, prec=prec, inner_degree=(deg or pkg.ST_PTHETA_DEFAULT_DEGREE) if dim >= 2 else None))
    B = pkg.BatchSolver(specs)
    fHs = [B.instance(i).st_assemble_rhs(_d(w.f), _d(w.u0)) for i, w in enumerate(ws)]
    outs, stats = B.st_solve_batch(fHs, tol=1e-10, maxit=600)
    for i, (w, p) in enumerate(zip(ws, probs)):
        fH = H.rhs(p, w.f, w.u0)
        x_ref, _ = H.solve(p, fH, tol=1e-13, maxit=600)
        u = outs[i].cpu().numpy().reshape(p.n, p.m)
        assert stats[i]["status"] == 0 and stats[i]["true_rel_res"] <= 1e-10, (i, stats[i])
        assert _rel(u, x_ref) <= 1e-8, (i, _rel(u, x_ref))
        single = pkg.Solver(specs[i])
        _, st1 = single.st_solve(fHs[i], tol=1e-10, maxit=600)
        assert abs(st1["iterations"] - stats[i]["iterations"]) <= 2, (i, st1, stats[i])
        single.close()
    B.close()


def test_batch_loops_end_on_budget_and_zero_rhs(pkg):
    """Each instance's device-side loop ends by itself: an instance whose iteration budget runs out
    reports ST_ERR_NOT_CONVERGED with its iterations capped, a zero right-hand side is done at
    once with u = 0, and the other instances of the same graph still converge."""
    ws = _instances(SMALL[:3], seed0=70)
    specs = [pkg.ProblemSpec(2, w.mx, w.my, w.n, w.T, w.scheme, w.theta, w.a_nodal, "PH", "mixed")
             for w in ws]
    B = pkg.BatchSolver(specs)
    fHs = [B.instance(i).st_assemble_rhs(_d(w.f), _d(w.u0)) for i, w in enumerate(ws)]
    fHs[1] = torch.zeros_like(fHs[1])
    outs, stats = B.st_solve_batch(fHs, tol=1e-10, maxit=600)
    assert stats[0]["status"] == 0 and stats[2]["status"] == 0
    assert stats[1]["status"] == 0 and stats[1]["iterations"] == 0
    assert float(outs[1].abs().max()) == 0.0
    # a budget of 3 iterations: no instance converges, each stops at the budget
    outs3, stats3 = B.st_solve_batch(fHs, tol=1e-10, maxit=3, allow_not_converged=True)
    for i in (0, 2):
        assert stats3[i]["status"] == pkg.ST_ERR_NOT_CONVERGED, stats3[i]
        assert stats3[i]["iterations"] <= 4, stats3[i]
    assert stats3[1]["status"] == 0
    # and the graph built for the full budget still solves afterwards
    outs4, stats4 = B.st_solve_batch(fHs, tol=1e-10, maxit=600)
    for a, b in zip(outs, outs4):
        assert torch.equal(a, b)
    B.close()
