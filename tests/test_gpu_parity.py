"""Parity of the CUDA path (through the C ABI) with the CPU oracle on the same seeded inputs."""
import json
import math
import os

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


def _spec(P, w, prec="PH", precision="fp64"):
    return P.ProblemSpec(w.dim, w.mx, w.my, w.n, w.T, w.scheme, w.theta, w.a_nodal, prec, precision)


def _d(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _h(t):
    return t.detach().cpu().numpy()


def _rel_max(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _rel2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


EPS = np.finfo(np.float64).eps


def _prec_tol(p, engine="dd"):
    """Tolerance for the float64 path's P^-1 v against the oracle.  The float64 engine: a
    log-depth FFT plus an n/2-term dense sum, 1e-12.  The double-float engine (the default): the
    same operations with 48-bit significands (unit roundoff 2^-48, 32 times float64's), 1e-11;
    it measured 1.0e-12 on the full 255^2 x 256 vector.  With a varying coefficient the averaged-K
    eigenvalues d - 2 e_x cos - 2 e_y cos cancel by max(mu)/min(mu) at the lowest modes, so
    last-bit differences in the averages (summation order) are amplified by that ratio."""
    base = 1e-11 if engine == "dd" else 1e-12
    if p.a_nodal is None:
        return base
    mu = H.averaged_stiffness_eigs(p)
    return max(base, 16 * EPS * mu.max() / mu.min())


def _ptheta_tol32(p):
    """float32 P_theta tolerance: the per-frequency matrices lam_H + lam_Htheta tau K have
    condition number up to about (2 + tau mu_max)/(lam_H,min + lam_Htheta,min tau mu_min)."""
    K = H.stiffness(p)
    ev = np.linalg.eigvalsh(K.toarray()) if p.m <= 1100 else None
    lh, lt = H.ptheta_time_eigs(p.n, p.theta)
    mu_min, mu_max = ev.min(), ev.max()
    cond = max((lh + lt * p.tau * mu_max) / (lh + lt * p.tau * mu_min))
    return max(2e-5, 4 * 2.0 ** -24 * cond)


# (dim, mx, my, n, scheme, theta, varcoef): ragged tiles (mx odd vs 32-wide blocks), odd and
# even n, n = 1 and 2, 1D and 2D, constant and varying a.
CASES = [
    (1, 7, 1, 5, "theta", 1.0, False),
    (1, 63, 1, 64, "theta", 1.0, False),
    (1, 127, 1, 37, "theta", 0.5, True),
    (1, 31, 1, 1, "theta", 0.5, True),
    (1, 15, 1, 2, "bdf2", 1.0, True),
    (2, 3, 3, 1, "theta", 0.5, False),
    (2, 15, 15, 16, "theta", 0.5, True),
    (2, 31, 7, 33, "theta", 1.0, False),
    (2, 7, 31, 2, "bdf2", 1.0, True),
    (2, 63, 63, 40, "bdf2", 1.0, True),
    (2, 63, 31, 65, "theta", 0.3, True),
]


def _ids(c):
    return f"{c[0]}d-{c[1]}x{c[2]}-n{c[3]}-{c[4]}{c[5]}-{'var' if c[6] else 'const'}"


@pytest.mark.parametrize("case", CASES, ids=[_ids(c) for c in CASES])
def test_apply_op_and_rhs(pkg, case):
    dim, mx, my, n, scheme, theta, var = case
    w = W.small_case(dim, mx, my, n, scheme=scheme, theta=theta, varcoef=var, seed=mx + n)
    p = H.Problem.from_workload(w)
    s = pkg.Solver(_spec(pkg, w))
    v = np.random.default_rng(1).standard_normal((n, p.m))
    y = _h(s.st_apply_op(_d(v))).reshape(n, p.m)
    assert _rel_max(y, H.apply_op(p, v)) <= 1e-13
    up = _d(w.u_prev) if w.u_prev is not None else None
    fH = _h(s.st_assemble_rhs(_d(w.f), _d(w.u0), up)).reshape(n, p.m)
    assert _rel_max(fH, H.rhs(p, w.f, w.u0, w.u_prev)) <= 1e-13
    s.close()


@pytest.mark.parametrize("case", CASES, ids=[_ids(c) for c in CASES])
def test_apply_prec_fp64_and_fp32(pkg, case):
    dim, mx, my, n, scheme, theta, var = case
    w = W.small_case(dim, mx, my, n, scheme=scheme, theta=theta, varcoef=var, seed=2 * mx + n)
    p = H.Problem.from_workload(w)
    s = pkg.Solver(_spec(pkg, w))
    v = np.random.default_rng(2).standard_normal((n, p.m))
    ref = H.apply_prec(p, v)
    z = _h(s.st_apply_prec(_d(v))).reshape(n, p.m)
    assert _rel_max(z, ref) <= _prec_tol(p)
    z32 = _h(s.st_apply_prec_f32(_d(v))).astype(np.float64).reshape(n, p.m)
    assert _rel2(z32, ref) <= 2e-5
    # in place
    vd = _d(v)
    s.st_apply_prec(vd, out=vd)
    assert _rel_max(_h(vd).reshape(n, p.m), ref) <= _prec_tol(p)
    s.close()


@pytest.mark.parametrize("case", [
    (1, 63, 1, 64, "theta", 1.0, False),
    (2, 31, 31, 32, "theta", 0.5, True),
    (2, 63, 15, 24, "bdf2", 1.0, True),
    (2, 15, 31, 17, "theta", 1.0, False),
], ids=_ids)
def test_solve_equal_iterations(pkg, case):
    """Same number of MINRES iterations on both sides: solutions agree to 1e-10 (relative 2-norm)."""
    dim, mx, my, n, scheme, theta, var = case
    w = W.small_case(dim, mx, my, n, scheme=scheme, theta=theta, varcoef=var, seed=5)
    p = H.Problem.from_workload(w)
    fH = H.rhs(p, w.f, w.u0, w.u_prev)
    s = pkg.Solver(_spec(pkg, w))
    for K in (1, 2, 7, 15):
        u, st = s.st_solve(_d(fH), tol=0.0, maxit=K, allow_not_converged=True)
        x_or, info = H.solve(p, fH, tol=0.0, maxit=K, rule="est")
        assert st["iterations"] == info["iterations"] == K
        assert _rel2(_h(u).reshape(n, p.m), x_or) <= 1e-10, K
        assert abs(st["est_rel_res"] - info["est"][-1]) <= 1e-9 * max(info["est"][-1], 1e-12) + 1e-14
    s.close()


@pytest.mark.parametrize("tol", [1e-6, 1e-8])
def test_solve_natural_stop(pkg, tol):
    """Stopping rule on the true residual: iteration counts within one of the oracle's."""
    for w in (W.config_1d_sine(), W.small_case(2, 31, 31, 48, theta=0.5, varcoef=True, seed=9)):
        p = H.Problem.from_workload(w)
        fH = H.rhs(p, w.f, w.u0, w.u_prev)
        s = pkg.Solver(_spec(pkg, w))
        u, st = s.st_solve(_d(fH), tol=tol, maxit=300)
        x_or, info = H.solve(p, fH, tol=tol, maxit=300)
        assert abs(st["iterations"] - info["iterations"]) <= 1, (st, info["iterations"])
        assert st["true_rel_res"] <= tol
        r = H.flip(fH, p.n) - H.apply_op(p, _h(u).reshape(p.n, p.m))
        assert np.linalg.norm(r) / np.linalg.norm(fH) <= tol * (1 + 1e-6)
        s.close()


def test_mixed_precision_solve(pkg):
    """float32 preconditioner in float64 refinement: error vs the oracle's converged solution."""
    w = W.small_case(2, 63, 63, 64, theta=0.5, varcoef=True, seed=13)
    p = H.Problem.from_workload(w)
    fH = H.rhs(p, w.f, w.u0, w.u_prev)
    x_ref, info = H.solve(p, fH, tol=1e-13, maxit=500)
    s = pkg.Solver(_spec(pkg, w, precision="mixed"))
    u, st = s.st_solve(_d(fH), tol=1e-10, maxit=500)
    assert st["true_rel_res"] <= 1e-10
    assert _rel2(_h(u).reshape(p.n, p.m), x_ref) <= 1e-8
    u8, st8 = s.st_solve(_d(fH), tol=1e-8, maxit=500)
    assert st8["true_rel_res"] <= 1e-8
    s.close()


def test_transpose_solve_and_grad_a(pkg):
    """T^T lam = g via (Y T)(Y lam) = g, and the a-gradient contraction, against the oracle."""
    w = W.small_case(2, 15, 31, 20, theta=1.0, varcoef=True, seed=17)
    p = H.Problem.from_workload(w)
    rng = np.random.default_rng(3)
    g = rng.standard_normal((p.n, p.m))
    s = pkg.Solver(_spec(pkg, w))
    lam, st = s.st_solve_transpose(_d(g), tol=1e-13, maxit=400)
    lam_or, info = H.solve_transpose(p, g, tol=1e-13, maxit=400)
    assert _rel2(_h(lam).reshape(p.n, p.m), lam_or) <= 1e-10
    u = rng.standard_normal((p.n, p.m))
    ga = _h(s.st_grad_a(_d(lam_or), _d(u), _d(w.u0))).reshape(w.a_nodal.shape)
    _, _, ga_or = H.adjoint_gradients(p, u, lam_or, w.u0)
    assert _rel_max(ga, ga_or) <= 1e-12
    s.close()


def test_zero_rhs(pkg):
    w = W.small_case(2, 7, 7, 4, seed=1)
    s = pkg.Solver(_spec(pkg, w))
    u, st = s.st_solve(torch.zeros(w.N, dtype=torch.float64, device="cuda"), tol=1e-8, maxit=10)
    assert st["iterations"] == 0 and float(u.abs().max()) == 0.0
    s.close()


# ------------------------------------------------------------------ full-size workloads
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_full_size_2d_crank_nicolson(pkg, precision):
    """2D 255^2, n = 256, theta = 1/2, manufactured rhs + seeded noise: operator and
    preconditioner parity on the whole vector, solve residual checked by the oracle's operator."""
    w = W.config_2d_sine_cn()
    p = H.Problem.from_workload(w)
    s = pkg.Solver(_spec(pkg, w, precision=precision))
    fH_or = H.rhs(p, w.f, w.u0) + w.noise
    fH = s.st_assemble_rhs(_d(w.f), _d(w.u0), extra=_d(w.noise))
    assert _rel_max(_h(fH).reshape(p.n, p.m), fH_or) <= 1e-13
    if precision == "fp64":
        v = np.random.default_rng(4).standard_normal((p.n, p.m))
        assert _rel_max(_h(s.st_apply_op(_d(v))).reshape(p.n, p.m), H.apply_op(p, v)) <= 1e-13
        assert _rel_max(_h(s.st_apply_prec(_d(v))).reshape(p.n, p.m), H.apply_prec(p, v)) <= _prec_tol(p)
    u, st = s.st_solve(fH, tol=1e-8, maxit=500)
    u_h = _h(u).reshape(p.n, p.m)
    r = H.flip(fH_or, p.n) - H.apply_op(p, u_h)
    assert np.linalg.norm(r) / np.linalg.norm(fH_or) <= 1e-8 * (1 + 1e-6)
    # discretisation error of the manufactured solution stays at the O(tau^2 + h^2) level
    assert np.max(np.abs(u_h - w.u_exact)) < 1e-3
    s.close()


# ------------------------------------------------------------------ full size against the oracle
DIGEST = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_digest.json")


def _digest(name):
    with open(DIGEST) as fh:
        return json.load(fh)["workloads"][name]


def _sampled_rel(u, d):
    """||u[idx] - x*[idx]|| / ||x*[idx]|| on the digest's seeded indices (x* the oracle's direct
    solve, tests/golden/make_oracle_digest.py)."""
    idx = np.asarray(d["idx"])
    ref = np.asarray(d["val"])
    return float(np.linalg.norm(np.asarray(u).reshape(-1)[idx] - ref) / np.linalg.norm(ref))


def test_full_size_equal_iterations_fp64(pkg):
    """The bench workload (2D 255^2 x 256, Crank-Nicolson, manufactured rhs + noise): the float64
    solve and the oracle's MINRES, stopped after the same K iterations on the estimate alone,
    agree on the whole vector to 1e-10 (relative 2-norm), with the same residual estimate."""
    w = W.config_2d_sine_cn()
    p = H.Problem.from_workload(w)
    fH = H.rhs(p, w.f, w.u0) + w.noise
    s = pkg.Solver(_spec(pkg, w))
    for K in (4,):
        u, st = s.st_solve(_d(fH), tol=0.0, maxit=K, allow_not_converged=True)
        x_or, info = H.solve(p, fH, tol=0.0, maxit=K, rule="est")
        assert st["iterations"] == info["iterations"] == K
        assert _rel2(_h(u).reshape(p.n, p.m), x_or) <= 1e-10, K
        assert abs(st["est_rel_res"] - info["est"][-1]) <= 1e-9 * info["est"][-1]
    s.close()


FULL_SIZE = {
    "1d_sine_63_n64": lambda: (W.config_1d_sine(), None),
    "2d_cn_255_n256": lambda: (W.config_2d_sine_cn(), "noise"),
    "2d_bdf2var_511_n128": lambda: (W.config_2d_varcoef_bdf2(), None),
}


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("name", list(FULL_SIZE))
def test_full_size_solution_against_oracle(pkg, name, precision):
    """Every measured single-instance workload at its full size, solved to the bench tolerance
    (true relative residual 1e-8): the solution's relative error against the oracle's direct
    solve, sampled at the digest's seeded indices, stays within 1e-8 (the mixed-precision target;
    the float64 path, which takes the oracle's own iterations, lands within 1e-10 of the oracle's
    MINRES solution, test_full_size_equal_iterations_fp64).  The oracle's own MINRES at this
    tolerance is 3.5e-11 from the direct solve on the 2D Crank-Nicolson workload."""
    w, extra = FULL_SIZE[name]()
    d = _digest(name)
    assert d["N"] == w.N
    s = pkg.Solver(_spec(pkg, w, precision=precision))
    up = _d(w.u_prev) if w.u_prev is not None else None
    ex = _d(w.noise) if extra == "noise" else None
    fH = s.st_assemble_rhs(_d(w.f), _d(w.u0), up, ex)
    u, st = s.st_solve(fH, tol=1e-8, maxit=600)
    assert st["true_rel_res"] <= 1e-8
    err = _sampled_rel(_h(u), d["u"])
    assert err <= 1e-8, (name, precision, err)
    if name == "2d_cn_255_n256" and precision == "fp64":
        # the same iterations as the oracle's MINRES: the same distance from the direct solve
        ref = d["oracle_minres_tol1e-8"]
        assert st["iterations"] == ref["iterations"]
        assert abs(err - ref["sampled_rel_err"]) <= 1e-10
    s.close()


# ------------------------------------------------------------------ P_theta (Sec. 3.1.4)
PTHETA_CASES = [
    (1, 63, 1, 16, 1.0, True),    # varying a in 1D: per-frequency tridiagonal solves (PCR)
    (1, 255, 1, 33, 0.5, True),
    (1, 1023, 1, 8, 0.3, True),
    (1, 31, 1, 24, 0.5, False),   # constant a: spectral scaling
    (2, 31, 15, 20, 1.0, False),
]


@pytest.mark.parametrize("case", PTHETA_CASES, ids=lambda c: f"{c[0]}d-{c[1]}x{c[2]}-n{c[3]}-th{c[4]}-{'var' if c[5] else 'const'}")
def test_ptheta_apply(pkg, case):
    dim, mx, my, n, theta, var = case
    w = W.small_case(dim, mx, my, n, theta=theta, varcoef=var, seed=mx + 3 * n)
    p = H.Problem.from_workload(w, prec="Ptheta")
    s = pkg.Solver(_spec(pkg, w, prec="Ptheta"))
    v = np.random.default_rng(7).standard_normal((n, p.m))
    ref = H.apply_ptheta(p, v)
    z = _h(s.st_apply_prec(_d(v))).reshape(n, p.m)
    assert _rel_max(z, ref) <= 1e-11
    z32 = _h(s.st_apply_prec_f32(_d(v))).astype(np.float64).reshape(n, p.m)
    assert _rel2(z32, ref) <= (_ptheta_tol32(p) if var else 2e-5)
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_ptheta_solve(pkg, precision):
    """P_theta-preconditioned MINRES with a varying 1D coefficient: equal-iteration parity (float64)
    and error against the converged oracle solution (mixed)."""
    w = W.small_case(1, 255, 1, 64, theta=1.0, varcoef=True, seed=41)
    p = H.Problem.from_workload(w, prec="Ptheta")
    fH = H.rhs(p, w.f, w.u0)
    s = pkg.Solver(_spec(pkg, w, prec="Ptheta", precision=precision))
    if precision == "fp64":
        u, st = s.st_solve(_d(fH), tol=0.0, maxit=9, allow_not_converged=True)
        x_or, info = H.solve(p, fH, tol=0.0, maxit=9, rule="est")
        assert st["iterations"] == info["iterations"] == 9
        assert _rel2(_h(u).reshape(p.n, p.m), x_or) <= 1e-10
        u, st = s.st_solve(_d(fH), tol=1e-8, maxit=200)
        x_or, info = H.solve(p, fH, tol=1e-8, maxit=200)
        assert abs(st["iterations"] - info["iterations"]) <= 1
    else:
        x_ref, info = H.solve(p, fH, tol=1e-13, maxit=400)
        u, st = s.st_solve(_d(fH), tol=1e-10, maxit=400)
        assert st["true_rel_res"] <= 1e-10
        assert _rel2(_h(u).reshape(p.n, p.m), x_ref) <= 1e-8
    s.close()


# P_theta with a varying 2D coefficient: per-frequency Chebyshev inner map (degree 0 = the
# library default); ragged sizes, n = 1, degree 1 (no residual pass)
CHEB_CASES = [
    (15, 15, 8, 0.5, 3),
    (31, 15, 12, 1.0, 1),
    (63, 31, 5, 0.3, 5),
    (7, 7, 1, 0.5, 2),
    (127, 127, 16, 0.5, 0),
]


def _cheb_tol32(p, degree):
    """float32 tolerance of the Chebyshev map: each step forms r - A_k d, whose rounding relative
    to the result grows with the condition of A_k, at most (lam_H + c a_max mu0_max) /
    (lam_H + c a_min mu0_min), c = lam_Htheta tau; the steps add their errors."""
    ax, ay = H.face_values(p)
    fmin = min(ax.min(), ay.min())
    fmax = max(ax.max(), ay.max())
    mu = H.constant_stiffness_eigs(p)
    lh, lt = H.ptheta_time_eigs(p.n, p.theta)
    cond = max((lh + lt * p.tau * fmax * mu.max()) / (lh + lt * p.tau * fmin * mu.min()))
    return max(2e-5, 4 * 2.0 ** -24 * cond * degree)


@pytest.mark.parametrize("case", CHEB_CASES, ids=lambda c: f"{c[0]}x{c[1]}-n{c[2]}-th{c[3]}-d{c[4]}")
def test_ptheta_cheb_apply(pkg, case):
    mx, my, n, theta, deg = case
    w = W.small_case(2, mx, my, n, theta=theta, varcoef=True, seed=mx + 5 * n)
    d_used = deg if deg else pkg.ST_PTHETA_DEFAULT_DEGREE
    p = H.Problem.from_workload(w, prec="Ptheta", inner_degree=d_used)
    spec = _spec(pkg, w, prec="Ptheta")
    spec.inner_degree = deg
    s = pkg.Solver(spec)
    v = np.random.default_rng(9).standard_normal((n, p.m))
    ref = H.apply_ptheta(p, v)
    z = _h(s.st_apply_prec(_d(v))).reshape(n, p.m)
    assert _rel_max(z, ref) <= 1e-11
    z32 = _h(s.st_apply_prec_f32(_d(v))).astype(np.float64).reshape(n, p.m)
    assert _rel2(z32, ref) <= _cheb_tol32(p, d_used)
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_ptheta_cheb_solve(pkg, precision):
    """MINRES with the Chebyshev P_theta (2D varying a, degree 3): equal-iteration parity and
    iteration count within one of the oracle (float64), error against the converged oracle
    solution (mixed)."""
    w = W.small_case(2, 31, 31, 16, theta=0.5, varcoef=True, seed=43)
    p = H.Problem.from_workload(w, prec="Ptheta", inner_degree=3)
    fH = H.rhs(p, w.f, w.u0)
    spec = _spec(pkg, w, prec="Ptheta", precision=precision)
    spec.inner_degree = 3
    s = pkg.Solver(spec)
    if precision == "fp64":
        u, st = s.st_solve(_d(fH), tol=0.0, maxit=9, allow_not_converged=True)
        x_or, info = H.solve(p, fH, tol=0.0, maxit=9, rule="est")
        assert st["iterations"] == info["iterations"] == 9
        assert _rel2(_h(u).reshape(p.n, p.m), x_or) <= 1e-10
        u, st = s.st_solve(_d(fH), tol=1e-8, maxit=200)
        x_or, info = H.solve(p, fH, tol=1e-8, maxit=200)
        assert abs(st["iterations"] - info["iterations"]) <= 1
        assert _rel2(_h(u).reshape(p.n, p.m), x_or) <= 1e-6
    else:
        x_ref, info = H.solve(p, fH, tol=1e-13, maxit=400)
        u, st = s.st_solve(_d(fH), tol=1e-10, maxit=400)
        assert st["true_rel_res"] <= 1e-10
        assert _rel2(_h(u).reshape(p.n, p.m), x_ref) <= 1e-8
    s.close()


def test_ptheta_cheb_constant_field_is_one_step(pkg):
    """A constant field given as a_nodal: B_k = A_k, every later Chebyshev step adds zero, and the
    handle applies one step; degrees 1 and 4 agree exactly and match the exact solve."""
    w = W.small_case(2, 31, 15, 8, theta=0.5, varcoef=True, seed=5)
    w.a_nodal = np.full_like(w.a_nodal, 1.3)
    p = H.Problem.from_workload(w, prec="Ptheta")
    v = np.random.default_rng(11).standard_normal((p.n, p.m))
    ref = H.apply_ptheta(p, v)
    out = []
    for deg in (1, 4):
        spec = _spec(pkg, w, prec="Ptheta")
        spec.inner_degree = deg
        s = pkg.Solver(spec)
        out.append(_h(s.st_apply_prec(_d(v))).reshape(p.n, p.m))
        s.close()
    assert np.array_equal(out[0], out[1])
    assert _rel_max(out[0], ref) <= 1e-11


def test_ptheta_cheb_full_size(pkg):
    """2D 255^2, n = 256, theta = 1, seeded 8x8-mode coefficient field (the adjoint problem's
    shape) with the Chebyshev P_theta: full-vector apply parity (float64), and a mixed-precision
    solve that reaches 1e-8, checked with the oracle's operator."""
    w = W.config_2d_varcoef_theta(255, 256, 1.0, seed=5)
    p = H.Problem.from_workload(w, prec="Ptheta", inner_degree=pkg.ST_PTHETA_DEFAULT_DEGREE)
    s = pkg.Solver(_spec(pkg, w, prec="Ptheta"))
    v = np.random.default_rng(10).standard_normal((p.n, p.m))
    assert _rel_max(_h(s.st_apply_prec(_d(v))).reshape(p.n, p.m), H.apply_ptheta(p, v)) <= 1e-11
    s.close()
    s = pkg.Solver(_spec(pkg, w, prec="Ptheta", precision="mixed"))
    fH = s.st_assemble_rhs(_d(w.f), _d(w.u0))
    u, st = s.st_solve(fH, tol=1e-8, maxit=400)
    fH_or = H.rhs(p, w.f, w.u0)
    r = H.flip(fH_or, p.n) - H.apply_op(p, _h(u).reshape(p.n, p.m))
    assert np.linalg.norm(r) / np.linalg.norm(fH_or) <= 1e-8 * (1 + 1e-6)
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_full_size_2d_varcoef_bdf2(pkg, precision):
    """2D 511^2, n = 128, BDF2, seeded 8x8-mode coefficient field: the solve reaches 1e-8 (checked
    with the oracle's operator) and the manufactured solution is recovered to discretisation
    accuracy; sampled operator / preconditioner parity on the full vector (float64 handle)."""
    w = W.config_2d_varcoef_bdf2()
    p = H.Problem.from_workload(w)
    s = pkg.Solver(_spec(pkg, w, precision=precision))
    fH = s.st_assemble_rhs(_d(w.f), _d(w.u0), _d(w.u_prev))
    fH_or = H.rhs(p, w.f, w.u0, w.u_prev)
    assert _rel_max(_h(fH).reshape(p.n, p.m), fH_or) <= 1e-13
    if precision == "fp64":
        v = np.random.default_rng(8).standard_normal((p.n, p.m))
        assert _rel_max(_h(s.st_apply_op(_d(v))).reshape(p.n, p.m), H.apply_op(p, v)) <= 1e-13
        assert _rel_max(_h(s.st_apply_prec(_d(v))).reshape(p.n, p.m), H.apply_prec(p, v)) <= _prec_tol(p)
    u, st = s.st_solve(fH, tol=1e-8, maxit=400)
    u_h = _h(u).reshape(p.n, p.m)
    r = H.flip(fH_or, p.n) - H.apply_op(p, u_h)
    assert np.linalg.norm(r) / np.linalg.norm(fH_or) <= 1e-8 * (1 + 1e-6)
    assert np.max(np.abs(u_h - w.u_exact)) < 1e-3
    s.close()


# ------------------------------------------------------------------ autotuned launch shapes
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", [(2, 63, 31, 65, "theta", 0.5, True), (2, 127, 127, 64, "theta", 1.0, True),
                                  (1, 255, 1, 40, "bdf2", 1.0, True)],
                         ids=["2d-63x31-n65", "2d-127-n64", "1d-255-n40-bdf2"])
def test_autotune_keeps_results(pkg, case, precision):
    """The tuned knobs change launch shapes and may move a preconditioner stage to another engine
    (float32: tensor-core or CUDA-core kernels; float64: double-float or float64 transforms): the
    float64 operator stays bit-identical, the float64 preconditioner agrees far inside its oracle
    tolerance (each engine is within 1e-12 of the oracle), the float32 preconditioner agrees to
    float32 accuracy (each engine within 2e-5 of the oracle), and the solve still meets the
    oracle's residual with the same iteration count up to one (the dot-product partial sums are
    grouped differently)."""
    dim, mx, my, n, scheme, theta, var = case
    w = W.small_case(dim, mx, my, n, scheme=scheme, theta=theta, varcoef=var, seed=77)
    p = H.Problem.from_workload(w)
    s = pkg.Solver(_spec(pkg, w, precision=precision))
    v = _d(np.random.default_rng(5).standard_normal((p.n, p.m)))
    op0, pr0 = s.st_apply_op(v).clone(), s.st_apply_prec(v).clone()
    pf0 = s.st_apply_prec_f32(v).clone()
    fH = s.st_assemble_rhs(_d(w.f), _d(w.u0), None if w.u_prev is None else _d(w.u_prev))
    u0, st0 = s.st_solve(fH, tol=1e-9, maxit=600)
    u0 = u0.clone()
    s.st_autotune(reps=2)
    s.st_autotune(reps=2)  # second call is served from the per-shape cache
    assert torch.equal(s.st_apply_op(v), op0)
    assert _rel_max(_h(s.st_apply_prec(v)), _h(pr0)) <= 2e-13
    assert _rel2(_h(s.st_apply_prec_f32(v)).astype(np.float64), _h(pf0).astype(np.float64)) <= 4e-5
    u1, st1 = s.st_solve(fH, tol=1e-9, maxit=600)
    assert abs(st1["iterations"] - st0["iterations"]) <= 1, (st0, st1)
    fH_or = H.rhs(p, w.f, w.u0, w.u_prev)
    r = H.flip(fH_or, p.n) - H.apply_op(p, _h(u1).reshape(p.n, p.m))
    assert np.linalg.norm(r) / np.linalg.norm(fH_or) <= 1e-9 * (1 + 1e-6)
    assert _rel2(_h(u1), _h(u0)) <= 1e-6
    s.close()


# ------------------------------------------------------------------ float64 preconditioner engines
@pytest.mark.parametrize("case", [
    (1, 63, 1, 64, "theta", 1.0, False),
    (2, 31, 31, 32, "theta", 0.5, True),
    (2, 63, 15, 24, "bdf2", 1.0, True),
    (2, 127, 63, 17, "theta", 0.7, False),
], ids=_ids)
def test_fp64_engines_match_oracle(pkg, case, monkeypatch):
    """The float64 preconditioner's two engines (transforms in double-float arithmetic, the
    default, and in float64, ST_FP64_ENGINE=dfma): each P^-1 v within the oracle tolerance, and the
    same MINRES iterates as the oracle at equal iteration count (1e-10)."""
    dim, mx, my, n, scheme, theta, var = case
    w = W.small_case(dim, mx, my, n, scheme=scheme, theta=theta, varcoef=var, seed=21)
    p = H.Problem.from_workload(w)
    v = np.random.default_rng(6).standard_normal((p.n, p.m))
    ref = H.apply_prec(p, v)
    fH = H.rhs(p, w.f, w.u0, w.u_prev)
    K = 7
    x_or, info = H.solve(p, fH, tol=0.0, maxit=K, rule="est")
    outs = {}
    for engine in ("dd", "dfma"):
        monkeypatch.setenv("ST_FP64_ENGINE", engine)
        s = pkg.Solver(_spec(pkg, w))
        z = _h(s.st_apply_prec(_d(v))).reshape(n, p.m)
        assert _rel_max(z, ref) <= _prec_tol(p, engine), engine
        u, st = s.st_solve(_d(fH), tol=0.0, maxit=K, allow_not_converged=True)
        assert st["iterations"] == K
        assert _rel2(_h(u).reshape(n, p.m), x_or) <= 1e-10, engine
        outs[engine] = z
        s.close()
    # the engines differ: double-float rounding is not float64 rounding
    assert not np.array_equal(outs["dd"], outs["dfma"])


# ------------------------------------------------------------------ grouped update
@pytest.mark.parametrize("maxit", [600, 13])
def test_grouped_update_matches_per_iteration(pkg, monkeypatch, maxit):
    """The mixed single solve applies the MINRES direction/solution updates G iterations at a time
    (default 8; ST_UPDATE_GROUP sets G).  The Lanczos recurrence does not read d or x, so every G
    gives the same iterations, and each element goes through the same float32 operations in the
    same order: the solutions are bitwise equal to the per-iteration ones (G = 1), whether the
    solve stops at a multiple of G or in between (maxit = 13 stops mid-group and exercises the
    flush at the end of each inner run), and the converged one meets the oracle's residual."""
    w = W.small_case(2, 63, 63, 40, scheme="theta", theta=0.5, varcoef=True, seed=90)
    p = H.Problem.from_workload(w)
    spec = _spec(pkg, w, precision="mixed")
    res = {}
    fH = None
    for G in (1, 3, 8):
        monkeypatch.setenv("ST_UPDATE_GROUP", str(G))
        s = pkg.Solver(spec)
        if fH is None:
            fH = s.st_assemble_rhs(_d(w.f), _d(w.u0))
        u, st = s.st_solve(fH, tol=1e-9, maxit=maxit, allow_not_converged=True)
        res[G] = (u.clone(), st["iterations"], st["outer_steps"], st["status"])
        s.close()
    for G in (3, 8):
        assert res[G][1:] == res[1][1:], G
        assert torch.equal(res[G][0], res[1][0]), G
    if maxit == 600:
        assert res[8][3] == 0
        fH_or = H.rhs(p, w.f, w.u0)
        r = H.flip(fH_or, p.n) - H.apply_op(p, _h(res[8][0]).reshape(p.n, p.m))
        assert np.linalg.norm(r) / np.linalg.norm(fH_or) <= 1e-9 * (1 + 1e-6)
    else:
        assert res[8][1] == 13


@pytest.mark.parametrize("dim,mx,n,theta", [(2, 63, 40, 0.5), (1, 127, 33, 1.0), (2, 31, 24, 0.7)])
def test_uniform_and_general_double_float_stencil(pkg, dim, mx, n, theta, monkeypatch):
    """A constant coefficient on a grid with equal spacing gives one face coefficient everywhere,
    and the double-float stencil then takes its uniform form (one exact neighbour sum and one
    product per node).  The mixed solve with it and with the general form (ST_STENCIL_GENERAL=1)
    both reach the oracle's converged solution to 1e-8 in the same number of iterations (within
    one)."""
    my = mx if dim == 2 else 1
    w = W.small_case(dim, mx, my, n, scheme="theta", theta=theta, varcoef=False, seed=41)
    p = H.Problem.from_workload(w)
    fH = H.rhs(p, w.f, w.u0)
    x_ref, _ = H.solve(p, fH, tol=1e-13, maxit=500)
    its = {}
    for form in ("uniform", "general"):
        if form == "general":
            monkeypatch.setenv("ST_STENCIL_GENERAL", "1")
        else:
            monkeypatch.delenv("ST_STENCIL_GENERAL", raising=False)
        s = pkg.Solver(_spec(pkg, w, precision="mixed"))
        u, st = s.st_solve(_d(fH), tol=1e-10, maxit=500)
        assert st["true_rel_res"] <= 1e-10
        assert _rel2(_h(u).reshape(p.n, p.m), x_ref) <= 1e-8, form
        its[form] = st["iterations"]
        s.close()
    assert abs(its["uniform"] - its["general"]) <= 1, its
