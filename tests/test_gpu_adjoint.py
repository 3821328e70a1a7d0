"""Adjoint gradients through the all-at-once solve (transposed MINRES solve + gradient kernels)
against the oracle's adjoint and against central finite differences of the GPU forward solve."""
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
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("dim,mx,my,n,scheme,theta", [
    (2, 15, 31, 12, "theta", 1.0),
    (2, 31, 15, 9, "theta", 0.5),
    (1, 63, 1, 16, "bdf2", 1.0),
])
def test_gradients_match_oracle_adjoint(pkg, dim, mx, my, n, scheme, theta):
    from paper_2201_10062_gb300.autograd import heat_solve

    w = W.small_case(dim, mx, my, n, scheme=scheme, theta=theta, varcoef=True, seed=51)
    p = H.Problem.from_workload(w)
    u_obs = np.random.default_rng(2).standard_normal((n, p.m))
    spec = pkg.ProblemSpec(dim, mx, my, n, w.T, scheme, theta)
    f = _d(w.f).requires_grad_(True)
    u0 = _d(w.u0).requires_grad_(True)
    a = _d(w.a_nodal).requires_grad_(True)
    up = _d(w.u_prev).requires_grad_(True) if w.u_prev is not None else None
    u = heat_solve(f, u0, spec, a_nodal=a, u_prev=up, tol=1e-13)
    loss = 0.5 * ((u - _d(u_obs)) ** 2).sum()
    loss.backward()
    u_or = H.march(p, w.f, w.u0, w.u_prev)
    assert _rel(u.detach().cpu().numpy(), u_or) <= 1e-10
    lam = H.solve_transpose(p, u_or - u_obs, tol=1e-14, maxit=500)[0]
    gf, gu0, ga = H.adjoint_gradients(p, u_or, lam, w.u0)
    assert _rel(f.grad.cpu().numpy(), gf) <= 1e-9
    if scheme == "theta":
        assert _rel(u0.grad.cpu().numpy(), gu0) <= 1e-9
    else:
        # oracle: u^(-1) is a separate input; its gradient is -lam_1/2
        assert _rel(u0.grad.cpu().numpy(), 2 * lam[0] - 0.5 * lam[1]) <= 1e-9
        assert _rel(up.grad.cpu().numpy(), -0.5 * lam[0]) <= 1e-9
    assert _rel(a.grad.cpu().numpy(), ga) <= 1e-9


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_adjoint_workload_finite_differences(pkg, precision):
    """2D 255^2, n = 256, backward Euler; u_obs is the oracle's solution for a seeded true a plus
    1% Gaussian noise; gradients at a different a against central differences (rel <= 1e-5)."""
    from paper_2201_10062_gb300.autograd import heat_solve

    w = W.config_adjoint()
    p_true = H.Problem.from_workload(w)
    u_true = H.march(p_true, w.f, w.u0)
    noise = w.extra["obs_normal"]
    u_obs = u_true + 0.01 * np.sqrt(np.mean(u_true ** 2)) * noise
    a_eval = 0.5 * (w.a_nodal + 1.0)
    spec = pkg.ProblemSpec(2, w.mx, w.my, w.n, w.T, "theta", 1.0, None, "PH", precision)
    uo = _d(u_obs)
    # the attainable relative residual of this system is about 1e-12 (condition ~1e5)
    tol = 3e-11

    def loss_of(f, u0, a):
        with torch.no_grad():
            u = heat_solve(f, u0, spec, a_nodal=a, tol=tol)
            return float(0.5 * ((u - uo) ** 2).sum())

    f = _d(w.f).requires_grad_(True)
    u0 = _d(w.u0).requires_grad_(True)
    a = _d(a_eval).requires_grad_(True)
    u = heat_solve(f, u0, spec, a_nodal=a, tol=tol)
    loss = 0.5 * ((u - uo) ** 2).sum()
    loss.backward()
    rng = np.random.default_rng(11)
    X, Y = W.nodal_grid(w.mx, w.my)
    checks = {
        "f": (rng.standard_normal(w.f.shape), f.grad),
        "u0": (rng.standard_normal(w.u0.shape), u0.grad),
        # smooth perturbation of a that keeps a > 0
        "a": (np.sin(np.pi * X) * np.sin(2 * np.pi * Y), a.grad),
    }
    for name, (d, g) in checks.items():
        eps = 1e-4 * float(np.abs(a_eval).max()) if name == "a" else 1e-3
        dd = _d(d)
        fp = [f.detach(), u0.detach(), a.detach()]
        fm = [f.detach(), u0.detach(), a.detach()]
        idx = {"f": 0, "u0": 1, "a": 2}[name]
        fp[idx] = fp[idx] + eps * dd
        fm[idx] = fm[idx] - eps * dd
        fd = (loss_of(*fp) - loss_of(*fm)) / (2 * eps)
        ad = float((g * dd).sum())
        assert abs(fd - ad) <= 1e-5 * abs(ad), (name, fd, ad)


def _sampled_rel(u, d):
    idx = np.asarray(d["idx"])
    ref = np.asarray(d["val"])
    return float(np.linalg.norm(np.asarray(u).reshape(-1)[idx] - ref) / np.linalg.norm(ref))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_adjoint_workload_against_oracle_direct_solves(pkg, precision):
    """The adjoint workload at full size (2D 255^2 x 256, backward Euler): forward solution,
    adjoint lam = T^-T (u - u_obs) and the f, u0 and a gradients of L = 1/2 ||u - u_obs||^2,
    each against the oracle's direct solves (tests/golden/oracle_digest.json, sampled at seeded
    indices), relative error <= 1e-8 with both solves at a true relative residual of 1e-10."""
    import json
    import os

    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                           "oracle_digest.json")) as fh:
        d = json.load(fh)["workloads"]["adjoint_255_n256"]
    w = W.config_adjoint()
    p_true = H.Problem.from_workload(w)
    u_true = H.march(p_true, w.f, w.u0)
    u_obs = u_true + 0.01 * np.sqrt(np.mean(u_true ** 2)) * w.extra["obs_normal"]
    a_eval = 0.5 * (w.a_nodal + 1.0)
    spec = pkg.ProblemSpec(2, w.mx, w.my, w.n, w.T, "theta", 1.0, a_eval, "PH", precision)
    s = pkg.Solver(spec)
    fH = s.st_assemble_rhs(_d(w.f), _d(w.u0))
    u, st = s.st_solve(fH, tol=1e-10, maxit=800)
    g = u.reshape(-1) - _d(u_obs).reshape(-1)
    lam, st2 = s.st_solve_transpose(g, tol=1e-10, maxit=800)
    gf, gu0, _ = s.st_grad_rhs(lam)
    ga = s.st_grad_a(lam, u, _d(w.u0))
    got = {"u": u, "lam": lam, "grad_f": gf, "grad_u0": gu0, "grad_a": ga}
    for k, v in got.items():
        err = _sampled_rel(v.detach().cpu().numpy(), d[k])
        assert err <= 1e-8, (precision, k, err)
    loss = 0.5 * float((g ** 2).sum())
    assert abs(loss - d["loss"]) <= 1e-8 * d["loss"]
    s.close()
