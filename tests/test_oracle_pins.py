"""Pins for the CPU oracle: each check ties an oracle function to the paper or to mathematics
it cannot reproduce by construction (invariants, closed forms, printed values, brute force)."""
import json
import math
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import heat as H
from workloads import synthetic as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _tiny(dim, scheme, theta=0.5, varcoef=True, mx=4, my=3, n=6, seed=11, mz=3):
    my = 1 if dim == 1 else my
    w = W.small_case(dim, mx, my, n, scheme=scheme, theta=theta, varcoef=varcoef, seed=seed, mz=mz)
    return w, H.Problem.from_workload(w)


# ----------------------------------------------------------------------------- transforms
@pytest.mark.parametrize("n", [1, 2, 5, 16, 33, 64])
def test_dst_matrix_invariants(n):
    """S_n symmetric, orthogonal, involutory and S_n P_n S_n = D_n (Sec. 3.1.1)."""
    S = H.dst_matrix(n)
    assert np.allclose(S, S.T, atol=1e-15)
    assert np.allclose(S @ S, np.eye(n), atol=1e-13)
    Pn = 0.5 * (np.eye(n, k=1) + np.eye(n, k=-1))
    D = S @ Pn @ S
    assert np.allclose(D, np.diag(H.time_cos(n)), atol=1e-13)
    # eigenvalues of tridiag(-1,2,-1): 2 - 2 cos(k pi/(n+1)) = 4 sin^2(k pi/(2(n+1)))
    L = 2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    k = np.arange(1, n + 1)
    assert np.allclose(np.diag(S @ L @ S), 4 * np.sin(k * math.pi / (2 * (n + 1))) ** 2, atol=1e-12)


@pytest.mark.parametrize("n,axis", [(7, 0), (16, 1), (31, 0)])
def test_dst_routine_is_sine_matrix(n, axis):
    """The library transform the oracle calls equals the matrix S_n of Sec. 3.1.1."""
    rng = np.random.default_rng(n)
    V = rng.standard_normal((n, 5)) if axis == 0 else rng.standard_normal((5, n))
    ref = H.dst_matrix(n) @ V if axis == 0 else V @ H.dst_matrix(n)
    assert np.allclose(H.dst(V, axis=axis), ref, atol=1e-13)


# ----------------------------------------------------------------------------- space operator
@pytest.mark.parametrize("dim", [1, 2, 3])
def test_stiffness_energy_form(dim):
    """v^T K v = sum over faces a_f (v_p - v_q)^2 / h^2 with zero boundary values (eq. matrix_Km_va)."""
    w, p = _tiny(dim, "theta", mx=6, my=5, mz=4)
    K = H.stiffness(p).toarray()
    assert np.allclose(K, K.T)
    rng = np.random.default_rng(1)
    v = rng.standard_normal(p.m)
    a = w.a_nodal
    e = 0.0
    if dim == 1:
        vp = np.concatenate([[0.0], v, [0.0]])
        for i in range(p.mx + 1):
            af = 0.5 * (a[i] + a[i + 1])
            e += af * (vp[i + 1] - vp[i]) ** 2 / p.hx ** 2
    elif dim == 3:
        V = np.zeros((p.mz + 2, p.my + 2, p.mx + 2))
        V[1:-1, 1:-1, 1:-1] = v.reshape(p.mz, p.my, p.mx)
        for k in range(p.mz + 2):
            for j in range(p.my + 2):
                for i in range(p.mx + 2):
                    # the face towards +x, +y, +z of node (k, j, i) when both ends lie on a line
                    # of interior nodes of the other two axes
                    if i <= p.mx and 1 <= j <= p.my and 1 <= k <= p.mz:
                        af = 0.5 * (a[k, j, i] + a[k, j, i + 1])
                        e += af * (V[k, j, i + 1] - V[k, j, i]) ** 2 / p.hx ** 2
                    if j <= p.my and 1 <= i <= p.mx and 1 <= k <= p.mz:
                        af = 0.5 * (a[k, j, i] + a[k, j + 1, i])
                        e += af * (V[k, j + 1, i] - V[k, j, i]) ** 2 / p.hy ** 2
                    if k <= p.mz and 1 <= i <= p.mx and 1 <= j <= p.my:
                        af = 0.5 * (a[k, j, i] + a[k + 1, j, i])
                        e += af * (V[k + 1, j, i] - V[k, j, i]) ** 2 / p.hz ** 2
    else:
        V = np.zeros((p.my + 2, p.mx + 2))
        V[1:-1, 1:-1] = v.reshape(p.my, p.mx)
        for j in range(1, p.my + 1):
            for i in range(p.mx + 1):
                af = 0.5 * (a[j, i] + a[j, i + 1])
                e += af * (V[j, i + 1] - V[j, i]) ** 2 / p.hx ** 2
        for j in range(p.my + 1):
            for i in range(1, p.mx + 1):
                af = 0.5 * (a[j, i] + a[j + 1, i])
                e += af * (V[j + 1, i] - V[j, i]) ** 2 / p.hy ** 2
    assert np.isclose(v @ K @ v, e, rtol=1e-12)
    assert np.all(np.linalg.eigvalsh(K) > 0)


def test_stiffness_constant_eigenvectors():
    """For a = 1 the sine modes are eigenvectors: K s_p = (2 - 2cos(p pi h))/h^2 s_p (+ y term)."""
    p = H.Problem(2, 7, 5, 3)
    K = H.stiffness(p)
    X, Y = W.interior_grid(7, 5)
    for (a, b) in [(1, 1), (3, 2), (7, 5)]:
        s = (np.sin(a * math.pi * X) * np.sin(b * math.pi * Y)).reshape(-1)
        lam = (2 - 2 * math.cos(a * math.pi * p.hx)) / p.hx ** 2 + (2 - 2 * math.cos(b * math.pi * p.hy)) / p.hy ** 2
        assert np.allclose(K @ s, lam * s, atol=1e-9)
    mu = H.averaged_stiffness_eigs(p)
    assert np.allclose(np.sort(mu), np.sort(np.linalg.eigvalsh(K.toarray())), rtol=1e-12)


def test_stiffness_3d_constant_is_kronecker_sum():
    """3D, constant a: K = a (T_z/hz^2 (x) I (x) I + I (x) T_y/hy^2 (x) I + I (x) I (x) T_x/hx^2)
    with T = tridiag(-1, 2, -1), built here by Kronecker products; its eigenvalues are the sums
    of the three 1D ones, which the a = 1 and the averaged spectra reproduce."""
    mx, my, mz, c = 5, 4, 3, 1.7
    p = H.Problem(3, mx, my, 2, a_nodal=np.full((mz + 2, my + 2, mx + 2), c), mz=mz)
    T = lambda k: 2 * np.eye(k) - np.eye(k, k=1) - np.eye(k, k=-1)  # noqa: E731
    I = np.eye
    ref = c * (np.kron(np.kron(T(mz), I(my)), I(mx)) / p.hz ** 2
               + np.kron(np.kron(I(mz), T(my)), I(mx)) / p.hy ** 2
               + np.kron(np.kron(I(mz), I(my)), T(mx)) / p.hx ** 2)
    assert np.allclose(H.stiffness(p).toarray(), ref, rtol=1e-13, atol=1e-9)
    ev = np.sort(np.linalg.eigvalsh(ref))
    assert np.allclose(np.sort(H.averaged_stiffness_eigs(p)), ev, rtol=1e-12)
    assert np.allclose(np.sort(c * H.constant_stiffness_eigs(p)), ev, rtol=1e-12)
    # the 3D transform diagonalises it in the stated order (x fastest)
    S = np.kron(np.kron(H.dst_matrix(mz), H.dst_matrix(my)), H.dst_matrix(mx))
    assert np.allclose(S @ ref @ S, np.diag(c * H.constant_stiffness_eigs(p)), atol=1e-8)
    v = np.random.default_rng(2).standard_normal((2, p.m))
    assert np.allclose(H.spatial_dst(p, v), v @ S, atol=1e-12)


# ----------------------------------------------------------------------------- all-at-once system
@pytest.mark.parametrize("dim", [1, 2, 3])
@pytest.mark.parametrize("scheme", ["theta", "bdf2"])
def test_flipped_operator_symmetric(dim, scheme):
    """Y T is symmetric (eq. main_system / main_system_gem_sym) and T^T = Y T Y."""
    w, p = _tiny(dim, scheme)
    Nn = p.N
    E = np.eye(Nn)
    YT = np.stack([H.apply_op(p, E[i]).reshape(-1) for i in range(Nn)], axis=1)
    assert np.allclose(YT, YT.T, atol=1e-12)
    T = H.all_at_once_matrix(p).toarray()
    Y = H.flip_matrix(p.n, p.m).toarray()
    assert np.allclose(Y @ T, YT, atol=1e-12)
    assert np.allclose(T.T, Y @ T @ Y, atol=1e-12)
    # transpose application
    v = np.random.default_rng(3).standard_normal(Nn)
    assert np.allclose(H.apply_T_transpose(p, v).reshape(-1), T.T @ v, atol=1e-12)


@pytest.mark.parametrize("dim", [1, 2, 3])
@pytest.mark.parametrize("scheme,theta", [("theta", 1.0), ("theta", 0.5), ("theta", 0.3), ("bdf2", 1.0)])
def test_all_at_once_equals_time_marching(dim, scheme, theta):
    """Solving T u = f_H at once equals stepping the scheme sequentially (Sec. 1)."""
    w, p = _tiny(dim, scheme, theta=theta, mx=5, my=4, n=7)
    fH = H.rhs(p, w.f, w.u0, w.u_prev)
    T = H.all_at_once_matrix(p).tocsc()
    u_direct = spla.spsolve(T, fH.reshape(-1)).reshape(p.n, p.m)
    u_march = H.march(p, w.f, w.u0, w.u_prev)
    assert np.allclose(u_direct, u_march, rtol=1e-11, atol=1e-11)


@pytest.mark.parametrize("dim", [1, 2, 3])
@pytest.mark.parametrize("scheme,theta", [("theta", 1.0), ("theta", 0.5), ("theta", 0.3), ("bdf2", 1.0)])
def test_forward_substitution_is_the_direct_solve(dim, scheme, theta):
    """The block forward substitution solves T u = f_H exactly for any f_H: it equals the sparse
    LU solve of the explicit all-at-once matrix (Sec. 1) for an arbitrary right-hand side, and the
    sequential time stepping for f_H = rhs(f, u0).  A dropped block, a sign error on A1 or A2 or
    a wrong block index fails the first comparison."""
    w, p = _tiny(dim, scheme, theta=theta, mx=5, my=4, n=7)
    T = H.all_at_once_matrix(p).tocsc()
    g = np.random.default_rng(8).standard_normal((p.n, p.m))
    ref = spla.spsolve(T, g.reshape(-1)).reshape(p.n, p.m)
    assert np.allclose(H.forward_substitution(p, g), ref, rtol=1e-11, atol=1e-11)
    fH = H.rhs(p, w.f, w.u0, w.u_prev)
    assert np.allclose(H.forward_substitution(p, fH), H.march(p, w.f, w.u0, w.u_prev),
                       rtol=1e-11, atol=1e-11)
    # the transposed system through T^T = Y T Y: lam = Y T^-1 Y g
    lam = H.flip(H.forward_substitution(p, H.flip(g, p.n)), p.n)
    assert np.allclose(T.T @ lam.reshape(-1), g.reshape(-1), rtol=1e-10, atol=1e-10)


def _error_1d(scheme, theta, mx, n):
    if scheme == "bdf2":
        w = W.config_1d_sine(mx, n, theta=1.0)
        w.scheme = "bdf2"
        w.u_prev = math.exp(-w.tau) * w.u0
    else:
        w = W.config_1d_sine(mx, n, theta=theta)
    p = H.Problem.from_workload(w)
    u = H.march(p, w.f, w.u0, w.u_prev)
    return np.abs(u - w.u_exact).max()


@pytest.mark.parametrize("scheme,theta,order", [("theta", 1.0, 1), ("theta", 0.5, 2), ("bdf2", 1.0, 2)])
def test_time_order(scheme, theta, order):
    """Manufactured solution: backward Euler is first order, Crank-Nicolson and BDF2 second."""
    mx = 2047  # spatial error ~ h^2 far below the time error at these n
    e1 = _error_1d(scheme, theta, mx, 16)
    e2 = _error_1d(scheme, theta, mx, 32)
    rate = math.log2(e1 / e2)
    assert abs(rate - order) < 0.15, rate


def test_space_order():
    """Second order in space (Crank-Nicolson with many steps isolates the spatial error)."""
    e = [_error_1d("theta", 0.5, mx, 4096) for mx in (15, 31)]
    assert abs(math.log2(e[0] / e[1]) - 2.0) < 0.1


def test_space_order_3d():
    """Second order in space on the 3D 7-point grid (Crank-Nicolson with many steps isolates the
    spatial error): u = sin(pi x) sin(pi y) sin(pi z) e^t."""
    e = []
    for mx in (7, 15):
        w = W.config_3d_sine(mx, 512, theta=0.5)
        p = H.Problem.from_workload(w)
        e.append(np.abs(H.march(p, w.f, w.u0) - w.u_exact).max())
    assert abs(math.log2(e[0] / e[1]) - 2.0) < 0.1


def test_table5_backward_euler_errors():
    """Example 2 errors printed in Table 5 (backward Euler, m+1 = 32), three digits."""
    g = json.load(open(os.path.join(GOLDEN, "table5_backward_euler.json")))
    for n, ref in zip(g["n"], g["error"]):
        w = W.paper_example2(g["m_plus_1"] - 1, n, 1.0)
        p = H.Problem.from_workload(w)
        fH = H.rhs(p, w.f, w.u0)
        x, info = H.solve(p, fH, tol=1e-6, maxit=100)
        err = np.abs(x - w.u_exact).max()
        assert float(f"{err:.2e}") == ref, (n, err, ref)


def test_table_iteration_counts_3d():
    """Example 3 (3D) iteration counts of Tables 6-7 (P_H, P_theta), within one."""
    g = json.load(open(os.path.join(GOLDEN, "table_iterations_3d.json")))
    for c in g["cases"]:
        w = W.paper_example3(c["m_plus_1"] - 1, c["n"], c["theta"])
        p = H.Problem.from_workload(w, prec=c["prec"])
        fH = H.rhs(p, w.f, w.u0)
        x, info = H.solve(p, fH, tol=1e-6, maxit=100)
        assert abs(info["iterations"] - c["iter"]) <= g["tolerance_iterations"], (c, info["iterations"])


def test_table_iteration_counts():
    """Iteration counts of Tables 1-3 (P_H, P_theta) within +-2 (stopping-rule details differ)."""
    g = json.load(open(os.path.join(GOLDEN, "table_iterations.json")))
    for c in g["cases"]:
        mx = c["m_plus_1"] - 1
        if c["example"] == 1:
            w = W.paper_example1(mx, c["n"], c["theta"])
        else:
            w = W.paper_example2(mx, c["n"], c["theta"])
        p = H.Problem.from_workload(w, prec=c["prec"])
        fH = H.rhs(p, w.f, w.u0)
        x, info = H.solve(p, fH, tol=1e-6, maxit=100)
        assert abs(info["iterations"] - c["iter"]) <= g["tolerance_iterations"], (c, info["iterations"])


# ----------------------------------------------------------------------------- preconditioners
def _averaged_dense_K(p):
    """Average K's entries along each of its diagonals (Sec. 3.1.1), 2D: x- and y-couplings apart."""
    K = H.stiffness(p).toarray()
    m, mx = p.m, p.mx
    d = np.mean(np.diag(K))
    offx = np.diag(K, 1)
    ex = np.mean(offx[np.arange(m - 1) % mx != mx - 1]) if mx > 1 else 0.0
    Kb = d * np.eye(m)
    for i in range(m - 1):
        if (i % mx) != mx - 1:
            Kb[i, i + 1] = Kb[i + 1, i] = ex
    if p.dim >= 2:
        # y-couplings exist between rows of one z-plane only
        pl = mx * p.my
        cols = [i for i in range(m - mx) if (i % pl) < pl - mx]
        ey = np.mean([K[i, i + mx] for i in cols])
        for i in cols:
            Kb[i, i + mx] = Kb[i + mx, i] = ey
    if p.dim == 3:
        pl = mx * p.my
        ez = np.mean(np.diag(K, pl))
        for i in range(m - pl):
            Kb[i, i + pl] = Kb[i + pl, i] = ez
    return Kb


@pytest.mark.parametrize("dim", [1, 2, 3])
@pytest.mark.parametrize("scheme", ["theta", "bdf2"])
@pytest.mark.parametrize("varcoef", [False, True])
def test_prec_squared_is_block_matrix(dim, scheme, varcoef):
    """P^{-1} P^{-1} (P^2 v) = v with P^2 built entry by entry from eq. def:matrix_P / def:matrix_P_gen."""
    w, p = _tiny(dim, scheme, theta=0.7, varcoef=varcoef, mx=5, my=4, n=7)
    Kb = _averaged_dense_K(p)
    P2 = H.dense_PH_squared(p, Kb)
    v = np.random.default_rng(5).standard_normal((p.n, p.m))
    z = H.apply_prec(p, H.apply_prec(p, (P2 @ v.reshape(-1)).reshape(p.n, p.m)))
    assert np.allclose(z, v, rtol=1e-11, atol=1e-11)
    # and the dense principal square root gives the same preconditioner
    Pd = H.sqrtm_spd(P2)
    assert np.allclose(H.apply_prec(p, v).reshape(-1), np.linalg.solve(Pd, v.reshape(-1)), atol=1e-11)


def test_lemma_rank_difference():
    """T^T T - P_H^2 = diag(0, ..., 0, -A1^2) (Lemma rankC_P), constant a."""
    p = H.Problem(2, 3, 3, 6, 1.0, "theta", 0.5)
    T = H.all_at_once_matrix(p).toarray()
    P2 = H.dense_PH_squared(p)
    D = T.T @ T - P2
    m = p.m
    K = H.stiffness(p).toarray()
    A1 = -np.eye(m) + (1 - p.theta) * p.tau * K
    expect = np.zeros_like(D)
    expect[-m:, -m:] = -A1 @ A1
    assert np.allclose(D, expect, atol=1e-9)


def test_normal_equations_unit_eigenvalues():
    """P^{-1} T^T T P^{-1} has at least m(n-1) eigenvalues equal to one (Theorem main_P_normal)."""
    p = H.Problem(1, 4, 1, 7, 1.0, "theta", 1.0)
    T = H.all_at_once_matrix(p).toarray()
    Pinv = np.linalg.inv(H.sqrtm_spd(H.dense_PH_squared(p)))
    ev = np.linalg.eigvalsh(Pinv @ T.T @ T @ Pinv)
    assert np.sum(np.abs(ev - 1.0) < 1e-9) >= p.m * (p.n - 1)


def test_bdf2_rank():
    """rank(T[|g|^2] - P-hat^2) = 2m for BDF2 (Sec. 4, Lemma rankC_P_gen with l = 2)."""
    p = H.Problem(1, 3, 1, 9, 1.0, "bdf2")
    D = H.dense_symbol_toeplitz_sq(p) - H.dense_PH_squared(p)
    assert np.linalg.matrix_rank(D, tol=1e-9) == 2 * p.m


@pytest.mark.parametrize("varcoef", [False, True])
def test_ptheta_matches_dense(varcoef):
    """P_theta^{-1} v equals the dense solve with H (x) I + H_theta (x) tau K (eq. def:matrix_mod_P)."""
    w, p = _tiny(2, "theta", theta=0.5, varcoef=varcoef, mx=4, my=3, n=6)
    p.prec = "Ptheta"
    v = np.random.default_rng(2).standard_normal((p.n, p.m))
    ref = np.linalg.solve(H.dense_Ptheta(p), v.reshape(-1))
    assert np.allclose(H.apply_ptheta(p, v).reshape(-1), ref, atol=1e-11)


# ------------------------------------------------ P_theta, 2D varying a: Chebyshev inner map
def _cheb_case(mx=7, my=5, n=4, theta=0.5, seed=21, const=None):
    w = W.small_case(2, mx, my, n, scheme="theta", theta=theta, varcoef=True, seed=seed)
    a = w.a_nodal if const is None else np.full_like(w.a_nodal, const)
    return H.Problem(2, mx, my, n, w.T, "theta", theta, a, "Ptheta")


def _dense_space_dst(p):
    return np.kron(H.dst_matrix(p.my), H.dst_matrix(p.mx))


def _cheb_map_dense(p, k, degree):
    """The per-frequency inner map as a dense matrix, column by column."""
    Ak, bk = H.ptheta_cheb_blocks(p, k)
    _, al, be = H.ptheta_cheb_bounds(p)
    cols = [H.chebyshev_solve(lambda u: Ak @ u, lambda r: H.space_dst(p, H.space_dst(p, r) / bk),
                              e, al[k], be[k], degree) for e in np.eye(p.m)]
    return np.array(cols).T, Ak.toarray(), bk


def test_cheb_interval_holds_generalised_spectrum():
    """a_min K0 <= K <= a_max K0 gives the interval of the pencil (A_k, B_k): every generalised
    eigenvalue (dense, scipy.linalg.eigh) lies in [alpha_k, beta_k]."""
    import scipy.linalg as sla
    p = _cheb_case()
    _, al, be = H.ptheta_cheb_bounds(p)
    S = _dense_space_dst(p)
    for k in range(p.n):
        _, Ak, bk = _cheb_map_dense(p, k, 1)
        lam = sla.eigh(Ak, S @ np.diag(bk) @ S, eigvals_only=True)
        assert lam.min() >= al[k] * (1 - 1e-12) and lam.max() <= be[k] * (1 + 1e-12)
        assert lam.max() / lam.min() > 1.2  # the field is not constant: a real interval


def test_cheb_interval_is_attained_by_comparison_operators():
    """B_k is lam_H,k I + lam_Htheta,k tau abar K0 with abar the mean face value and K0 the a = 1
    stiffness matrix (built densely here by the oracle's own K with a = 1).  alpha_k and beta_k are
    the extreme generalised eigenvalues of the comparison pencils (lam I + c a_min K0, B_k) and
    (lam I + c a_max K0, B_k), c = lam_Htheta,k tau, which bound the pencil (A_k, B_k)."""
    import scipy.linalg as sla
    p = _cheb_case()
    K0 = H.stiffness(H.Problem(2, p.mx, p.my, p.n, p.T, "theta", p.theta)).toarray()
    ax, ay = H.face_values(p)
    faces = np.concatenate([ax.reshape(-1), ay.reshape(-1)])
    lam_h, lam_ht = H.ptheta_time_eigs(p.n, p.theta)
    abar, al, be = H.ptheta_cheb_bounds(p)
    assert abar == pytest.approx(faces.mean(), rel=1e-14)
    S = _dense_space_dst(p)
    I = np.eye(p.m)
    for k in range(p.n):
        c = lam_ht[k] * p.tau
        _, _, bk = _cheb_map_dense(p, k, 1)
        B = S @ np.diag(bk) @ S
        assert np.allclose(B, lam_h[k] * I + c * faces.mean() * K0, rtol=0, atol=1e-10 * np.abs(B).max())
        lo = sla.eigh(lam_h[k] * I + c * faces.min() * K0, B, eigvals_only=True).min()
        hi = sla.eigh(lam_h[k] * I + c * faces.max() * K0, B, eigvals_only=True).max()
        assert al[k] == pytest.approx(lo, rel=1e-12) and be[k] == pytest.approx(hi, rel=1e-12)


@pytest.mark.parametrize("degree", [1, 2, 3, 5])
def test_cheb_map_is_the_chebyshev_polynomial(degree):
    """The inner map M_k of degree d satisfies M_k A_k = I - p_d(B_k^-1 A_k), with p_d the
    Chebyshev polynomial T_d of the first kind mapped from [alpha_k, beta_k] onto [-1, 1] and scaled
    to p_d(0) = 1 (evaluated by numpy's Chebyshev series, independent of the recurrence).  M_k is
    symmetric and positive definite."""
    import numpy.polynomial.chebyshev as C
    import scipy.linalg as sla
    p = _cheb_case()
    _, al, be = H.ptheta_cheb_bounds(p)
    S = _dense_space_dst(p)
    coef = [0.0] * degree + [1.0]
    for k in (0, p.n - 1):
        M, Ak, bk = _cheb_map_dense(p, k, degree)
        assert np.abs(M - M.T).max() <= 1e-12 * np.abs(M).max()
        assert np.linalg.eigvalsh(0.5 * (M + M.T)).min() > 0
        lam = sla.eigh(Ak, S @ np.diag(bk) @ S, eigvals_only=True)
        a, b = al[k], be[k]
        pd = C.chebval((b + a - 2 * lam) / (b - a), coef) / C.chebval((b + a) / (b - a), coef)
        got = np.sort(np.linalg.eigvals(M @ Ak).real)
        assert np.allclose(got, np.sort(1.0 - pd), atol=1e-11)


def test_cheb_high_degree_is_the_exact_solve():
    """With degree 40 the Chebyshev error (about 0.25^40 here) is below rounding: P_theta^-1 v
    equals the exact per-frequency sparse LU solve."""
    p = _cheb_case(mx=15, my=7, n=5)
    v = np.random.default_rng(4).standard_normal((p.n, p.m))
    exact = H.apply_ptheta(p, v)
    p.inner_degree = 40
    assert np.linalg.norm(H.apply_ptheta(p, v) - exact) <= 1e-12 * np.linalg.norm(exact)


def test_cheb_3d_interval_and_limit():
    """3D (faces along z as well): the interval holds the dense generalised spectrum of
    (A_k, B_k), and degree 40 reproduces the exact per-frequency solve."""
    import scipy.linalg as sla
    w = W.small_case(3, 5, 4, 3, scheme="theta", theta=0.5, varcoef=True, seed=23, mz=3)
    p = H.Problem.from_workload(w, prec="Ptheta")
    _, al, be = H.ptheta_cheb_bounds(p)
    S = np.kron(np.kron(H.dst_matrix(p.mz), H.dst_matrix(p.my)), H.dst_matrix(p.mx))
    for k in range(p.n):
        Ak, bk = H.ptheta_cheb_blocks(p, k)
        lam = sla.eigh(Ak.toarray(), S @ np.diag(bk) @ S, eigvals_only=True)
        assert lam.min() >= al[k] * (1 - 1e-12) and lam.max() <= be[k] * (1 + 1e-12)
    v = np.random.default_rng(6).standard_normal((p.n, p.m))
    exact = H.apply_ptheta(p, v)
    p.inner_degree = 40
    assert np.linalg.norm(H.apply_ptheta(p, v) - exact) <= 1e-12 * np.linalg.norm(exact)


def test_cheb_constant_field_is_exact_at_any_degree():
    """A constant a makes B_k = A_k (abar = a): the first step is exact, and the map equals the
    exact solve for every degree."""
    p = _cheb_case(const=1.3)
    v = np.random.default_rng(5).standard_normal((p.n, p.m))
    exact = H.apply_ptheta(p, v)
    for d in (1, 3):
        p.inner_degree = d
        assert np.linalg.norm(H.apply_ptheta(p, v) - exact) <= 1e-12 * np.linalg.norm(exact)
        p.inner_degree = None


def test_cheb_ptheta_spd_and_close_to_exact():
    """The whole P_theta^-1 with the inner map (degree 3) is symmetric positive definite, and its
    product with the exact P_theta has eigenvalues within the Chebyshev bound 1/T_3((b+a)/(b-a))
    of one, with the widest interval over the frequencies."""
    p = _cheb_case(mx=3, my=3, n=4)
    _, al, be = H.ptheta_cheb_bounds(p)
    p.inner_degree = 3
    E = np.eye(p.N)
    Mc = np.array([H.apply_ptheta(p, e.reshape(p.n, p.m)).reshape(-1) for e in E]).T
    assert np.abs(Mc - Mc.T).max() <= 1e-12 * np.abs(Mc).max()
    assert np.linalg.eigvalsh(0.5 * (Mc + Mc.T)).min() > 0
    ev = np.linalg.eigvals(Mc @ H.dense_Ptheta(p)).real
    t = ((be + al) / (be - al)).min()
    eps = 1.0 / math.cosh(3 * math.acosh(t))
    assert np.abs(ev - 1).max() <= eps * (1 + 1e-9)
    assert np.abs(ev - 1).max() > 1e-3 * eps  # the map is not exact


def test_preconditioned_spectrum_clusters():
    """Eigenvalues of P^{-1} Y T cluster at +-1 with a number of outliers that does not depend on n
    (Theorem absP_main). The blocks A0, A1 are held fixed (fixed tau) while n grows."""
    for th in (1.0, 0.5):
        outl = []
        for n in (32, 64, 128):
            p = H.Problem(1, 3, 1, n, n / 32.0, "theta", th)
            T = H.all_at_once_matrix(p).toarray()
            Y = H.flip_matrix(n, p.m).toarray()
            Pinv = np.linalg.inv(H.sqrtm_spd(H.dense_PH_squared(p)))
            ev = np.linalg.eigvals(Pinv @ Y @ T).real
            dist = np.minimum(np.abs(ev - 1), np.abs(ev + 1))
            outl.append(int(np.sum(dist > 0.01)))
        assert len(set(outl)) == 1 and outl[0] <= 3 * p.m, (th, outl)


# ----------------------------------------------------------------------------- MINRES
def test_ideal_preconditioner_two_steps():
    """With sqrt(T^T T) as preconditioner MINRES converges in at most two steps (Proposition absC)."""
    p = H.Problem(2, 3, 2, 5, 1.0, "theta", 0.5)
    T = H.all_at_once_matrix(p).toarray()
    Y = H.flip_matrix(p.n, p.m).toarray()
    Pinv = np.linalg.inv(H.sqrtm_spd(T.T @ T))
    b = np.random.default_rng(4).standard_normal(p.N)
    x, info = H.minres(lambda v: Y @ T @ v, lambda v: Pinv @ v, b, 1e-12, 10)
    assert info["iterations"] <= 2
    assert np.linalg.norm(Y @ T @ x - b) <= 1e-10 * np.linalg.norm(b)


def test_minres_iterates_are_krylov_minimisers():
    """Iterate k minimises ||b - A x||_{M^{-1}} over x in span{M^{-1}b, (M^{-1}A) M^{-1}b, ...}."""
    w, p = _tiny(1, "theta", theta=1.0, mx=4, n=5)
    T = H.all_at_once_matrix(p).toarray()
    Y = H.flip_matrix(p.n, p.m).toarray()
    A = Y @ T
    Pd = H.sqrtm_spd(H.dense_PH_squared(p, _averaged_dense_K(p)))
    Minv = np.linalg.inv(Pd)
    b = np.random.default_rng(8).standard_normal(p.N)
    iterates = {}
    H.minres(lambda v: A @ v, lambda v: Minv @ v, b, 0.0, 8,
             callback=lambda k, x, est: iterates.__setitem__(k, (x.copy(), est)))
    L = np.linalg.cholesky(Minv)  # ||r||_{M^{-1}} = ||L^T r||
    basis = [Minv @ b]
    for k in range(1, 9):
        Q, _ = np.linalg.qr(np.stack(basis, axis=1))
        c, *_ = np.linalg.lstsq(L.T @ A @ Q, L.T @ b, rcond=None)
        xk = Q @ c
        x_or, est = iterates[k]
        assert np.allclose(x_or, xk, rtol=1e-7, atol=1e-9), k
        rn = np.linalg.norm(L.T @ (b - A @ xk)) / np.linalg.norm(L.T @ b)
        assert np.isclose(est, rn, rtol=1e-6, atol=1e-12), (k, est, rn)
        basis.append(Minv @ (A @ basis[-1]))
    ests = [iterates[k][1] for k in sorted(iterates)]
    assert all(b2 <= b1 * (1 + 1e-12) for b1, b2 in zip(ests, ests[1:]))


@pytest.mark.parametrize("scheme", ["theta", "bdf2"])
def test_solve_matches_direct(scheme):
    w, p = _tiny(2, scheme, theta=0.5, mx=6, my=5, n=8)
    fH = H.rhs(p, w.f, w.u0, w.u_prev)
    x, info = H.solve(p, fH, tol=1e-13, maxit=200)
    ref = spla.spsolve(H.all_at_once_matrix(p).tocsc(), fH.reshape(-1)).reshape(p.n, p.m)
    assert np.linalg.norm(x - ref) <= 1e-10 * np.linalg.norm(ref)


# ----------------------------------------------------------------------------- adjoint
@pytest.mark.parametrize("dim,theta", [(1, 1.0), (2, 1.0), (2, 0.5)])
def test_adjoint_gradients_vs_finite_differences(dim, theta):
    """dL/d(f, u0, a) from the transposed solve equals central differences of the forward march."""
    w, p = _tiny(dim, "theta", theta=theta, varcoef=True, mx=5, my=4, n=6, seed=21)
    rng = np.random.default_rng(9)
    u_obs = rng.standard_normal((p.n, p.m))

    def loss(f, u0, a):
        q = H.Problem(p.dim, p.mx, p.my, p.n, p.T, p.scheme, p.theta, a)
        u = H.march(q, f, u0)
        return 0.5 * np.sum((u - u_obs) ** 2)

    u = H.march(p, w.f, w.u0)
    lam, info = H.solve_transpose(p, u - u_obs, tol=1e-14, maxit=400)
    T = H.all_at_once_matrix(p).tocsc()
    lam_direct = spla.spsolve(T.T.tocsc(), (u - u_obs).reshape(-1)).reshape(p.n, p.m)
    assert np.allclose(lam, lam_direct, rtol=1e-9, atol=1e-10)
    gf, gu0, ga = H.adjoint_gradients(p, u, lam_direct, w.u0)
    for target in ("f", "u0", "a"):
        if target == "f":
            d = rng.standard_normal(w.f.shape); g = np.sum(gf * d)
            Lp = loss(w.f + 1e-5 * d, w.u0, w.a_nodal); Lm = loss(w.f - 1e-5 * d, w.u0, w.a_nodal)
        elif target == "u0":
            d = rng.standard_normal(w.u0.shape); g = np.sum(gu0 * d)
            Lp = loss(w.f, w.u0 + 1e-5 * d, w.a_nodal); Lm = loss(w.f, w.u0 - 1e-5 * d, w.a_nodal)
        else:
            d = rng.standard_normal(w.a_nodal.shape); g = np.sum(ga * d)
            Lp = loss(w.f, w.u0, w.a_nodal + 1e-5 * d); Lm = loss(w.f, w.u0, w.a_nodal - 1e-5 * d)
        fd = (Lp - Lm) / 2e-5
        assert abs(fd - g) <= 1e-6 * max(1.0, abs(g)), (target, fd, g)
