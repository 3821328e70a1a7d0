"""Plain FP64 CPU oracle for sine-transform preconditioned MINRES on all-at-once heat systems.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this module. It shares
no code with the CUDA path (``paper_2201_10062_gb300``) and imports nothing from
it; the only common input is the seeded data from ``workloads``.

Every function states the passage of the paper (Hon, Fung, Dong,
Serra-Capizzano, "A sine transform based preconditioned MINRES method for
all-at-once systems from constant and variable-coefficient evolutionary PDEs",
arXiv 2201.10062) it writes out. Library primitives used as single steps:
scipy.sparse matrix products and sparse LU solves, scipy.fft.dst (type I,
orthonormal) for the transform S_n, numpy.linalg.eigh for dense square roots.

Pins (tests/test_oracle_*.py) tie each function to something other than itself:
  * dst / dst_matrix: S_n symmetric, orthogonal, involutory, diagonalises the
    tridiagonal P_n with eigenvalues cos(k pi/(n+1)) (Sec. 3.1.1).
  * stiffness / apply_T / apply_op: Y*T symmetric (Sec. 1, eq. main_system),
    T^T = Y T Y, all-at-once solution equals sequential time marching (Sec. 1),
    manufactured-solution orders (BE 1, CN 2, BDF2 2, space 2) and the Table 5
    backward-Euler errors of Example 2 (Sec. 5).
  * ph_spectrum / apply_prec: P_H^2 equals the block tridiagonal matrix of
    eq. def:matrix_P built entry by entry; the dense square root agrees; the
    difference T^T T - P_H^2 is zero except the last block, -A1^2 (Lemma
    rankC_P); P^-1 T^T T P^-1 has at least m(n-1) unit eigenvalues (Theorem
    main_P_normal); BDF2: rank(T[|g|^2] - P^2) = 2m (Sec. 4, Lemma rankC_P_gen).
  * apply_ptheta: equals the dense H (x) I + H_theta (x) tau K of eq.
    def:matrix_mod_P with matrix square roots from eigh (Sec. 3.1.4).
  * apply_ptheta_cheb (2D varying a, Chebyshev inner map of step 2): the interval
    [alpha_k, beta_k] holds the dense generalised spectrum of (A_k, B_k) and its ends are
    the extreme eigenvalues of the comparison pencils a_min K0, a_max K0; the map of degree
    d equals I - T_d-polynomial (numpy Chebyshev series) on that spectrum, symmetric
    positive definite; degree 40 reproduces the sparse LU solve; a constant field is
    exact at any degree; the whole P_theta^-1 stays within the Chebyshev bound of exact.
  * 3D (Sec. 5, Example 3): the 7-point K equals the Kronecker sum of 1D second
    differences for constant a and the face energy form for varying a; the 3D
    transform diagonalises it in the stated order; Y T symmetric, marching, the
    block matrix of P_H^2 and the Chebyshev interval in 3D; second-order spatial
    convergence on a manufactured 3D solution; the iteration counts of Tables 6-7 within one.
  * minres: the ideal preconditioner sqrt(T^T T) converges in at most two
    steps (Proposition absC); each iterate's preconditioned residual equals the
    brute-force least-squares minimum over the explicit Krylov basis; residual
    estimate monotone; iteration counts of Tables 1-3 within +-2.
  * forward_substitution: equals the sparse LU solve of the explicit all-at-once matrix on
    tiny sizes and the sequential time stepping of march when f_H = rhs(f, u0).
  * adjoint_gradients: central finite differences of the forward solve.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Callable, Optional

import numpy as np
import scipy.fft
import scipy.sparse as sp
import scipy.sparse.linalg as spla


# --------------------------------------------------------------------------------------
# Problem description
# --------------------------------------------------------------------------------------
@dataclass
class Problem:
    """Discretised heat problem on (0,1)^dim x (0,T], zero Dirichlet data (Sec. 1, eq. heat).

    Finite differences on a uniform grid, so the mass matrix M_m is the identity
    (Sec. 5).  scheme is "theta" (Sec. 1) or "bdf2" (Sec. 4).
    """

    dim: int
    mx: int
    my: int
    n: int
    T: float = 1.0
    scheme: str = "theta"
    theta: float = 1.0
    a_nodal: Optional[np.ndarray] = None
    prec: str = "PH"  # "PH" (eq. def:matrix_P / def:matrix_P_gen) or "Ptheta" (eq. def:matrix_mod_P)
    # P_theta with a 2D or 3D varying a: degree of the Chebyshev inner map of step 2 (Sec. 3.1.4);
    # None solves every per-frequency system exactly (sparse LU)
    inner_degree: Optional[int] = None
    mz: int = 1  # interior points along z (3D, Sec. 5 Example 3); 1 in 1D and 2D

    @property
    def m(self) -> int:
        return self.mx * self.my * self.mz

    @property
    def N(self) -> int:
        return self.m * self.n

    @property
    def tau(self) -> float:
        return self.T / self.n

    @property
    def hx(self) -> float:
        return 1.0 / (self.mx + 1)

    @property
    def hy(self) -> float:
        return 1.0 / (self.my + 1)

    @property
    def hz(self) -> float:
        return 1.0 / (self.mz + 1)

    @staticmethod
    def from_workload(w, prec: str = "PH", inner_degree: Optional[int] = None) -> "Problem":
        return Problem(w.dim, w.mx, w.my, w.n, w.T, w.scheme, w.theta, w.a_nodal, prec,
                       inner_degree, getattr(w, "mz", 1))


# --------------------------------------------------------------------------------------
# Space: stiffness matrix K_m (Sec. 3.1.1, eq. matrix_Km_va) and its 2D analogue
# --------------------------------------------------------------------------------------
def nodal_a(prob: Problem) -> np.ndarray:
    if prob.a_nodal is not None:
        return np.asarray(prob.a_nodal, dtype=np.float64)
    shape = ((prob.mx + 2,) if prob.dim == 1 else (prob.my + 2, prob.mx + 2) if prob.dim == 2
             else (prob.mz + 2, prob.my + 2, prob.mx + 2))
    return np.ones(shape)


def face_values(prob: Problem):
    """Diffusion coefficient at cell faces, a_{i+1/2} = (a_i + a_{i+1})/2.

    eq. matrix_Km_va uses a at the half-grid points; the nodal field is averaged
    onto them. Returns (ax, ay): ax[j, i] is the face between x-nodes i and i+1
    (node index 0 and mx+1 are boundary nodes) on interior row j, shape
    (my, mx+1); ay[j, i] the face between y-nodes j and j+1 on interior column
    i, shape (my+1, mx). In 1D ay is None and ax has shape (1, mx+1).  In 3D (the same reading
    along a third axis) the result is (ax, ay, az) with shapes (mz, my, mx+1), (mz, my+1, mx) and
    (mz+1, my, mx), each face between two nodes of its axis on interior lines of the others.
    """
    a = nodal_a(prob)
    if prob.dim == 3:
        ax = 0.5 * (a[1:-1, 1:-1, :-1] + a[1:-1, 1:-1, 1:])
        ay = 0.5 * (a[1:-1, :-1, 1:-1] + a[1:-1, 1:, 1:-1])
        az = 0.5 * (a[:-1, 1:-1, 1:-1] + a[1:, 1:-1, 1:-1])
        return ax, ay, az
    if prob.dim == 1:
        ax = 0.5 * (a[:-1] + a[1:])
        return ax[None, :], None
    ax = 0.5 * (a[1:-1, :-1] + a[1:-1, 1:])
    ay = 0.5 * (a[:-1, 1:-1] + a[1:, 1:-1])
    return ax, ay


def stiffness(prob: Problem) -> sp.csr_matrix:
    """K_m approximating -div(a grad .) with zero Dirichlet data.

    1D: the tridiagonal matrix of eq. matrix_Km_va,
    (1/h^2) [ -a_{i-1/2}, a_{i-1/2} + a_{i+1/2}, -a_{i+1/2} ].
    2D: the same three-point form along x and along y, summed (5-point).
    3D: the same along x, y and z (7-point), assembled with array indexing.
    """
    if prob.dim == 3:
        return _stiffness_3d(prob)
    mx, my = prob.mx, prob.my
    ax, ay = face_values(prob)
    m = mx * my
    rows, cols, vals = [], [], []

    def idx(i, j):
        return j * mx + i

    for j in range(my):
        for i in range(mx):
            p = idx(i, j)
            w, e = ax[j, i] / prob.hx ** 2, ax[j, i + 1] / prob.hx ** 2
            diag = w + e
            if i > 0:
                rows.append(p); cols.append(idx(i - 1, j)); vals.append(-w)
            if i < mx - 1:
                rows.append(p); cols.append(idx(i + 1, j)); vals.append(-e)
            if prob.dim == 2:
                s, nn = ay[j, i] / prob.hy ** 2, ay[j + 1, i] / prob.hy ** 2
                diag += s + nn
                if j > 0:
                    rows.append(p); cols.append(idx(i, j - 1)); vals.append(-s)
                if j < my - 1:
                    rows.append(p); cols.append(idx(i, j + 1)); vals.append(-nn)
            rows.append(p); cols.append(p); vals.append(diag)
    return sp.csr_matrix((vals, (rows, cols)), shape=(m, m))


def _stiffness_3d(prob: Problem) -> sp.csr_matrix:
    """7-point K: node p couples to its neighbour q across face f with -a_f/h^2 and its diagonal
    is the sum of a_f/h^2 over its six faces (faces on the boundary included)."""
    mx, my, mz = prob.mx, prob.my, prob.mz
    ax, ay, az = face_values(prob)
    wx, wy, wz = ax / prob.hx ** 2, ay / prob.hy ** 2, az / prob.hz ** 2
    idx = np.arange(prob.m).reshape(mz, my, mx)
    diag = (wx[:, :, :-1] + wx[:, :, 1:]) + (wy[:, :-1, :] + wy[:, 1:, :]) + (wz[:-1] + wz[1:])
    rows, cols, vals = [idx.ravel()], [idx.ravel()], [diag.ravel()]
    for c, p, q in ((wx[:, :, 1:-1], idx[:, :, :-1], idx[:, :, 1:]),
                    (wy[:, 1:-1, :], idx[:, :-1, :], idx[:, 1:, :]),
                    (wz[1:-1], idx[:-1], idx[1:])):
        rows += [p.ravel(), q.ravel()]
        cols += [q.ravel(), p.ravel()]
        vals += [-c.ravel(), -c.ravel()]
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(prob.m, prob.m))


def time_blocks(prob: Problem, K: Optional[sp.csr_matrix] = None):
    """Blocks A_(r) of the all-at-once matrix.

    theta-method (Sec. 1, eq. theta / symbol_h): A0 = M + theta tau K,
    A1 = -M + (1-theta) tau K.
    BDF2 (Sec. 4, eq. matrix_gen; coefficients are the standard two-step BDF):
    A0 = 3/2 M + tau K, A1 = -2 M, A2 = 1/2 M.
    """
    if K is None:
        K = stiffness(prob)
    I = sp.identity(prob.m, format="csr")
    tau = prob.tau
    if prob.scheme == "theta":
        th = prob.theta
        return [(I + th * tau * K).tocsr(), (-I + (1 - th) * tau * K).tocsr()]
    if prob.scheme == "bdf2":
        return [(1.5 * I + tau * K).tocsr(), (-2.0 * I).tocsr(), (0.5 * I).tocsr()]
    raise ValueError(prob.scheme)


# --------------------------------------------------------------------------------------
# All-at-once operator, flip and right-hand side (Sec. 1 eq. theta, main_system; Sec. 4)
# --------------------------------------------------------------------------------------
def apply_T(prob: Problem, v: np.ndarray, blocks=None) -> np.ndarray:
    """(T v)_k = sum_r A_(r) v_{k-r}, block lower-triangular Toeplitz (eq. theta / matrix_gen)."""
    A = blocks if blocks is not None else time_blocks(prob)
    V = np.asarray(v, dtype=np.float64).reshape(prob.n, prob.m)
    out = np.zeros_like(V)
    for r, Ar in enumerate(A):
        if r == 0:
            out += (Ar @ V.T).T
        elif r < prob.n:
            out[r:] += (Ar @ V[:-r].T).T
    return out


def apply_T_transpose(prob: Problem, v: np.ndarray, blocks=None) -> np.ndarray:
    """(T^T v)_k = sum_r A_(r) v_{k+r} (the blocks are symmetric)."""
    A = blocks if blocks is not None else time_blocks(prob)
    V = np.asarray(v, dtype=np.float64).reshape(prob.n, prob.m)
    out = np.zeros_like(V)
    for r, Ar in enumerate(A):
        if r == 0:
            out += (Ar @ V.T).T
        elif r < prob.n:
            out[:-r] += (Ar @ V[r:].T).T
    return out


def flip(v: np.ndarray, n: int) -> np.ndarray:
    """Y = Y_n (x) I_m: reverse the order of the n time blocks (Sec. 1)."""
    V = np.asarray(v).reshape(n, -1)
    return V[::-1].copy()


def apply_op(prob: Problem, v: np.ndarray, blocks=None) -> np.ndarray:
    """Y T v, the symmetric (indefinite) all-at-once operator (eq. main_system)."""
    return flip(apply_T(prob, v, blocks), prob.n)


def rhs(prob: Problem, f: np.ndarray, u0: np.ndarray, u_prev: Optional[np.ndarray] = None,
        K: Optional[sp.csr_matrix] = None) -> np.ndarray:
    """All-at-once right-hand side f_H.

    theta (Sec. 1): block k = theta tau f^(k) + (1-theta) tau f^(k-1), block 1 also
    gets (M - (1-theta) tau K) u^(0).
    BDF2 (Sec. 4 leaves f-hat open): block k = tau f^(k); the start-up history
    moves to the rhs so that T stays exactly Toeplitz: block 1 += 2 u^(0) - 1/2 u^(-1),
    block 2 += -1/2 u^(0). Without u^(-1) the start uses u^(-1) = u^(0).
    """
    n, m, tau = prob.n, prob.m, prob.tau
    F = np.asarray(f, dtype=np.float64).reshape(n + 1, m)
    u0 = np.asarray(u0, dtype=np.float64).reshape(m)
    if prob.scheme == "theta":
        th = prob.theta
        fH = th * tau * F[1:] + (1 - th) * tau * F[:-1]
        if K is None:
            K = stiffness(prob)
        fH[0] += u0 - (1 - th) * tau * (K @ u0)
        return fH
    fH = tau * F[1:].copy()
    up = u0 if u_prev is None else np.asarray(u_prev, dtype=np.float64).reshape(m)
    fH[0] += 2.0 * u0 - 0.5 * up
    if n > 1:
        fH[1] += -0.5 * u0
    return fH


def all_at_once_matrix(prob: Problem) -> sp.csr_matrix:
    """Explicit sparse T (tiny sizes only), Kronecker form of eq. theta / matrix_gen."""
    A = time_blocks(prob)
    n = prob.n
    T = sp.csr_matrix((prob.N, prob.N))
    for r, Ar in enumerate(A):
        if r < n:
            T = T + sp.kron(sp.eye(n, k=-r), Ar)
    return T.tocsr()


def flip_matrix(n: int, m: int) -> sp.csr_matrix:
    Yn = sp.csr_matrix(np.fliplr(np.eye(n)))
    return sp.kron(Yn, sp.identity(m)).tocsr()


# --------------------------------------------------------------------------------------
# Sine transform S_n (Sec. 3.1.1, eq. matrix_tri_p)
# --------------------------------------------------------------------------------------
def dst_matrix(n: int) -> np.ndarray:
    """S_n = sqrt(2/(n+1)) [sin(i j pi/(n+1))]_{i,j=1..n}."""
    i = np.arange(1, n + 1)
    return math.sqrt(2.0 / (n + 1)) * np.sin(np.outer(i, i) * math.pi / (n + 1))


def dst(v: np.ndarray, axis: int) -> np.ndarray:
    """Apply S along one axis (library DST-I, orthonormal scaling)."""
    return scipy.fft.dst(v, type=1, norm="ortho", axis=axis)


def spatial_dst(prob: Problem, V: np.ndarray) -> np.ndarray:
    """(I_n (x) U_m) with U_m = S_my (x) S_mx (x fastest), S_mz (x) S_my (x) S_mx in 3D; S is its
    own inverse."""
    W = np.asarray(V, dtype=np.float64).reshape(prob.n, prob.mz, prob.my, prob.mx)
    W = dst(W, axis=3)
    if prob.dim >= 2:
        W = dst(W, axis=2)
    if prob.dim == 3:
        W = dst(W, axis=1)
    return W.reshape(prob.n, prob.m)


def time_dst(prob: Problem, V: np.ndarray) -> np.ndarray:
    """(S_n (x) I_m)."""
    return dst(np.asarray(V, dtype=np.float64).reshape(prob.n, prob.m), axis=0)


# --------------------------------------------------------------------------------------
# Spatial spectrum used by the preconditioners
# --------------------------------------------------------------------------------------
def averaged_stiffness_eigs(prob: Problem) -> np.ndarray:
    """Eigenvalues (shape (m,), x fastest) of the diagonal-averaged stiffness matrix.

    Sec. 3.1.1 (after eq. matrix_Km_va): K is replaced by the symmetric Toeplitz
    matrix whose diagonals are the averages of K's diagonals, which S diagonalises.
    Reading for 2D: average the main diagonal, the x-couplings and the
    y-couplings separately (only couplings that exist), giving
    Kbar = d I - e_x (shift_x + shift_x^T) - e_y (shift_y + shift_y^T), whose
    eigenvalues are d - 2 e_x cos(i pi/(mx+1)) - 2 e_y cos(j pi/(my+1)).
    For constant a this is exactly K.  3D: the z-couplings are averaged apart as well.
    """
    K = stiffness(prob).tocoo()
    mx = prob.mx
    r, c, v = K.row, K.col, K.data
    d = v[r == c].mean()
    xmask = np.abs(r - c) == 1
    ex = -v[xmask].mean() if np.any(xmask) else 0.0
    ey = ez = 0.0
    if prob.dim >= 2:
        ymask = np.abs(r - c) == mx
        ey = -v[ymask].mean() if np.any(ymask) else 0.0
    if prob.dim == 3:
        zmask = np.abs(r - c) == mx * prob.my
        ez = -v[zmask].mean() if np.any(zmask) else 0.0
    cx = np.cos(np.arange(1, mx + 1) * math.pi / (mx + 1))
    if prob.dim == 1:
        return d - 2.0 * ex * cx
    cy = np.cos(np.arange(1, prob.my + 1) * math.pi / (prob.my + 1))
    if prob.dim == 2:
        return (d - 2.0 * ex * cx[None, :] - 2.0 * ey * cy[:, None]).reshape(-1)
    cz = np.cos(np.arange(1, prob.mz + 1) * math.pi / (prob.mz + 1))
    return (d - 2.0 * ex * cx[None, None, :] - 2.0 * ey * cy[None, :, None]
            - 2.0 * ez * cz[:, None, None]).reshape(-1)


def time_cos(n: int) -> np.ndarray:
    """Diagonal of D_n: cos(k pi/(n+1)), k = 1..n, paired with column k of S_n."""
    return np.cos(np.arange(1, n + 1) * math.pi / (n + 1))


def ph_spectrum_sq(prob: Problem, mu: Optional[np.ndarray] = None) -> np.ndarray:
    """Eigenvalues (n, m) of P_H^2 (theta) or P-hat^2 (BDF), in the transformed basis.

    theta (Sec. 3.1.1): I_n (x) (L0^2 + L1^2) + D_n (x) 2 L0 L1 with
    L0 = 1 + theta tau mu, L1 = -1 + (1-theta) tau mu.
    BDF2 (Sec. 4, eq. symbol_h_gen_poly / def:matrix_P_gen): with
    q0 = A0^2 + A1^2 + A2^2, q1 = A0 A1 + A1 A2, q2 = A0 A2, writing
    2 cos 2x = 4 cos^2 x - 2 gives qbar0 = q0 - 2 q2, qbar1 = 2 q1, qbar2 = 4 q2
    and the spectrum qbar0 + qbar1 cos x_k + qbar2 cos^2 x_k.
    """
    if mu is None:
        mu = averaged_stiffness_eigs(prob)
    ck = time_cos(prob.n)[:, None]
    tau = prob.tau
    if prob.scheme == "theta":
        th = prob.theta
        L0 = 1.0 + th * tau * mu
        L1 = -1.0 + (1 - th) * tau * mu
        return (L0 ** 2 + L1 ** 2)[None, :] + ck * (2.0 * L0 * L1)[None, :]
    A0 = 1.5 + tau * mu
    A1 = -2.0 * np.ones_like(mu)
    A2 = 0.5 * np.ones_like(mu)
    q0 = A0 ** 2 + A1 ** 2 + A2 ** 2
    q1 = A0 * A1 + A1 * A2
    q2 = A0 * A2
    qb0, qb1, qb2 = q0 - 2 * q2, 2 * q1, 4 * q2
    return qb0[None, :] + ck * qb1[None, :] + ck ** 2 * qb2[None, :]


def apply_prec(prob: Problem, v: np.ndarray) -> np.ndarray:
    """z = P_H^{-1} v by the three steps of Sec. 3.1.1: transform, scale, transform back.

    (S_n (x) U_m) is symmetric and involutory, so both transforms are the same map.
    """
    if prob.prec == "Ptheta":
        return apply_ptheta(prob, v)
    d = ph_spectrum_sq(prob)
    vt = time_dst(prob, spatial_dst(prob, v))
    zt = vt / np.sqrt(d)
    return spatial_dst(prob, time_dst(prob, zt))


# --------------------------------------------------------------------------------------
# Modified preconditioner P_theta (Sec. 1 eq. def:matrix_mod_P; Sec. 3.1.4)
# --------------------------------------------------------------------------------------
def ptheta_time_eigs(n: int, theta: float):
    """Eigenvalues of H = sqrt(tridiag(-1,2,-1)) and H_theta (Sec. 1), in S_n's order.

    tridiag(-1,2,-1) = S_n diag(2 - 2cos x_k) S_n and the theta matrix
    tridiag(th(1-th), th^2+(1-th)^2, th(1-th)) = S_n diag(th^2+(1-th)^2+2th(1-th)cos x_k) S_n.
    """
    ck = time_cos(n)
    lam_h = np.sqrt(2.0 - 2.0 * ck)
    lam_ht = np.sqrt(theta ** 2 + (1 - theta) ** 2 + 2.0 * theta * (1 - theta) * ck)
    return lam_h, lam_ht


def apply_ptheta(prob: Problem, v: np.ndarray, K: Optional[sp.csr_matrix] = None) -> np.ndarray:
    """z = P_theta^{-1} v (Sec. 3.1.4): time DST, per-frequency solve with
    (lam_H,k M + lam_Htheta,k tau K), inverse time DST. Uses the true K (tau
    restored in the second term, as in the definition eq. def:matrix_mod_P)."""
    if K is None:
        K = stiffness(prob)
    if prob.dim >= 2 and prob.a_nodal is not None and prob.inner_degree is not None:
        return apply_ptheta_cheb(prob, v, prob.inner_degree, K)
    lam_h, lam_ht = ptheta_time_eigs(prob.n, prob.theta)
    vt = time_dst(prob, v)
    zt = np.empty_like(vt)
    I = sp.identity(prob.m, format="csc")
    for k in range(prob.n):
        Ak = (lam_h[k] * I + lam_ht[k] * prob.tau * K).tocsc()
        zt[k] = spla.spsolve(Ak, vt[k])
    return time_dst(prob, zt)


# Step 2 of Sec. 3.1.4 leaves the solver of the shifted systems open (the paper names multigrid).
# For a 2D varying a each system A_k = lam_H,k I + lam_Htheta,k tau K is approximated here by a
# fixed number of Chebyshev steps preconditioned with B_k = lam_H,k I + lam_Htheta,k tau abar K0,
# K0 the a = 1 stiffness matrix (diagonalised by the spatial DST) and abar the mean face value of
# a.  A fixed polynomial in B_k^-1 A_k times B_k^-1 is a fixed symmetric linear map, positive
# definite when the polynomial's error stays below one on the spectrum, so P_theta stays SPD and
# MINRES applies unchanged.
def constant_stiffness_eigs(prob: Problem) -> np.ndarray:
    """Eigenvalues of K0 (a = 1) in S's order, x fastest: (2 - 2cos(i pi/(mx+1)))/hx^2 plus the
    same term along y in 2D (the 3-point matrix tridiag(-1, 2, -1)/h^2 per axis), evaluated as
    4 sin^2(i pi/(2(mx+1))), which is the same number without the cancellation at small i."""
    ex = 4.0 * np.sin(np.arange(1, prob.mx + 1) * math.pi / (2 * (prob.mx + 1))) ** 2 / prob.hx ** 2
    if prob.dim == 1:
        return ex
    ey = 4.0 * np.sin(np.arange(1, prob.my + 1) * math.pi / (2 * (prob.my + 1))) ** 2 / prob.hy ** 2
    if prob.dim == 2:
        return (ey[:, None] + ex[None, :]).reshape(-1)
    ez = 4.0 * np.sin(np.arange(1, prob.mz + 1) * math.pi / (2 * (prob.mz + 1))) ** 2 / prob.hz ** 2
    return (ez[:, None, None] + ey[None, :, None] + ex[None, None, :]).reshape(-1)


def ptheta_cheb_bounds(prob: Problem):
    """abar and, per time frequency k, the interval [alpha_k, beta_k] holding the eigenvalues of
    B_k^-1 A_k.

    K's quadratic form is the sum over cell faces of a_f (u_p - u_q)^2 / h_f^2 (u = 0 beyond the
    boundary) and K0's the same with a_f = 1, so a_min K0 <= K <= a_max K0 with a_min, a_max over
    the faces.  B_k commutes with K0, and the ratio (lam + c a mu)/(lam + c abar mu) is monotone in
    mu and equals 1 at mu = 0, so with mu_max = the largest eigenvalue of K0 and c = lam_Htheta,k
    tau the generalised eigenvalues of (A_k, B_k) lie in
      [(lam + c a_min mu_max)/(lam + c abar mu_max), (lam + c a_max mu_max)/(lam + c abar mu_max)].
    """
    faces = np.concatenate([f.reshape(-1) for f in face_values(prob) if f is not None])
    amin, amax, abar = float(faces.min()), float(faces.max()), float(faces.mean())
    lam_h, lam_ht = ptheta_time_eigs(prob.n, prob.theta)
    mu_max = float(constant_stiffness_eigs(prob).max())
    c = lam_ht * prob.tau
    den = lam_h + c * abar * mu_max
    alpha = (lam_h + c * min(amin, abar) * mu_max) / den
    beta = (lam_h + c * max(amax, abar) * mu_max) / den
    return abar, alpha, beta


def chebyshev_solve(apply_A: Callable, apply_Binv: Callable, b: np.ndarray, alpha: float,
                    beta: float, degree: int) -> np.ndarray:
    """x ~ A^-1 b by `degree` steps of the Chebyshev iteration for B^-1 A with spectrum in
    [alpha, beta], from x = 0 (Saad, Iterative Methods for Sparse Linear Systems, Alg. 12.1, with
    the preconditioner B).  The error is x - A^-1 b = -p(B^-1 A) A^-1 b with p the Chebyshev
    polynomial of degree `degree` on [alpha, beta] scaled to p(0) = 1.  When alpha = beta up to
    rounding (B = A) the first step is already exact and the later ones are skipped."""
    centre, half = 0.5 * (beta + alpha), 0.5 * (beta - alpha)
    x = np.zeros_like(b)
    r = b.copy()
    d = apply_Binv(r) / centre
    if half <= 1e-14 * centre:
        return d
    sigma1 = centre / half
    rho = 1.0 / sigma1
    for j in range(degree):
        x = x + d
        if j == degree - 1:
            break
        r = r - apply_A(d)
        rho_next = 1.0 / (2.0 * sigma1 - rho)
        d = rho_next * rho * d + (2.0 * rho_next / half) * apply_Binv(r)
        rho = rho_next
    return x


def ptheta_cheb_blocks(prob: Problem, k: int, K: Optional[sp.csr_matrix] = None):
    """(A_k as a sparse matrix, the diagonal of B_k in the spatial DST basis) for frequency k."""
    if K is None:
        K = stiffness(prob)
    abar, _, _ = ptheta_cheb_bounds(prob)
    lam_h, lam_ht = ptheta_time_eigs(prob.n, prob.theta)
    Ak = (lam_h[k] * sp.identity(prob.m, format="csr") + lam_ht[k] * prob.tau * K).tocsr()
    bk = lam_h[k] + lam_ht[k] * prob.tau * abar * constant_stiffness_eigs(prob)
    return Ak, bk


def space_dst(prob: Problem, r: np.ndarray) -> np.ndarray:
    """U_m r for one space vector (S_my (x) S_mx, x fastest; S_mz (x) S_my (x) S_mx in 3D)."""
    R = dst(np.asarray(r, dtype=np.float64).reshape(prob.mz, prob.my, prob.mx), axis=2)
    if prob.dim >= 2:
        R = dst(R, axis=1)
    if prob.dim == 3:
        R = dst(R, axis=0)
    return R.reshape(-1)


def apply_ptheta_cheb(prob: Problem, v: np.ndarray, degree: int,
                      K: Optional[sp.csr_matrix] = None) -> np.ndarray:
    """z = P_theta^-1 v (Sec. 3.1.4) with step 2 done by `degree` Chebyshev steps per frequency
    (see ptheta_cheb_bounds / chebyshev_solve)."""
    if K is None:
        K = stiffness(prob)
    _, alpha, beta = ptheta_cheb_bounds(prob)
    vt = time_dst(prob, v)
    zt = np.empty_like(vt)
    for k in range(prob.n):
        Ak, bk = ptheta_cheb_blocks(prob, k, K)
        zt[k] = chebyshev_solve(lambda u: Ak @ u, lambda r: space_dst(prob, space_dst(prob, r) / bk),
                                vt[k], alpha[k], beta[k], degree)
    return time_dst(prob, zt)


# --------------------------------------------------------------------------------------
# Dense versions for tiny sizes (pins only)
# --------------------------------------------------------------------------------------
def sqrtm_spd(A: np.ndarray) -> np.ndarray:
    w, Q = np.linalg.eigh(0.5 * (A + A.T))
    return (Q * np.sqrt(w)) @ Q.T


def dense_PH_squared(prob: Problem, K_used: Optional[np.ndarray] = None) -> np.ndarray:
    """Block matrix under the root in eq. def:matrix_P (theta) / def:matrix_P_gen (BDF2).

    Built entry by entry from the blocks: theta: diagonal A0^2 + A1^2, off-diagonals
    A0 A1. BDF2: I (x) qbar0 + P_n (x) qbar1 + P_n^2 (x) qbar2 with
    P_n = tridiag(1/2, 0, 1/2) (eq. matrix_tri_p).
    """
    n, m, tau = prob.n, prob.m, prob.tau
    if K_used is None:
        K_used = stiffness(prob).toarray()
    I = np.eye(m)
    if prob.scheme == "theta":
        th = prob.theta
        A0 = I + th * tau * K_used
        A1 = -I + (1 - th) * tau * K_used
        out = np.zeros((n * m, n * m))
        for k in range(n):
            out[k * m:(k + 1) * m, k * m:(k + 1) * m] = A0 @ A0 + A1 @ A1
            if k + 1 < n:
                out[k * m:(k + 1) * m, (k + 1) * m:(k + 2) * m] = A0 @ A1
                out[(k + 1) * m:(k + 2) * m, k * m:(k + 1) * m] = A0 @ A1
        return out
    A0 = 1.5 * I + tau * K_used
    A1 = -2.0 * I
    A2 = 0.5 * I
    q0 = A0 @ A0 + A1 @ A1 + A2 @ A2
    q1 = A0 @ A1 + A1 @ A2
    q2 = A0 @ A2
    Pn = 0.5 * (np.eye(n, k=1) + np.eye(n, k=-1))
    return np.kron(np.eye(n), q0 - 2 * q2) + np.kron(Pn, 2 * q1) + np.kron(Pn @ Pn, 4 * q2)


def dense_symbol_toeplitz_sq(prob: Problem, K_used: Optional[np.ndarray] = None) -> np.ndarray:
    """T_(n,m)[|g|^2] for BDF2: block Toeplitz with blocks q0 (diag), q1 (+-1), q2 (+-2).

    Sec. 4, eq. symbol_h_gen_poly: |g|^2 = q0 + q1 2cos x + q2 2cos 2x, whose
    Fourier coefficients are q0, q1 (at +-1) and q2 (at +-2).
    """
    n, m, tau = prob.n, prob.m, prob.tau
    if K_used is None:
        K_used = stiffness(prob).toarray()
    I = np.eye(m)
    A0 = 1.5 * I + tau * K_used
    A1 = -2.0 * I
    A2 = 0.5 * I
    q0 = A0 @ A0 + A1 @ A1 + A2 @ A2
    q1 = A0 @ A1 + A1 @ A2
    q2 = A0 @ A2
    return (np.kron(np.eye(n), q0) + np.kron(np.eye(n, k=1) + np.eye(n, k=-1), q1)
            + np.kron(np.eye(n, k=2) + np.eye(n, k=-2), q2))


def dense_Ptheta(prob: Problem) -> np.ndarray:
    """P_theta = H (x) M + H_theta (x) tau K (eq. def:matrix_mod_P), square roots by eigh."""
    n, th = prob.n, prob.theta
    K = stiffness(prob).toarray()
    H = sqrtm_spd(2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1))
    od = th * (1 - th)
    Ht = sqrtm_spd((th ** 2 + (1 - th) ** 2) * np.eye(n) + od * (np.eye(n, k=1) + np.eye(n, k=-1)))
    return np.kron(H, np.eye(prob.m)) + np.kron(Ht, prob.tau * K)


# --------------------------------------------------------------------------------------
# MINRES (Paige & Saunders 1975), preconditioned, zero initial guess (Sec. 5)
# --------------------------------------------------------------------------------------
def minres(apply_A: Callable, apply_Minv: Callable, b: np.ndarray, tol: float, maxit: int,
           x0: Optional[np.ndarray] = None, callback: Optional[Callable] = None,
           stop: Optional[Callable] = None):
    """Preconditioned MINRES for symmetric A and SPD M.

    Lanczos in the M^{-1} inner product: with z_k = M^{-1} vhat_k and
    beta_k = sqrt(<vhat_k, z_k>), the basis is q_k = z_k / beta_k and
      p_k = A q_k,  alpha_k = <p_k, q_k>,
      vhat_{k+1} = p_k - (alpha_k/beta_k) vhat_k - (beta_k/beta_{k-1}) vhat_{k-1}.
    The tridiagonal matrix is reduced by Givens rotations; the solution is
    updated with the directions d_k = (q_k - delta_k d_{k-1} - eps_k d_{k-2})/rho_k.
    Stops when |eta_{k+1}| / beta_1 (the M^{-1}-norm relative residual) <= tol, or, when
    ``stop`` is given, when stop(k, x, est) returns True.
    Returns (x, info) with info["iterations"], info["est"] (history).
    """
    shape = b.shape
    bb = np.asarray(b, dtype=np.float64).reshape(-1)
    x = np.zeros_like(bb) if x0 is None else np.asarray(x0, dtype=np.float64).reshape(-1).copy()
    r = bb - (apply_A(x.reshape(shape)).reshape(-1) if x0 is not None else 0.0)
    vhat = r.copy()
    z = apply_Minv(vhat.reshape(shape)).reshape(-1)
    beta_sq = float(np.dot(vhat, z))
    info = {"iterations": 0, "est": [1.0], "status": "ok"}
    if beta_sq < 0 or not np.isfinite(beta_sq):
        info["status"] = "breakdown"
        return x.reshape(shape), info
    beta = math.sqrt(beta_sq)
    beta1 = beta
    if beta1 == 0.0:
        return x.reshape(shape), info
    vhat_prev = np.zeros_like(vhat)
    beta_prev = 1.0
    d_prev = np.zeros_like(vhat)  # d_{k-1}
    d_prev2 = np.zeros_like(vhat)  # d_{k-2}
    c_prev, s_prev = 1.0, 0.0  # rotation k-1
    c_prev2, s_prev2 = 1.0, 0.0  # rotation k-2
    eta = beta1
    for k in range(1, maxit + 1):
        q = z / beta
        p = apply_A(q.reshape(shape)).reshape(-1)
        alpha = float(np.dot(p, q))
        vnext = p - (alpha / beta) * vhat - ((beta / beta_prev) if k > 1 else 0.0) * vhat_prev
        znext = apply_Minv(vnext.reshape(shape)).reshape(-1)
        bnext_sq = float(np.dot(vnext, znext))
        if bnext_sq < 0 or not np.isfinite(bnext_sq):
            info["status"] = "breakdown"
            break
        bnext = math.sqrt(bnext_sq)
        # Column k of the tridiagonal: (beta_k above the diagonal for k > 1, alpha_k, beta_{k+1}).
        off = beta if k > 1 else 0.0
        eps = s_prev2 * off
        delta_bar = c_prev2 * off
        delta = c_prev * delta_bar + s_prev * alpha
        gamma_bar = -s_prev * delta_bar + c_prev * alpha
        rho = math.hypot(gamma_bar, bnext)
        if rho == 0.0:
            info["status"] = "breakdown"
            break
        c, s = gamma_bar / rho, bnext / rho
        tk = c * eta
        eta = -s * eta
        d = (q - delta * d_prev - eps * d_prev2) / rho
        x = x + tk * d
        d_prev2, d_prev = d_prev, d
        c_prev2, s_prev2 = c_prev, s_prev
        c_prev, s_prev = c, s
        vhat_prev, vhat = vhat, vnext
        z = znext
        beta_prev, beta = beta, bnext
        info["iterations"] = k
        est = abs(eta) / beta1
        info["est"].append(est)
        if callback is not None:
            callback(k, x.reshape(shape), est)
        if bnext == 0.0:
            break
        if (stop(k, x.reshape(shape), est) if stop is not None else est <= tol):
            break
    return x.reshape(shape), info


# --------------------------------------------------------------------------------------
# Solves
# --------------------------------------------------------------------------------------
def _prec_apply(prob: Problem, K):
    if prob.prec == "Ptheta":
        return lambda v: apply_ptheta(prob, v, K)  # noqa: E731
    sq = np.sqrt(ph_spectrum_sq(prob))

    def Minv(v):
        vt = time_dst(prob, spatial_dst(prob, v))
        return spatial_dst(prob, time_dst(prob, vt / sq))
    return Minv


def true_residual_rule(apply_A: Callable, b: np.ndarray, tol: float):
    """Stopping rule on the 2-norm relative residual (Sec. 5 stops on the relative residual).

    MINRES monitors est = ||r||_{M^-1}/||b||_{M^-1}. When est <= target (first target = tol)
    the true rho = ||b - A x||_2/||b||_2 is computed; the solve stops if rho <= tol, otherwise
    the target becomes target * tol / rho and the iteration continues.
    """
    state = {"target": tol, "checks": 0, "true": None}
    bn = float(np.linalg.norm(b))

    def stop(k, x, est):
        if est > state["target"]:
            return False
        rho = float(np.linalg.norm(b - apply_A(x)) / bn)
        state["checks"] += 1
        state["true"] = rho
        if rho <= tol:
            return True
        state["target"] = state["target"] * tol / rho
        return False
    return stop, state


def solve(prob: Problem, fH: np.ndarray, tol: float = 1e-8, maxit: int = 200, callback=None,
          rule: str = "true"):
    """Solve T u = f_H through MINRES on Y T u = Y f_H with P_H or P_theta (Sec. 3.1).

    rule "true": stop on the 2-norm relative residual (true_residual_rule); rule "est": stop on
    the preconditioned estimate alone.
    """
    K = stiffness(prob)
    A = time_blocks(prob, K)
    b = flip(fH, prob.n)
    Aop = lambda v: apply_op(prob, v, A)  # noqa: E731
    stop, state = (true_residual_rule(Aop, b, tol) if rule == "true" else (None, {}))
    x, info = minres(Aop, _prec_apply(prob, K), b, tol, maxit, callback=callback, stop=stop)
    r = b - apply_op(prob, x, A)
    info["true_rel_res"] = float(np.linalg.norm(r) / np.linalg.norm(b))
    info["true_checks"] = state.get("checks", 0)
    return x, info


def solve_transpose(prob: Problem, g: np.ndarray, tol: float = 1e-8, maxit: int = 200):
    """Solve T^T lam = g: T^T = Y T Y, so (Y T)(Y lam) = g and lam = Y mu."""
    K = stiffness(prob)
    A = time_blocks(prob, K)
    g = np.asarray(g, dtype=np.float64).reshape(prob.n, prob.m)
    Aop = lambda v: apply_op(prob, v, A)  # noqa: E731
    stop, state = true_residual_rule(Aop, g, tol)
    mu, info = minres(Aop, _prec_apply(prob, K), g, tol, maxit, stop=stop)
    return flip(mu, prob.n), info


def forward_substitution(prob: Problem, fH: np.ndarray) -> np.ndarray:
    """Direct solve of T u = f_H (the reference solution of the all-at-once system, Sec. 1).

    T is block lower triangular and Toeplitz with the blocks of time_blocks (eq. theta; Sec. 4
    for BDF2), so block row k reads A0 u_k + A1 u_{k-1} (+ A2 u_{k-2}) = f_H,k and the unknown
    blocks follow one after the other: u_k = A0^{-1} (f_H,k - A1 u_{k-1} - A2 u_{k-2}), with one
    sparse LU factorisation of the SPD block A0.  For f_H = rhs(f, u0) this is the sequential
    time stepping of march; for any other f_H (e.g. one with added noise) it is still exact up
    to the rounding of the LU solves.
    """
    n, m = prob.n, prob.m
    A = time_blocks(prob)
    F = np.asarray(fH, dtype=np.float64).reshape(n, m)
    lu = spla.splu(A[0].tocsc())
    U = np.zeros((n, m))
    for k in range(n):
        r = F[k].copy()
        for d in range(1, len(A)):
            if k - d >= 0:
                r -= A[d] @ U[k - d]
        U[k] = lu.solve(r)
    return U


def march(prob: Problem, f: np.ndarray, u0: np.ndarray, u_prev: Optional[np.ndarray] = None):
    """Sequential time stepping, the system the all-at-once form is equivalent to (Sec. 1).

    theta: (M + theta tau K) u^k = (M - (1-theta) tau K) u^{k-1} + theta tau f^k + (1-theta) tau f^{k-1}.
    BDF2:  (3/2 M + tau K) u^k = 2 u^{k-1} - 1/2 u^{k-2} + tau f^k.
    """
    n, m, tau = prob.n, prob.m, prob.tau
    K = stiffness(prob)
    I = sp.identity(m, format="csc")
    F = np.asarray(f, dtype=np.float64).reshape(n + 1, m)
    U = np.zeros((n, m))
    if prob.scheme == "theta":
        th = prob.theta
        lu = spla.splu((I + th * tau * K).tocsc())
        prev = np.asarray(u0, dtype=np.float64).reshape(m)
        for k in range(1, n + 1):
            r = prev - (1 - th) * tau * (K @ prev) + th * tau * F[k] + (1 - th) * tau * F[k - 1]
            prev = lu.solve(r)
            U[k - 1] = prev
        return U
    lu = spla.splu((1.5 * I + tau * K).tocsc())
    um1 = np.asarray(u0 if u_prev is None else u_prev, dtype=np.float64).reshape(m)
    u_0 = np.asarray(u0, dtype=np.float64).reshape(m)
    hist = [um1, u_0]
    for k in range(1, n + 1):
        r = 2.0 * hist[-1] - 0.5 * hist[-2] + tau * F[k]
        uk = lu.solve(r)
        U[k - 1] = uk
        hist.append(uk)
    return U


# --------------------------------------------------------------------------------------
# Adjoint gradients of L = 1/2 ||u - u_obs||^2 (chain rule through T u = f_H(f, u0))
# --------------------------------------------------------------------------------------
def adjoint_gradients(prob: Problem, u: np.ndarray, lam: np.ndarray, u0: np.ndarray):
    """Given the forward solution u and the adjoint lam = T^{-T} (u - u_obs):

    dL/df_H = lam. theta: f_H block k = theta tau f^(k) + (1-theta) tau f^(k-1),
    block 1 += (M - (1-theta) tau K) u0, hence
      dL/df^(k) = theta tau lam_k + (1-theta) tau lam_{k+1}  (lam_0 = lam_{n+1} = 0),
      dL/du0   = (M - (1-theta) tau K) lam_1.
    BDF2: dL/df^(k) = tau lam_k (k >= 1), dL/du0 = 2 lam_1 - 1/2 lam_2 (u^(-1) tied to u0 is not
    differentiated).
    dL/da: the residual block k is A0 u_k + A1 u_{k-1} - rhs_k and only tau K depends on a, so
      dL/da = -tau sum_k lam_k^T (dK/da) w_k, w_k = theta u_k + (1-theta) u_{k-1} (u_0 = u0),
    (BDF2: w_k = u_k). For the face value a_f between nodes p and q (q may be a boundary node
    with value 0), lam^T (dK/da_f) w = (lam_p - lam_q)(w_p - w_q)/h^2. Each face value is the mean
    of its two nodal values, so half of each face gradient goes to each node.
    Returns (grad_f (n+1, m), grad_u0 (m,), grad_a_nodal (nodal shape)).
    """
    n, m, tau = prob.n, prob.m, prob.tau
    U = np.asarray(u, dtype=np.float64).reshape(n, m)
    L = np.asarray(lam, dtype=np.float64).reshape(n, m)
    u0 = np.asarray(u0, dtype=np.float64).reshape(m)
    K = stiffness(prob)
    gf = np.zeros((n + 1, m))
    if prob.scheme == "theta":
        th = prob.theta
        gf[1:] += th * tau * L
        gf[:-1] += (1 - th) * tau * L
        gu0 = L[0] - (1 - th) * tau * (K @ L[0])
        Uprev = np.vstack([u0[None, :], U[:-1]])
        W = th * U + (1 - th) * Uprev
    else:
        gf[1:] += tau * L
        gu0 = 2.0 * L[0] - (0.5 * L[1] if n > 1 else 0.0)
        W = U
    if prob.dim == 3:
        raise NotImplementedError("the a-gradient is written for 1D and 2D grids")
    mx, my = prob.mx, prob.my
    Lg = L.reshape(n, my, mx)
    Wg = W.reshape(n, my, mx)
    # pad with the zero boundary values
    Lp = np.zeros((n, my + 2, mx + 2))
    Wp = np.zeros((n, my + 2, mx + 2))
    Lp[:, 1:-1, 1:-1] = Lg
    Wp[:, 1:-1, 1:-1] = Wg
    if prob.dim == 1:
        Lp1 = Lp[:, 1, :]
        Wp1 = Wp[:, 1, :]
        gx = (np.diff(Lp1, axis=1) * np.diff(Wp1, axis=1)).sum(axis=0) / prob.hx ** 2  # (mx+1,)
        gface_x = -tau * gx
        ga = np.zeros(mx + 2)
        ga[:-1] += 0.5 * gface_x
        ga[1:] += 0.5 * gface_x
        return gf, gu0, ga
    # x-faces on interior rows: between (j, i) and (j, i+1), i = 0..mx
    dLx = np.diff(Lp[:, 1:-1, :], axis=2)
    dWx = np.diff(Wp[:, 1:-1, :], axis=2)
    gface_x = -tau * (dLx * dWx).sum(axis=0) / prob.hx ** 2  # (my, mx+1)
    dLy = np.diff(Lp[:, :, 1:-1], axis=1)
    dWy = np.diff(Wp[:, :, 1:-1], axis=1)
    gface_y = -tau * (dLy * dWy).sum(axis=0) / prob.hy ** 2  # (my+1, mx)
    ga = np.zeros((my + 2, mx + 2))
    ga[1:-1, :-1] += 0.5 * gface_x
    ga[1:-1, 1:] += 0.5 * gface_x
    ga[:-1, 1:-1] += 0.5 * gface_y
    ga[1:, 1:-1] += 0.5 * gface_y
    return gf, gu0, ga
