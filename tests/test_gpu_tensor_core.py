"""The tensor-core (tcgen05) kernels of the mixed-precision preconditioner (time DST with the
spectral scaling; spatial DST along y) against the oracle and against the float32 FFMA /
shared-memory FFT kernels they replace (ST_DISABLE_TENSOR_CORES=1), on the lengths they support."""
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


def _rel2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# n supported by the tensor-core time path (multiples of 32 up to 256) and my + 1 in
# {32, ..., 256} for the tensor-core y-DST; spatial sizes with ragged 32-column tiles
# (m = 63, 15*31, 63*63, 127*127, 31*255); n = 40 keeps the FFMA time kernel
@pytest.mark.parametrize("dim,mx,my,n,scheme,theta", [
    (1, 63, 1, 32, "theta", 1.0),
    (2, 15, 31, 64, "theta", 0.5),
    (2, 63, 63, 128, "bdf2", 1.0),
    (2, 127, 127, 256, "theta", 0.5),
    (2, 31, 31, 96, "theta", 0.3),
    (2, 31, 255, 40, "theta", 0.5),
    # 256 < n <= 512: the kernel that streams S_n through shared memory (K padded to 256)
    (2, 15, 15, 512, "theta", 0.5),
    (1, 63, 1, 320, "theta", 1.0),
    (2, 31, 15, 384, "bdf2", 1.0),
])
def test_tc_time_dst_matches_oracle_and_ffma(pkg, dim, mx, my, n, scheme, theta):
    w = W.small_case(dim, mx, my, n, scheme=scheme, theta=theta, varcoef=True, seed=n + mx)
    p = H.Problem.from_workload(w)
    v = np.random.default_rng(6).standard_normal((n, p.m))
    ref = H.apply_prec(p, v)
    spec = pkg.ProblemSpec(w.dim, w.mx, w.my, w.n, w.T, w.scheme, w.theta, w.a_nodal, "PH", "mixed")
    s_tc = pkg.Solver(spec)
    z_tc = s_tc.st_apply_prec_f32(torch.tensor(v, device="cuda")).cpu().numpy().astype(np.float64)
    os.environ["ST_DISABLE_TENSOR_CORES"] = "1"
    try:
        s_ff = pkg.Solver(spec)
    finally:
        del os.environ["ST_DISABLE_TENSOR_CORES"]
    z_ff = s_ff.st_apply_prec_f32(torch.tensor(v, device="cuda")).cpu().numpy().astype(np.float64)
    assert _rel2(z_tc.reshape(n, p.m), ref) <= 2e-5
    assert _rel2(z_ff.reshape(n, p.m), ref) <= 2e-5
    assert _rel2(z_tc, z_ff) <= 2e-5
    s_tc.close()
    s_ff.close()


# The P_theta paths with a varying coefficient transform time alone (no scaling); for n a
# multiple of 32 up to 256 that transform runs on the tensor cores.  1D: PCR blocks; 2D: the
# Chebyshev inner map (degree 0 = the library default).
@pytest.mark.parametrize("dim,mx,my,n,theta,deg", [
    (1, 127, 1, 64, 1.0, 0),
    (2, 31, 15, 32, 0.5, 2),
    (2, 15, 15, 256, 0.5, 2),
    (2, 63, 63, 96, 1.0, 3),
])
def test_tc_single_time_transform_ptheta(pkg, dim, mx, my, n, theta, deg):
    w = W.small_case(dim, mx, my, n, scheme="theta", theta=theta, varcoef=True, seed=n + mx)
    d_used = (deg if deg else pkg.ST_PTHETA_DEFAULT_DEGREE) if dim == 2 else None
    p = H.Problem.from_workload(w, prec="Ptheta", inner_degree=d_used)
    v = np.random.default_rng(8).standard_normal((n, p.m))
    ref = H.apply_ptheta(p, v)
    spec = pkg.ProblemSpec(w.dim, w.mx, w.my, w.n, w.T, w.scheme, w.theta, w.a_nodal, "Ptheta",
                           "mixed", deg)
    s_tc = pkg.Solver(spec)
    z_tc = s_tc.st_apply_prec_f32(torch.tensor(v, device="cuda")).cpu().numpy().astype(np.float64)
    os.environ["ST_DISABLE_TENSOR_CORES"] = "1"
    try:
        s_ff = pkg.Solver(spec)
    finally:
        del os.environ["ST_DISABLE_TENSOR_CORES"]
    z_ff = s_ff.st_apply_prec_f32(torch.tensor(v, device="cuda")).cpu().numpy().astype(np.float64)
    # float32 errors of the per-frequency solves dominate and are the same on both paths; the
    # tensor-core transform adds float32-level rounding of its own
    e_ff = _rel2(z_ff.reshape(n, p.m), ref)
    assert _rel2(z_tc.reshape(n, p.m), ref) <= max(2e-5, 2 * e_ff)
    assert _rel2(z_tc, z_ff) <= max(2e-5, 2 * e_ff)
    s_tc.close()
    s_ff.close()


def _prec_tol64(p):
    """float64 path with double-float transforms: 1e-11 (48-bit significands), widened for a
    varying coefficient by the spread of the averaged-K eigenvalues (the lowest modes cancel)."""
    if p.a_nodal is None:
        return 1e-11
    mu = H.averaged_stiffness_eigs(p)
    return max(1e-11, 16 * 2.220446049250313e-16 * mu.max() / mu.min())


# n supported by the float64 tensor-core time stage (multiples of 32 with n/2 <= 64, and 256),
# ragged 32-column tiles, theta, BDF2 and the constant-coefficient P_theta
@pytest.mark.parametrize("dim,mx,my,n,scheme,theta,var,prec", [
    (1, 63, 1, 32, "theta", 1.0, False, "PH"),
    (2, 15, 31, 64, "theta", 0.5, True, "PH"),
    (2, 31, 31, 96, "bdf2", 1.0, True, "PH"),
    (1, 127, 1, 128, "theta", 0.5, False, "PH"),
    (2, 63, 63, 256, "theta", 0.5, True, "PH"),
    (2, 31, 15, 64, "theta", 0.5, False, "Ptheta"),
])
def test_fp64_time_digits_match_oracle(pkg, dim, mx, my, n, scheme, theta, var, prec):
    """The float64 path's time stage on the tensor cores (S_n and the double-float data cut into
    seven 7-bit integer digits, each digit group accumulated exactly in float32): P^-1 v within
    the float64 path's oracle tolerance, within 1e-12 of the CUDA-core double-float kernel
    (ST_DISABLE_TENSOR_CORES=1) but not bitwise equal to it (a different kernel ran), and the same
    MINRES iterates as the oracle at equal iteration count (1e-10)."""
    w = W.small_case(dim, mx, my, n, scheme=scheme, theta=theta, varcoef=var, seed=3 * n + mx)
    p = H.Problem.from_workload(w, prec=prec)
    v = np.random.default_rng(8).standard_normal((n, p.m))
    ref = H.apply_prec(p, v)
    spec = pkg.ProblemSpec(w.dim, w.mx, w.my, w.n, w.T, w.scheme, w.theta, w.a_nodal, prec, "fp64")
    s_tc = pkg.Solver(spec)
    z_tc = s_tc.st_apply_prec(torch.tensor(v, device="cuda")).cpu().numpy()
    os.environ["ST_DISABLE_TENSOR_CORES"] = "1"
    try:
        s_cc = pkg.Solver(spec)
    finally:
        del os.environ["ST_DISABLE_TENSOR_CORES"]
    z_cc = s_cc.st_apply_prec(torch.tensor(v, device="cuda")).cpu().numpy()
    scale = np.abs(ref).max()
    assert np.abs(z_tc - ref).max() / scale <= _prec_tol64(p)
    assert np.abs(z_tc - z_cc).max() / scale <= max(1e-12, _prec_tol64(p) / 10)
    assert not np.array_equal(z_tc, z_cc)
    fH = H.rhs(p, w.f, w.u0, w.u_prev)
    K = 5
    x_or, _ = H.solve(p, fH, tol=0.0, maxit=K, rule="est")
    u, st = s_tc.st_solve(torch.tensor(fH, device="cuda").reshape(-1), tol=0.0, maxit=K,
                          allow_not_converged=True)
    assert st["iterations"] == K
    assert _rel2(u.cpu().numpy().reshape(n, p.m), x_or) <= 1e-10
    s_tc.close()
    s_cc.close()


# The last x pass of the preconditioner on the tensor cores (k_dst_tc_yw over contiguous x-lines,
# 32 lines per tile), which a handle takes by default where mx + 1 allows, against the
# shared-memory FFT that ST_X_TENSOR_CORES=0 selects.  mx + 1 in {32, 64, 128, 256}; line counts n my mz with a ragged
# last tile (40 * 15 = 600, 24 * 7 * 7 = 1176) and whole tiles; 1D, 2D and 3D.
@pytest.mark.parametrize("dim,mx,my,n,scheme,theta", [
    (1, 63, 1, 40, "theta", 1.0),
    (2, 31, 15, 40, "theta", 0.5),
    (2, 127, 63, 64, "bdf2", 1.0),
    (2, 255, 31, 32, "theta", 0.5),
    (3, 31, 7, 24, "theta", 1.0),
])
def test_tc_x_pass_matches_oracle_and_fft(pkg, dim, mx, my, n, scheme, theta):
    w = W.small_case(dim, mx, my, n, scheme=scheme, theta=theta, varcoef=True, seed=3 * n + my,
                     mz=my)
    p = H.Problem.from_workload(w)
    v = np.random.default_rng(10).standard_normal((n, p.m))
    ref = H.apply_prec(p, v)
    spec = pkg.ProblemSpec(w.dim, w.mx, w.my, w.n, w.T, w.scheme, w.theta, w.a_nodal, "PH", "mixed",
                           0, w.mz)
    s_tc = pkg.Solver(spec)
    z_tc = s_tc.st_apply_prec_f32(torch.tensor(v, device="cuda")).cpu().numpy().astype(np.float64)
    os.environ["ST_X_TENSOR_CORES"] = "0"
    try:
        s_fft = pkg.Solver(spec)
    finally:
        del os.environ["ST_X_TENSOR_CORES"]
    z_fft = s_fft.st_apply_prec_f32(torch.tensor(v, device="cuda")).cpu().numpy().astype(np.float64)
    assert _rel2(z_tc.reshape(n, p.m), ref) <= 2e-5
    assert _rel2(z_fft.reshape(n, p.m), ref) <= 2e-5
    assert _rel2(z_tc, z_fft) <= 2e-5
    assert not np.array_equal(z_tc, z_fft)  # a different kernel ran
    # a mixed solve through it reaches the oracle's converged solution
    fH = H.rhs(p, w.f, w.u0, w.u_prev)
    x_ref, _ = H.solve(p, fH, tol=1e-13, maxit=800)
    u, st = s_tc.st_solve(torch.tensor(fH, device="cuda").reshape(-1), tol=1e-9, maxit=800)
    assert st["true_rel_res"] <= 1e-9
    assert _rel2(u.cpu().numpy().reshape(n, p.m), x_ref) <= 1e-8
    s_fft.close()
    s_tc.close()
