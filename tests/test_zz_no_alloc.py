"""st_residual_noalloc: the residual check for callers that cannot allocate device memory.

Callers recording a CUDA graph, running latency-critical loops (cudaFree synchronises the
device) or owning all device memory in their own arena cannot let a library allocate.  This
entry point serves them from a static device array; here it must agree with the regular path
(st_apply_op through a handle) and with the oracle's Y f_H - Y T u on two calls in a row, which
also shows the shared scratch is left in a usable state.  Collected last so that a failure here
stops the run after the rest.
"""
import ctypes

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


@pytest.mark.parametrize("case", [(2, 63, 31, 37, "theta", 0.5), (1, 127, 1, 20, "bdf2", 1.0)])
def test_noalloc_residual_matches_regular_path(pkg, case):
    dim, mx, my, n, scheme, theta = case
    w = W.small_case(dim, mx, my, n, scheme=scheme, theta=theta, varcoef=True, seed=31)
    dev = torch.device("cuda")
    fH = torch.tensor(np.random.default_rng(1).standard_normal((n, w.m)), device=dev)
    u = torch.tensor(np.random.default_rng(2).standard_normal((n, w.m)), device=dev)
    a_dev = torch.tensor(w.a_nodal, device=dev)
    # regular path: a handle and st_apply_op
    s = pkg.Solver(pkg.ProblemSpec(dim, mx, my, n, w.T, scheme, theta, w.a_nodal))
    r_ref = torch.flip(fH, dims=[0]) - s.st_apply_op(u).reshape(n, w.m)
    torch.cuda.synchronize()
    s.close()
    sums_ref = np.array([float((r_ref * r_ref).sum()), float((fH * fH).sum())])
    # the oracle's residual on the same inputs
    po = H.Problem.from_workload(w)
    r_or = H.flip(fH.cpu().numpy(), n) - H.apply_op(po, u.cpu().numpy())
    sums_or = np.array([float(np.sum(r_or * r_or)), float(np.sum(fH.cpu().numpy() ** 2))])
    spec = pkg.ProblemSpec(dim, mx, my, n, w.T, scheme, theta, None)
    p, keep = spec.to_c(torch.cuda.current_stream().cuda_stream)
    lib = pkg.load_library()
    for call in range(2):
        r = torch.full_like(fH, float("nan"))
        sums = torch.full((2,), float("nan"), dtype=torch.float64, device=dev)
        rc = lib.st_residual_noalloc(ctypes.byref(p), ctypes.c_void_p(a_dev.data_ptr()),
                                     ctypes.c_void_p(fH.data_ptr()), ctypes.c_void_p(u.data_ptr()),
                                     ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(sums.data_ptr()))
        assert rc == pkg.ST_OK, pkg.strerror(rc)
        torch.cuda.synchronize()
        rel = float((r - r_ref).abs().max() / r_ref.abs().max())
        assert rel <= 1e-13, (call, rel)
        r_h = r.cpu().numpy()
        assert np.max(np.abs(r_h - r_or)) / np.max(np.abs(r_or)) <= 1e-13, call
        got = sums.cpu().numpy()
        assert np.allclose(got, sums_ref, rtol=1e-12, atol=0.0), (call, got, sums_ref)
        assert np.allclose(got, sums_or, rtol=1e-12, atol=0.0), (call, got, sums_or)


def test_noalloc_rejects_what_it_cannot_hold(pkg):
    lib = pkg.load_library()
    bad = pkg.ProblemSpec(2, 2047, 2047, 4)
    p, keep = bad.to_c()
    z = ctypes.c_void_p(1)
    assert lib.st_residual_noalloc(ctypes.byref(p), None, z, z, None, z) == pkg.ST_ERR_ARG
    host_a = pkg.ProblemSpec(2, 15, 15, 4, a_nodal=np.ones((17, 17)))
    p2, keep2 = host_a.to_c()
    assert lib.st_residual_noalloc(ctypes.byref(p2), None, z, z, None, z) == pkg.ST_ERR_ARG


def test_noalloc_rejects_overlapping_output(pkg):
    """r must not share memory with f_H or u: every block reads both inputs across time levels
    while other blocks write r.  The call refuses before it launches anything."""
    lib = pkg.load_library()
    spec = pkg.ProblemSpec(2, 15, 15, 4)
    p, keep = spec.to_c()
    n_bytes = spec.N * 8
    base = 1 << 20  # fake addresses: the call must reject them before touching the device
    fH, u = ctypes.c_void_p(base), ctypes.c_void_p(base + 4 * n_bytes)
    sums = ctypes.c_void_p(base + 8 * n_bytes)
    for r in (base, base + n_bytes // 2, base + 4 * n_bytes + 8, base + 4 * n_bytes - 8):
        rc = lib.st_residual_noalloc(ctypes.byref(p), None, fH, u, ctypes.c_void_p(r), sums)
        assert rc == pkg.ST_ERR_ARG, r
