"""The C-ABI library builds, loads and exports every symbol include/st_minres.h declares
(no GPU needed: no compute call is made here)."""
import ctypes
import os
import re

import numpy as np

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2201_10062_gb300 import build, load_library

    build.build()
    return load_library()


def _declared():
    src = open(os.path.join(ROOT, "include", "st_minres.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(st_[a-z0-9_]+)\s*\(", src)))


def test_header_matches_binding_exports():
    from paper_2201_10062_gb300 import EXPORTS

    assert _declared() == sorted(EXPORTS)


def test_every_declared_symbol_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_strerror_and_version(lib):
    from paper_2201_10062_gb300 import strerror

    assert lib.st_version() >= 1
    for c in range(7):
        assert isinstance(strerror(c), str) and strerror(c)
    assert strerror(99) == "unknown status"


def _spec(**kw):
    from paper_2201_10062_gb300 import ProblemSpec

    base = dict(dim=2, mx=15, my=15, n=8)
    base.update(kw)
    return ProblemSpec(**base)


@pytest.mark.parametrize("bad", [
    dict(mx=14), dict(my=16), dict(dim=3), dict(n=0), dict(n=2000), dict(T=0.0), dict(theta=1.5),
    dict(dim=1, my=3), dict(mx=2047), dict(prec="Ptheta", scheme="bdf2"),
    dict(prec="Ptheta", a_nodal=np.ones((17, 17)), inner_degree=17),
    dict(prec="Ptheta", a_nodal=np.ones((17, 17)), inner_degree=-1),
    dict(inner_degree=2), dict(prec="Ptheta", inner_degree=2),
    dict(dim=1, my=1, prec="Ptheta", a_nodal=np.ones(17), inner_degree=2),
    dict(dim=3, mz=14), dict(dim=3, mz=1), dict(dim=4),
    dict(dim=3, mx=1023, my=1023, mz=1023, n=4),  # n*m beyond 2^31
    dict(dim=3, mx=3, my=1023, mz=1023, n=2),  # my*mz beyond the stencil grid's row axis
])
def test_setup_rejects_bad_problems_before_touching_the_gpu(lib, bad):
    from paper_2201_10062_gb300 import ST_ERR_ARG

    spec = _spec(**bad)
    p, keep = spec.to_c()
    h = ctypes.c_void_p()
    assert lib.st_setup(ctypes.byref(p), ctypes.byref(h)) == ST_ERR_ARG
    assert not h.value


def test_setup_rejects_nonpositive_a(lib):
    """a must be finite and >= 0, with every face (mean of two nodes on an interior line) > 0."""
    import numpy as np
    from paper_2201_10062_gb300 import ST_ERR_ARG, st_workspace_bytes

    for bad in ("negative", "zero face", "nan"):
        a = np.ones((17, 17))
        if bad == "negative":
            a[3, 4] = -1e-3
        elif bad == "zero face":
            a[3, 4] = a[3, 5] = 0.0  # the x face between them is zero
        else:
            a[8, 8] = np.nan
        p, keep = _spec(a_nodal=a).to_c()
        h = ctypes.c_void_p()
        assert lib.st_setup(ctypes.byref(p), ctypes.byref(h)) == ST_ERR_ARG, bad
    # a vanishing on the boundary nodes (the paper's Example 2, a = 1e-5 sin(pi x y)) is valid
    x = np.linspace(0.0, 1.0, 17)
    a = 1e-5 * np.sin(np.pi * np.outer(x, x))
    assert st_workspace_bytes(_spec(a_nodal=a)) > 0


def test_workspace_bytes(lib):
    from paper_2201_10062_gb300 import st_workspace_bytes

    b64 = st_workspace_bytes(_spec(mx=255, my=255, n=256))
    b32 = st_workspace_bytes(_spec(mx=255, my=255, n=256, precision="mixed"))
    N = 255 * 255 * 256
    assert 9 * 8 * N <= b64 <= 9 * 8 * N + (64 << 20)
    # float32 z vectors, plus a double-float x accumulator, the tensor-core S_n image and the
    # seven float32 z vectors a grouped update of 8 iterations keeps pending
    assert b32 <= b64 + 7 * 4 * N + (1 << 20)


def test_workspace_bytes_follow_the_update_group(lib, monkeypatch):
    """Each iteration of the update group beyond the first keeps one more float32 z vector
    (mixed precision only)."""
    from paper_2201_10062_gb300 import st_workspace_bytes

    N = 255 * 255 * 256
    got = {}
    for G in (1, 4, 8):
        monkeypatch.setenv("ST_UPDATE_GROUP", str(G))
        got[G] = (st_workspace_bytes(_spec(mx=255, my=255, n=256, precision="mixed")),
                  st_workspace_bytes(_spec(mx=255, my=255, n=256)))
    assert got[4][0] - got[1][0] == 3 * 4 * N
    assert got[8][0] - got[1][0] == 7 * 4 * N
    assert got[1][1] == got[4][1] == got[8][1]


def test_workspace_bytes_chebyshev_ptheta(lib):
    """P_theta with a 2D varying a adds five float64 scratch vectors and the step scalars."""
    from paper_2201_10062_gb300 import st_workspace_bytes

    a = np.ones((257, 257))
    N = 255 * 255 * 64
    base = st_workspace_bytes(_spec(mx=255, my=255, n=64, a_nodal=a))
    for deg in (0, 1, 16):
        b = st_workspace_bytes(_spec(mx=255, my=255, n=64, a_nodal=a, prec="Ptheta", inner_degree=deg))
        assert 5 * 8 * N <= b - base <= 5 * 8 * N + (1 << 20)


def test_c_abi_rejects_mz_below_3d(lib):
    """st_problem.mz must be 0 or 1 for dim 1 and 2 (the binding always passes 1 there)."""
    from paper_2201_10062_gb300 import ST_ERR_ARG

    p, keep = _spec(dim=2).to_c()
    p.mz = 7
    h = ctypes.c_void_p()
    assert lib.st_setup(ctypes.byref(p), ctypes.byref(h)) == ST_ERR_ARG
    size = ctypes.c_size_t(0)
    assert lib.st_workspace_bytes(ctypes.byref(p), ctypes.byref(size)) == ST_ERR_ARG


def test_setup_rejects_nonpositive_a_3d(lib):
    from paper_2201_10062_gb300 import ST_ERR_ARG

    a = np.ones((9, 17, 17))
    a[2, 3, 4] = -1.0
    p, keep = _spec(dim=3, mz=7, a_nodal=a).to_c()
    h = ctypes.c_void_p()
    assert lib.st_setup(ctypes.byref(p), ctypes.byref(h)) == ST_ERR_ARG


def test_workspace_bytes_3d(lib):
    """3D: the same vectors over m = mx*my*mz; the Chebyshev P_theta adds its five scratch
    vectors."""
    from paper_2201_10062_gb300 import st_workspace_bytes

    N = 63 * 63 * 63 * 64
    b64 = st_workspace_bytes(_spec(dim=3, mx=63, my=63, mz=63, n=64))
    assert 9 * 8 * N <= b64 <= 9 * 8 * N + (64 << 20)
    a = np.ones((65, 65, 65))
    bc = st_workspace_bytes(_spec(dim=3, mx=63, my=63, mz=63, n=64, a_nodal=a, prec="Ptheta"))
    base = st_workspace_bytes(_spec(dim=3, mx=63, my=63, mz=63, n=64, a_nodal=a))
    assert 5 * 8 * N <= bc - base <= 5 * 8 * N + (1 << 20)


def test_null_arguments(lib):
    from paper_2201_10062_gb300 import ST_ERR_ARG

    assert lib.st_setup(None, None) == ST_ERR_ARG
    assert lib.st_apply_op(None, None, None) == ST_ERR_ARG
    assert lib.st_solve(None, None, None, 1e-8, 10, None) == ST_ERR_ARG
    lib.st_destroy(None)
