"""GB300 (sm_103a) sine-transform preconditioned MINRES for all-at-once heat systems.

Python binding of the C ABI in ``include/st_minres.h`` (libstminres.so, built in-tree by
``paper_2201_10062_gb300.build``).  This module only marshals arguments: every step of the
solve runs in the library's CUDA kernels.  PyTorch provides device memory and streams.
The functions ``st_setup``, ``st_apply_op``, ... carry the C names; ``Solver`` wraps a handle.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libstminres.so")

ST_OK, ST_ERR_ARG, ST_ERR_CUDA, ST_ERR_NOT_CONVERGED, ST_ERR_BREAKDOWN, ST_ERR_TIMEOUT, ST_ERR_OOM = range(7)
ST_THETA, ST_BDF2 = 0, 1
ST_PREC_PH, ST_PREC_PTHETA = 0, 1
ST_FP64, ST_MIXED = 0, 1
ST_PTHETA_DEFAULT_DEGREE, ST_PTHETA_MAX_DEGREE = 2, 16

# Every symbol declared in include/st_minres.h.
EXPORTS = (
    "st_setup", "st_destroy", "st_workspace_bytes", "st_assemble_rhs", "st_apply_op",
    "st_apply_prec", "st_apply_prec_f32", "st_solve", "st_solve_host", "st_solve_transpose",
    "st_grad_a", "st_strerror", "st_version", "st_profile_begin", "st_profile_end",
    "st_kernel_class_name", "st_residual_noalloc", "st_grad_rhs", "st_setup_batch",
    "st_solve_batch", "st_batch_instance", "st_destroy_batch", "st_autotune",
)
KERNEL_CLASSES = ("stencil", "lanczos_dst_x", "dst_x", "dst_y", "time_dst_scale", "update", "residual",
                  "aux")
# Most MINRES iterations one grouped direction/solution update applies (the library's ring).
UPDATE_GROUP_MAX = 8


def update_group() -> int:
    """Iterations per grouped update of a mixed single solve, as st_setup reads it: the
    ST_UPDATE_GROUP environment variable when it holds 1..8, else 8."""
    try:
        g = int(os.environ.get("ST_UPDATE_GROUP", "0"))
    except ValueError:
        g = 0
    return g if 1 <= g <= UPDATE_GROUP_MAX else UPDATE_GROUP_MAX


class StProblem(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("mx", ctypes.c_int), ("my", ctypes.c_int), ("n", ctypes.c_int),
        ("T", ctypes.c_double), ("scheme", ctypes.c_int), ("theta", ctypes.c_double),
        ("a_nodal", ctypes.POINTER(ctypes.c_double)), ("prec", ctypes.c_int),
        ("precision", ctypes.c_int), ("stream", ctypes.c_void_p), ("inner_degree", ctypes.c_int),
        ("mz", ctypes.c_int),
    ]


class StStats(ctypes.Structure):
    _fields_ = [
        ("iterations", ctypes.c_int), ("outer_steps", ctypes.c_int), ("true_checks", ctypes.c_int),
        ("status", ctypes.c_int), ("est_rel_res", ctypes.c_double),
        ("true_rel_res", ctypes.c_double), ("seconds", ctypes.c_double),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class StKernelTime(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int), ("timed", ctypes.c_int), ("ms", ctypes.c_double)]


class SolverError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {strerror(code)} (status {code})")


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libstminres.so (raises if it has not been built: there is no fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing; build it with `python -m paper_2201_10062_gb300.build`")
    lib = ctypes.CDLL(path)
    P, D, I = ctypes.c_void_p, ctypes.c_double, ctypes.c_int
    lib.st_setup.argtypes = [ctypes.POINTER(StProblem), ctypes.POINTER(P)]
    lib.st_setup.restype = I
    lib.st_destroy.argtypes = [P]
    lib.st_destroy.restype = None
    lib.st_workspace_bytes.argtypes = [ctypes.POINTER(StProblem), ctypes.POINTER(ctypes.c_size_t)]
    lib.st_workspace_bytes.restype = I
    lib.st_assemble_rhs.argtypes = [P, P, P, P, P, P]
    lib.st_assemble_rhs.restype = I
    for name in ("st_apply_op", "st_apply_prec", "st_apply_prec_f32"):
        getattr(lib, name).argtypes = [P, P, P]
        getattr(lib, name).restype = I
    for name in ("st_solve", "st_solve_host", "st_solve_transpose"):
        getattr(lib, name).argtypes = [P, P, P, D, I, ctypes.POINTER(StStats)]
        getattr(lib, name).restype = I
    lib.st_autotune.argtypes = [P, I]
    lib.st_autotune.restype = I
    lib.st_setup_batch.argtypes = [ctypes.POINTER(StProblem), I, P, ctypes.POINTER(P)]
    lib.st_setup_batch.restype = I
    lib.st_solve_batch.argtypes = [P, ctypes.POINTER(P), ctypes.POINTER(P), D, I,
                                   ctypes.POINTER(StStats)]
    lib.st_solve_batch.restype = I
    lib.st_batch_instance.argtypes = [P, I, ctypes.POINTER(P)]
    lib.st_batch_instance.restype = I
    lib.st_destroy_batch.argtypes = [P]
    lib.st_destroy_batch.restype = None
    lib.st_grad_rhs.argtypes = [P, P, P, P, P]
    lib.st_grad_rhs.restype = I
    lib.st_grad_a.argtypes = [P, P, P, P, P]
    lib.st_grad_a.restype = I
    lib.st_strerror.argtypes = [I]
    lib.st_strerror.restype = ctypes.c_char_p
    lib.st_version.argtypes = []
    lib.st_version.restype = I
    lib.st_profile_begin.argtypes = [P, I]
    lib.st_profile_begin.restype = I
    lib.st_profile_end.argtypes = [P, ctypes.POINTER(StKernelTime), I]
    lib.st_profile_end.restype = I
    lib.st_residual_noalloc.argtypes = [ctypes.POINTER(StProblem), P, P, P, P, P]
    lib.st_residual_noalloc.restype = I
    lib.st_kernel_class_name.argtypes = [I]
    lib.st_kernel_class_name.restype = ctypes.c_char_p
    _lib = lib
    return lib


def strerror(code: int) -> str:
    return load_library().st_strerror(int(code)).decode()


def _check(code: int, where: str, ok=(ST_OK,)):
    if code not in ok:
        raise SolverError(code, where)
    return code


def _dev_ptr(t, dtype=None, numel=None):
    import torch

    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"expected dtype {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"expected {numel} elements, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


@dataclass
class ProblemSpec:
    dim: int
    mx: int
    my: int
    n: int
    T: float = 1.0
    scheme: str = "theta"  # "theta" | "bdf2"
    theta: float = 1.0
    a_nodal: Optional[np.ndarray] = None
    prec: str = "PH"  # "PH" | "Ptheta"
    precision: str = "fp64"  # "fp64" | "mixed"
    inner_degree: int = 0  # Ptheta with a 2D/3D a_nodal: Chebyshev steps (0 = library default)
    mz: int = 1  # dim 3: interior points along z

    @property
    def m(self):
        return self.mx * self.my * (self.mz if self.dim == 3 else 1)

    @property
    def N(self):
        return self.m * self.n

    def to_c(self, stream_ptr=None):
        a = None
        keep = None
        if self.a_nodal is not None:
            keep = np.ascontiguousarray(self.a_nodal, dtype=np.float64)
            a = keep.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        p = StProblem(
            self.dim, self.mx, self.my, self.n, float(self.T),
            ST_THETA if self.scheme == "theta" else ST_BDF2, float(self.theta),
            a, ST_PREC_PH if self.prec == "PH" else ST_PREC_PTHETA,
            ST_FP64 if self.precision == "fp64" else ST_MIXED,
            ctypes.c_void_p(stream_ptr) if stream_ptr else None, int(self.inner_degree),
            int(self.mz if self.dim == 3 else 1),
        )
        return p, keep


def st_workspace_bytes(spec: ProblemSpec) -> int:
    p, keep = spec.to_c()
    out = ctypes.c_size_t(0)
    _check(load_library().st_workspace_bytes(ctypes.byref(p), ctypes.byref(out)), "st_workspace_bytes")
    return int(out.value)


def st_setup(spec: ProblemSpec, stream=None):
    import torch

    lib = load_library()
    if stream is None:
        stream = torch.cuda.current_stream()
    p, keep = spec.to_c(stream.cuda_stream)
    h = ctypes.c_void_p()
    _check(lib.st_setup(ctypes.byref(p), ctypes.byref(h)), "st_setup")
    return h


def st_destroy(h):
    load_library().st_destroy(h)


class Solver:
    """One problem instance on the current CUDA device and stream."""

    def __init__(self, spec: ProblemSpec, stream=None):
        import torch

        self.spec = spec
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.h = st_setup(spec, self.stream)
        self.lib = load_library()

    def close(self):
        if getattr(self, "h", None):
            self.lib.st_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- allocation helpers (torch owns device memory)
    def empty(self, *shape, dtype=None):
        import torch

        return torch.empty(*shape, dtype=dtype or torch.float64, device=self.device)

    def st_assemble_rhs(self, f, u0, uprev=None, extra=None, out=None):
        import torch

        s = self.spec
        out = out if out is not None else self.empty(s.n, s.m)
        up = _dev_ptr(uprev, torch.float64, s.m) if uprev is not None else None
        ex = _dev_ptr(extra, torch.float64, s.N) if extra is not None else None
        _check(self.lib.st_assemble_rhs(self.h, _dev_ptr(f, torch.float64, (s.n + 1) * s.m),
                                        _dev_ptr(u0, torch.float64, s.m), up, ex,
                                        _dev_ptr(out, torch.float64, s.N)), "st_assemble_rhs")
        return out

    def st_apply_op(self, v, out=None):
        import torch

        out = out if out is not None else torch.empty_like(v)
        _check(self.lib.st_apply_op(self.h, _dev_ptr(v, torch.float64, self.spec.N),
                                    _dev_ptr(out, torch.float64, self.spec.N)), "st_apply_op")
        return out

    def st_apply_prec(self, v, out=None):
        import torch

        out = out if out is not None else torch.empty_like(v)
        _check(self.lib.st_apply_prec(self.h, _dev_ptr(v, torch.float64, self.spec.N),
                                      _dev_ptr(out, torch.float64, self.spec.N)), "st_apply_prec")
        return out

    def st_apply_prec_f32(self, v, out=None):
        import torch

        out = out if out is not None else torch.empty(v.shape, dtype=torch.float32, device=v.device)
        _check(self.lib.st_apply_prec_f32(self.h, _dev_ptr(v, torch.float64, self.spec.N),
                                          _dev_ptr(out, torch.float32, self.spec.N)),
               "st_apply_prec_f32")
        return out

    def st_solve(self, fH, tol=1e-8, maxit=500, out=None, allow_not_converged=False):
        import torch

        out = out if out is not None else torch.empty_like(fH)
        st = StStats()
        ok = (ST_OK, ST_ERR_NOT_CONVERGED) if allow_not_converged else (ST_OK,)
        _check(self.lib.st_solve(self.h, _dev_ptr(fH, torch.float64, self.spec.N),
                                 _dev_ptr(out, torch.float64, self.spec.N), float(tol), int(maxit),
                                 ctypes.byref(st)), "st_solve", ok)
        return out, st.as_dict()

    def st_solve_host(self, fH_host: np.ndarray, u_host: np.ndarray, tol=1e-8, maxit=500,
                      allow_not_converged=False):
        """Host buffers (numpy float64 or pinned CPU torch tensors); copies inside the call."""
        def ptr(a):
            if isinstance(a, np.ndarray):
                assert a.dtype == np.float64 and a.flags.c_contiguous and a.size == self.spec.N
                return ctypes.c_void_p(a.ctypes.data)
            assert (not a.is_cuda) and a.is_contiguous() and a.numel() == self.spec.N
            return ctypes.c_void_p(a.data_ptr())
        st = StStats()
        ok = (ST_OK, ST_ERR_NOT_CONVERGED) if allow_not_converged else (ST_OK,)
        _check(self.lib.st_solve_host(self.h, ptr(fH_host), ptr(u_host), float(tol), int(maxit),
                                      ctypes.byref(st)), "st_solve_host", ok)
        return st.as_dict()

    def st_solve_transpose(self, g, tol=1e-8, maxit=500, out=None, allow_not_converged=False):
        import torch

        out = out if out is not None else torch.empty_like(g)
        st = StStats()
        ok = (ST_OK, ST_ERR_NOT_CONVERGED) if allow_not_converged else (ST_OK,)
        _check(self.lib.st_solve_transpose(self.h, _dev_ptr(g, torch.float64, self.spec.N),
                                           _dev_ptr(out, torch.float64, self.spec.N), float(tol),
                                           int(maxit), ctypes.byref(st)), "st_solve_transpose", ok)
        return out, st.as_dict()

    def st_autotune(self, reps=5):
        _check(self.lib.st_autotune(self.h, int(reps)), "st_autotune")

    def st_profile_begin(self, capacity=1 << 16):
        _check(self.lib.st_profile_begin(self.h, int(capacity)), "st_profile_begin")

    def st_profile_end(self):
        """Per kernel class: launches, timed launches and summed CUDA-event milliseconds."""
        arr = (StKernelTime * len(KERNEL_CLASSES))()
        _check(self.lib.st_profile_end(self.h, arr, len(KERNEL_CLASSES)), "st_profile_end")
        return {KERNEL_CLASSES[i]: {"launches": arr[i].launches, "timed": arr[i].timed,
                                    "ms": arr[i].ms} for i in range(len(KERNEL_CLASSES))}

    def st_grad_rhs(self, lam):
        """(dL/df (n+1, m), dL/du0 (m,), dL/du^(-1) (m,)) from lam = dL/df_H."""
        import torch

        s = self.spec
        gf = self.empty(s.n + 1, s.m)
        gu0 = self.empty(s.m)
        gup = self.empty(s.m)
        _check(self.lib.st_grad_rhs(self.h, _dev_ptr(lam, torch.float64, s.N),
                                    _dev_ptr(gf, torch.float64), _dev_ptr(gu0, torch.float64),
                                    _dev_ptr(gup, torch.float64)), "st_grad_rhs")
        return gf, gu0, gup

    def st_grad_a(self, lam, u, u0, out=None):
        import torch

        s = self.spec
        nn = (s.mx + 2) if s.dim == 1 else (s.mx + 2) * (s.my + 2)
        out = out if out is not None else self.empty(nn)
        _check(self.lib.st_grad_a(self.h, _dev_ptr(lam, torch.float64, s.N),
                                  _dev_ptr(u, torch.float64, s.N), _dev_ptr(u0, torch.float64, s.m),
                                  _dev_ptr(out, torch.float64, nn)), "st_grad_a")
        return out


class _InstanceView(Solver):
    """A Solver whose handle belongs to a BatchSolver (not destroyed on close)."""

    def __init__(self, spec, handle, stream, device):
        self.spec = spec
        self.stream = stream
        self.device = device
        self.h = handle
        self.lib = load_library()

    def close(self):
        self.h = None


class BatchSolver:
    """Many independent mixed-precision instances solved by one captured CUDA graph."""

    def __init__(self, specs, stream=None):
        import torch

        self.lib = load_library()
        self.specs = list(specs)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.device = torch.device("cuda", torch.cuda.current_device())
        arr = (StProblem * len(self.specs))()
        self._keep = []
        for i, sp in enumerate(self.specs):
            if sp.precision != "mixed":
                raise ValueError("batched solves run in mixed precision")
            p, keep = sp.to_c()
            arr[i] = p
            self._keep.append(keep)
        self.b = ctypes.c_void_p()
        _check(self.lib.st_setup_batch(arr, len(self.specs), ctypes.c_void_p(self.stream.cuda_stream),
                                       ctypes.byref(self.b)), "st_setup_batch")

    def instance(self, i) -> Solver:
        h = ctypes.c_void_p()
        _check(self.lib.st_batch_instance(self.b, int(i), ctypes.byref(h)), "st_batch_instance")
        return _InstanceView(self.specs[i], h, self.stream, self.device)

    def st_solve_batch(self, fHs, tol=1e-8, maxit=500, outs=None, allow_not_converged=False):
        import torch

        n = len(self.specs)
        outs = outs if outs is not None else [torch.empty_like(f) for f in fHs]
        fp = (ctypes.c_void_p * n)(*[_dev_ptr(f, torch.float64, sp.N).value for f, sp in zip(fHs, self.specs)])
        up = (ctypes.c_void_p * n)(*[_dev_ptr(u, torch.float64, sp.N).value for u, sp in zip(outs, self.specs)])
        stats = (StStats * n)()
        ok = (ST_OK, ST_ERR_NOT_CONVERGED) if allow_not_converged else (ST_OK,)
        _check(self.lib.st_solve_batch(self.b, fp, up, float(tol), int(maxit), stats),
               "st_solve_batch", ok)
        return outs, [stats[i].as_dict() for i in range(n)]

    def close(self):
        if getattr(self, "b", None):
            self.lib.st_destroy_batch(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


__all__ = [
    "ProblemSpec", "Solver", "BatchSolver", "SolverError", "StProblem", "StStats", "load_library", "strerror",
    "st_setup", "st_destroy", "st_workspace_bytes", "EXPORTS", "LIB_PATH",
]
