"""Seeded synthetic workloads shaped like the paper's examples and the bench configurations.

Everything here samples closed-form PDE data for the heat equation
u_t = div(a grad u) + f on the unit interval/square with u = 0 on the boundary
(Sec. 1, eq. heat): nodal diffusion a(x), forcing f at the time levels
t_k = k*tau (k = 0..n), the initial value u0 and, where one exists, the exact
solution. Random numbers come from numpy's PCG64 (``numpy.random.default_rng``)
with an explicit seed. No discretisation, assembly or solver step lives here.

Array layout: a spatial grid vector is indexed [j*mx + i] (x fastest), with
interior nodes x_i = (i+1) h_x, y_j = (j+1) h_y, h = 1/(m_axis+1). Space-time
arrays are [k][j*mx+i]. Nodal a is given on the full (my+2) x (mx+2) grid,
boundary nodes included (1D: shape (mx+2,)).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

__all__ = [
    "Workload",
    "interior_grid",
    "nodal_grid",
    "random_field",
    "random_field_1d",
    "config_1d_sine",
    "config_2d_sine_cn",
    "config_2d_varcoef_bdf2",
    "config_2d_varcoef_theta",
    "config_adjoint",
    "batch_draws",
    "paper_example1",
    "paper_example2",
    "small_case",
]


@dataclass
class Workload:
    """One heat-equation instance: grid, time stepping and sampled data."""

    name: str
    dim: int
    mx: int
    my: int
    n: int
    T: float
    scheme: str  # "theta" or "bdf2"
    theta: float
    a_nodal: Optional[np.ndarray]  # None means a == 1
    f: np.ndarray  # (n+1, m): f(x, t_k) for k = 0..n
    u0: np.ndarray  # (m,)
    u_prev: Optional[np.ndarray] = None  # (m,) u(x, -tau) for BDF2 start-up
    u_exact: Optional[np.ndarray] = None  # (n, m) exact solution at t_1..t_n
    noise: Optional[np.ndarray] = None  # (n, m) added to the all-at-once rhs
    extra: dict = field(default_factory=dict)
    mz: int = 1  # interior points along z (3D); 1 in 1D and 2D

    @property
    def m(self) -> int:
        return self.mx * self.my * self.mz

    @property
    def N(self) -> int:
        return self.m * self.n

    @property
    def tau(self) -> float:
        return self.T / self.n


def interior_grid(mx: int, my: int):
    """Interior node coordinates as 2D arrays [j, i] (1D: my == 1, y unused)."""
    hx = 1.0 / (mx + 1)
    x = hx * np.arange(1, mx + 1)
    if my == 1:
        return x[None, :], np.zeros((1, mx))
    hy = 1.0 / (my + 1)
    y = hy * np.arange(1, my + 1)
    X, Y = np.meshgrid(x, y, indexing="xy")
    return X, Y


def nodal_grid(mx: int, my: int):
    """All node coordinates including the boundary, [j, i] of shape (my+2, mx+2)."""
    x = np.linspace(0.0, 1.0, mx + 2)
    y = np.linspace(0.0, 1.0, my + 2)
    X, Y = np.meshgrid(x, y, indexing="xy")
    return X, Y


class _SineField2D:
    """F(x,y) = sum_{p,q=1..K} c_pq sin(p pi x) sin(q pi y), c_pq ~ U(-1,1), scaled.

    a = 1 + amp * F / Fmax where Fmax = max |F| over the nodal grid it is
    sampled on, so a lies in [1-amp, 1+amp] at every node (the clip to
    [1-amp, 1+amp] is then the identity on the nodes).
    """

    def __init__(self, seed: int, modes: int = 8, amp: float = 0.5):
        rng = np.random.default_rng(seed)
        self.c = rng.uniform(-1.0, 1.0, size=(modes, modes))
        self.p = np.arange(1, modes + 1)
        self.amp = amp
        self.scale = 1.0

    def _raw(self, X, Y, dx=0, dy=0):
        out = np.zeros_like(X, dtype=np.float64)
        for ip, p in enumerate(self.p):
            if dx == 0:
                sx = np.sin(p * math.pi * X)
            else:
                sx = p * math.pi * np.cos(p * math.pi * X)
            for iq, q in enumerate(self.p):
                if dy == 0:
                    sy = np.sin(q * math.pi * Y)
                else:
                    sy = q * math.pi * np.cos(q * math.pi * Y)
                out += self.c[ip, iq] * sx * sy
        return out

    def calibrate(self, mx: int, my: int):
        X, Y = nodal_grid(mx, my)
        self.scale = 1.0 / np.max(np.abs(self._raw(X, Y)))
        return self

    def a(self, X, Y):
        return np.clip(1.0 + self.amp * self.scale * self._raw(X, Y), 1.0 - self.amp, 1.0 + self.amp)

    def grad(self, X, Y):
        s = self.amp * self.scale
        return s * self._raw(X, Y, dx=1), s * self._raw(X, Y, dy=1)


class _SineField1D:
    def __init__(self, seed: int, modes: int = 8, amp: float = 0.5):
        rng = np.random.default_rng(seed)
        self.c = rng.uniform(-1.0, 1.0, size=modes)
        self.p = np.arange(1, modes + 1)
        self.amp = amp
        self.scale = 1.0

    def _raw(self, x, d=0):
        out = np.zeros_like(x, dtype=np.float64)
        for c, p in zip(self.c, self.p):
            out += c * (np.sin(p * math.pi * x) if d == 0 else p * math.pi * np.cos(p * math.pi * x))
        return out

    def calibrate(self, mx: int):
        x = np.linspace(0.0, 1.0, mx + 2)
        self.scale = 1.0 / np.max(np.abs(self._raw(x)))
        return self

    def a(self, x):
        return np.clip(1.0 + self.amp * self.scale * self._raw(x), 1.0 - self.amp, 1.0 + self.amp)

    def grad(self, x):
        return self.amp * self.scale * self._raw(x, d=1)


def random_field(mx: int, my: int, seed: int, modes: int = 8, amp: float = 0.5) -> np.ndarray:
    """Nodal a on the (my+2, mx+2) grid: 1 + amp * (seeded 8x8 sine-mode field)/max."""
    fld = _SineField2D(seed, modes, amp).calibrate(mx, my)
    X, Y = nodal_grid(mx, my)
    return np.ascontiguousarray(fld.a(X, Y))


def random_field_1d(mx: int, seed: int, modes: int = 8, amp: float = 0.5) -> np.ndarray:
    fld = _SineField1D(seed, modes, amp).calibrate(mx)
    x = np.linspace(0.0, 1.0, mx + 2)
    return np.ascontiguousarray(fld.a(x))


def _times(n: int, T: float):
    return (T / n) * np.arange(0, n + 1)


def config_1d_sine(mx: int = 63, n: int = 64, T: float = 1.0, theta: float = 1.0) -> Workload:
    """1D, a = 1, u = sin(pi x) e^t, f = (1 + pi^2) u, u0 = sin(pi x)."""
    X, _ = interior_grid(mx, 1)
    s = np.sin(math.pi * X[0])
    t = _times(n, T)
    f = (1.0 + math.pi ** 2) * np.exp(t)[:, None] * s[None, :]
    u_exact = np.exp(t[1:])[:, None] * s[None, :]
    return Workload("1d_sine", 1, mx, 1, n, T, "theta", theta, None, f, s.copy(), None, u_exact)


def config_2d_sine_cn(mx: int = 255, n: int = 256, T: float = 1.0, theta: float = 0.5,
                      noise_sigma: float = 1e-3, seed: int = 2) -> Workload:
    """2D, a = 1, u = sin(pi x) sin(pi y) e^t, f = (1 + 2 pi^2) u, plus seeded N(0, sigma) rhs noise."""
    my = mx
    X, Y = interior_grid(mx, my)
    s = (np.sin(math.pi * X) * np.sin(math.pi * Y)).reshape(-1)
    t = _times(n, T)
    f = (1.0 + 2.0 * math.pi ** 2) * np.exp(t)[:, None] * s[None, :]
    u_exact = np.exp(t[1:])[:, None] * s[None, :]
    noise = None
    if noise_sigma > 0:
        rng = np.random.default_rng(seed)
        noise = rng.normal(0.0, noise_sigma, size=(n, mx * my))
    return Workload("2d_sine_cn", 2, mx, my, n, T, "theta", theta, None, f, s.copy(), None,
                    u_exact, noise)


def _varcoef_forcing(fld: _SineField2D, X, Y, t):
    """f = u_t - div(a grad u) for u = sin(pi x) sin(pi y) e^t with smooth a."""
    sx, sy = np.sin(math.pi * X), np.sin(math.pi * Y)
    cx, cy = np.cos(math.pi * X), np.cos(math.pi * Y)
    a = fld.a(X, Y)
    ax, ay = fld.grad(X, Y)
    space = (-2.0 * math.pi ** 2 * a * sx * sy + ax * math.pi * cx * sy + ay * math.pi * sx * cy)
    base = (sx * sy).reshape(-1)
    spat = space.reshape(-1)
    et = np.exp(t)
    return et[:, None] * (base[None, :] - spat[None, :]), base


def config_2d_varcoef_bdf2(mx: int = 511, n: int = 128, T: float = 1.0, seed: int = 3) -> Workload:
    """2D variable a (seeded 8x8 sine-mode field), BDF2, u = sin(pi x) sin(pi y) e^t."""
    my = mx
    fld = _SineField2D(seed).calibrate(mx, my)
    Xn, Yn = nodal_grid(mx, my)
    a_nodal = np.ascontiguousarray(fld.a(Xn, Yn))
    X, Y = interior_grid(mx, my)
    t = _times(n, T)
    f, base = _varcoef_forcing(fld, X, Y, t)
    tau = T / n
    u_exact = np.exp(t[1:])[:, None] * base[None, :]
    return Workload("2d_varcoef_bdf2", 2, mx, my, n, T, "bdf2", 1.0, a_nodal, f, base.copy(),
                    math.exp(-tau) * base, u_exact)


def config_2d_varcoef_theta(mx: int, n: int, theta: float, seed: int, T: float = 1.0) -> Workload:
    """2D variable a, theta-method, same manufactured solution as the BDF2 case."""
    my = mx
    fld = _SineField2D(seed).calibrate(mx, my)
    Xn, Yn = nodal_grid(mx, my)
    a_nodal = np.ascontiguousarray(fld.a(Xn, Yn))
    X, Y = interior_grid(mx, my)
    t = _times(n, T)
    f, base = _varcoef_forcing(fld, X, Y, t)
    u_exact = np.exp(t[1:])[:, None] * base[None, :]
    return Workload(f"2d_varcoef_theta_{mx}_{n}", 2, mx, my, n, T, "theta", theta, a_nodal, f,
                    base.copy(), None, u_exact)


def config_adjoint(mx: int = 255, n: int = 256, T: float = 1.0, seed: int = 5):
    """Adjoint workload: true nodal a (seeded field), f and u0 of the sine solution,
    and a standard-normal array the caller scales into observation noise."""
    w = config_2d_sine_cn(mx, n, T, theta=1.0, noise_sigma=0.0)
    w.name = "adjoint"
    w.a_nodal = random_field(mx, mx, seed)
    rng = np.random.default_rng(seed + 1000)
    w.extra["obs_normal"] = rng.standard_normal(size=(n, mx * mx))
    return w


def batch_draws(count: int = 64, seed: int = 4):
    """Seeded instance list: mx+1 in {64,128,256}, n in {32..512}, theta in {1/2, 1}, own a-seed."""
    rng = np.random.default_rng(seed)
    mxs = np.array([63, 127, 255])
    ns = np.array([32, 64, 128, 256, 512])
    thetas = np.array([0.5, 1.0])
    out = []
    for b in range(count):
        out.append(dict(mx=int(rng.choice(mxs)), n=int(rng.choice(ns)),
                        theta=float(rng.choice(thetas)), seed=int(rng.integers(0, 2 ** 31 - 1))))
    return out


def paper_example1(mx: int, n: int, theta: float, a_const: float = 1e-5, T: float = 1.0) -> Workload:
    """Example 1 shape: a = 1e-5, u0 = x(x-1)y(y-1), f = 0 (Sec. 5, Example 1)."""
    my = mx
    X, Y = interior_grid(mx, my)
    u0 = (X * (X - 1) * Y * (Y - 1)).reshape(-1)
    a_nodal = np.full((my + 2, mx + 2), a_const)
    f = np.zeros((n + 1, mx * my))
    return Workload("paper_ex1", 2, mx, my, n, T, "theta", theta, a_nodal, f, u0)


def paper_example2(mx: int, n: int, theta: float, T: float = 1.0) -> Workload:
    """Example 2 shape: a = 1e-5 sin(pi x y), u = e^{-t} x(1-x) y(1-y) (Sec. 5, Example 2).

    The forcing is f = u_t - div(a grad u) evaluated from the closed forms.
    """
    my = mx
    eps = 1e-5
    Xn, Yn = nodal_grid(mx, my)
    a_nodal = eps * np.sin(math.pi * Xn * Yn)
    X, Y = interior_grid(mx, my)
    P = X * (1 - X)
    Q = Y * (1 - Y)
    a = eps * np.sin(math.pi * X * Y)
    ax = eps * math.pi * Y * np.cos(math.pi * X * Y)
    ay = eps * math.pi * X * np.cos(math.pi * X * Y)
    # u = e^{-t} P Q: u_x = (1-2x) Q, u_xx = -2 Q (times e^{-t}), likewise in y.
    div = a * (-2.0 * Q - 2.0 * P) + ax * (1 - 2 * X) * Q + ay * (1 - 2 * Y) * P
    base = (P * Q).reshape(-1)
    t = _times(n, T)
    f = np.exp(-t)[:, None] * (-base[None, :] - div.reshape(-1)[None, :])
    u_exact = np.exp(-t[1:])[:, None] * base[None, :]
    return Workload("paper_ex2", 2, mx, my, n, T, "theta", theta, a_nodal, f, base.copy(), None,
                    u_exact)


def small_case(dim: int, mx: int, my: int, n: int, scheme: str = "theta", theta: float = 1.0,
               varcoef: bool = False, seed: int = 7, T: float = 1.0, mz: int = 1) -> Workload:
    """Small random instance for parity tests: seeded f, u0 (and a if varcoef).  dim = 3 takes
    mz interior points along z."""
    rng = np.random.default_rng(seed)
    mz = mz if dim == 3 else 1
    m = mx * my * mz
    f = rng.standard_normal((n + 1, m))
    u0 = rng.standard_normal(m)
    u_prev = rng.standard_normal(m) if scheme == "bdf2" else None
    a = None
    if varcoef:
        if dim == 3:
            a = random_field_3d(mx, my, mz, seed + 1)
        else:
            a = random_field(mx, my, seed + 1) if dim == 2 else random_field_1d(mx, seed + 1)
    name = f"small_{dim}d_{mx}x{my}" + (f"x{mz}" if dim == 3 else "") + f"x{n}_{scheme}"
    return Workload(name, dim, mx, my, n, T, scheme, theta, a, f, u0, u_prev, mz=mz)


def random_field_3d(mx: int, my: int, mz: int, seed: int, modes: int = 4,
                    amp: float = 0.5) -> np.ndarray:
    """Nodal a on the (mz+2, my+2, mx+2) grid (boundary nodes included): 1 + amp F / max|F| with
    F = sum_{p,q,r <= modes} c_pqr sin(p pi x) sin(q pi y) sin(r pi z), c_pqr ~ U(-1, 1)."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(-1.0, 1.0, (modes, modes, modes))
    x = np.linspace(0.0, 1.0, mx + 2)
    y = np.linspace(0.0, 1.0, my + 2)
    z = np.linspace(0.0, 1.0, mz + 2)
    k = np.arange(1, modes + 1)
    sx = np.sin(math.pi * k[:, None] * x[None, :])  # (modes, mx+2)
    sy = np.sin(math.pi * k[:, None] * y[None, :])
    sz = np.sin(math.pi * k[:, None] * z[None, :])
    F = np.einsum("pqr,rk,qj,pi->kji", c, sz, sy, sx)
    fmax = np.abs(F).max()
    return np.ascontiguousarray(1.0 + amp * F / fmax if fmax > 0 else np.ones_like(F))


def interior_grid_3d(mx: int, my: int, mz: int):
    """Interior node coordinates as 3D arrays [k, j, i] (x fastest)."""
    x = np.arange(1, mx + 1) / (mx + 1)
    y = np.arange(1, my + 1) / (my + 1)
    z = np.arange(1, mz + 1) / (mz + 1)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return X, Y, Z


def paper_example3(mx: int, n: int, theta: float, a_const: float = 1e-3, T: float = 1.0) -> Workload:
    """Example 3 shape: the unit cube, a = 1e-3, u0 = x(x-1)y(y-1)z(z-1), f = 0 (Sec. 5,
    Example 3)."""
    X, Y, Z = interior_grid_3d(mx, mx, mx)
    u0 = (X * (X - 1) * Y * (Y - 1) * Z * (Z - 1)).reshape(-1)
    a_nodal = np.full((mx + 2, mx + 2, mx + 2), a_const)
    f = np.zeros((n + 1, mx ** 3))
    return Workload("paper_ex3", 3, mx, mx, n, T, "theta", theta, a_nodal, f, u0, mz=mx)


def config_3d_sine(mx: int = 63, n: int = 64, T: float = 1.0, theta: float = 0.5) -> Workload:
    """3D, a = 1, u = sin(pi x) sin(pi y) sin(pi z) e^t, f = (1 + 3 pi^2) u."""
    X, Y, Z = interior_grid_3d(mx, mx, mx)
    base = (np.sin(math.pi * X) * np.sin(math.pi * Y) * np.sin(math.pi * Z)).reshape(-1)
    t = _times(n, T)
    f = (1.0 + 3.0 * math.pi ** 2) * np.exp(t)[:, None] * base[None, :]
    u_exact = np.exp(t[1:])[:, None] * base[None, :]
    return Workload(f"3d_sine_{mx}_{n}", 3, mx, mx, n, T, "theta", theta, None, f, base.copy(),
                    None, u_exact, mz=mx)
