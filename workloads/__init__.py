"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This package holds no arithmetic of the solver method: it samples analytic
fields (the PDE data f, u0, a and exact solutions) on the grid and draws
seeded random numbers. Both the CUDA path and the CPU oracle receive these
arrays and assemble everything else themselves.
"""
from .synthetic import *  # noqa: F401,F403
