"""Shared helpers of the GPU tests: seeded problems and the tolerances.

Tolerances (derived from the arithmetic, stated once here):
  a complete 3D FFT (forward + inverse) in precision eps has a relative
  rounding error of about eps * log2(N); term i of the order-2k expansion
  applies i of them and is scaled by |c_i|, so the propagated block carries
  an error of about  eps * log2(N) * sum_i i |c_i|  relative to the largest
  value.  The tests allow 8x that (FP64) and 2x (FP32, where the bound is
  already pessimistic because the terms' errors are independent).
"""
import math

import numpy as np

from itp_workloads import Grid, gaussian_wells_potential, normal_states
from oracle import itp_oracle as O

EPS64 = 2.0 ** -53
EPS32 = 2.0 ** -24


def propagate_tolerance(order: int, n_points: int, precision: str) -> float:
    c = O.mp_coefficients_float(order // 2)
    weight = sum((i + 1) * abs(ci) for i, ci in enumerate(c))
    lg = math.log2(n_points)
    if precision == "fp64":
        return max(8 * EPS64 * lg * weight, 1e-13)
    return 2 * EPS32 * lg * weight + 1e-6


def wells_problem(g: Grid, n_wells: int = 5, seed: int = 3):
    """A non-separable potential: a few Gaussian wells inside the box."""
    rng = np.random.default_rng(seed)
    L = np.array([g.lx, g.ly, g.lz])
    centres = rng.uniform(-0.25, 0.25, (n_wells, 3)) * L
    depths = rng.uniform(0.5, 3.0, n_wells)
    sigmas = rng.uniform(0.5, 1.2, n_wells) * min(L) / 8.0
    return gaussian_wells_potential(g, centres, depths, sigmas)


def seeded_states(g: Grid, m: int, seed: int = 1234):
    return normal_states(m, g.n_points, seed)


def report(name: str, err: float, tol: float) -> None:
    """Print an observed error beside its bound (shown with pytest -s), so
    that every parity check leaves the margin it passed with on record."""
    print(f"[parity] {name}: err={err:.3e} tol={tol:.3e} err/tol={err / tol:.3g}", flush=True)
