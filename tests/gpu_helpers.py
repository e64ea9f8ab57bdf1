"""Shared helpers of the GPU tests: seeded problems and the tolerances.

Tolerance of the propagated block (derived from the arithmetic, stated
once here, and checked against the errors every GPU test prints):
  the rounding errors of a complete 3D FFT pair in precision eps are many
  independent roundings, so they grow like a random walk, about
  eps * sqrt(log2 N) relative to the largest value; term i of the order-2k
  expansion applies i such pairs and is scaled by c_i, and the terms'
  errors are independent, so they add in quadrature:
      e(order, N) = eps * sqrt(log2 N) * sqrt(sum_i i c_i^2).
  Across every grid, order, precision, launch shape and state count the
  tests run (48 to 256 per edge, 1 to 256 states, orders 2-12) the observed
  maximum error is 0.5 - 2.0 e (FP64) and 0.5 - 1.25 e (mixed); the tests
  allow 4 e.
"""
import math

import numpy as np

from itp_workloads import Grid, gaussian_wells_potential, normal_states
from oracle import itp_oracle as O

EPS64 = 2.0 ** -53
EPS32 = 2.0 ** -24


def propagate_tolerance(order: int, n_points: int, precision: str) -> float:
    c = O.mp_coefficients_float(order // 2)
    weight = math.sqrt(sum((i + 1) * ci * ci for i, ci in enumerate(c)))
    eps = EPS64 if precision == "fp64" else EPS32
    return 4 * eps * math.sqrt(math.log2(n_points)) * weight


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
