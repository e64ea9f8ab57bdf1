"""Planes too large for one CTA (row + column passes) and the 256^3 workload.

A 256 x 256 FP32 half-spectrum plane (265 KB) or a 192 x 192 FP64 one does
not fit one CTA's shared memory; those grids run the x transform in row
passes over blocks of row pairs and the y transform in column passes.  The
mixed path then accumulates the terms as error-free FP32 pairs.
"""
import numpy as np
import pytest

from itp_workloads import Grid, c60_like_potential, cubic, normal_states
from oracle import itp_oracle as O

from gpu_helpers import propagate_tolerance, report, seeded_states, wells_problem

pytestmark = pytest.mark.gpu

import paper_0809_3739_gb300 as P  # noqa: E402

PREC = {"fp64": P.ITP_FP64, "mixed": P.ITP_MIXED}


def _relerr(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


@pytest.mark.parametrize("dims,prec", [((256, 256, 8), "mixed"), ((256, 256, 8), "fp64"),
                                       ((192, 192, 6), "fp64"), ((128, 256, 4), "fp64")])
def test_split_plane_step_matches_oracle(dims, prec):
    nx, ny, nz = dims
    g = Grid(nx, ny, nz, 20.0, 18.0, 6.0)
    V = wells_problem(g)
    m = 4
    psi = seeded_states(g, m)
    order, tau = 6, 0.25
    with P.ItpGrid(nx, ny, nz, g.lx, g.ly, g.lz, m, 0, PREC[prec]) as h:
        h.set_potential(V)
        h.set_states(psi)
        h.propagate(order, tau)
        phi = h.get_phi()
        h.orthonormalize()
        E = h.energies("values")
        got = h.get_states()
    phi_ref = O.propagate(psi, V, g, order, tau)
    report(f"{nx}x{ny}x{nz} {prec} propagate order {order} (split planes)",
           _relerr(phi, phi_ref), propagate_tolerance(order, g.n_points, prec))
    assert _relerr(phi, phi_ref) < propagate_tolerance(order, g.n_points, prec)
    psi_ref, _ = O.cholesky_orthonormalize(phi_ref, g.dV)
    assert _relerr(got, psi_ref) < (1e-11 if prec == "fp64" else 2e-4)
    E_ref, _, _ = O.energies(psi_ref, V, g, ritz=True)
    assert np.max(np.abs(E - E_ref)) < (1e-11 if prec == "fp64" else 1e-5) * np.max(np.abs(E_ref))


def test_c60_256_cubed_sampled():
    """The 256^3 C60-like workload (box 32 bohr, order 8, mixed), 16 states:
    the first two propagated states element by element against the oracle,
    and the first two orthonormalised states, which depend on phi_1, phi_2
    alone (Eq. 4 with a triangular L^{-1})."""
    g = cubic(256, 32.0)
    V = c60_like_potential(g)
    m = 16
    psi = normal_states(m, g.n_points, seed=1234)
    order, tau = 8, 0.25
    with P.ItpGrid(256, 256, 256, 32.0, 32.0, 32.0, m, 0, P.ITP_MIXED) as h:
        h.set_potential(V)
        h.set_states(psi)
        h.propagate(order, tau)
        phi = h.get_phi()[:2]
        h.orthonormalize()
        got = h.get_states()[:2]
    phi_ref = O.propagate(psi[:2], V, g, order, tau)
    tol = propagate_tolerance(order, g.n_points, "mixed")
    report(f"256^3 mixed propagate order {order} (sampled states)", _relerr(phi, phi_ref), tol)
    assert _relerr(phi, phi_ref) < tol
    psi_ref, _ = O.cholesky_orthonormalize(phi_ref, g.dV)
    # L^{-1} amplifies the error of phi by up to sqrt(cond(S)) of the block
    kappa = np.sqrt(np.linalg.cond(O.overlap(phi_ref, g.dV)))
    assert _relerr(got, psi_ref) < 2 * tol * kappa


def test_mixed_overlap_long_chunks():
    """Orthonormalised FP32 states over 256^3 points: each tensor-core CTA
    sums ~10^5 points of the overlap (Eq. 4's S), and psi^T psi dV must come
    out as the identity to FP32 accuracy, not to the tensor core's
    accumulation error."""
    g = cubic(256, 32.0)
    m = 8
    psi = normal_states(m, g.n_points, seed=99)
    with P.ItpGrid(256, 256, 256, 32.0, 32.0, 32.0, m, 0, P.ITP_MIXED) as h:
        h.set_potential(np.zeros(g.n_points))
        h.set_states(psi)
        h.propagate(2, 1e-3)   # orthonormalisation works on the propagated block
        h.orthonormalize()
        got = h.get_states()
    S = got @ got.T * g.dV
    assert np.max(np.abs(S - np.eye(m))) < 1e-5
