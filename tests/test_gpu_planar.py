"""The planar case (nz = 1): 2D grids through the same C ABI, against the
oracle (which treats them as 3D grids with one z plane)."""
import numpy as np
import pytest

from itp_workloads import Grid, harmonic_potential_2d, normal_states, planar, quantum_dot_array
from oracle import itp_oracle as O

from gpu_helpers import propagate_tolerance

pytestmark = pytest.mark.gpu

import paper_0809_3739_gb300 as P  # noqa: E402

PREC = {"fp64": P.ITP_FP64, "mixed": P.ITP_MIXED}


def _relerr(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("dims,order", [((64, 48), 8), ((96, 96), 12), ((256, 256), 6)])
def test_planar_propagate_and_step_match_oracle(prec, dims, order):
    nx, ny = dims
    g = planar(nx, ny, 0.25 * nx, 0.25 * ny)
    V = quantum_dot_array(g, n_side=3, spacing=0.06 * nx)
    m = 5
    psi = normal_states(m, g.n_points, seed=31)
    tau = 0.3
    with P.ItpGrid(nx, ny, 1, g.lx, g.ly, g.lz, m, 0, PREC[prec]) as h:
        h.set_potential(V)
        h.set_states(psi)
        h.propagate(order, tau)
        phi = h.get_phi()
        h.orthonormalize()
        E = h.energies("values")
    ref = O.propagate(psi, V, g, order, tau)
    assert _relerr(phi, ref) < propagate_tolerance(order, g.n_points, prec)
    psi_ref, _ = O.cholesky_orthonormalize(ref, g.dV)
    E_ref, _, _ = O.energies(psi_ref, V, g, ritz=True)
    assert np.max(np.abs(E - E_ref)) < (1e-11 if prec == "fp64" else 1e-5) * np.max(np.abs(E_ref))


def test_planar_oscillator_spectrum_on_gpu():
    """FP64 steps on the 2D oscillator converge to 1, 2, 2, 3, 3, 3."""
    g = planar(32, 32, 16.0, 16.0)
    V = harmonic_potential_2d(g)
    psi = normal_states(8, g.n_points, seed=21)
    with P.ItpGrid(32, 32, 1, 16.0, 16.0, 1.0, 6, 2, P.ITP_FP64) as h:
        h.set_potential(V)
        h.set_states(psi)
        for _ in range(120):
            E = h.step_graph(8, 0.4)
    assert np.max(np.abs(E[:6] - np.array([1, 2, 2, 3, 3, 3]))) < 1e-9
