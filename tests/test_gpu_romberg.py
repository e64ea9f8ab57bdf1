"""Eq. (sixp), the Romberg-type T_6 comparator (itp_propagate_romberg6),
against the oracle's romberg_t6, element by element."""
import numpy as np
import pytest

from itp_workloads import Grid
from oracle import itp_oracle as O

from gpu_helpers import propagate_tolerance, seeded_states, wells_problem

pytestmark = pytest.mark.gpu

import paper_0809_3739_gb300 as P  # noqa: E402

PREC = {"fp64": P.ITP_FP64, "mixed": P.ITP_MIXED}


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("dims", [(24, 16, 12), (32, 32, 32)])
def test_romberg6_matches_oracle(prec, dims):
    g = Grid(*dims, 9.0, 7.0, 6.0)
    V = wells_problem(g)
    m = 4
    psi = seeded_states(g, m)
    tau = 0.3
    with P.ItpGrid(g.nx, g.ny, g.nz, g.lx, g.ly, g.lz, m, 0, PREC[prec]) as h:
        h.set_potential(V)
        h.set_states(psi)
        h.propagate_romberg6(tau)
        phi = h.get_phi()
        h.orthonormalize()   # the propagated block feeds Eq. (4) as usual
        h.synchronize()
    k2 = O.kinetic_k2(g.shape, (g.lz, g.ly, g.lx))
    ref = np.stack([O.romberg_t6(p.reshape(g.shape), V, tau, k2).ravel() for p in psi])
    err = np.max(np.abs(phi - ref)) / np.max(np.abs(ref))
    # three order-4 applications, two of them chained, combined with 16/15 and 1/15
    tol = 3 * propagate_tolerance(4, g.n_points, prec)
    assert err < tol, (err, tol)
