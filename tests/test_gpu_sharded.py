"""The arithmetic backend of the sharded step (paper_0809_3739_gb300.sharded
.AbiBackend) on one GPU: the rank's propagation on an ItpGrid of its
states, the replicated orthonormalisation (itp_orthonormalize_noalloc) and
the Ritz step on an ItpGrid of all states, driven by ShardedStep in a single
process, against the oracle's steps (FP64 path).  The exchange itself is
checked on CPU gloo ranks (test_sharded.py)."""
import numpy as np
import pytest

from itp_workloads import Grid, gaussian_wells_potential, normal_states
from oracle import itp_oracle as O

pytestmark = pytest.mark.gpu

import paper_0809_3739_gb300 as P  # noqa: E402,F401
from paper_0809_3739_gb300.sharded import AbiBackend, ShardedStep  # noqa: E402


@pytest.mark.parametrize("ritz", [False, True])
def test_abi_backend_steps_match_oracle(ritz):
    g = Grid(24, 16, 12, 9.0, 7.0, 6.0)
    V = gaussian_wells_potential(g, np.array([[0.5, 0.2, -0.3], [-1.0, 0.4, 0.6]]),
                                 [2.0, 1.5], [0.9, 0.7])
    m = 5
    psi = normal_states(m, g.n_points, seed=909)
    be = AbiBackend((g.nx, g.ny, g.nz), (g.lx, g.ly, g.lz), V, m, m)
    try:
        st = ShardedStep(be, m)
        st.set_states(psi)
        ref = psi
        for _ in range(2):
            E, p = st.step(6, 0.3, ritz=ritz)
            ref, E_ref = O.itp_step(ref, V, g, 6, 0.3, ritz=ritz)
            assert np.max(np.abs(E - E_ref)) < 1e-11 * np.max(np.abs(E_ref))
            if ritz:
                # Ritz vectors are unique up to sign (the eigenvalues here
                # are simple): compare after aligning each state's sign
                sign = np.sign(np.sum(p * ref, axis=1))
                p = p * sign[:, None]
            assert np.max(np.abs(p - ref)) < 1e-10 * np.max(np.abs(ref))
    finally:
        be.close()
