"""Edge cases of the state count: a single state (1 x 1 overlap, Cholesky and
eigenproblem) and the largest block (128 states), against the oracle; and the
degenerate block (a zero state: singular overlap, ITP_ERR_NOT_PD)."""
import numpy as np
import pytest

from itp_workloads import Grid
from oracle import itp_oracle as O

from gpu_helpers import propagate_tolerance, report, seeded_states, wells_problem

pytestmark = pytest.mark.gpu

import paper_0809_3739_gb300 as P  # noqa: E402

PREC = {"fp64": P.ITP_FP64, "mixed": P.ITP_MIXED}


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("m", [1, 128, 129, 200, 256])
def test_state_count_extremes(prec, m):
    """One state; the largest single 128-state block; and m > 128, where the
    n x n work runs in 128-state blocks (129: a one-row second block; 256:
    the largest handle), through propagation, Cholesky orthonormalisation
    and Ritz values."""
    g = Grid(16, 12, 8, 8.0, 7.0, 6.0)
    V = wells_problem(g)
    psi = seeded_states(g, m)
    order, tau = 8, 0.05   # a short step keeps 128 states of 1536 points well conditioned
    with P.ItpGrid(g.nx, g.ny, g.nz, g.lx, g.ly, g.lz, m, 0, PREC[prec]) as h:
        h.set_potential(V)
        h.set_states(psi)
        h.propagate(order, tau)
        phi = h.get_phi()
        h.orthonormalize()
        E = h.energies("values")
        got = h.get_states()
    ref = O.propagate(psi, V, g, order, tau)
    err = np.max(np.abs(phi - ref)) / np.max(np.abs(ref))
    report(f"m={m} {prec} propagate order {order}", err,
           propagate_tolerance(order, g.n_points, prec))
    assert err < propagate_tolerance(order, g.n_points, prec)
    psi_ref, _ = O.cholesky_orthonormalize(ref, g.dV)
    E_ref, _, _ = O.energies(psi_ref, V, g, ritz=True)
    assert np.max(np.abs(E - E_ref)) < (1e-11 if prec == "fp64" else 1e-5) * np.max(np.abs(E_ref))
    S = got @ got.T * g.dV
    assert np.max(np.abs(S - np.eye(m))) < (1e-12 if prec == "fp64" else 2e-5)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_zero_state_reports_not_positive_definite(prec):
    """A state that is zero everywhere makes the overlap matrix singular
    (first pivot exactly 0): the Cholesky kernel records it, the next
    synchronising call returns ITP_ERR_NOT_PD, and the handle then steps
    valid states normally."""
    g = Grid(16, 16, 8, 8.0, 8.0, 6.0)
    V = wells_problem(g)
    psi = seeded_states(g, 3)
    psi[0] = 0.0
    with P.ItpGrid(g.nx, g.ny, g.nz, g.lx, g.ly, g.lz, 3, 0, PREC[prec]) as h:
        h.set_potential(V)
        h.set_states(psi)
        h.propagate(4, 0.2)
        h.orthonormalize()
        with pytest.raises(P.ItpError) as ei:
            h.energies("values")
        assert ei.value.code == P.itp.ITP_ERR_NOT_PD
        h.set_states(seeded_states(g, 3))
        E = h.step_graph(4, 0.2)
        assert np.all(np.isfinite(E))


@pytest.mark.parametrize("which", ["overlap", "update", "subspace"])
def test_expired_wait_reports_timeout_and_handle_recovers(which):
    """The bounded-wait expiry path of the tensor-core kernels, made to run
    without any fault: itp_test_expire_waits makes a launch wait, before it
    issues any copy or MMA, on an mbarrier phase nothing completes, with a
    2 ms limit.  The kernel leaves its output unwritten, frees its tensor
    memory and records the timeout; the next synchronising call returns
    ITP_ERR_TIMEOUT, and the same handle then steps normally and matches the
    oracle."""
    g = Grid(16, 16, 8, 8.0, 8.0, 6.0)
    V = wells_problem(g)
    m = 4
    psi = seeded_states(g, m)
    with P.ItpGrid(g.nx, g.ny, g.nz, g.lx, g.ly, g.lz, m, 0, P.ITP_MIXED) as h:
        h.set_potential(V)
        h.set_states(psi)
        h.propagate(4, 0.2)
        if which == "overlap":        # the first tensor-core launch: the overlap Gram
            h.test_expire_waits(1)
            h.orthonormalize()
        elif which == "update":       # the second: psi = L^{-1} phi
            h.orthonormalize()        # (queued, not synchronised)
            h.synchronize()
            h.set_states(psi)
            h.propagate(4, 0.2)
            h.test_expire_waits(2)
            h.orthonormalize()        # Gram expires, then the update
        else:                         # the subspace matrix of the energies
            h.orthonormalize()
            h.synchronize()
            h.test_expire_waits(1)
        with pytest.raises(P.ItpError) as ei:
            h.energies("values")
        assert ei.value.code == P.itp.ITP_ERR_TIMEOUT
        assert "expired" in P.itp_last_error(h.h)
        # the hook is spent; the handle is usable and correct again
        h.set_states(psi)
        ref = psi.copy()
        for _ in range(2):
            E = h.step_graph(4, 0.2)
            ref, E_ref = O.itp_step(ref, V, g, 4, 0.2)
            assert np.max(np.abs(E - E_ref)) < 1e-5 * np.max(np.abs(E_ref))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("m", [160, 256])
def test_ritz_rotation_beyond_one_block(prec, m):
    """The Ritz rotation (parallel Jacobi; above ~166 states its working
    matrix lives in global memory) and the block-wise update with a full
    (not triangular) matrix: the Ritz values match the oracle, the rotated
    states stay orthonormal and diagonalise the subspace matrix, and graph
    steps continue from them in agreement with the oracle."""
    g = Grid(24, 16, 12, 9.0, 7.0, 6.0)
    V = wells_problem(g)
    psi = seeded_states(g, m, seed=11)
    with P.ItpGrid(g.nx, g.ny, g.nz, g.lx, g.ly, g.lz, m, 0, PREC[prec]) as h:
        h.set_potential(V)
        h.set_states(psi)
        h.propagate(6, 0.1)
        h.orthonormalize()
        start = h.get_states()
        E = h.energies(True)
        rot = h.get_states()
        E_diag = h.energies(False)
        E_next = h.step_graph(6, 0.1)
    E_ref, _, _ = O.energies(start, V, g, ritz=True)
    tolE = (1e-11 if prec == "fp64" else 1e-5) * np.max(np.abs(E_ref))
    assert np.max(np.abs(E - E_ref)) < tolE
    assert np.max(np.abs(E_diag - E)) < tolE
    S = rot @ rot.T * g.dV
    assert np.max(np.abs(S - np.eye(m))) < (1e-11 if prec == "fp64" else 2e-5)
    _, E_ref2 = O.itp_step(rot, V, g, 6, 0.1)
    assert np.max(np.abs(E_next - E_ref2)) < tolE
