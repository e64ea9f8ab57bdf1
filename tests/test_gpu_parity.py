"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Small grids: every output element is compared.  The grids are non-cubic,
include factors of 3, and have half-spectrum widths that leave ragged pencil
blocks.  All inputs come from the seeded generators.
"""
import numpy as np
import pytest

from itp_workloads import Grid, cubic, harmonic_potential
from oracle import itp_oracle as O

from gpu_helpers import propagate_tolerance, report, seeded_states, wells_problem

pytestmark = pytest.mark.gpu

import paper_0809_3739_gb300 as P  # noqa: E402  (fails loudly without libitp.so)

GRIDS = [
    Grid(8, 6, 4, 4.0, 3.5, 3.0),
    Grid(24, 16, 12, 9.0, 7.0, 6.0),
    Grid(32, 32, 32, 12.0, 12.0, 12.0),
    Grid(48, 24, 16, 14.0, 10.0, 8.0),
    Grid(96, 32, 32, 20.0, 10.0, 10.0),
]
PREC = {"fp64": P.ITP_FP64, "mixed": P.ITP_MIXED}


def _grid_handle(g, m, prec, V, psi, n_guard=0):
    h = P.ItpGrid(g.nx, g.ny, g.nz, g.lx, g.ly, g.lz, m - n_guard, n_guard, PREC[prec])
    h.set_potential(V)
    h.set_states(psi)
    return h


def _relerr(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("gi", range(len(GRIDS)))
@pytest.mark.parametrize("order", [2, 4, 8, 12])
def test_propagate_matches_oracle(prec, gi, order):
    g = GRIDS[gi]
    V = wells_problem(g)
    m = 5
    psi = seeded_states(g, m)
    tau = 0.3
    with _grid_handle(g, m, prec, V, psi) as h:
        h.propagate(order, tau)
        phi = h.get_phi()
    ref = O.propagate(psi, V, g, order, tau)
    err = _relerr(phi, ref)
    tol = propagate_tolerance(order, g.n_points, prec)
    report(f"{g.nx}x{g.ny}x{g.nz} {prec} propagate order {order}", err, tol)
    assert err < tol, (err, tol)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_orthonormalize_matches_oracle(prec):
    g = GRIDS[2]
    V = wells_problem(g)
    m = 7
    psi = seeded_states(g, m)
    with _grid_handle(g, m, prec, V, psi) as h:
        h.propagate(6, 0.25)
        h.orthonormalize()
        got = h.get_states()
    phi = O.propagate(psi, V, g, 6, 0.25)
    want, _ = O.cholesky_orthonormalize(phi, g.dV)
    tol = 1e-11 if prec == "fp64" else 2e-4
    assert _relerr(got, want) < tol
    ov = got @ got.T * g.dV
    assert np.max(np.abs(ov - np.eye(m))) < (1e-12 if prec == "fp64" else 1e-5)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("ritz", [False, True, "values"])
def test_energies_match_oracle(prec, ritz):
    g = GRIDS[1]
    V = wells_problem(g)
    m = 6
    psi0 = seeded_states(g, m)
    psi, _ = O.cholesky_orthonormalize(psi0, g.dV)
    with _grid_handle(g, m, prec, V, psi) as h:
        E = h.energies(ritz)
        got = h.get_states()
    E_ref, psi_ref, _ = O.energies(psi, V, g, bool(ritz))
    scale = np.max(np.abs(E_ref))
    tol = 1e-12 if prec == "fp64" else 1e-5
    assert np.max(np.abs(E - E_ref)) < tol * scale
    if ritz == "values":
        # Ritz values only: the states are left as they were
        assert np.max(np.abs(got - psi)) < (1e-14 if prec == "fp64" else 1e-6) * np.max(np.abs(psi))
    elif ritz:
        # the rotated states agree up to sign (random states: simple spectrum)
        for j in range(m):
            d = abs(np.dot(got[j], psi_ref[j]) * g.dV)
            assert abs(d - 1.0) < (1e-10 if prec == "fp64" else 1e-4)


def test_ho_spectrum_fp64_path():
    """32^3 HO, [-8,8)^3, n = 10 (+2 guard), order 4, tau = 0.1: the FP64 GPU
    iteration converges to E = 3/2, 5/2 (x3), 7/2 (x6) within 1e-10 Ha."""
    g = cubic(32, 16.0)
    V = harmonic_potential(g)
    psi = seeded_states(g, 12)
    want = np.array([1.5] + [2.5] * 3 + [3.5] * 6)
    with _grid_handle(g, 12, "fp64", V, psi, n_guard=2) as h:
        prev = None
        for it in range(400):
            E = h.step(4, 0.1, ritz="values")
            if prev is not None and np.max(np.abs(E[:10] - prev[:10])) < 1e-12:
                break
            prev = E
        E = h.energies(True)
        psi_out = h.get_states()
    assert np.max(np.abs(E[:10] - want)) < 1e-10, E[:10] - want
    # the Ritz vectors of the ground state and the 2p shell: orthonormal and
    # eigenvectors of H to the same accuracy
    ov = psi_out @ psi_out.T * g.dV
    assert np.max(np.abs(ov - np.eye(12))) < 1e-11


def test_ho_spectrum_mixed_path_with_polish():
    """Same problem, FP32 iterations to their plateau, then FP64 polish: the
    mixed path reaches 1e-8 Ha."""
    g = cubic(32, 16.0)
    V = harmonic_potential(g)
    psi = seeded_states(g, 12)
    want = np.array([1.5] + [2.5] * 3 + [3.5] * 6)
    with _grid_handle(g, 12, "mixed", V, psi, n_guard=2) as h:
        prev = None
        for it in range(300):
            E = h.step(4, 0.1, ritz="values")
            if prev is not None and np.max(np.abs(E[:10] - prev[:10])) < 1e-6:
                break
            prev = E
        steps, E = h.polish(4, 0.1, 1e-11, 60)
    assert np.max(np.abs(E[:10] - want)) < 1e-8, (steps, E[:10] - want)


@pytest.mark.parametrize("ritz", [True, "values"])
def test_itp_sequence_matches_oracle_iterations(ritz):
    """Five full iterations (propagate, Cholesky, Ritz) from identical inputs
    give the oracle's energies, with or without rotating the states each
    step (the Ritz values depend only on the span)."""
    g = GRIDS[1]
    V = wells_problem(g)
    m = 6
    psi = seeded_states(g, m)
    ref = psi.copy()
    with _grid_handle(g, m, "fp64", V, psi) as h:
        for _ in range(5):
            E = h.step(8, 0.4, ritz=ritz)
            ref, E_ref = O.itp_step(ref, V, g, 8, 0.4)
            assert np.max(np.abs(E - E_ref)) < 1e-11 * np.max(np.abs(E_ref))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_graph_step_matches_plain_steps(prec):
    """itp_step replays the same kernels from a CUDA graph: the energies of
    every step equal those of the plain call sequence, also across a change
    of tau (which captures a new graph)."""
    g = GRIDS[2]
    V = wells_problem(g)
    m = 6
    psi = seeded_states(g, m)
    plan = [(8, 0.3)] * 3 + [(8, 0.2)] * 2
    with _grid_handle(g, m, prec, V, psi) as a, _grid_handle(g, m, prec, V, psi) as b:
        for order, tau in plan:
            Ea = a.step(order, tau, ritz="values")
            Eb = b.step_graph(order, tau)
            assert np.max(np.abs(Ea - Eb)) <= 1e-13 * np.max(np.abs(Ea))
        assert _relerr(b.get_states(), a.get_states()) < 1e-12


def test_not_positive_definite_is_reported():
    g = GRIDS[0]
    V = wells_problem(g)
    psi = seeded_states(g, 4)
    psi[2] = 0.0   # a vanished state makes S singular
    with _grid_handle(g, 4, "fp64", V, psi) as h:
        h.propagate(4, 0.2)
        h.orthonormalize()
        with pytest.raises(P.ItpError) as ei:
            h.synchronize()
        assert ei.value.code == 3
        # the handle stays usable
        h.set_states(seeded_states(g, 4))
        h.propagate(4, 0.2)
        h.orthonormalize()
        h.synchronize()


def test_argument_errors():
    g = GRIDS[0]
    with pytest.raises(P.ItpError) as ei:
        P.ItpGrid(10, 8, 8, 1.0, 1.0, 1.0, 2)
    assert ei.value.code == 1
    h = P.ItpGrid(g.nx, g.ny, g.nz, g.lx, g.ly, g.lz, 2)
    with pytest.raises(P.ItpError) as ei:
        h.propagate(4, 0.1)
    assert ei.value.code == 6   # no potential / states yet
    h.set_potential(wells_problem(g))
    h.set_states(seeded_states(g, 2))
    for order, tau in ((3, 0.1), (14, 0.1), (4, 0.0), (4, -1.0)):
        with pytest.raises(P.ItpError) as ei:
            h.propagate(order, tau)
        assert ei.value.code == 1
    with pytest.raises(P.ItpError) as ei:
        h.orthonormalize()
    assert ei.value.code == 6
    h.close()


def test_kernel_launch_count():
    """One order-2k step launches k(k+2) FFT passes (2i+1 per term i; the
    paper's k(k+1)/2 complete FFTs, Sec. II), plus the table set-up once."""
    g = GRIDS[0]
    with _grid_handle(g, 3, "fp64", wells_problem(g), seeded_states(g, 3)) as h:
        h.propagate(8, 0.2)   # builds the tables of (8, 0.2)
        n0 = h.kernel_launches
        h.propagate(8, 0.2)
        k = 4
        assert h.kernel_launches - n0 == k * (k + 2)


def test_mixed_dense_steps_at_full_state_count():
    """m = 128 states (the tensor-core tile height) on a small grid: the
    mixed path's overlap, Cholesky update and Ritz values match the oracle,
    and the states come out orthonormal to FP32 accuracy."""
    g = Grid(32, 32, 32, 14.0, 14.0, 14.0)
    V = wells_problem(g, n_wells=8)
    m = 128
    psi = seeded_states(g, m)
    with _grid_handle(g, m, "mixed", V, psi, n_guard=8) as h:
        h.propagate(4, 0.2)
        phi = h.get_phi()
        h.orthonormalize()
        got = h.get_states()
        E = h.energies("values")
    phi_ref = O.propagate(psi, V, g, 4, 0.2)
    assert _relerr(phi, phi_ref) < propagate_tolerance(4, g.n_points, "mixed")
    ov = got @ got.T * g.dV
    assert np.max(np.abs(ov - np.eye(m))) < 2e-5
    # psi = L^{-1} phi: the first states follow from the leading block alone
    want, _ = O.cholesky_orthonormalize(phi_ref[:4], g.dV)
    assert _relerr(got[:4], want) < 1e-4
    E_ref, _, _ = O.energies(got, V, g, ritz=True)
    assert np.max(np.abs(E - E_ref)) < 1e-5 * np.max(np.abs(E_ref))


def test_fp64_evaluation_of_fp32_states_matches_oracle():
    """ITP_EVAL_FP64 on a mixed handle: the FP32 states, rounded up to FP64,
    orthonormalised again in FP64 and their Ritz values taken in FP64, equal
    the oracle's orthonormalisation and Ritz values of the same FP32 values
    to FP64 accuracy."""
    g = GRIDS[1]
    V = wells_problem(g)
    m = 6
    psi = seeded_states(g, m)
    with _grid_handle(g, m, "mixed", V, psi) as h:
        h.step(6, 0.3, ritz="values")
        psi32 = h.get_states()            # the FP32 states, as FP64 values
        E = h.energies("values", fp64=True)
        got = h.get_states()
        E2 = h.step(6, 0.3, ritz="values")   # FP32 steps continue
    want, _ = O.cholesky_orthonormalize(psi32, g.dV)
    E_ref, _, _ = O.energies(want, V, g, ritz=True)
    assert np.max(np.abs(E - E_ref)) < 1e-12 * np.max(np.abs(E_ref))
    assert _relerr(got, want) < 1e-11   # the states are FP64 after the evaluation
    assert np.all(np.isfinite(E2))
