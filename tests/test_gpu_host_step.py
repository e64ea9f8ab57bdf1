"""itp_step_host: one step between host buffers with the copies overlapped
with the device work.

It runs the kernels of itp_set_states + itp_step + itp_get_states on the
same values, only chunked over states (the propagation of a state needs no
other state), so its states and energies must equal theirs bit for bit; the
step itself is anchored to the oracle once.  Ragged chunks (m not a
multiple of 4, m < 4), in-place buffers, page-locked buffers, the planar
grids and the split plane passes are covered.
"""
import numpy as np
import pytest

from itp_workloads import Grid, planar
from oracle import itp_oracle as O

from gpu_helpers import propagate_tolerance, seeded_states, wells_problem

pytestmark = pytest.mark.gpu

import paper_0809_3739_gb300 as P  # noqa: E402

PREC = {"fp64": P.ITP_FP64, "mixed": P.ITP_MIXED}


def _pair(g, m, prec):
    mk = lambda: P.ItpGrid(g.nx, g.ny, g.nz, g.lx, g.ly, g.lz, m, 0, PREC[prec])  # noqa: E731
    return mk(), mk()


def _graph_step(h, psi, order, tau, ritz="values"):
    h.set_states(psi)
    E = h.step_graph(order, tau, ritz)
    return h.get_states(), E


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("m", [7, 3, 1])
def test_equals_set_step_get(prec, m):
    g = Grid(32, 24, 16, 10.0, 9.0, 7.0)
    V = wells_problem(g)
    psi = seeded_states(g, m)
    order, tau = 8, 0.2
    a, b = _pair(g, m, prec)
    with a, b:
        for h in (a, b):
            h.set_potential(V)
        want, E_want = _graph_step(a, psi, order, tau)
        got, E_got = b.step_host(order, tau, psi)
        assert np.array_equal(got, want)
        assert np.array_equal(E_got, E_want)
        # a second step continues from the returned states
        want2, E_want2 = _graph_step(a, want, order, tau)
        got2, E_got2 = b.step_host(order, tau, got)
        assert np.array_equal(got2, want2)
        assert np.array_equal(E_got2, E_want2)
    # the step itself, against the oracle
    ref = O.propagate(psi, V, g, order, tau)
    psi_ref, _ = O.cholesky_orthonormalize(ref, g.dV)
    E_ref, _, _ = O.energies(psi_ref, V, g, ritz=True)
    assert np.max(np.abs(E_got - E_ref)) < (1e-11 if prec == "fp64" else 1e-5) * np.max(np.abs(E_ref))
    S = got @ got.T * g.dV
    assert np.max(np.abs(S - np.eye(m))) < (1e-12 if prec == "fp64" else 2e-5)


def test_in_place_page_locked_buffers():
    """psi_out may be psi_in; page-locked (torch pinned) buffers passed as
    raw addresses, as a caller that owns its host memory would."""
    torch = pytest.importorskip("torch")
    g = Grid(48, 32, 24, 12.0, 10.0, 8.0)
    V = wells_problem(g)
    m = 10
    psi = seeded_states(g, m)
    a, b = _pair(g, m, "mixed")
    with a, b:
        for h in (a, b):
            h.set_potential(V)
        buf = torch.from_numpy(psi.copy()).pin_memory()
        E = np.empty(m)
        want = psi
        for _ in range(3):
            want, E_want = _graph_step(a, want, 12, 0.25)
            P.itp_step_host(b.h, m, g.n_points, 12, 0.25, buf.data_ptr(), buf.data_ptr(),
                            P.ITP_RITZ_VALUES, E)
            assert np.array_equal(buf.numpy(), want)
            assert np.array_equal(E, E_want)


@pytest.mark.parametrize("case", ["planar", "split_planes", "diag_energies"])
def test_other_paths(case):
    if case == "planar":
        g, prec, ritz = planar(64, 48, 16.0, 12.0), "mixed", "values"
    elif case == "split_planes":   # 256 x 256 FP32 planes: row + column passes
        g, prec, ritz = Grid(256, 256, 4, 20.0, 18.0, 6.0), "mixed", "values"
    else:
        g, prec, ritz = Grid(24, 24, 24, 9.0, 9.0, 9.0), "fp64", False
    V = wells_problem(g)
    m = 5
    psi = seeded_states(g, m)
    a, b = _pair(g, m, prec)
    with a, b:
        for h in (a, b):
            h.set_potential(V)
        want, E_want = _graph_step(a, psi, 6, 0.3, ritz)
        got, E_got = b.step_host(6, 0.3, psi, ritz=ritz)
        assert np.array_equal(got, want)
        assert np.array_equal(E_got, E_want)
    ref = O.propagate(psi, V, g, 6, 0.3)
    psi_ref, _ = O.cholesky_orthonormalize(ref, g.dV)
    tol = 1e-11 if prec == "fp64" else 2e-4
    assert np.max(np.abs(got - psi_ref)) / np.max(np.abs(psi_ref)) < max(
        tol, 4 * propagate_tolerance(6, g.n_points, prec))


def test_arguments_rejected():
    g = Grid(16, 16, 16, 8.0, 8.0, 8.0)
    with P.ItpGrid(16, 16, 16, 8.0, 8.0, 8.0, 2, 0, P.ITP_MIXED) as h:
        psi = seeded_states(g, 2)
        with pytest.raises(P.ItpError) as ei:   # no potential yet
            h.step_host(4, 0.2, psi)
        assert ei.value.code == P.itp.ITP_ERR_STATE
        h.set_potential(np.zeros((16, 16, 16)))
        out = np.empty_like(psi)
        for order, tau, flags in ((5, 0.2, 0), (4, 0.0, 0), (4, 0.2, P.ITP_RITZ)):
            with pytest.raises(P.ItpError) as ei:
                P.itp_step_host(h.h, 2, g.n_points, order, tau, psi, out, flags)
            assert ei.value.code == P.itp.ITP_ERR_ARG
        with pytest.raises(P.ItpError) as ei:
            P.itp_step_host(h.h, 2, g.n_points, 4, 0.2, 0, out)
        assert ei.value.code == P.itp.ITP_ERR_ARG
        with pytest.raises(ValueError):
            h.step_host(4, 0.2, psi[:1])
        # the handle still works
        got, E = h.step_host(4, 0.2, psi)
        assert np.all(np.isfinite(E))
