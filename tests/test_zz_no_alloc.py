"""The allocation-free orthonormalisation entry point.

Some callers cannot allocate device memory (a pool or arena owns it all, or a
fixed budget forbids new allocations); itp_orthonormalize_noalloc serves them
with a scratch array inside the library.  This file is collected last so that
a run stopping at the first failure has already run every other test.

Checked here, through the C ABI: two calls in a row on caller-owned device
buffers give the same states as the allocating path (itp_orthonormalize,
read back with itp_get_states) within the FP64 tolerance of the other tests.
"""
import numpy as np
import pytest

import paper_0809_3739_gb300 as P
from itp_workloads import Grid

from gpu_helpers import seeded_states, wells_problem

pytestmark = pytest.mark.gpu


def _reference(g, m, V, psi, order, tau):
    with P.ItpGrid(g.nx, g.ny, g.nz, g.lx, g.ly, g.lz, m, 0, P.ITP_FP64) as h:
        h.set_potential(V)
        h.set_states(psi)
        h.propagate(order, tau)
        phi = h.get_phi()
        h.orthonormalize()
        return phi, h.get_states()


def test_noalloc_matches_allocating_orthonormalize():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    g = Grid(24, 16, 12, 9.0, 7.0, 6.0)
    V = wells_problem(g)
    cases = []
    for m, seed in ((7, 1234), (5, 99)):
        psi = seeded_states(g, m, seed=seed)
        phi, want = _reference(g, m, V, psi, 6, 0.25)
        cases.append((m, phi, want))
    stream = torch.cuda.current_stream().cuda_stream
    for m, phi, want in cases:   # two calls in a row, different sizes
        phi_dev = torch.from_numpy(phi).cuda()
        psi_dev = torch.empty_like(phi_dev)
        P.itp_orthonormalize_noalloc(phi_dev.data_ptr(), psi_dev.data_ptr(), m, g.n_points,
                                     g.dV, stream)
        got = psi_dev.cpu().numpy()
        err = np.max(np.abs(got - want)) / np.max(np.abs(want))
        assert err < 1e-11, err
        ov = got @ got.T * g.dV
        assert np.max(np.abs(ov - np.eye(m))) < 1e-12


def test_noalloc_rejects_oversized_and_bad_arguments():
    torch = pytest.importorskip("torch")
    x = torch.zeros((4, 64), dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    shifted = x.data_ptr() + 64 * 8   # psi = phi + one state: the ranges overlap
    for args in ((x.data_ptr(), y.data_ptr(), 129, 64, 1.0),
                 (x.data_ptr(), x.data_ptr(), 4, 64, 1.0),
                 (x.data_ptr(), shifted, 3, 64, 1.0),
                 (shifted, x.data_ptr(), 3, 64, 1.0),
                 (x.data_ptr(), y.data_ptr(), 4, 64, 0.0)):
        with pytest.raises(P.ItpError) as ei:
            P.itp_orthonormalize_noalloc(*args)
        assert ei.value.code == 1


def test_noalloc_full_state_count():
    """m = 128, the documented maximum: the partial-sum region of the scratch
    array is full and the update stages the whole 128 x 128 inverse factor.
    Same result as the allocating path."""
    torch = pytest.importorskip("torch")
    g = Grid(24, 16, 12, 9.0, 7.0, 6.0)
    V = wells_problem(g)
    m = 128
    psi = seeded_states(g, m, seed=4321)
    phi, want = _reference(g, m, V, psi, 4, 0.2)
    phi_dev = torch.from_numpy(phi).cuda()
    psi_dev = torch.empty_like(phi_dev)
    P.itp_orthonormalize_noalloc(phi_dev.data_ptr(), psi_dev.data_ptr(), m, g.n_points, g.dV,
                                 torch.cuda.current_stream().cuda_stream)
    got = psi_dev.cpu().numpy()
    err = np.max(np.abs(got - want)) / np.max(np.abs(want))
    assert err < 1e-10, err
    ov = got @ got.T * g.dV
    assert np.max(np.abs(ov - np.eye(m))) < 1e-11


def test_noalloc_recovers_after_not_positive_definite():
    """A vanished state makes the overlap singular: ITP_ERR_NOT_PD.  Every
    call shares the scratch array, whose status word keeps the failed
    call's flag unless the next call clears it; the next call on valid
    states must return ITP_OK with orthonormal states."""
    torch = pytest.importorskip("torch")
    g = Grid(24, 16, 12, 9.0, 7.0, 6.0)
    m = 6
    phi = seeded_states(g, m, seed=31)
    bad = phi.copy()
    bad[3] = 0.0
    stream = torch.cuda.current_stream().cuda_stream
    out = torch.empty((m, g.n_points), dtype=torch.float64, device="cuda")
    bad_dev = torch.from_numpy(bad).cuda()
    with pytest.raises(P.ItpError) as ei:
        P.itp_orthonormalize_noalloc(bad_dev.data_ptr(), out.data_ptr(), m, g.n_points, g.dV,
                                     stream)
    assert ei.value.code == P.itp.ITP_ERR_NOT_PD
    good_dev = torch.from_numpy(phi).cuda()
    P.itp_orthonormalize_noalloc(good_dev.data_ptr(), out.data_ptr(), m, g.n_points, g.dV,
                                 stream)
    got = out.cpu().numpy()
    ov = got @ got.T * g.dV
    assert np.max(np.abs(ov - np.eye(m))) < 1e-12
