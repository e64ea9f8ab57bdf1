"""Pins of the oracle's reference-eigenvalue solver (oracle/eigensolver.py).

The block eigensolver supplies E_ref, the exact eigenvalues of the grid
Hamiltonian that the imaginary-time iteration converges to, where no closed
form exists (the C60-like well).  It is pinned against values fixed from
outside it: the separable oscillator's grid spectrum (sums of 1D dense
eigenvalues), and a dense eigendecomposition of the Hamiltonian built from
the DFT definition (oracle/dense_reference.py, no FFT), both on a random
Gaussian-well potential and on the C60-like well itself on a small grid.
"""
import numpy as np
import pytest

from itp_workloads import Grid, c60_like_potential, cubic, harmonic_potential
from oracle.dense_reference import dense_hamiltonian, ho_grid_spectrum
from oracle.eigensolver import certify, interpolate_states, lobpcg_lowest

from gpu_helpers import wells_problem


def test_oscillator_grid_spectrum():
    """16^3 oscillator, box 12: the lowest 10 eigenvalues (the 1s, 1p, 1d+2s
    shells) equal the separable grid spectrum."""
    g = cubic(16, 12.0)
    V = harmonic_potential(g).reshape(g.shape)
    th, X, res, it = lobpcg_lowest(V, g, 10, block=16, tol=1e-9)
    want = ho_grid_spectrum(g, 10)
    assert np.max(np.abs(th - want)) < 1e-10, th - want
    assert np.all(res < 1e-9)


def test_wells_against_dense_eigh():
    """A non-separable potential on a 10 x 8 x 6 grid: the lowest 12
    eigenvalues equal those of the dense Hamiltonian (DFT definition)."""
    g = Grid(10, 8, 6, 6.0, 5.0, 4.0)
    V = wells_problem(g).reshape(g.shape)
    want = np.linalg.eigvalsh(dense_hamiltonian(g, V))[:12]
    th, X, res, it = lobpcg_lowest(V, g, 12, block=20, tol=1e-10)
    assert np.max(np.abs(th - want)) < 1e-11, th - want


def test_c60_like_against_dense_eigh():
    """The C60-like well itself on a 12^3 grid in its 32 bohr box (too
    coarse to resolve it, but an exact grid problem): the lowest 24
    eigenvalues, including its degenerate multiplets, equal the dense
    eigendecomposition; certify() recomputes residuals from scratch and its
    Kato-Temple bounds hold."""
    g = cubic(12, 32.0)
    V = c60_like_potential(g).reshape(g.shape)
    want = np.linalg.eigvalsh(dense_hamiltonian(g, V))[:24]
    th, X, res, it = lobpcg_lowest(V, g, 24, block=36, tol=1e-10)
    assert np.max(np.abs(th - want)) < 1e-11, th - want
    th2, r, bound = certify(th, X, V, g)
    assert np.max(np.abs(th2 - th)) < 1e-12
    assert np.all(r < 1e-9)
    assert np.all(np.abs(th2 - want) <= bound + 1e-12)


def test_certify_catches_a_wrong_eigenvalue():
    """certify() reports a large residual when the vectors are not
    eigenvectors (here: a random block)."""
    g = cubic(8, 6.0)
    V = harmonic_potential(g).reshape(g.shape)
    X = np.random.default_rng(0).standard_normal((g.n_points, 4))
    th, r, _ = certify(np.zeros(4), X, V, g)
    assert np.all(r > 1e-2)


def test_interpolated_start_converges_faster():
    """A coarse-grid solution interpolated to a finer grid of the same box is
    a better start than random vectors (fewer iterations, same values)."""
    gc, gf = cubic(12, 12.0), cubic(24, 12.0)
    Vc = harmonic_potential(gc).reshape(gc.shape)
    Vf = harmonic_potential(gf).reshape(gf.shape)
    _, Xc, _, _ = lobpcg_lowest(Vc, gc, 4, block=8, tol=1e-6)
    X0 = np.concatenate([interpolate_states(Xc, gc, gf),
                         np.random.default_rng(1).standard_normal((gf.n_points, 4))], axis=1)
    th1, _, _, it1 = lobpcg_lowest(Vf, gf, 4, block=8, X0=X0, tol=1e-9)
    th2, _, _, it2 = lobpcg_lowest(Vf, gf, 4, block=8, tol=1e-9)
    assert np.max(np.abs(th1 - th2)) < 1e-11
    assert np.max(np.abs(th1 - ho_grid_spectrum(gf, 4))) < 1e-10
    assert it1 < it2
