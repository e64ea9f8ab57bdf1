"""Dense-matrix statements of the grid Hamiltonian, for pinning the oracle.

TEST INFRASTRUCTURE ONLY (see oracle/itp_oracle.py).  Nothing here uses an
FFT: the discrete Fourier transform is the explicit matrix
F[k, n] = exp(-2 pi i k n / N) written from its definition, so these
routines check the oracle's use of numpy.fft (axes, wave-number order,
Nyquist handling, normalisation) from outside.

The spectral grid Hamiltonian is H = F^-1 diag(|k|^2 / 2) F + diag(V)
(Eq. 2 with hbar = m = 1).  Its kinetic part is a Kronecker sum of 1D
matrices, so on a separable potential the exact grid spectrum is the sum of
1D spectra, and e^{-tau T} is the Kronecker product of 1D propagators.
"""
from __future__ import annotations

import numpy as np

__all__ = ["dft_matrix", "wave_numbers", "kinetic_1d", "kinetic_propagator_1d",
           "dense_hamiltonian", "dense_t2", "ho_grid_spectrum"]


def dft_matrix(n: int) -> np.ndarray:
    """F[k, m] = exp(-2 pi i k m / n) (unnormalised forward DFT)."""
    k = np.arange(n)
    return np.exp(-2j * np.pi * np.outer(k, k) / n)


def wave_numbers(n: int, length: float) -> np.ndarray:
    """k_m = 2 pi m / L for m = 0..n/2, then 2 pi (m - n) / L."""
    m = np.arange(n)
    m = np.where(m <= n // 2, m, m - n)
    return 2.0 * np.pi * m / length


def _spectral_1d(n: int, length: float, diag: np.ndarray) -> np.ndarray:
    F = dft_matrix(n)
    M = np.conj(F).T @ (diag[:, None] * F) / n
    assert np.max(np.abs(M.imag)) < 1e-10 * max(1.0, np.max(np.abs(M.real)))
    return M.real


def kinetic_1d(n: int, length: float) -> np.ndarray:
    """Dense 1D kinetic matrix F^-1 diag(k^2/2) F."""
    return _spectral_1d(n, length, 0.5 * wave_numbers(n, length) ** 2)


def kinetic_propagator_1d(n: int, length: float, tau: float) -> np.ndarray:
    """Dense 1D e^{-tau T} = F^-1 diag(exp(-tau k^2/2)) F."""
    return _spectral_1d(n, length, np.exp(-0.5 * tau * wave_numbers(n, length) ** 2))


def dense_hamiltonian(grid, V: np.ndarray) -> np.ndarray:
    """Full N x N H for a grid with x fastest (index = (z*ny + y)*nx + x)."""
    Tx = kinetic_1d(grid.nx, grid.lx)
    Ty = kinetic_1d(grid.ny, grid.ly)
    Tz = kinetic_1d(grid.nz, grid.lz)
    Ix, Iy, Iz = np.eye(grid.nx), np.eye(grid.ny), np.eye(grid.nz)
    H = (np.kron(Tz, np.kron(Iy, Ix)) + np.kron(Iz, np.kron(Ty, Ix))
         + np.kron(Iz, np.kron(Iy, Tx)))
    H[np.diag_indices_from(H)] += V.ravel()
    return H


def dense_t2(grid, V: np.ndarray, tau: float) -> np.ndarray:
    """Dense T_2(tau) = diag(e^{-tau V/2}) (Pz (x) Py (x) Px) diag(e^{-tau V/2})."""
    P = np.kron(kinetic_propagator_1d(grid.nz, grid.lz, tau),
                np.kron(kinetic_propagator_1d(grid.ny, grid.ly, tau),
                        kinetic_propagator_1d(grid.nx, grid.lx, tau)))
    h = np.exp(-0.5 * tau * V.ravel())
    return h[:, None] * P * h[None, :]


def ho_grid_spectrum(grid, n_lowest: int, omega: float = 1.0) -> np.ndarray:
    """Exact lowest eigenvalues of the spectral grid Hamiltonian for
    V = omega^2 r^2 / 2: sums of the three 1D dense spectra (separable)."""
    axes = []
    for n, L in ((grid.nx, grid.lx), (grid.ny, grid.ly), (grid.nz, grid.lz)):
        x = -0.5 * L + (L / n) * np.arange(n)
        h1 = kinetic_1d(n, L) + np.diag(0.5 * omega ** 2 * x ** 2)
        axes.append(np.linalg.eigvalsh(h1)[: n_lowest + 2])
    tot = (axes[0][:, None, None] + axes[1][None, :, None]
           + axes[2][None, None, :]).ravel()
    return np.sort(tot)[:n_lowest]
