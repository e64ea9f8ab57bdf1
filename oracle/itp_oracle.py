"""FP64 CPU oracle of the multi-product imaginary-time propagation method.

TEST INFRASTRUCTURE ONLY.  This module is the plain, slow, obviously correct
statement of what the GPU library computes.  Only the tests, the smoke check
and the CPU-baseline leg of the benchmark may import it; the library itself
never does, and this module imports nothing from the library.

Everything is float64 numpy.  The FFT (numpy.fft) and the dense linear
algebra (numpy.linalg) are library primitives used as single steps; nothing
is blocked, fused or reordered beyond the paper's own statement.

Notation (Chin, Janecek, Krotscheck, "Any order imaginary time propagation
method for solving the Schroedinger equation"):
  * H = T + V, T = -(1/2) nabla^2 in Hartree units (hbar = m = 1)  [Eq. 2];
  * tau = Delta t > 0 is the imaginary time step; the paper's eps = -tau
    [Eq. 3], so T_2 applies exp(-tau V/2) exp(-tau T) exp(-tau V/2)  [Eq. so];
  * the order-2k multi-product propagator is
    T_2k(tau) = sum_{i=1..k} c_i T_2(tau/i)^i with
    c_i = prod_{j != i} i^2 / (i^2 - j^2)                  [Eqs. mcomp, coef];
  * one iteration: phi_j = T_2k(tau) psi_j for every state      [Eq. 3],
    then orthonormalise the phi_j                                [Eq. 4].

Grid conventions (the paper is silent): periodic box [-L/2, L/2) per axis,
x_i = -L/2 + i h, h = L/N; wave numbers k = (2 pi / L) * {0..N/2, -N/2+1..-1}
(the Nyquist mode uses |k| = pi/h); forward FFT unnormalised, inverse scaled
by 1/N; states normalised as sum psi^2 dV = 1.  States are stored as rows of
an (n, N) array, a state reshaped to (nz, ny, nx) with x fastest.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

__all__ = [
    "mp_coefficients", "mp_coefficients_float", "kinetic_k2", "t2", "t2_power",
    "t2k", "romberg_t6", "overlap", "cholesky_orthonormalize", "apply_h",
    "subspace_matrix", "energies", "itp_step", "solve", "residual_h", "residual_e",
    "solve_adaptive", "propagator_eigenvalue", "fft_count",
]


# ---------------------------------------------------------------------------
# Eq. (coef): closed-form multi-product coefficients with k_i = i.
def mp_coefficients(k: int) -> list[Fraction]:
    """Exact c_1..c_k of the order-2k expansion, c_i = prod_{j!=i} i^2/(i^2-j^2)."""
    if k < 1:
        raise ValueError("k >= 1")
    out = []
    for i in range(1, k + 1):
        c = Fraction(1)
        for j in range(1, k + 1):
            if j != i:
                c *= Fraction(i * i, i * i - j * j)
        out.append(c)
    return out


def mp_coefficients_float(k: int) -> np.ndarray:
    return np.array([float(c) for c in mp_coefficients(k)], dtype=np.float64)


def fft_count(k: int) -> int:
    """Complete FFTs per order-2k step: one per T_2 factor, sum_i i = k(k+1)/2
    (Sec. II, after Eq. ten)."""
    return k * (k + 1) // 2


# ---------------------------------------------------------------------------
# Kinetic energy on the half spectrum produced by rfftn over (z, y, x).
def kinetic_k2(shape, box) -> np.ndarray:
    """|k|^2 on the (nz, ny, nx//2+1) half spectrum; shape = (nz, ny, nx),
    box = (lz, ly, lx)."""
    nz, ny, nx = shape
    lz, ly, lx = box
    kz = 2.0 * np.pi * np.fft.fftfreq(nz, d=lz / nz)
    ky = 2.0 * np.pi * np.fft.fftfreq(ny, d=ly / ny)
    kx = 2.0 * np.pi * np.fft.rfftfreq(nx, d=lx / nx)
    return kz[:, None, None] ** 2 + ky[None, :, None] ** 2 + kx[None, None, :] ** 2


def _box(grid):
    return (grid.lz, grid.ly, grid.lx)


# ---------------------------------------------------------------------------
# Eq. (so): second-order split operator on one state, tau > 0.
def t2(psi: np.ndarray, V: np.ndarray, tau: float, k2: np.ndarray) -> np.ndarray:
    """T_2(tau) psi = e^{-tau V/2} F^-1[ e^{-tau |k|^2/2} F[ e^{-tau V/2} psi ] ].

    psi and V have shape (nz, ny, nx); k2 is kinetic_k2 of that grid.
    """
    half = np.exp(-0.5 * tau * V)
    u = half * psi
    spec = np.fft.rfftn(u, axes=(0, 1, 2))
    spec *= np.exp(-0.5 * tau * k2)
    u = np.fft.irfftn(spec, s=psi.shape, axes=(0, 1, 2))
    return half * u


def t2_power(psi, V, tau, k2, p: int):
    """T_2(tau)^p psi: p successive applications."""
    u = psi
    for _ in range(p):
        u = t2(u, V, tau, k2)
    return u


# Eqs. (mcomp), (coef), with the signed sum of Sec. II (negative c_i subtract).
def t2k(psi, V, tau, k2, k: int):
    """T_2k(tau) psi = sum_{i=1..k} c_i T_2(tau/i)^i psi."""
    c = mp_coefficients_float(k)
    acc = np.zeros_like(psi)
    for i in range(1, k + 1):
        acc += c[i - 1] * t2_power(psi, V, tau / i, k2, i)
    return acc


def romberg_t6(psi, V, tau, k2):
    """Eq. (sixp): -1/15 T_4(tau) + 16/15 T_4(tau/2)^2, with T_4 the order-4
    multi-product expansion.  This cancels the tau^5 term of T_4 only: T_4 is
    a sum of products, not time-symmetric, so a tau^6 local error remains."""
    a = t2k(psi, V, tau, k2, 2)
    b = t2k(t2k(psi, V, 0.5 * tau, k2, 2), V, 0.5 * tau, k2, 2)
    return -a / 15.0 + 16.0 * b / 15.0


# ---------------------------------------------------------------------------
# Eq. (4): orthonormalisation of the propagated states.
def overlap(Phi: np.ndarray, dV: float) -> np.ndarray:
    """S_ij = (phi_i | phi_j) = sum_r phi_i(r) phi_j(r) dV; Phi is (n, N)."""
    return (Phi @ Phi.T) * dV


def cholesky_orthonormalize(Phi: np.ndarray, dV: float):
    """psi = L^{-1} phi with S = L L^T: the c_ji of Eq. (4) form L^{-1}, a
    lower-triangular matrix, so psi_j lies in span(phi_1..phi_j).

    Returns (Psi, L).  Raises numpy.linalg.LinAlgError if S is not positive
    definite.
    """
    S = overlap(Phi, dV)
    L = np.linalg.cholesky(S)
    Psi = np.linalg.solve(L, Phi)
    return Psi, L


# ---------------------------------------------------------------------------
# Eq. (2): H psi and the subspace (Rayleigh-Ritz) matrix.
def apply_h(psi, V, k2):
    """H psi = F^-1[ |k|^2/2 F psi ] + V psi for one (nz, ny, nx) state."""
    spec = np.fft.rfftn(psi, axes=(0, 1, 2))
    spec *= 0.5 * k2
    return np.fft.irfftn(spec, s=psi.shape, axes=(0, 1, 2)) + V * psi


def subspace_matrix(Psi, V, grid):
    """H_sub = (psi_i | H | psi_j) dV for the rows of Psi (n, N); symmetrised."""
    k2 = kinetic_k2(grid.shape, _box(grid))
    HPsi = np.stack([apply_h(p.reshape(grid.shape), V, k2).ravel() for p in Psi])
    Hs = (Psi @ HPsi.T) * grid.dV
    return 0.5 * (Hs + Hs.T), HPsi


def energies(Psi, V, grid, ritz: bool = True):
    """Energies of orthonormal states.

    ritz=True: eigenvalues of the subspace matrix (ascending) and the rotated
    states Psi <- U^T Psi (the subspace step of Sec. III); ritz=False: the
    expectation values (psi_j|H|psi_j) dV with the states unchanged.
    Returns (E, Psi_out, HPsi) where HPsi belongs to the returned Psi.
    """
    Hs, HPsi = subspace_matrix(Psi, V, grid)
    if not ritz:
        return np.diag(Hs).copy(), Psi, HPsi
    E, U = np.linalg.eigh(Hs)
    return E, U.T @ Psi, U.T @ HPsi


def residual_h(Psi, HPsi, E, dV):
    """R^H_j = sum_r |H psi_j - E_j psi_j|^2 dV (Sec. III, with E_j for E_i)."""
    return ((HPsi - E[:, None] * Psi) ** 2).sum(axis=1) * dV


def residual_e(Phi, Psi, E, tau, dV):
    """R^E_j = sum_r |phi_j - exp(-tau E_j) psi_j|^2 dV with phi_j = T_2k(tau)
    psi_j: the variance of psi_j with respect to the evolution operator
    (Sec. III; the paper's exp(eps E) with eps = -tau, E_j for E_i, and the
    volume element so that the value does not depend on the grid)."""
    return ((Phi - np.exp(-tau * np.asarray(E))[:, None] * Psi) ** 2).sum(axis=1) * dV


# ---------------------------------------------------------------------------
def propagate(Psi, V, grid, order: int, tau: float):
    """Phi = T_2k(tau) Psi for every row of Psi (Eq. 3), k = order/2."""
    if order < 2 or order % 2:
        raise ValueError("order must be even and >= 2")
    k2 = kinetic_k2(grid.shape, _box(grid))
    out = np.empty_like(Psi)
    for j in range(Psi.shape[0]):
        out[j] = t2k(Psi[j].reshape(grid.shape), V, tau, k2, order // 2).ravel()
    return out


def itp_step(Psi, V, grid, order, tau, ritz=True):
    """One iteration: propagate (Eq. 3), orthonormalise (Eq. 4), energies."""
    Phi = propagate(Psi, V, grid, order, tau)
    Psi, _ = cholesky_orthonormalize(Phi, grid.dV)
    E, Psi, _ = energies(Psi, V, grid, ritz)
    return Psi, E


def solve(Psi0, V, grid, order, tau, n_report, tol=1e-10, max_iter=1000,
          ritz=True):
    """Iterate until max_j |E_j^(l) - E_j^(l-1)| < tol over the n_report
    lowest states.  Returns (E, Psi, iterations)."""
    Psi = np.array(Psi0, dtype=np.float64, copy=True)
    E_prev = None
    for it in range(1, max_iter + 1):
        Psi, E = itp_step(Psi, V, grid, order, tau, ritz)
        if E_prev is not None and np.max(np.abs(E[:n_report] - E_prev[:n_report])) < tol:
            return E, Psi, it
        E_prev = E
    return E, Psi, max_iter


def solve_adaptive(Psi0, V, grid, order, tau0, reduce, gamma, n_report, max_steps=200,
                   max_levels=12):
    """The adaptive iteration of Sec. III.

    The initial states are orthonormalised (Eq. 4) and their diagonal
    energies E_j = (psi_j|H|psi_j) dV taken.  Then, at a fixed tau (first
    tau0), steps repeat: the states not yet converged are propagated (Eq. 3),
    R^E_j is evaluated for them, all states are orthonormalised (Eq. 4) and
    the diagonal energies taken again.  A state has converged at this tau
    once R^E_j < gamma tau^2 / 10: for small tau, phi_j - exp(-tau E_j) psi_j
    = -tau (H - E_j) psi_j + O(tau^2), so R^E_j / tau^2 is on the scale of
    R^H_j, and one bound gamma serves both tests as the text has it (with
    R^E_j < gamma literally, a reduced tau passes the test after one step
    whatever R^H_j is, and the iteration stalls); the factor 1/10 makes the
    states that pass it pass the final R^H_j < gamma too, instead of ending
    each level just above it.  The states kept fixed are the leading ones up to the
    first unconverged state, since a fixed state must precede the propagated
    ones in the Cholesky order of Eq. (4) to stay unchanged.  When the first
    n_report states have converged (or after max_steps steps), the states are
    rotated onto the Ritz vectors of their span (the subspace step of Sec.
    III) and R^H_j is evaluated for them with the Ritz values: if R^H_j <
    gamma for all j < n_report the iteration ends; else tau *= reduce and
    the steps repeat from the current states, all of them propagated again.

    Returns a dict: E (Ritz values), Psi (Ritz vectors), RH (R^H_j of the
    last basis), levels = [(tau, steps, propagated state-steps), ...] and
    converged (R^H below gamma before max_levels levels).
    """
    m = np.asarray(Psi0).shape[0]
    Psi, _ = cholesky_orthonormalize(np.array(Psi0, dtype=np.float64), grid.dV)
    E, Psi, HPsi = energies(Psi, V, grid, ritz=False)
    tau = tau0
    levels = []
    RH = residual_h(Psi, HPsi, E, grid.dV)
    converged = False
    for _ in range(max_levels):
        c = 0
        steps = props = 0
        while steps < max_steps and c < n_report:
            Phi = Psi.copy()
            Phi[c:] = propagate(Psi[c:], V, grid, order, tau)
            RE = residual_e(Phi[c:], Psi[c:], E[c:], tau, grid.dV)
            props += m - c
            steps += 1
            Psi, _ = cholesky_orthonormalize(Phi, grid.dV)
            E, Psi, HPsi = energies(Psi, V, grid, ritz=False)
            j = 0
            while j < len(RE) and RE[j] < 0.1 * gamma * tau * tau:
                j += 1
            c += j
        # R^H of the Ritz vectors: within a nearly degenerate group only the
        # spanned subspace converges at the rate of the gap to the unwanted
        # states, and the Ritz vectors of that subspace are its eigenvectors
        E, Psi, HPsi = energies(Psi, V, grid, ritz=True)
        RH = residual_h(Psi, HPsi, E, grid.dV)
        levels.append((tau, steps, props))
        if np.all(RH[:n_report] < gamma):
            converged = True
            break
        tau *= reduce
    E, Psi, _ = energies(Psi, V, grid, ritz=True)
    return dict(E=E, Psi=Psi, RH=RH, levels=levels, converged=converged)


def propagator_eigenvalue(psi, V, grid, order, tau):
    """E_T = -ln((psi|T_2k(tau)|psi) dV) / tau for a normalised state psi: the
    eigenvalue that the propagator itself assigns (Fig. 1 shows its error
    falling as Delta t^order)."""
    k2 = kinetic_k2(grid.shape, _box(grid))
    tp = t2k(psi.reshape(grid.shape), V, tau, k2, order // 2).ravel()
    return -np.log(np.dot(psi, tp) * grid.dV) / tau
