"""Reference eigenvalues of the grid Hamiltonian by a block eigensolver.

TEST INFRASTRUCTURE ONLY (see oracle/itp_oracle.py): used by the tests and
by the script that writes the stored reference eigenvalues, never by the
library, and independent of the imaginary-time method it checks.

What it computes has a plain definition: the lowest eigenvalues of the
spectral grid Hamiltonian H = F^-1 diag(|k|^2/2) F + diag(V) (Eq. 2,
hbar = m = 1) that the imaginary-time iteration of Eqs. (3)-(4) converges
to.  On grids too large for a dense eigendecomposition they are found with
LOBPCG (Knyazev, "Toward the optimal preconditioned eigensolver: locally
optimal block preconditioned conjugate gradient method", SIAM J. Sci.
Comput. 23, 517 (2001)): each iteration takes the Rayleigh-Ritz
approximation of H on span[X, W, P] -- the current block X, the
preconditioned residuals W = K (H X - X Theta), and the previous search
directions P -- with K = (|k|^2/2 + sigma)^-1 applied in Fourier space.
numpy / scipy FFTs and dense symmetric eigendecompositions are the library
steps.  The result is certified from outside the solver by the residual
norms |H x_j - theta_j x_j| of the returned orthonormal vectors, computed
with the oracle's own H application: each interval
[theta_j - r_j, theta_j + r_j] holds an eigenvalue of H (Weinstein), the
Ritz values bound the eigenvalues from above (Courant-Fischer), and for
well separated values |theta_j - lambda_j| <= r_j^2 / gap_j (Kato-Temple).
"""
from __future__ import annotations

import os

import numpy as np

try:   # multi-threaded FFTs when scipy is there; numpy.fft otherwise
    import scipy.fft as _sfft

    def _rfftn(a):
        return _sfft.rfftn(a, axes=(1, 2, 3), workers=os.cpu_count())

    def _irfftn(a, shape):
        return _sfft.irfftn(a, s=shape, axes=(1, 2, 3), workers=os.cpu_count())
except ImportError:   # pragma: no cover
    def _rfftn(a):
        return np.fft.rfftn(a, axes=(1, 2, 3))

    def _irfftn(a, shape):
        return np.fft.irfftn(a, s=shape, axes=(1, 2, 3))

from .itp_oracle import kinetic_k2

__all__ = ["apply_h_block", "lobpcg_lowest", "residual_norms", "certify", "interpolate_states"]


def _k2(grid):
    return kinetic_k2(grid.shape, (grid.lz, grid.ly, grid.lx))


def apply_h_block(Xt, V, k2, shape, chunk=16):
    """H applied to the columns of Xt (N, b): F^-1[|k|^2/2 F x] + V x,
    chunk columns at a time."""
    N, b = Xt.shape
    out = np.empty_like(Xt)
    v = V.ravel()
    for c0 in range(0, b, chunk):
        c1 = min(b, c0 + chunk)
        blk = np.ascontiguousarray(Xt[:, c0:c1].T).reshape((c1 - c0,) + tuple(shape))
        spec = _rfftn(blk)
        spec *= 0.5 * k2
        hx = _irfftn(spec, tuple(shape)).reshape(c1 - c0, N)
        hx += v[None, :] * blk.reshape(c1 - c0, N)
        out[:, c0:c1] = hx.T
    return out


def _precondition(R, k2, shape, sigma, chunk=16):
    """W = (|k|^2/2 + sigma)^-1 R, column by column in Fourier space."""
    N, b = R.shape
    out = np.empty_like(R)
    inv = 1.0 / (0.5 * k2 + sigma)
    for c0 in range(0, b, chunk):
        c1 = min(b, c0 + chunk)
        blk = np.ascontiguousarray(R[:, c0:c1].T).reshape((c1 - c0,) + tuple(shape))
        spec = _rfftn(blk)
        spec *= inv
        out[:, c0:c1] = _irfftn(spec, tuple(shape)).reshape(c1 - c0, N).T
    return out


def _orthonormal_basis(B, against=(), drop=1e-10):
    """Columns of B made orthogonal to the orthonormal blocks in `against`
    (twice, classical Gram-Schmidt) and then orthonormal among themselves
    through the eigendecomposition of their Gram matrix; directions whose
    norm falls below `drop` (relative) are dropped.  Returns (Q, T) with
    Q = B' T, B' the projected B."""
    for _ in range(2):
        for A in against:
            B = B - A @ (A.T @ B)
    nrm = np.sqrt(np.einsum("ij,ij->j", B, B))
    keep = nrm > drop * max(1e-300, nrm.max(initial=0.0))
    B = B[:, keep] / nrm[keep]
    if B.shape[1] == 0:
        return B, None
    G = B.T @ B
    w, U = np.linalg.eigh(0.5 * (G + G.T))
    good = w > drop
    T = U[:, good] / np.sqrt(w[good])
    return B @ T, (keep, T)


def residual_norms(X, HX, theta):
    """|H x_j - theta_j x_j| for orthonormal columns x_j (Euclidean norm)."""
    R = HX - X * theta[None, :]
    return np.sqrt(np.einsum("ij,ij->j", R, R))


def lobpcg_lowest(V, grid, n_eig, block=None, X0=None, tol=1e-9, max_iter=400,
                  sigma=1.0, log=None):
    """Lowest n_eig eigenpairs of the grid Hamiltonian.

    V: potential (nz, ny, nx); grid: itp_workloads.Grid; block: vectors
    iterated (default n_eig + 16: the extra ones speed up the convergence
    of the highest wanted pairs); X0: (N, block) start vectors (default
    seeded random normal).  Iterates until the residual norms of the first
    n_eig pairs are below tol (Euclidean norm of unit vectors, Hartree).
    Returns (theta, X, res, iterations): Ritz values (ascending), the
    orthonormal Ritz vectors (N, n_eig) in the Euclidean inner product
    (divide by sqrt(dV) for sum psi^2 dV = 1), residual norms.
    """
    shape = grid.shape
    N = grid.n_points
    b = block or (n_eig + 16)
    k2 = _k2(grid)
    if X0 is None:
        rng = np.random.default_rng(20240917)
        X0 = rng.standard_normal((N, b))
    X, _ = _orthonormal_basis(np.asarray(X0, dtype=np.float64))
    b = X.shape[1]
    HX = apply_h_block(X, V, k2, shape)
    G = X.T @ HX
    theta, C = np.linalg.eigh(0.5 * (G + G.T))
    X, HX = X @ C, HX @ C
    P = None
    res = residual_norms(X, HX, theta)
    it = 0
    for it in range(1, max_iter + 1):
        act = np.nonzero(res > 0.1 * tol)[0]   # soft locking of converged pairs
        if np.all(res[:n_eig] < tol):
            break
        R = HX[:, act] - X[:, act] * theta[act][None, :]
        W = _precondition(R, k2, shape, sigma)
        W, _ = _orthonormal_basis(W, against=(X,))
        HW = apply_h_block(W, V, k2, shape)
        blocks, hblocks = [X, W], [HX, HW]
        if P is not None:
            # the previous directions, orthonormalised against X and W; H
            # is applied to the new basis itself rather than updated, so
            # no rounding accumulates in H P
            Pn, _ = _orthonormal_basis(P, against=(X, W))
            if Pn.shape[1]:
                blocks.append(Pn)
                hblocks.append(apply_h_block(Pn, V, k2, shape))
        nb = len(blocks)
        G = np.zeros((sum(B.shape[1] for B in blocks),) * 2)
        offs = np.cumsum([0] + [B.shape[1] for B in blocks])
        for i in range(nb):
            for j in range(i, nb):
                g = blocks[i].T @ hblocks[j]
                G[offs[i]:offs[i + 1], offs[j]:offs[j + 1]] = g
                G[offs[j]:offs[j + 1], offs[i]:offs[i + 1]] = g.T
        w, U = np.linalg.eigh(0.5 * (G + G.T))
        C = U[:, :b]
        theta = w[:b]
        Xn = sum(blocks[i] @ C[offs[i]:offs[i + 1]] for i in range(nb))
        HXn = sum(hblocks[i] @ C[offs[i]:offs[i + 1]] for i in range(nb))
        P = sum(blocks[i] @ C[offs[i]:offs[i + 1]] for i in range(1, nb))
        X, HX = Xn, HXn
        res = residual_norms(X, HX, theta)
        if log:
            log(it, theta, res)
    return theta[:n_eig], X[:, :n_eig], res[:n_eig], it


def certify(theta, X, V, grid):
    """Residual norms r_j = |H x_j - theta_j x_j| recomputed from scratch
    with the oracle's H (itp_oracle.apply_h, one state at a time) after
    re-orthonormalising X, and the Kato-Temple estimate r_j^2 / gap_j of
    |theta_j - lambda_j|, gap_j the distance from theta_j to the nearest
    other Ritz value outside its own cluster (values within 10 r of it).
    Returns (theta, r, bound)."""
    from .itp_oracle import apply_h
    k2 = _k2(grid)
    Q, _ = np.linalg.qr(X)
    HQ = np.stack([apply_h(Q[:, j].reshape(grid.shape), V, k2).ravel()
                   for j in range(Q.shape[1])], axis=1)
    G = Q.T @ HQ
    th, U = np.linalg.eigh(0.5 * (G + G.T))
    Q, HQ = Q @ U, HQ @ U
    r = residual_norms(Q, HQ, th)
    bound = np.empty_like(th)
    for j in range(len(th)):
        far = np.abs(th - th[j]) > 10 * max(r[j], 1e-14)
        gap = np.min(np.abs(th[far] - th[j])) if np.any(far) else np.inf
        bound[j] = r[j] ** 2 / gap
    return th, r, bound


def interpolate_states(X, grid_from, grid_to):
    """Trigonometric interpolation of the columns of X (N_from, b) from one
    grid to a finer one over the same box: the half spectrum is copied into
    the larger one (zero padding; the Nyquist planes of the coarse grid are
    dropped) and scaled by N_to / N_from.  Used only to start the solver on
    a fine grid from a coarse solution."""
    sf, st = grid_from.shape, grid_to.shape
    b = X.shape[1]
    out = np.empty((grid_to.n_points, b))
    scale = grid_to.n_points / grid_from.n_points
    for j in range(b):
        spec = np.fft.rfftn(X[:, j].reshape(sf), axes=(0, 1, 2))
        big = np.zeros((st[0], st[1], st[2] // 2 + 1), dtype=complex)
        hz, hy, hx = sf[0] // 2, sf[1] // 2, sf[2] // 2
        for zs in (slice(0, hz), slice(-hz + 1, None) if hz > 1 else slice(0, 0)):
            for ys in (slice(0, hy), slice(-hy + 1, None) if hy > 1 else slice(0, 0)):
                big[zs, ys, :hx] = spec[zs, ys, :hx]
        out[:, j] = np.fft.irfftn(big * scale, s=st, axes=(0, 1, 2)).ravel()
    return out
