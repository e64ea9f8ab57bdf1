"""Write the reference eigenvalues of the C60-like workloads.

Run:  python tests/golden/make_c60_eref.py [edge ...]      (default: 64 128)

For each grid edge (box 32 bohr, the C60-like Gaussian well of the input
module: 60 wells of depth 2.0 Ha and width 0.8 bohr on a truncated
icosahedron of radius 6.7 bohr) this computes the lowest N_EIG eigenvalues
of the grid Hamiltonian H = F^-1 diag(|k|^2/2) F + diag(V) (Eq. 2) with the
oracle's block eigensolver, certifies them from outside the solver
(residual norms recomputed with the oracle's own H application), and writes
tests/golden/c60_<edge>_eref.txt.  It imports only oracle/ and
itp_workloads/; no value comes from the CUDA library.  The 128^3 grid is
started from the 64^3 solution, trigonometrically interpolated.
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from itp_workloads import c60_like_potential, cubic  # noqa: E402
from oracle.eigensolver import certify, interpolate_states, lobpcg_lowest  # noqa: E402

BOX = 32.0
N_EIG = 128          # the 120 wanted states of the workload and 8 beyond
BLOCK = 144          # iterated vectors (N_EIG + 16)


def solve(edge, X0=None, tol=1e-9):
    g = cubic(edge, BOX)
    V = c60_like_potential(g).reshape(g.shape)
    t0 = time.time()

    def log(it, th, res):
        print(f"  {edge}^3 iteration {it}: {time.time() - t0:.0f} s, max residual of the "
              f"first {N_EIG}: {res[:N_EIG].max():.2e}", flush=True)

    th, X, res, it = lobpcg_lowest(V, g, N_EIG, block=BLOCK, X0=X0, tol=tol, log=log)
    return g, V, th, X, res, it, time.time() - t0


def write(edge, g, V, th, X, it, secs):
    th2, r, bound = certify(th, X, V, g)
    path = os.path.join(HERE, f"c60_{edge}_eref.txt")
    with open(path, "w") as f:
        f.write(f"# Lowest {N_EIG} eigenvalues (Hartree) of the grid Hamiltonian of the C60-like\n"
                f"# well on a {edge}^3 periodic grid, box {BOX:g} bohr (the BASELINE C60-like\n"
                "# workload: 60 Gaussian wells, depth 2.0 Ha, sigma 0.8 bohr, truncated-icosahedron\n"
                "# vertices at radius 6.7 bohr).  Written by tests/golden/make_c60_eref.py with the\n"
                f"# oracle's LOBPCG eigensolver ({it} iterations, {secs:.0f} s, block {BLOCK}),\n"
                "# certified by residual norms r_j = |H x_j - E_j x_j| (unit vectors, Hartree)\n"
                "# recomputed with the oracle's H; bound_j = r_j^2 / gap_j (Kato-Temple).\n"
                "# Columns: j  E_j  r_j  bound_j\n")
        for j, (e, rr, b) in enumerate(zip(th2, r, bound)):
            f.write(f"{j + 1:4d}  {e:+.15f}  {rr:.3e}  {b:.3e}\n")
    print(f"wrote {path}: max residual {r.max():.2e}, max bound {bound.max():.2e}", flush=True)


def main(edges):
    coarse = None
    for edge in edges:
        X0 = None
        if coarse is not None:
            gc, Xc = coarse
            X0 = interpolate_states(Xc, gc, cubic(edge, BOX))
            extra = np.random.default_rng(edge).standard_normal((X0.shape[0], BLOCK - X0.shape[1]))
            X0 = np.concatenate([X0, extra], axis=1)
        g, V, th, X, res, it, secs = solve(edge, X0)
        write(edge, g, V, th, X, it, secs)
        coarse = (g, X)


if __name__ == "__main__":
    main([int(a) for a in sys.argv[1:]] or [64, 128])
