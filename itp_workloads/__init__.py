"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module generates *inputs only*: grid coordinates, model potentials and
random initial states.  It holds none of the propagation, orthonormalisation
or energy arithmetic of the imaginary-time method, so that the CPU oracle and
the CUDA path can both draw byte-identical inputs from it without sharing any
of the method.

Random numbers come from the counter-based generator Philox4x32-10 (Salmon,
Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11),
implemented from its published definition, followed by the Box-Muller
transform.  A draw is keyed by (seed, problem) and addressed by
(point pair, state, stream tag), so any state of any problem can be
regenerated on its own.

Workloads (the paper's own C60 potential is not usable as printed, Sec. III;
the Gaussian C60-like well stands in for it):
  * harmonic oscillator V = r^2/2 (hbar = m = 1, Hartree units);
  * C60-like well: 60 Gaussian wells of depth 2.0 Ha, width 0.8 bohr on the
    vertices of a truncated icosahedron scaled to radius 6.7 bohr;
  * random Gaussian-well problems for the batched workload;
  * planar problems (nz = 1): the 2D oscillator and a square array of
    quantum dots with the paper's sech well shape.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np

__all__ = [
    "philox4x32_10", "uniform53", "normal_states", "Grid", "grid_axes",
    "harmonic_potential", "truncated_icosahedron", "gaussian_wells_potential",
    "c60_like_potential", "random_wells_problem", "supported_dim", "planar",
    "harmonic_potential_2d", "quantum_dot_array",
]

# ---------------------------------------------------------------------------
# Philox4x32-10 (SC'11, Sec. 5): 10 rounds of two 32x32->64 multiplies with a
# Weyl-sequence key schedule.
_PHILOX_M0 = np.uint64(0xD2511F53)
_PHILOX_M1 = np.uint64(0xCD9E8D57)
_PHILOX_W0 = 0x9E3779B9
_PHILOX_W1 = 0xBB67AE85
_U32 = 0xFFFFFFFF


def philox4x32_10(c0, c1, c2, c3, k0: int, k1: int):
    """Philox4x32 with 10 rounds on vectors of 32-bit counters.

    Each round: (hi0, lo0) = M0*c0, (hi1, lo1) = M1*c2 and the new counter is
    (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0); the key is bumped by the Weyl
    constants between rounds.  Returns four uint32 arrays.
    """
    c0 = np.asarray(c0, dtype=np.uint32)
    c1 = np.broadcast_to(np.asarray(c1, dtype=np.uint32), c0.shape)
    c2 = np.broadcast_to(np.asarray(c2, dtype=np.uint32), c0.shape)
    c3 = np.broadcast_to(np.asarray(c3, dtype=np.uint32), c0.shape)
    key0, key1 = int(k0) & _U32, int(k1) & _U32
    shift = np.uint64(32)
    for rnd in range(10):
        p0 = _PHILOX_M0 * c0.astype(np.uint64)
        p1 = _PHILOX_M1 * c2.astype(np.uint64)
        hi0 = (p0 >> shift).astype(np.uint32)
        lo0 = p0.astype(np.uint32)
        hi1 = (p1 >> shift).astype(np.uint32)
        lo1 = p1.astype(np.uint32)
        c0, c1, c2, c3 = (hi1 ^ c1 ^ np.uint32(key0), lo1,
                          hi0 ^ c3 ^ np.uint32(key1), lo0)
        if rnd < 9:
            key0 = (key0 + _PHILOX_W0) & _U32
            key1 = (key1 + _PHILOX_W1) & _U32
    return c0, c1, c2, c3


def uniform53(hi, lo):
    """Two uint32 words -> doubles in (0, 1) with 53 random bits (never 0)."""
    a = (np.asarray(hi, dtype=np.uint64) >> np.uint64(5)).astype(np.float64)
    b = (np.asarray(lo, dtype=np.uint64) >> np.uint64(6)).astype(np.float64)
    return (a * 67108864.0 + b + 0.5) / 9007199254740992.0


_TAG_STATES = 0x5157A7E5  # stream tag of the initial-state draws

_HERE = os.path.dirname(os.path.abspath(__file__))
_NATIVE = os.path.join(_HERE, "libphilox.so")
_native_lib = None


def build_native() -> str:
    """Compile philox.c (the same generator in C, for large inputs)."""
    src = os.path.join(_HERE, "philox.c")
    if not os.path.exists(_NATIVE) or os.path.getmtime(_NATIVE) < os.path.getmtime(src):
        subprocess.run(["gcc", "-O2", "-shared", "-fPIC", "-o", _NATIVE + ".tmp", src],
                       check=True)
        os.replace(_NATIVE + ".tmp", _NATIVE)
    return _NATIVE


def _native():
    global _native_lib
    if _native_lib is None and os.path.exists(_NATIVE):
        lib = ctypes.CDLL(_NATIVE)
        lib.philox_uniform_pairs.restype = None
        lib.philox_uniform_pairs.argtypes = [ctypes.c_uint64] + [ctypes.c_uint32] * 6 + [
            ctypes.c_void_p]
        _native_lib = lib
    return _native_lib


def _state_uniforms(npairs, state, problem, k0, k1, use_native=True):
    """(u1, u2) of the Philox draws (pair, state, problem, states tag)."""
    lib = _native() if use_native else None
    if lib is not None:
        u = np.empty(2 * npairs)
        lib.philox_uniform_pairs(npairs, 0, state & _U32, problem & _U32, _TAG_STATES, k0, k1,
                                 u.ctypes.data)
        return u[0::2], u[1::2]
    pairs = np.arange(npairs, dtype=np.uint32)
    r0, r1, r2, r3 = philox4x32_10(pairs, state, problem, _TAG_STATES, k0, k1)
    return uniform53(r0, r1), uniform53(r2, r3)


def normal_states(n_states: int, n_points: int, seed: int, problem: int = 0,
                  first_state: int = 0, use_native: bool = True) -> np.ndarray:
    """Random-normal initial states, shape (n_states, n_points), float64.

    State j (global index first_state + j), point p takes the Box-Muller
    normal number (p % 2) of the Philox draw at counter
    (p // 2, j, problem, tag) under key (seed, seed >> 32).  The C and numpy
    Philox give identical uniforms; the Box-Muller step is numpy in both.
    """
    if n_points % 2:
        raise ValueError("n_points must be even")
    out = np.empty((n_states, n_points), dtype=np.float64)
    k0, k1 = int(seed) & _U32, (int(seed) >> 32) & _U32
    for j in range(n_states):
        u1, u2 = _state_uniforms(n_points // 2, first_state + j, problem, k0, k1, use_native)
        rad = np.sqrt(-2.0 * np.log(u1))
        ang = 2.0 * np.pi * u2
        out[j, 0::2] = rad * np.cos(ang)
        out[j, 1::2] = rad * np.sin(ang)
    return out


def _uniforms(count: int, seed: int, problem: int, tag: int) -> np.ndarray:
    """`count` uniform doubles in (0,1) from the Philox stream (problem, tag)."""
    npairs = (count + 1) // 2
    ctr = np.arange(npairs, dtype=np.uint32)
    r0, r1, r2, r3 = philox4x32_10(ctr, 0, problem, tag, int(seed) & _U32,
                                   (int(seed) >> 32) & _U32)
    u = np.empty(2 * npairs)
    u[0::2] = uniform53(r0, r1)
    u[1::2] = uniform53(r2, r3)
    return u[:count]


# ---------------------------------------------------------------------------
# Grids.  Periodic box [-L/2, L/2) per axis, x_i = -L/2 + i*h, h = L/N.
@dataclass(frozen=True)
class Grid:
    nx: int
    ny: int
    nz: int
    lx: float
    ly: float
    lz: float

    @property
    def shape(self):
        """Array shape of one state, (nz, ny, nx): x is the fastest axis."""
        return (self.nz, self.ny, self.nx)

    @property
    def n_points(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def dV(self) -> float:
        return (self.lx / self.nx) * (self.ly / self.ny) * (self.lz / self.nz)


def cubic(n: int, box: float) -> Grid:
    return Grid(n, n, n, box, box, box)


def supported_dim(n: int) -> bool:
    """Axis lengths the CUDA FFT passes take: even, 2 <= n <= 256, and a
    product of two factors from {1,2,3,4,6,8,12,16}."""
    radices = (1, 2, 3, 4, 6, 8, 12, 16)
    if n < 2 or n > 256 or n % 2:
        return False
    return any(n % a == 0 and (n // a) in radices for a in radices)


def grid_axes(g: Grid):
    """Coordinates (z, y, x) of the grid points along each axis."""
    ax = [-0.5 * L + (L / N) * np.arange(N)
          for N, L in ((g.nz, g.lz), (g.ny, g.ly), (g.nx, g.lx))]
    return ax[0], ax[1], ax[2]


def harmonic_potential(g: Grid, omega: float = 1.0) -> np.ndarray:
    """V = omega^2 r^2 / 2 on the grid, shape (nz, ny, nx)."""
    z, y, x = grid_axes(g)
    return 0.5 * omega ** 2 * (z[:, None, None] ** 2 + y[None, :, None] ** 2
                               + x[None, None, :] ** 2)


def truncated_icosahedron(radius: float = 6.7) -> np.ndarray:
    """The 60 vertices of a truncated icosahedron, scaled to `radius`.

    Cyclic (even) permutations of (0, +-1, +-3phi), (+-1, +-(2+phi), +-2phi)
    and (+-phi, +-2, +-phi^3), with phi the golden ratio.
    """
    phi = (1.0 + math.sqrt(5.0)) / 2.0
    bases = [(0.0, 1.0, 3 * phi), (1.0, 2 + phi, 2 * phi), (phi, 2.0, phi ** 3)]
    pts = set()
    for b in bases:
        for sx in (1, -1):
            for sy in (1, -1):
                for sz in (1, -1):
                    v = (sx * b[0], sy * b[1], sz * b[2])
                    for r in range(3):
                        p = tuple(round(v[(i + r) % 3], 12) + 0.0 for i in range(3))
                        pts.add(p)
    arr = np.array(sorted(pts), dtype=np.float64)
    assert arr.shape == (60, 3)
    rad = np.sqrt((arr ** 2).sum(axis=1))
    return arr * (radius / rad[:, None])


def gaussian_wells_potential(g: Grid, centres: np.ndarray, depths, sigmas,
                             chunk: int = 8) -> np.ndarray:
    """V(r) = -sum_a depth_a * exp(-|r - R_a|^2 / (2 sigma_a^2)), Hartree.

    Distances are the plain (non-periodic) ones inside the box.
    """
    z, y, x = grid_axes(g)
    depths = np.broadcast_to(np.asarray(depths, dtype=np.float64), (len(centres),))
    sigmas = np.broadcast_to(np.asarray(sigmas, dtype=np.float64), (len(centres),))
    V = np.zeros(g.shape)
    for a, (cx, cy, cz) in enumerate(centres):
        s2 = 2.0 * sigmas[a] ** 2
        ez = np.exp(-(z - cz) ** 2 / s2)
        ey = np.exp(-(y - cy) ** 2 / s2)
        ex = np.exp(-(x - cx) ** 2 / s2)
        V -= depths[a] * (ez[:, None, None] * ey[None, :, None] * ex[None, None, :])
    return V


def c60_like_potential(g: Grid, depth: float = 2.0, sigma: float = 0.8,
                       radius: float = 6.7) -> np.ndarray:
    """Gaussian C60-like well: 60 wells on the truncated-icosahedron vertices."""
    return gaussian_wells_potential(g, truncated_icosahedron(radius), depth, sigma)


def planar(nx: int, ny: int, lx: float, ly: float) -> Grid:
    """A two-dimensional grid: nz = 1 and lz = 1, so the volume element is
    dx*dy and the z coordinate plays no part (the potentials below for
    planar problems depend on x and y only)."""
    return Grid(nx, ny, 1, lx, ly, 1.0)


def harmonic_potential_2d(g: Grid, omega: float = 1.0) -> np.ndarray:
    """V = omega^2 (x^2 + y^2) / 2 on a planar grid, shape (1, ny, nx)."""
    _, y, x = grid_axes(g)
    return (0.5 * omega ** 2 * (y[:, None] ** 2 + x[None, :] ** 2))[None, :, :]


def quantum_dot_array(g: Grid, n_side: int = 9, spacing: float = 3.0, depth: float = 2.0,
                      width: float = 0.6) -> np.ndarray:
    """The planar case of the method's demonstration: a square n_side x
    n_side array of quantum dots centred in the box, each with the paper's
    well shape V = -depth / cosh(|r - R|/width) (Hartree, bohr; the printed
    strength and width are not usable, so depth and width are chosen here),
    summed over the dots.  Shape (1, ny, nx)."""
    _, y, x = grid_axes(g)
    c = (np.arange(n_side) - 0.5 * (n_side - 1)) * spacing
    V = np.zeros((g.ny, g.nx))
    for cy in c:
        for cx in c:
            r = np.sqrt((y[:, None] - cy) ** 2 + (x[None, :] - cx) ** 2)
            V -= depth / np.cosh(r / width)
    return V[None, :, :]


_TAG_WELLS = 0x3E11C0DE


def random_wells_problem(seed: int, problem: int,
                         sizes=(32, 48, 64, 96), box: float = 32.0,
                         n_range=(8, 64), wells_range=(4, 60)):
    """One problem of the batched workload.

    Drawn from the Philox stream (problem, wells tag): the grid edge from
    `sizes`, the state count n ~ U{n_range}, the well count ~ U{wells_range},
    depths U[0.5, 3] Ha, widths U[0.5, 1.2] bohr and centres uniform in a
    ball of radius 8 bohr.  Returns (grid, V, n_states).
    """
    head = _uniforms(3, seed, problem, _TAG_WELLS)
    N = sizes[int(head[0] * len(sizes))]
    n_states = n_range[0] + int(head[1] * (n_range[1] - n_range[0] + 1))
    n_wells = wells_range[0] + int(head[2] * (wells_range[1] - wells_range[0] + 1))
    u = _uniforms(3 + 6 * n_wells, seed, problem, _TAG_WELLS)[3:].reshape(n_wells, 6)
    depths = 0.5 + 2.5 * u[:, 0]
    sigmas = 0.5 + 0.7 * u[:, 1]
    # uniform in the ball: radius ~ 8 * u^(1/3), direction from (cos theta, phi)
    rad = 8.0 * np.cbrt(u[:, 2])
    cos_t = 2.0 * u[:, 3] - 1.0
    sin_t = np.sqrt(np.maximum(0.0, 1.0 - cos_t ** 2))
    ph = 2.0 * np.pi * u[:, 4]
    centres = np.stack([rad * sin_t * np.cos(ph), rad * sin_t * np.sin(ph),
                        rad * cos_t], axis=1)
    g = cubic(N, box)
    return g, gaussian_wells_potential(g, centres, depths, sigmas), n_states
