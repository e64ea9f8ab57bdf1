"""The Sturm count of the Ritz-value bisection (csrc/dense.cu, sturm_count),
compiled for the host: the same function text with the three bit-cast
intrinsics it uses supplied as plain C++.  The count of eigenvalues below x
of a symmetric tridiagonal (the eigenvalues of the subspace matrix, Sec. III)
must equal the count from LAPACK's tridiagonal eigenvalues, away from points
within rounding of an eigenvalue, on the matrices where a division-free
recurrence can go wrong: zero and tiny couplings, degenerate clusters, x at a
diagonal entry or an eigenvalue, graded and extreme scales, Wilkinson
matrices.  The multisection over 128 points per round, written out here as
the kernel runs it, must then give the eigenvalues within a few ulps of the
norm."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

scipy_linalg = pytest.importorskip("scipy.linalg")

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "..", "paper_0809_3739_gb300", "csrc", "dense.cu")
FIRST = "__device__ __forceinline__ int dexp(double v)"
AFTER = "// One CTA per eigenvalue index j (ascending)"

SHIM = r"""
#include <cmath>
#include <cstdint>
#include <cstring>
using std::fabs;
using std::fma;
#define __device__
#define __forceinline__ inline
#define __restrict__ __restrict
static inline int __double2hiint(double v) {
  uint64_t u; std::memcpy(&u, &v, 8); return (int)(uint32_t)(u >> 32);
}
static inline int __double2loint(double v) {
  uint64_t u; std::memcpy(&u, &v, 8); return (int)(uint32_t)u;
}
static inline double __hiloint2double(int hi, int lo) {
  uint64_t u = ((uint64_t)(uint32_t)hi << 32) | (uint32_t)lo;
  double v; std::memcpy(&v, &u, 8); return v;
}
"""
EXPORT = r"""
extern "C" int host_sturm_count(const double* d, const double* e2, int m, double x) {
  return sturm_count(d, e2, m, x);
}
"""


@pytest.fixture(scope="module")
def count(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    src = open(SRC).read()
    a, b = src.index(FIRST), src.index(AFTER)
    d = tmp_path_factory.mktemp("sturm")
    cpp, so = d / "sturm.cpp", d / "libsturm.so"
    cpp.write_text(SHIM + src[a:b] + EXPORT)
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", str(so),
                           str(cpp)])
    lib = ctypes.CDLL(str(so))
    dp = ctypes.POINTER(ctypes.c_double)
    lib.host_sturm_count.restype = ctypes.c_int
    lib.host_sturm_count.argtypes = [dp, dp, ctypes.c_int, ctypes.c_double]

    def f(sd, se2, x):
        return lib.host_sturm_count(sd.ctypes.data_as(dp), se2.ctypes.data_as(dp), len(sd),
                                    float(x))
    return f


def _scaled(d, e):
    """The kernel's set-up: Gershgorin interval with a small margin, then a
    power of two that brings it into (-1, 1); e2 the squared couplings."""
    m = len(d)
    r = np.zeros(m)
    r[1:] += np.abs(e[:m - 1])
    r[:m - 1] += np.abs(e[:m - 1])
    lo, hi = min(d[0], (d - r).min()), max(d[0], (d + r).max())
    span = max(hi - lo, 1e-300)
    lo -= 1e-14 * span + 1e-300
    hi += 1e-14 * span + 1e-300
    g = np.ldexp(1.0, -int(np.frexp(max(abs(lo), abs(hi)))[1]))
    ee = np.zeros(m)
    ee[:m - 1] = e[:m - 1] * g
    return np.ascontiguousarray(d * g), np.ascontiguousarray(ee * ee), lo * g, hi * g, g


def _matrices():
    rng = np.random.default_rng(2008)
    out = []
    for m in (1, 2, 3, 7, 64, 128, 256):
        out.append((f"random {m}", rng.normal(size=m), rng.normal(size=m)))
    m = 128
    out.append(("zero couplings", rng.normal(size=m), np.zeros(m)))
    out.append(("tiny couplings", rng.normal(size=m), 1e-30 * rng.normal(size=m)))
    out.append(("fourfold clusters", np.repeat(rng.normal(size=32), 4),
                1e-12 * rng.normal(size=m)))
    out.append(("fourfold, decoupled", np.repeat(rng.normal(size=32), 4), np.zeros(m)))
    out.append(("dyadic diagonal, decoupled", np.round(4 * rng.normal(size=m)) / 4, np.zeros(m)))
    out.append(("Wilkinson 21", np.abs(np.arange(21) - 10.0), np.ones(21)))
    out.append(("Wilkinson 201", np.abs(np.arange(201) - 100.0), np.ones(201)))
    glue = np.ones(126)
    glue[20::21] = 1e-10
    out.append(("glued Wilkinson", np.tile(np.abs(np.arange(21) - 10.0), 6), glue))
    out.append(("norm 1e150", 1e150 * rng.normal(size=m), 1e150 * rng.normal(size=m)))
    out.append(("norm 1e-150", 1e-150 * rng.normal(size=m), 1e-150 * rng.normal(size=m)))
    out.append(("graded", np.logspace(-12, 0, m), np.logspace(-13, -1, m)))
    out.append(("nearly diagonal spectrum", np.sort(rng.uniform(-0.52, -0.1, m)),
                1e-9 * rng.normal(size=m)))
    out.append(("tight cluster", -0.5 + 1e-13 * rng.normal(size=m), 1e-14 * rng.normal(size=m)))
    out.append(("zero matrix", np.zeros(m), np.zeros(m)))
    return out


def _prepare(d, e):
    d = np.ascontiguousarray(d, dtype=np.float64)
    m = len(d)
    e = np.ascontiguousarray(np.resize(np.asarray(e, dtype=np.float64), m))
    e[m - 1] = 0.0
    lam = scipy_linalg.eigvalsh_tridiagonal(d, e[:m - 1]) if m > 1 else d.copy()
    return d, e, lam


@pytest.mark.parametrize("name,d,e", _matrices(), ids=[c[0] for c in _matrices()])
def test_counts_equal_lapack_counts(count, name, d, e):
    d, e, lam = _prepare(d, e)
    sd, se2, lo, hi, g = _scaled(d, e)
    lam_s = lam * g
    tol = 1e-12 * max(np.abs(lam_s).max(), np.abs(e * g).max(), 1e-300)
    rng = np.random.default_rng(7)
    xs = np.concatenate([rng.uniform(lo, hi, 300), sd, lam_s, lam_s * (1 + 1e-9), [lo, hi]])
    for x in xs:
        if not lo <= x <= hi:
            continue
        c = count(sd, se2, x)
        # exact count of a matrix within rounding: between the counts at x -+ tol
        assert int(np.sum(lam_s < x - tol)) <= c <= int(np.sum(lam_s < x + tol)), (name, x)


@pytest.mark.parametrize("name,d,e", _matrices(), ids=[c[0] for c in _matrices()])
def test_multisection_gives_lapack_eigenvalues(count, name, d, e):
    d, e, lam = _prepare(d, e)
    sd, se2, lo0, hi0, g = _scaled(d, e)
    m, pts = len(d), 128
    E = np.empty(m)
    for j in range(m):
        lo, hi = lo0, hi0
        for _ in range(16):
            width = hi - lo
            if width <= 4.0 * 2.220446049250313e-16 * max(abs(lo), abs(hi)) + 2.0 ** -70:
                break
            first = pts - 1
            for t in range(pts - 1):   # the first point whose count exceeds j
                if count(sd, se2, lo + width * float(t + 1) / pts) > j:
                    first = t
                    break
            nlo = lo if first == 0 else lo + width * float(first) / pts
            nhi = hi if first == pts - 1 else lo + width * float(first + 1) / pts
            lo, hi = nlo, nhi
        E[j] = 0.5 * (lo + hi) / g
    nrm = max(np.abs(lam).max(), np.abs(e).max(), 1e-300)
    assert np.max(np.abs(E - lam)) <= 2e-14 * nrm, name


def test_exact_zero_minors(count):
    """Small-integer matrices at dyadic points: the arithmetic is exact, so
    leading minors vanish exactly (with nonzero couplings) wherever x is an
    eigenvalue of a leading block; away from the whole matrix's eigenvalues
    the count must still be LAPACK's."""
    rng = np.random.default_rng(31)
    zeros = checked = 0
    for _ in range(300):
        m = int(rng.integers(3, 14))
        d = rng.integers(-4, 5, size=m).astype(np.float64)
        e = rng.integers(-3, 4, size=m).astype(np.float64)
        d, e, lam = _prepare(d, e)
        sd, se2, lo, hi, g = _scaled(d, e)
        lam_s = lam * g
        for x in np.arange(-64, 65) / 8.0 * g:
            if not lo <= x <= hi or np.min(np.abs(lam_s - x)) < 1e-9 * g:
                continue
            # exact leading minors at x (integers scaled by powers of two)
            p0, p1, hit = 1.0, sd[0] - x, sd[0] == x
            for i in range(1, m):
                p0, p1 = p1, (sd[i] - x) * p1 - se2[i - 1] * p0
                hit |= p1 == 0.0 and i < m - 1
            zeros += hit
            checked += 1
            assert count(sd, se2, x) == int(np.sum(lam_s < x)), (d, e, x / g)
    assert checked > 1000 and zeros > 50
