// Plane and pencil passes of the 3D real FFT with the split-operator factors
// fused in (T_2 of Eq. (so) as point-wise multiplies around one complete
// FFT; Sec. I).
//
// Data layout in HBM (internal to the library):
//   real arrays     [m][nz][nx][ny]      per-plane transposed: y fastest, so a
//                                         "row pair" (rows y = 2r, 2r+1 at one
//                                         x) is one contiguous (re, im) pair
//   half spectrum   [m][nz][ny][nx/2+1]  complex, natural frequency order
//   FP64 accumulator and potential: same layout as the real arrays.
//
// Plane pass: one CTA per (state, z plane).  Rows 2r and 2r+1 travel as one
// complex row (re = row 2r, im = row 2r+1) of length nx, so the real
// transform along x is one complex FFT per row pair followed by the
// even/odd split; after the split, row pair r holds the half-spectrum rows
// of y = 2r and y = 2r+1 back to back.  The complex FFT along y runs down
// the nx/2+1 columns.  Global loads and stores are fused into the first and
// last FFT stage of each pass; with the transposed real layout every such
// access is coalesced (neighbouring lanes = neighbouring row pairs or
// columns).
//
// Pencil pass: one CTA per (state, ky, block of kx columns).  Forward FFT
// along z (first stage fused with the loads), then in registers the second
// forward stage, the kinetic factor exp(-tau |k|^2/2)/N and the first
// inverse stage, then the last inverse stage fused with the stores: two
// shared-memory round trips per pencil.
//
// Kernels are specialised at compile time for the common edge lengths
// (all index arithmetic folds to constants); a generic instantiation takes
// the sizes at run time.
#pragma once
#include <cooperative_groups.h>

#include "fft_common.cuh"
#include "itp_kernels.cuh"

namespace cg = cooperative_groups;

namespace itp {

namespace {

constexpr int kThreads = 256;

__host__ __device__ constexpr bool is_radix(int r) {
  return r == 1 || r == 2 || r == 3 || r == 4 || r == 6 || r == 8 || r == 12 || r == 16;
}
// r1 of the split L = r1 * r2 (r1 <= r2, most balanced; r1 = 1 if L <= 16).
__host__ __device__ constexpr int split_r1(int L) {
  if (L <= 16 && is_radix(L)) return 1;
  int best = 0;
  for (int a = 2; a <= 16; ++a) {
    if (!is_radix(a) || L % a) continue;
    const int b = L / a;
    if (!is_radix(b) || b < a) continue;
    if (best == 0 || (b - a) < (L / best - best)) best = a;
  }
  return best;
}

// Compile-time (N > 0) or run-time (N == 0) axis.
template <int N>
struct AxisT {
  static constexpr int L_ = N, R1_ = (N ? split_r1(N) : 0), R2_ = (N ? N / split_r1(N) : 0);
  int L, r1, r2;
  __device__ __forceinline__ AxisT(int l, int a, int b)
      : L(N ? L_ : l), r1(N ? R1_ : a), r2(N ? R2_ : b) {}
};

// Threads doing FFT tasks: a multiple of the column count w (= nx/2+1 or a
// pencil block) close to 256, so the column stages have no ragged last
// iteration; the CTA is launched with that count rounded up to whole warps.
__host__ __device__ constexpr int task_threads(int w) {
  return w <= 0 ? kThreads : w * ((kThreads + w / 2) / w < 1 ? 1 : (kThreads + w / 2) / w);
}
__host__ __device__ constexpr int launch_threads(int nt) { return (nt + 31) / 32 * 32; }

// Shared-memory pitch of a row pair: room for the padded packed row
// (nx + nx/16) and the two half-spectrum rows (nx + 2), odd.
__host__ __device__ constexpr int row_pitch(int nx) {
  return ((nx + nx / 16 + 2) % 2) ? nx + nx / 16 + 2 : nx + nx / 16 + 3;
}
// CTAs per SM that the shared memory of a specialised pass allows (the
// register budget follows from it through __launch_bounds__).
__host__ __device__ constexpr int min_blocks(long long smem_bytes, int cap) {
  return smem_bytes <= 0 ? 1
         : (227LL * 1024 / smem_bytes) < 1 ? 1
         : (227LL * 1024 / smem_bytes) > cap ? cap
         : (int)(227LL * 1024 / smem_bytes);
}
__host__ __device__ constexpr long long plane_smem_ct(int nx, int ny, int rbytes) {
  return nx ? ((long long)(ny / 2) * row_pitch(nx) + nx + ny) * 2 * rbytes : 0;
}
// CTAs per SM a specialised pencil pass asks the compiler to fit (the
// register budget follows): 3 for FP32, but 2 for 256-point pencils, whose
// radix-16 stages do not fit the 75 registers of three 288-thread CTAs.
__host__ __device__ constexpr int pencil_min_ctas(int nz, int rbytes) {
  return rbytes == 4 && nz < 256 ? 3 : 2;
}
__host__ __device__ constexpr long long pencil_smem_ct(int nz, int w, int rbytes) {
  return nz ? ((long long)nz * w + nz) * 2 * rbytes : 0;
}

// Padded position of element p of a packed row: one pad slot per 16 keeps
// the strided reads of the split/merge free of bank conflicts.
__device__ __forceinline__ int swz(int p) { return p + (p >> 4); }

// Task loop over NT threads: task = t + ntr * q, t fastest across lanes.
template <int NT, typename F>
__device__ __forceinline__ void for_tasks(int ntr, int nq, F&& f) {
  const int total = ntr * nq;
  if (threadIdx.x >= NT) return;
  for (int task = threadIdx.x; task < total; task += NT) {
    const int q = task / ntr;
    const int t = task - q * ntr;
    f(t, q);
  }
}

// Radix dispatch: FN<r>(args...) for the run-time radix r (folds to one case
// when r is a compile-time constant).
#define ITP_WITH_RADIX(r, FN, ...)          \
  switch (r) {                              \
    case 1: FN<1>(__VA_ARGS__); break;      \
    case 2: FN<2>(__VA_ARGS__); break;      \
    case 3: FN<3>(__VA_ARGS__); break;      \
    case 4: FN<4>(__VA_ARGS__); break;      \
    case 6: FN<6>(__VA_ARGS__); break;      \
    case 8: FN<8>(__VA_ARGS__); break;      \
    case 12: FN<12>(__VA_ARGS__); break;    \
    case 16: FN<16>(__VA_ARGS__); break;    \
    default: break;                         \
  }

template <typename C>
__device__ __forceinline__ C cscale(C a, decltype(a.x) s) {
  a.x *= s;
  a.y *= s;
  return a;
}
template <typename C>
__device__ __forceinline__ C cmulri(C a, C f) {  // (a.x * f.x, a.y * f.y)
  a.x *= f.x;
  a.y *= f.y;
  return a;
}
template <>
__device__ __forceinline__ float2 cmulri<float2>(float2 a, float2 f) {
  return __fmul2_rn(a, f);
}

// a[j] *= w^(q j) (CONJ: w^(-q j)), j = 1..R-1, from the table tw of
// roots.  For R = 8 and 16 the factor is w^(q j1) w^(4 q j2) with
// j = j1 + 4 j2: four or six table reads instead of seven or fifteen (the
// reads are shared-memory wavefronts, the passes' bound), each product
// within about an ulp of the table value.
template <int R, bool CONJ = false, typename C>
__device__ __forceinline__ void twiddle_stage(C (&a)[R], const C* tw, int q) {
  if constexpr (R == 8 || R == 16) {
    constexpr int NH = R / 4;   // hi factors w^(4 q j2), j2 = 1 .. NH-1
    C lo[4], hi[NH];
#pragma unroll
    for (int j = 1; j < 4; ++j) lo[j] = tw[q * j];
#pragma unroll
    for (int j = 1; j < NH; ++j) hi[j] = tw[4 * q * j];
#pragma unroll
    for (int j = 1; j < R; ++j) {
      const int j1 = j & 3, j2 = j >> 2;
      const C w = j2 == 0 ? lo[j1] : (j1 == 0 ? hi[j2] : cmul(lo[j1], hi[j2]));
      a[j] = CONJ ? cmulc(a[j], w) : cmul(a[j], w);
    }
  } else {
#pragma unroll
    for (int j = 1; j < R; ++j) a[j] = CONJ ? cmulc(a[j], tw[q * j]) : cmul(a[j], tw[q * j]);
  }
}

// ----------------------------------------------------------------------------
// Shared-memory geometry of one plane.
template <typename R, int NX, int NY, int NTT>
struct PlaneGeo {
  using C = typename CplxOf<R>::type;
  static constexpr int NT = NTT;
  AxisT<NX> ax;
  AxisT<NY> ay;
  int nx, ny, nxh, npair, pp;
  int gpair;   // row-pair stride of the global (transposed) real layout
  int srs;     // row stride of the global half spectrum (complex)
  int kym, kya;  // local spectrum row j holds ky = kym * j + kya
  __device__ __forceinline__ PlaneGeo(const GridDesc& g)
      : ax(g.nx, g.rx1, g.rx2), ay(g.ny, g.ry1, g.ry2) {
    nx = NX ? NX : g.nx;
    ny = NY ? NY : g.ny;
    nxh = nx / 2 + 1;
    npair = ny / 2;
    gpair = npair;
    pp = NX ? row_pitch(NX) : g.pp;
    srs = nxh;
    kym = 1;
    kya = 0;
  }
  // x rows: transform t = row pair, element e = x (padded)
  __device__ __forceinline__ int row(int t, int e) const { return t * pp + swz(e); }
  // y columns: transform t = kx, element e = y position
  __device__ __forceinline__ int col(int t, int e) const {
    return (e >> 1) * pp + (e & 1) * nxh + t;
  }
  // The same positions for the elements a stage touches: e = n1 + r1*j of a
  // stage-A task (n1 < r1), e = i + r1*b of a stage-B task (i < r1), with j
  // and i unrolled.  When r1 divides 16 (rows) or is even (columns) -- every
  // specialised edge but 48 -- the position is a per-task base plus a
  // compile-time offset, since n1 or i cannot carry into the pad term
  // (r1*j mod 16 <= 16 - r1) or the row-pair index; the shared-memory
  // accesses then need no address arithmetic per element.
  static constexpr int XR1 = NX ? AxisT<NX>::R1_ : 0;
  static constexpr int YR1 = NY ? AxisT<NY>::R1_ : 0;
  static constexpr bool kRowFast = XR1 > 0 && 16 % (XR1 > 0 ? XR1 : 1) == 0;
  static constexpr bool kColFast = YR1 > 0 && YR1 % 2 == 0;
  __device__ __forceinline__ int rowA(int t, int n1, int j) const {
    if constexpr (kRowFast) return (t * pp + n1) + (XR1 * j + ((XR1 * j) >> 4));
    else return row(t, n1 + ax.r1 * j);
  }
  __device__ __forceinline__ int rowB(int t, int b, int i) const {
    if constexpr (kRowFast) return (t * pp + XR1 * b + ((XR1 * b) >> 4)) + i;
    else return row(t, i + ax.r1 * b);
  }
  __device__ __forceinline__ int colA(int t, int n1, int j) const {
    if constexpr (kColFast) return ((n1 >> 1) * pp + (n1 & 1) * nxh + t) + (YR1 / 2) * j * pp;
    else return col(t, n1 + ay.r1 * j);
  }
  __device__ __forceinline__ int colB(int t, int b, int i) const {
    if constexpr (kColFast) return ((YR1 / 2) * b * pp + t) + ((i >> 1) * pp + (i & 1) * nxh);
    else return col(t, i + ay.r1 * b);
  }
};

// ---- x stages (rows), all in shared memory except the fused ends ------------
// Forward stage A with the global load fused in: element x of row pair t is
// the pair (psi[y=2t][x], psi[y=2t+1][x]) = src[x * npair + t] (transposed
// layout), times the factor pair f[x * npair + t].
template <int R2, typename R, int NX, int NY, int NTT, typename C>
__device__ __forceinline__ void xA_fwd_global_r(const PlaneGeo<R, NX, NY, NTT>& G, C* sm,
                                                const C* __restrict__ src,
                                                const C* __restrict__ f, const C* tw) {
  constexpr int NT = PlaneGeo<R, NX, NY, NTT>::NT;
  for_tasks<NT>(G.npair, G.ax.r1, [&](int t, int n1) {
    C a[R2];
#pragma unroll
    for (int j = 0; j < R2; ++j) {
      const int x = n1 + G.ax.r1 * j;
      a[j] = src[x * G.gpair + t];
      if (f) a[j] = cmulri(a[j], __ldg(&f[x * G.gpair + t]));
    }
    Dft<R2, -1, C>::run(a);
    if (G.ax.r1 > 1) {   // (the two-table twiddles measured slower here)
#pragma unroll
      for (int j = 1; j < R2; ++j) a[j] = cmul(a[j], tw[n1 * j]);
    }
#pragma unroll
    for (int j = 0; j < R2; ++j) sm[G.rowA(t, n1, j)] = a[j];
  });
}
template <typename R, int NX, int NY, int NTT, typename C>
__device__ __forceinline__ void xA_fwd_global(const PlaneGeo<R, NX, NY, NTT>& G, C* sm,
                                              const C* __restrict__ src,
                                              const C* __restrict__ f, const C* tw) {
  ITP_WITH_RADIX(G.ax.r2, xA_fwd_global_r, G, sm, src, f, tw)
}

// Stage B (DIR = -1 forward, +1 inverse with the conjugate twiddle after).
template <int R1, int DIR, typename R, int NX, int NY, int NTT, typename C>
__device__ __forceinline__ void xB_r(const PlaneGeo<R, NX, NY, NTT>& G, C* sm, const C* tw) {
  constexpr int NT = PlaneGeo<R, NX, NY, NTT>::NT;
  for_tasks<NT>(G.npair, G.ax.r2, [&](int t, int b) {
    C a[R1];
#pragma unroll
    for (int i = 0; i < R1; ++i) a[i] = sm[G.rowB(t, b, i)];
    Dft<R1, DIR, C>::run(a);
    if (DIR > 0) {
#pragma unroll
      for (int i = 1; i < R1; ++i) a[i] = cmulc(a[i], tw[i * b]);
    }
#pragma unroll
    for (int i = 0; i < R1; ++i) sm[G.rowB(t, b, i)] = a[i];
  });
}
template <int R1, typename G_, typename C>
__device__ __forceinline__ void xB_fwd_r(const G_& G, C* sm, const C* tw) { xB_r<R1, -1>(G, sm, tw); }
template <int R1, typename G_, typename C>
__device__ __forceinline__ void xB_inv_r(const G_& G, C* sm, const C* tw) { xB_r<R1, 1>(G, sm, tw); }
template <int DIR, typename R, int NX, int NY, int NTT, typename C>
__device__ __forceinline__ void xB(const PlaneGeo<R, NX, NY, NTT>& G, C* sm, const C* tw) {
  if (G.ax.r1 == 1) return;
  if (DIR < 0) {
    ITP_WITH_RADIX(G.ax.r1, xB_fwd_r, G, sm, tw)
  } else {
    ITP_WITH_RADIX(G.ax.r1, xB_inv_r, G, sm, tw)
  }
}

// Inverse stage A' followed by an epilogue on the natural-order row data:
// epi.apply<R2>(t, n1, a) receives a[j] = element x = n1 + r1*j of row pair
// t and either stores it somewhere (returns false) or transforms it and asks
// for the forward stage A to follow in registers (returns true).
template <int R2, typename R, int NX, int NY, int NTT, typename C, typename Epi>
__device__ __forceinline__ void xA_inv_then_r(const PlaneGeo<R, NX, NY, NTT>& G, C* sm, const C* tw,
                                              const Epi& epi) {
  constexpr int NT = PlaneGeo<R, NX, NY, NTT>::NT;
  for_tasks<NT>(G.npair, G.ax.r1, [&](int t, int n1) {
    C a[R2];
#pragma unroll
    for (int j = 0; j < R2; ++j) a[j] = sm[G.rowA(t, n1, j)];
    Dft<R2, 1, C>::run(a);
    if (epi.template apply<R2>(t, n1, a)) {
      Dft<R2, -1, C>::run(a);
      if (G.ax.r1 > 1) twiddle_stage<R2>(a, tw, n1);
#pragma unroll
      for (int j = 0; j < R2; ++j) sm[G.rowA(t, n1, j)] = a[j];
    }
  });
}
template <typename R, int NX, int NY, int NTT, typename C, typename Epi>
__device__ __forceinline__ void xA_inv_then(const PlaneGeo<R, NX, NY, NTT>& G, C* sm, const C* tw,
                                            const Epi& epi) {
  ITP_WITH_RADIX(G.ax.r2, xA_inv_then_r, G, sm, tw, epi)
}

// Real transform along x, forward: split the spectrum Z of each packed row
// (a + i b) into A = FFT(a), B = FFT(b), k = 0..nx/2.  One warp per row
// pair; Z is read in digit-swapped order.
template <typename R, int NX, int NY, int NTT>
__device__ __forceinline__ void x_split(const PlaneGeo<R, NX, NY, NTT>& G, typename CplxOf<R>::type* sm) {
  using C = typename CplxOf<R>::type;
  constexpr int MAXQ = NX ? (NX / 2 + 32) / 32 : 5;
  constexpr int NW = PlaneGeo<R, NX, NY, NTT>::NT / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int half = G.nx >> 1;
  const Axis ax{G.ax.L, G.ax.r1, G.ax.r2};
  if (warp >= NW) return;
  for (int r = warp; r < G.npair; r += NW) {
    C* row = sm + r * G.pp;
    C zp[MAXQ], zm[MAXQ];
#pragma unroll
    for (int q = 0; q < MAXQ; ++q) {
      const int k = lane + 32 * q;
      if (k <= half) {
        zp[q] = row[swz(spec_pos(ax, k))];
        zm[q] = row[swz(spec_pos(ax, k == 0 ? 0 : G.nx - k))];
      }
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < MAXQ; ++q) {
      const int k = lane + 32 * q;
      if (k <= half) {
        C A, B;
        A.x = (R)0.5 * (zp[q].x + zm[q].x);
        A.y = (R)0.5 * (zp[q].y - zm[q].y);
        B.x = (R)0.5 * (zp[q].y + zm[q].y);
        B.y = (R)0.5 * (zm[q].x - zp[q].x);
        row[k] = A;
        row[G.nxh + k] = B;
      }
    }
    __syncwarp();
  }
}

// Inverse of x_split (Hermitian extension; the imaginary parts of the
// self-conjugate bins k = 0, nx/2 are dropped, as a complex-to-real
// transform does), writing Z in digit-swapped order.
template <typename R, int NX, int NY, int NTT>
__device__ __forceinline__ void x_merge(const PlaneGeo<R, NX, NY, NTT>& G, typename CplxOf<R>::type* sm) {
  using C = typename CplxOf<R>::type;
  constexpr int MAXQ = NX ? (NX / 2 + 32) / 32 : 5;
  constexpr int NW = PlaneGeo<R, NX, NY, NTT>::NT / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int half = G.nx >> 1;
  const Axis ax{G.ax.L, G.ax.r1, G.ax.r2};
  if (warp >= NW) return;
  for (int r = warp; r < G.npair; r += NW) {
    C* row = sm + r * G.pp;
    C av[MAXQ], bv[MAXQ];
#pragma unroll
    for (int q = 0; q < MAXQ; ++q) {
      const int k = lane + 32 * q;
      if (k <= half) {
        av[q] = row[k];
        bv[q] = row[G.nxh + k];
      }
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < MAXQ; ++q) {
      const int k = lane + 32 * q;
      if (k <= half) {
        C A = av[q], B = bv[q];
        if (k == 0 || k == half) { A.y = 0; B.y = 0; }
        C Z;
        Z.x = A.x - B.y;
        Z.y = A.y + B.x;
        row[swz(spec_pos(ax, k))] = Z;
        if (k > 0 && k < half) {
          C Zm;
          Zm.x = A.x + B.y;
          Zm.y = B.x - A.y;
          row[swz(spec_pos(ax, G.nx - k))] = Zm;
        }
      }
    }
    __syncwarp();
  }
}

// ---- stage B of the x transform fused with the real-FFT split / merge --------
// One row pair per group of r2 lanes (32 / r2 rows per warp): lane b owns the
// frequencies k = b + r2*k1 (k1 < r1) of its row, which are exactly the
// outputs of its forward stage-B task; the partner frequencies nx - k sit in
// lane (r2 - b) % r2 of the same group and arrive by warp shuffles.
template <int R1, typename R, int NX, int NY, int NTT, typename C>
__device__ __forceinline__ void xB_fwd_split_r(const PlaneGeo<R, NX, NY, NTT>& G, C* sm) {
  constexpr int NW = PlaneGeo<R, NX, NY, NTT>::NT / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (warp >= NW) return;
  const int r2 = G.ax.r2, rpw = 32 / r2;
  const int grp = lane / r2, b = lane - grp * r2;
  const int ngroups = (G.npair + rpw - 1) / rpw;
  const int src = grp * r2 + (r2 - b) % r2;
  const int half = G.nx >> 1;
  for (int rg = warp; rg < ngroups; rg += NW) {
    const int t = rg * rpw + grp;
    const bool active = grp < rpw && t < G.npair;
    C* row = sm + (active ? t : 0) * G.pp;
    C a[R1];
#pragma unroll
    for (int i = 0; i < R1; ++i) a[i] = active ? sm[G.rowB(active ? t : 0, b, i)] : C{0, 0};
    Dft<R1, -1, C>::run(a);   // a[k1] = Z[b + r2*k1]
    C zm[R1];
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
      // the receiver wants Z[nx - k]; its sender (lane src) holds it at index
      // (R1 - k1) % R1 when b == 0 and R1 - 1 - k1 otherwise
      const C mine = (b == 0) ? a[(R1 - k1) % R1] : a[R1 - 1 - k1];
      zm[k1].x = __shfl_sync(0xffffffffu, mine.x, src);
      zm[k1].y = __shfl_sync(0xffffffffu, mine.y, src);
    }
    __syncwarp();
    if (active) {
#pragma unroll
      for (int k1 = 0; k1 < R1; ++k1) {
        const int k = b + r2 * k1;
        if (k <= half) {
          C A, B;
          A.x = (R)0.5 * (a[k1].x + zm[k1].x);
          A.y = (R)0.5 * (a[k1].y - zm[k1].y);
          B.x = (R)0.5 * (a[k1].y + zm[k1].y);
          B.y = (R)0.5 * (zm[k1].x - a[k1].x);
          row[k] = A;
          row[G.nxh + k] = B;
        }
      }
    }
    __syncwarp();
  }
}

// Inverse: each lane builds its stage-B' inputs Z[b + r2*a] (a < r1) from
// the half-spectrum rows A, B (Hermitian extension, imaginary parts of the
// self-conjugate bins dropped), the row's lanes synchronise, then stage B'.
template <int R1, typename R, int NX, int NY, int NTT, typename C>
__device__ __forceinline__ void xB_inv_merge_r(const PlaneGeo<R, NX, NY, NTT>& G, C* sm, const C* tw) {
  constexpr int NW = PlaneGeo<R, NX, NY, NTT>::NT / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (warp >= NW) return;
  const int r2 = G.ax.r2, rpw = 32 / r2;
  const int grp = lane / r2, b = lane - grp * r2;
  const int ngroups = (G.npair + rpw - 1) / rpw;
  const int half = G.nx >> 1;
  // the twiddles w^{-i b} depend on the lane only: for R1 <= 8 they are
  // loaded once into registers, not per row group (the row loop writes the
  // same shared array, so the compiler reloads them); at R1 = 16 the 30 more
  // registers would spill
  constexpr bool kHold = R1 <= 8;
  C twr[kHold ? R1 : 1];
  if constexpr (kHold) {
#pragma unroll
    for (int i = 1; i < R1; ++i) twr[i] = tw[i * b];
  }
  for (int rg = warp; rg < ngroups; rg += NW) {
    const int t = rg * rpw + grp;
    const bool active = grp < rpw && t < G.npair;
    C* row = sm + (active ? t : 0) * G.pp;
    C v[R1];
#pragma unroll
    for (int i = 0; i < R1; ++i) {
      const int k = b + r2 * i;
      C z = C{0, 0};
      if (active) {
        if (k <= half) {
          C A = row[k], B = row[G.nxh + k];
          if (k == 0 || k == half) { A.y = 0; B.y = 0; }
          z.x = A.x - B.y;
          z.y = A.y + B.x;
        } else {
          const C A = row[G.nx - k], B = row[G.nxh + G.nx - k];
          z.x = A.x + B.y;
          z.y = B.x - A.y;
        }
      }
      v[i] = z;
    }
    __syncwarp();
    Dft<R1, 1, C>::run(v);
    if (R1 > 1) {
#pragma unroll
      for (int i = 1; i < R1; ++i) {
        if constexpr (kHold) v[i] = cmulc(v[i], twr[i]);
        else v[i] = cmulc(v[i], tw[i * b]);
      }
    }
    if (active) {
#pragma unroll
      for (int i = 0; i < R1; ++i) sm[G.rowB(t, b, i)] = v[i];
    }
    __syncwarp();
  }
}

template <typename R, int NX, int NY, int NTT, typename C>
__device__ __forceinline__ void xB_fwd_split(const PlaneGeo<R, NX, NY, NTT>& G, C* sm, const C* tw) {
  if (G.ax.r1 == 1 || G.ax.r2 > 32) {   // single-stage rows: split on its own
    x_split(G, sm);
    return;
  }
  ITP_WITH_RADIX(G.ax.r1, xB_fwd_split_r, G, sm)
}
template <typename R, int NX, int NY, int NTT, typename C>
__device__ __forceinline__ void xB_inv_merge(const PlaneGeo<R, NX, NY, NTT>& G, C* sm, const C* tw) {
  if (G.ax.r1 == 1 || G.ax.r2 > 32) {
    x_merge(G, sm);
    __syncthreads();
    xB<1>(G, sm, tw);
    return;
  }
  ITP_WITH_RADIX(G.ax.r1, xB_inv_merge_r, G, sm, tw)
}

// ---- y stages (columns) -------------------------------------------------------
// Inverse stage B' with the global load fused in: column t, block b reads
// the frequencies ky = b + r2*a (a < r1) straight from the half spectrum.
template <int R1, typename R, int NX, int NY, int NTT, typename C>
__device__ __forceinline__ void yB_inv_global_r(const PlaneGeo<R, NX, NY, NTT>& G, C* sm,
                                                const C* __restrict__ spec, const C* tw) {
  constexpr int NT = PlaneGeo<R, NX, NY, NTT>::NT;
  for_tasks<NT>(G.nxh, G.ay.r2, [&](int t, int b) {
    C a[R1];
#pragma unroll
    for (int i = 0; i < R1; ++i) a[i] = spec[(b + G.ay.r2 * i) * G.srs + t];
    Dft<R1, 1, C>::run(a);
    if (R1 > 1) twiddle_stage<R1, true>(a, tw, b);
#pragma unroll
    for (int i = 0; i < R1; ++i) sm[G.colB(t, b, i)] = a[i];
  });
}
template <typename R, int NX, int NY, int NTT, typename C>
__device__ __forceinline__ void yB_inv_global(const PlaneGeo<R, NX, NY, NTT>& G, C* sm,
                                              const C* __restrict__ spec, const C* tw) {
  ITP_WITH_RADIX(G.ay.r1, yB_inv_global_r, G, sm, spec, tw)
}

// Stage A on columns (DIR = -1 forward with twiddle after; +1 inverse).
template <int R2, int DIR, typename R, int NX, int NY, int NTT, typename C>
__device__ __forceinline__ void yA_r(const PlaneGeo<R, NX, NY, NTT>& G, C* sm, const C* tw) {
  constexpr int NT = PlaneGeo<R, NX, NY, NTT>::NT;
  for_tasks<NT>(G.nxh, G.ay.r1, [&](int t, int n1) {
    C a[R2];
#pragma unroll
    for (int j = 0; j < R2; ++j) a[j] = sm[G.colA(t, n1, j)];
    Dft<R2, DIR, C>::run(a);
    if (DIR < 0 && G.ay.r1 > 1) twiddle_stage<R2>(a, tw, n1);
#pragma unroll
    for (int j = 0; j < R2; ++j) sm[G.colA(t, n1, j)] = a[j];
  });
}
template <int R2, typename G_, typename C>
__device__ __forceinline__ void yA_fwd_r(const G_& G, C* sm, const C* tw) { yA_r<R2, -1>(G, sm, tw); }
template <int R2, typename G_, typename C>
__device__ __forceinline__ void yA_inv_r(const G_& G, C* sm, const C* tw) { yA_r<R2, 1>(G, sm, tw); }
template <int DIR, typename R, int NX, int NY, int NTT, typename C>
__device__ __forceinline__ void yA(const PlaneGeo<R, NX, NY, NTT>& G, C* sm, const C* tw) {
  if (DIR < 0) {
    ITP_WITH_RADIX(G.ay.r2, yA_fwd_r, G, sm, tw)
  } else {
    ITP_WITH_RADIX(G.ay.r2, yA_inv_r, G, sm, tw)
  }
}

// Forward stage B with the global store fused in: column t, block b writes
// the frequencies ky = b + r2*k1 to the half spectrum.
// Kinetic factor of frequency (kx, ky) for planar grids (see KinFac).
template <typename R>
__device__ __forceinline__ R kin_factor(const KinFac<R>& k, int kx, int ky) {
  return k.mode == 0 ? k.fx[kx] * k.fy[ky] * k.fz[0] : (k.fx[kx] + k.fy[ky] + k.fz[0]) * k.scale;
}

template <int R1, typename R, int NX, int NY, int NTT, typename C>
__device__ __forceinline__ void yB_fwd_global_r(const PlaneGeo<R, NX, NY, NTT>& G, C* sm,
                                                C* __restrict__ spec, const KinFac<R>& kin) {
  constexpr int NT = PlaneGeo<R, NX, NY, NTT>::NT;
  for_tasks<NT>(G.nxh, G.ay.r2, [&](int t, int b) {
    C a[R1];
#pragma unroll
    for (int i = 0; i < R1; ++i) a[i] = sm[G.colB(t, b, i)];
    Dft<R1, -1, C>::run(a);
    if (kin.fx) {
#pragma unroll
      for (int k1 = 0; k1 < R1; ++k1) a[k1] = cscale(a[k1], kin_factor(kin, t, (b + G.ay.r2 * k1) * G.kym + G.kya));
    }
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) spec[(b + G.ay.r2 * k1) * G.srs + t] = a[k1];
  });
}
template <typename R, int NX, int NY, int NTT, typename C>
__device__ __forceinline__ void yB_fwd_global(const PlaneGeo<R, NX, NY, NTT>& G, C* sm,
                                              C* __restrict__ spec, const KinFac<R>& kin) {
  ITP_WITH_RADIX(G.ay.r1, yB_fwd_global_r, G, sm, spec, kin)
}

// ---- epilogues of the inverse x transform -------------------------------------
// PLANE_MERGED: multiply by exp(-tau_i V) (pairs in the transposed layout)
// and continue with the forward stage A.
template <typename R>
struct EpiMerged {
  using C = typename CplxOf<R>::type;
  const C* f;
  int npair, r1;
  template <int R2> __device__ __forceinline__ bool apply(int t, int n1, C* a) const {
#pragma unroll
    for (int j = 0; j < R2; ++j) a[j] = cmulri(a[j], __ldg(&f[(n1 + r1 * j) * npair + t]));
    return true;
  }
};
// PLANE_COMBINE: acc (=|+=) c * f_out * u in FP64; with phi set, the
// finished sum goes to phi in precision R instead of back to acc.
template <typename R>
struct EpiCombine {
  using C = typename CplxOf<R>::type;
  const C* f;
  double2* acc;
  C* phi;
  double c;
  int init, npair, r1;
  template <int R2> __device__ __forceinline__ bool apply(int t, int n1, C* a) const {
#pragma unroll
    for (int j = 0; j < R2; ++j) {
      const int idx = (n1 + r1 * j) * npair + t;
      const C u = cmulri(a[j], __ldg(&f[idx]));
      double2 v;
      v.x = c * (double)u.x;
      v.y = c * (double)u.y;
      if (!init) {
        const double2 o = acc[idx];
        v.x += o.x;
        v.y += o.y;
      }
      if (phi) {
        C w;
        w.x = (R)v.x;
        w.y = (R)v.y;
        phi[idx] = w;
      } else {
        acc[idx] = v;
      }
    }
    return false;
  }
};
// PLANE_COMBINE on planes that need split passes, mixed path: the running
// sum is an unevaluated pair (s, e) of FP32 values per point kept in the
// accumulator buffer and updated with the error-free TwoSum (Knuth), so the
// sum of the terms' FP32 contributions stays exact up to its final rounding.
__device__ __forceinline__ void two_sum_acc(float& s, float& e, float x) {
  const float t = s + x;
  const float bb = t - s;
  e += (s - (t - bb)) + (x - bb);
  s = t;
}
template <typename R>
struct EpiCombinePair {
  using C = typename CplxOf<R>::type;
  const C* f;
  float4* acc;   // per real pair: (s_re, e_re, s_im, e_im)
  C* phi;
  float c;
  int init, npair, r1;
  template <int R2> __device__ __forceinline__ bool apply(int t, int n1, C* a) const {
#pragma unroll
    for (int j = 0; j < R2; ++j) {
      const int idx = (n1 + r1 * j) * npair + t;
      const C fv = __ldg(&f[idx]);
      const float vx = c * ((float)a[j].x * (float)fv.x);
      const float vy = c * ((float)a[j].y * (float)fv.y);
      float4 q = init ? make_float4(0.f, 0.f, 0.f, 0.f) : acc[idx];
      two_sum_acc(q.x, q.y, vx);
      two_sum_acc(q.z, q.w, vy);
      if (phi) {
        C w;
        w.x = (R)(q.x + q.y);
        w.y = (R)(q.z + q.w);
        phi[idx] = w;
      } else {
        acc[idx] = q;
      }
    }
    return false;
  }
};

// PLANE_TERM: the term's scaled contribution c * f_out * u, rounded to
// precision R, written over the term's own spectrum plane (its real plane
// fits in the half-spectrum plane; all of the plane was read before).
template <typename R>
struct EpiTerm {
  using C = typename CplxOf<R>::type;
  const C* f;
  C* out;
  R c;   // c_i rounded to R: the term is an R value anyway
  int npair, r1;
  template <int R2> __device__ __forceinline__ bool apply(int t, int n1, C* a) const {
#pragma unroll
    for (int j = 0; j < R2; ++j) {
      const int idx = (n1 + r1 * j) * npair + t;
      const C fv = __ldg(&f[idx]);
      C w;
      w.x = c * (a[j].x * fv.x);
      w.y = c * (a[j].y * fv.y);
      out[idx] = w;
    }
    return false;
  }
};

// PLANE_HPSI: out = u + V * psi.  FP32 passes (the mixed path, whose
// subspace matrix is formed from FP32 data) write FP32 to outr with the FP32
// potential; FP64 passes write FP64 to out.  The choice is made at compile
// time: a run-time branch let the compiler predicate the FP64 arm, whose
// instructions then still occupied GB300's narrow FP64 pipe.
template <typename R>
struct EpiHpsi {
  using C = typename CplxOf<R>::type;
  const C* psi;
  const double2* V;
  double2* out;
  const C* Vr;
  C* outr;
  int npair, r1;
  template <int R2> __device__ __forceinline__ bool apply(int t, int n1, C* a) const {
#pragma unroll
    for (int j = 0; j < R2; ++j) {
      const int idx = (n1 + r1 * j) * npair + t;
      const C q = psi[idx];
      if constexpr (sizeof(R) == 4) {
        const C v = __ldg(&Vr[idx]);
        C h;
        h.x = a[j].x + v.x * q.x;
        h.y = a[j].y + v.y * q.y;
        outr[idx] = h;
      } else {
        const double2 v = __ldg(&V[idx]);
        double2 h;
        h.x = (double)a[j].x + v.x * (double)q.x;
        h.y = (double)a[j].y + v.y * (double)q.y;
        out[idx] = h;
      }
    }
    return false;
  }
};

// One plane pass over plane z of state s (the whole-plane kernels below
// take z, s from the grid; the grouped kernel from a table of rows).
template <typename R, int NX, int NY, int MODE>
__device__ __forceinline__ void plane_body(const GridDesc& g, const PlaneArgs<R>& a, int z,
                                           int s) {
  using C = typename CplxOf<R>::type;
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int NTT = kThreads;
  const PlaneGeo<R, NX, NY, NTT> G(g);
  C* sm = reinterpret_cast<C*>(smraw);
  C* twx = sm + G.npair * G.pp;   // nx roots
  C* twy = twx + G.nx;            // ny roots
  for (int i = threadIdx.x; i < G.nx; i += blockDim.x) twx[i] = static_cast<const C*>(a.twx)[i];
  for (int i = threadIdx.x; i < G.ny; i += blockDim.x) twy[i] = static_cast<const C*>(a.twy)[i];

  const long long plane_pts = (long long)G.nx * G.ny;
  const long long real_off = (long long)s * g.n_points + (long long)z * plane_pts;
  const long long spec_off = ((long long)s * g.nz + z) * (long long)G.ny * G.nxh;
  const long long fac_off = (long long)z * plane_pts;
  __syncthreads();

  if constexpr (MODE == PLANE_FWD_REAL) {
    const C* src = reinterpret_cast<const C*>(a.in_real + real_off);
    const C* f = a.f_in ? reinterpret_cast<const C*>(a.f_in + fac_off) : nullptr;
    xA_fwd_global(G, sm, src, f, twx);
    __syncthreads();
  } else {
    const C* spec = static_cast<const C*>(a.spec) + spec_off;
    yB_inv_global(G, sm, spec, twy);
    __syncthreads();
    yA<1>(G, sm, twy);
    __syncthreads();
    xB_inv_merge(G, sm, twx);
    __syncthreads();
    if constexpr (MODE == PLANE_MERGED) {
      EpiMerged<R> epi{reinterpret_cast<const C*>(a.f_mid + fac_off), G.npair, G.ax.r1};
      xA_inv_then(G, sm, twx, epi);
      __syncthreads();
    } else if constexpr (MODE == PLANE_TERM) {
      EpiTerm<R> epi{reinterpret_cast<const C*>(a.f_out + fac_off),
                     static_cast<C*>(a.spec) + spec_off, (R)a.coef, G.npair, G.ax.r1};
      xA_inv_then(G, sm, twx, epi);
      return;
    } else if constexpr (MODE == PLANE_COMBINE) {
      EpiCombine<R> epi{reinterpret_cast<const C*>(a.f_out + fac_off),
                        reinterpret_cast<double2*>(a.acc + real_off),
                        a.phi_out ? reinterpret_cast<C*>(a.phi_out + real_off) : nullptr,
                        a.coef, a.acc_init, G.npair, G.ax.r1};
      xA_inv_then(G, sm, twx, epi);
      return;
    } else {
      EpiHpsi<R> epi{reinterpret_cast<const C*>(a.in_real + real_off),
                     reinterpret_cast<const double2*>(a.V + fac_off),
                     reinterpret_cast<double2*>(a.acc + real_off),
                     a.V_r ? reinterpret_cast<const C*>(a.V_r + fac_off) : nullptr,
                     a.phi_out ? reinterpret_cast<C*>(a.phi_out + real_off) : nullptr,
                     G.npair, G.ax.r1};
      xA_inv_then(G, sm, twx, epi);
      return;
    }
  }
  // forward x (stage B fused with the split), forward y
  xB_fwd_split(G, sm, twx);
  __syncthreads();
  yA<-1>(G, sm, twy);
  __syncthreads();
  yB_fwd_global(G, sm, static_cast<C*>(a.spec) + spec_off, a.kin);
}

template <typename R, int NX, int NY, int MODE>
__global__ void __launch_bounds__(launch_threads(kThreads),
                                  min_blocks(plane_smem_ct(NX, NY, sizeof(R)),
                                             sizeof(R) == 4 ? 3 : 2))
    plane_kernel(const GridDesc g, const PlaneArgs<R> a) {
  plane_body<R, NX, NY, MODE>(g, a, blockIdx.x, blockIdx.y);
}

// Grouped plane pass: one launch over the states of several problems with
// the same grid (a batch of independent problems).  CTA row y of the grid
// is state rows[y].y of problem rows[y].x, whose arguments are args[rows[y].x].
template <typename R, int NX, int NY, int MODE>
__global__ void __launch_bounds__(launch_threads(kThreads),
                                  min_blocks(plane_smem_ct(NX, NY, sizeof(R)),
                                             sizeof(R) == 4 ? 3 : 2))
    plane_group_kernel(const GridDesc g, const PlaneArgs<R>* __restrict__ args,
                       const int2* __restrict__ rows) {
  const int2 r = rows[blockIdx.y];
  plane_body<R, NX, NY, MODE>(g, args[r.x], blockIdx.x, r.y);
}

// ----------------------------------------------------------------------------
// Pencil stages.  Slab element (z, column t) at shared position z * pw + t.
template <int M> struct mode_tag {};

// forward stage A, loads fused
template <int NT> struct nt_tag {};

template <int R2, typename C, int NT>
__device__ __forceinline__ void pencil_fwdA_r(nt_tag<NT>, C* sm, const C* __restrict__ base,
                                              const C* tw, long long zstride, int w, int pw,
                                              int r1) {
  for_tasks<NT>(pw, r1, [&](int t, int n1) {
    if (t >= w) return;
    C v[R2];
#pragma unroll
    for (int j = 0; j < R2; ++j) v[j] = base[(n1 + r1 * j) * zstride + t];
    Dft<R2, -1, C>::run(v);
    if (r1 > 1) {
#pragma unroll
      for (int j = 1; j < R2; ++j) v[j] = cmul(v[j], tw[n1 * j]);
    }
#pragma unroll
    for (int j = 0; j < R2; ++j) sm[(n1 + r1 * j) * pw + t] = v[j];
  });
}

// forward stage B, kinetic factor, inverse stage B' -- in registers
template <int R1, typename C, typename R, int MODE, int NT>
__device__ __forceinline__ void pencil_mid_r(nt_tag<NT>, C* sm, const C* tw,
                                             const R* __restrict__ kx_tab,
                                             const R* __restrict__ kz_tab, R fy, R scale, int w,
                                             int pw, int r2, int kx0, mode_tag<MODE>) {
  for_tasks<NT>(pw, r2, [&](int t, int b) {
    if (t >= w) return;
    C v[R1];
#pragma unroll
    for (int i = 0; i < R1; ++i) v[i] = sm[(i + R1 * b) * pw + t];
    Dft<R1, -1, C>::run(v);
    const R fx = __ldg(&kx_tab[kx0 + t]);
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
      const R fz = __ldg(&kz_tab[b + r2 * k1]);
      R f;
      if constexpr (MODE == PENCIL_PROPAGATE) f = fx * fy * fz;
      else f = (fx + fy + fz) * scale;
      v[k1] = cscale(v[k1], f);
    }
    Dft<R1, 1, C>::run(v);
    if (R1 > 1) {
#pragma unroll
      for (int i = 1; i < R1; ++i) v[i] = cmulc(v[i], tw[i * b]);
    }
#pragma unroll
    for (int i = 0; i < R1; ++i) sm[(i + R1 * b) * pw + t] = v[i];
  });
}

// inverse stage A', stores fused
template <int R2, typename C, int NT>
__device__ __forceinline__ void pencil_invA_r(nt_tag<NT>, const C* sm, C* __restrict__ base,
                                              long long zstride, int w, int pw, int r1) {
  for_tasks<NT>(pw, r1, [&](int t, int n1) {
    if (t >= w) return;
    C v[R2];
#pragma unroll
    for (int j = 0; j < R2; ++j) v[j] = sm[(n1 + r1 * j) * pw + t];
    Dft<R2, 1, C>::run(v);
#pragma unroll
    for (int j = 0; j < R2; ++j) base[(n1 + r1 * j) * zstride + t] = v[j];
  });
}

// ----------------------------------------------------------------------------
// 256 x 256 FP32 planes on a cluster of two CTAs (one HBM round trip per pass
// where the row + column passes below take three).  CTA r of the pair holds
// the real-space rows y = 128 r + n (n < 128) and the half-spectrum rows
// ky = 2 j + r (j < 128), each in the one-CTA layout with 64 row pairs.  The
// length-256 y transform is a radix-2 step across the pair plus local
// 128-point transforms:
//   forward  (decimation in frequency): X(2j)   = FFT128[x(n) + x(n+128)](j),
//                                       X(2j+1) = FFT128[(x(n) - x(n+128)) w^n](j);
//   inverse  (decimation in time):      x(n)     = E(n) + w^-n O(n),
//                                       x(n+128) = E(n) - w^-n O(n),
// E, O the inverse 128-point transforms of the even and odd rows, w = exp(-2 pi i/256).
// The radix-2 step reads the partner CTA's shared memory (distributed shared
// memory) in two halves: read the partner's values, cluster barrier, write
// the own values.
constexpr int kC2Threads = 512;

template <int DIR, typename G_>
__device__ __forceinline__ void c2_exchange(const G_& G, float2* sm, const float2* tw2,
                                            cg::cluster_group& cl, int rank) {
  constexpr int NT = G_::NT;
  const float2* psm = cl.map_shared_rank(sm, rank ^ 1);
  const int total = 128 * G.nxh;   // (n, t): 128 rows, nxh columns
  const int halfcnt = (total + 1) / 2;
  constexpr int MAXQ = (128 * 129 / 2 + 1 + NT - 1) / NT;
  cl.sync();   // the partner's local stage is complete
  for (int h = 0; h < 2; ++h) {
    const int e0 = h * halfcnt, e1 = min(total, e0 + halfcnt);
    float2 pv[MAXQ];
#pragma unroll
    for (int q = 0; q < MAXQ; ++q) {
      const int e = e0 + (int)threadIdx.x + NT * q;
      if (e < e1) {
        const int n = e / G.nxh, t = e - n * G.nxh;
        pv[q] = psm[G.col(t, n)];
      }
    }
    cl.sync();   // every remote read of this half is done before it is overwritten
#pragma unroll
    for (int q = 0; q < MAXQ; ++q) {
      const int e = e0 + (int)threadIdx.x + NT * q;
      if (e < e1) {
        const int n = e / G.nxh, t = e - n * G.nxh;
        const int pos = G.col(t, n);
        const float2 own = sm[pos];
        float2 r;
        if (DIR < 0) {   // forward: rank 0 x0 + x1, rank 1 (x0 - x1) w^n
          r = rank == 0 ? cadd(own, pv[q]) : cmul(csub(pv[q], own), tw2[n]);
        } else {         // inverse: rank 0 E + w^-n O, rank 1 E - w^-n O
          r = rank == 0 ? cadd(own, cmulc(pv[q], tw2[n])) : csub(pv[q], cmulc(own, tw2[n]));
        }
        sm[pos] = r;
      }
    }
  }
}

template <int MODE>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kC2Threads, 1)
    plane_c2_kernel(const GridDesc g, const PlaneArgs<float> a) {
  using R = float;
  using C = float2;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  extern __shared__ __align__(16) unsigned char smraw[];
  PlaneGeo<R, 256, 128, kC2Threads> G(g);
  G.gpair = 128;          // row pairs of the whole plane (global real layout)
  G.srs = 2 * G.nxh;      // this CTA's spectrum rows ky = 2 j + rank
  G.kym = 2;
  G.kya = rank;
  C* sm = reinterpret_cast<C*>(smraw);
  C* twx = sm + G.npair * G.pp;   // 256 roots
  C* twy = twx + 256;             // 128 roots of the local transforms: w^(2j)
  C* tw2 = twy + 128;             // w^n, n < 128, of the radix-2 step
  const C* tg = static_cast<const C*>(a.twy);
  for (int i = threadIdx.x; i < 256; i += blockDim.x) twx[i] = static_cast<const C*>(a.twx)[i];
  for (int i = threadIdx.x; i < 128; i += blockDim.x) {
    twy[i] = tg[2 * i];
    tw2[i] = tg[i];
  }
  const int z = blockIdx.x >> 1, s = blockIdx.y;
  const long long plane_pts = 256LL * 256;
  const long long real_off = (long long)s * g.n_points + (long long)z * plane_pts;
  const long long spec_off = ((long long)s * g.nz + z) * 256LL * G.nxh;
  const long long fac_off = (long long)z * plane_pts;
  const int t0 = 64 * rank;   // first (global) row pair of this CTA
  __syncthreads();

  if constexpr (MODE == PLANE_FWD_REAL) {
    const C* src = reinterpret_cast<const C*>(a.in_real + real_off) + t0;
    const C* f = a.f_in ? reinterpret_cast<const C*>(a.f_in + fac_off) + t0 : nullptr;
    xA_fwd_global(G, sm, src, f, twx);
    __syncthreads();
  } else {
    yB_inv_global(G, sm, static_cast<const C*>(a.spec) + spec_off + rank * G.nxh, twy);
    __syncthreads();
    yA<1>(G, sm, twy);
    __syncthreads();
    c2_exchange<1>(G, sm, tw2, cl, rank);
    __syncthreads();
    xB_inv_merge(G, sm, twx);
    __syncthreads();
    if constexpr (MODE == PLANE_MERGED) {
      EpiMerged<R> epi{reinterpret_cast<const C*>(a.f_mid + fac_off) + t0, G.gpair, G.ax.r1};
      xA_inv_then(G, sm, twx, epi);
      __syncthreads();
    } else if constexpr (MODE == PLANE_TERM) {
      EpiTerm<R> epi{reinterpret_cast<const C*>(a.f_out + fac_off) + t0,
                     static_cast<C*>(a.spec) + spec_off + t0, (R)a.coef, G.gpair, G.ax.r1};
      xA_inv_then(G, sm, twx, epi);
      return;
    } else if constexpr (MODE == PLANE_COMBINE) {
      EpiCombinePair<R> epi{reinterpret_cast<const C*>(a.f_out + fac_off) + t0,
                            reinterpret_cast<float4*>(a.acc + real_off) + t0,
                            a.phi_out ? reinterpret_cast<C*>(a.phi_out + real_off) + t0 : nullptr,
                            (float)a.coef, a.acc_init, G.gpair, G.ax.r1};
      xA_inv_then(G, sm, twx, epi);
      return;
    } else if constexpr (MODE == PLANE_HPSI) {
      EpiHpsi<R> epi{reinterpret_cast<const C*>(a.in_real + real_off) + t0,
                     reinterpret_cast<const double2*>(a.V + fac_off) + t0,
                     reinterpret_cast<double2*>(a.acc + real_off) + t0,
                     reinterpret_cast<const C*>(a.V_r + fac_off) + t0,
                     reinterpret_cast<C*>(a.phi_out + real_off) + t0, G.gpair, G.ax.r1};
      xA_inv_then(G, sm, twx, epi);
      return;
    } else {
      return;
    }
  }
  xB_fwd_split(G, sm, twx);
  __syncthreads();
  c2_exchange<-1>(G, sm, tw2, cl, rank);
  __syncthreads();
  yA<-1>(G, sm, twy);
  __syncthreads();
  yB_fwd_global(G, sm, static_cast<C*>(a.spec) + spec_off + rank * G.nxh, a.kin);
}

// The same planes on a cluster of four CTAs, each holding 64 real-space rows
// (y = 64 r + n) or the spectrum rows ky = 4 j + r, 75 KB of shared memory,
// so that three CTAs share an SM: a radix-4 step across the cluster plus
// local 64-point transforms,
//   forward:  X(4j+r) = FFT64[ w^(nr) sum_q x_q(n) (-i)^(qr) ](j),  x_q(n) = x(64q + n);
//   inverse:  x(64q+n) = sum_r i^(qr) w^(-nr) O_r(n),  O_r = IFFT64 of the rows 4j+r.
// The exchange reads all four CTAs' values of a chunk of elements, then a
// cluster barrier, then each CTA writes its own result for the chunk.
constexpr int kC4Threads = 256;

template <int DIR, typename G_>
__device__ __forceinline__ void c4_exchange(const G_& G, float2* sm, const float2* tw256,
                                            cg::cluster_group& cl, int rank) {
  constexpr int NT = G_::NT;
  constexpr int PER = 8;   // elements per thread and chunk
  const float2* rs[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) rs[q] = cl.map_shared_rank(sm, q);
  const int total = 64 * G.nxh;
  cl.sync();   // every CTA's local stage is complete
  for (int c0 = 0; c0 < total; c0 += NT * PER) {
    float2 v[PER][4];
#pragma unroll
    for (int p = 0; p < PER; ++p) {
      const int e = c0 + (int)threadIdx.x + NT * p;
      if (e < total) {
        const int n = e / G.nxh, t = e - n * G.nxh;
        const int pos = G.col(t, n);
#pragma unroll
        for (int q = 0; q < 4; ++q) v[p][q] = rs[q][pos];
      }
    }
    cl.sync();   // the chunk is read everywhere before any CTA overwrites it
#pragma unroll
    for (int p = 0; p < PER; ++p) {
      const int e = c0 + (int)threadIdx.x + NT * p;
      if (e < total) {
        const int n = e / G.nxh, t = e - n * G.nxh;
        float2 a0 = v[p][0], a1 = v[p][1], a2 = v[p][2], a3 = v[p][3];
        if (DIR > 0) {   // inverse: twiddle w^(-rn) first
          a1 = cmulc(a1, tw256[n]);
          a2 = cmulc(a2, tw256[2 * n]);
          a3 = cmulc(a3, tw256[3 * n]);
        }
        const float2 s02 = cadd(a0, a2), d02 = csub(a0, a2);
        const float2 s13 = cadd(a1, a3), d13 = csub(a1, a3);
        float2 r;
        // i*d = (-d.y, d.x), -i*d = (d.y, -d.x)
        const int k = DIR < 0 ? rank : (4 - rank) & 3;   // inverse uses i^(qr) = (-i)^(-qr)
        if (k == 0) r = cadd(s02, s13);
        else if (k == 2) r = csub(s02, s13);
        else if (k == 1) r = float2{d02.x + d13.y, d02.y - d13.x};
        else r = float2{d02.x - d13.y, d02.y + d13.x};
        if (DIR < 0 && rank > 0) r = cmul(r, tw256[rank * n]);
        sm[G.col(t, n)] = r;
      }
    }
  }
}

template <int MODE>
__global__ void __cluster_dims__(4, 1, 1) __launch_bounds__(kC4Threads, 3)
    plane_c4_kernel(const GridDesc g, const PlaneArgs<float> a) {
  using R = float;
  using C = float2;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  extern __shared__ __align__(16) unsigned char smraw[];
  PlaneGeo<R, 256, 64, kC4Threads> G(g);
  G.gpair = 128;
  G.srs = 4 * G.nxh;      // this CTA's spectrum rows ky = 4 j + rank
  G.kym = 4;
  G.kya = rank;
  C* sm = reinterpret_cast<C*>(smraw);
  C* twx = sm + G.npair * G.pp;   // 256 roots (x)
  C* twy = twx + 256;             // 64 roots of the local transforms: w^(4j)
  C* tw256 = twy + 64;            // 256 roots w^m of the radix-4 step
  const C* tg = static_cast<const C*>(a.twy);
  for (int i = threadIdx.x; i < 256; i += blockDim.x) {
    twx[i] = static_cast<const C*>(a.twx)[i];
    tw256[i] = tg[i];
  }
  for (int i = threadIdx.x; i < 64; i += blockDim.x) twy[i] = tg[4 * i];
  const int z = blockIdx.x >> 2, s = blockIdx.y;
  const long long plane_pts = 256LL * 256;
  const long long real_off = (long long)s * g.n_points + (long long)z * plane_pts;
  const long long spec_off = ((long long)s * g.nz + z) * 256LL * G.nxh;
  const long long fac_off = (long long)z * plane_pts;
  const int t0 = 32 * rank;   // first (global) row pair of this CTA
  __syncthreads();

  if constexpr (MODE == PLANE_FWD_REAL) {
    const C* src = reinterpret_cast<const C*>(a.in_real + real_off) + t0;
    const C* f = a.f_in ? reinterpret_cast<const C*>(a.f_in + fac_off) + t0 : nullptr;
    xA_fwd_global(G, sm, src, f, twx);
    __syncthreads();
  } else {
    yB_inv_global(G, sm, static_cast<const C*>(a.spec) + spec_off + rank * G.nxh, twy);
    __syncthreads();
    yA<1>(G, sm, twy);
    __syncthreads();
    c4_exchange<1>(G, sm, tw256, cl, rank);
    __syncthreads();
    xB_inv_merge(G, sm, twx);
    __syncthreads();
    if constexpr (MODE == PLANE_MERGED) {
      EpiMerged<R> epi{reinterpret_cast<const C*>(a.f_mid + fac_off) + t0, G.gpair, G.ax.r1};
      xA_inv_then(G, sm, twx, epi);
      __syncthreads();
    } else if constexpr (MODE == PLANE_TERM) {
      EpiTerm<R> epi{reinterpret_cast<const C*>(a.f_out + fac_off) + t0,
                     static_cast<C*>(a.spec) + spec_off + t0, (R)a.coef, G.gpair, G.ax.r1};
      xA_inv_then(G, sm, twx, epi);
      return;
    } else if constexpr (MODE == PLANE_COMBINE) {
      EpiCombinePair<R> epi{reinterpret_cast<const C*>(a.f_out + fac_off) + t0,
                            reinterpret_cast<float4*>(a.acc + real_off) + t0,
                            a.phi_out ? reinterpret_cast<C*>(a.phi_out + real_off) + t0 : nullptr,
                            (float)a.coef, a.acc_init, G.gpair, G.ax.r1};
      xA_inv_then(G, sm, twx, epi);
      return;
    } else if constexpr (MODE == PLANE_HPSI) {
      EpiHpsi<R> epi{reinterpret_cast<const C*>(a.in_real + real_off) + t0,
                     reinterpret_cast<const double2*>(a.V + fac_off) + t0,
                     reinterpret_cast<double2*>(a.acc + real_off) + t0,
                     reinterpret_cast<const C*>(a.V_r + fac_off) + t0,
                     reinterpret_cast<C*>(a.phi_out + real_off) + t0, G.gpair, G.ax.r1};
      xA_inv_then(G, sm, twx, epi);
      return;
    } else {
      return;
    }
  }
  xB_fwd_split(G, sm, twx);
  __syncthreads();
  c4_exchange<-1>(G, sm, tw256, cl, rank);
  __syncthreads();
  yA<-1>(G, sm, twy);
  __syncthreads();
  yB_fwd_global(G, sm, static_cast<C*>(a.spec) + spec_off + rank * G.nxh, a.kin);
}

// ----------------------------------------------------------------------------
// Split plane passes, for planes whose half spectrum does not fit one CTA's
// shared memory (nx = ny = 256 in FP32, >= 192 in FP64).  A row pass does
// the x transform (and the mode's point-wise epilogue) of a block of TB row
// pairs; column passes do the y transform.  Between them the data is kept
// in the half-spectrum layout [z][y][kx] with y not yet transformed.
template <typename R, int NX, int TB>
struct RowGeo : PlaneGeo<R, NX, 2 * TB, kThreads> {
  __device__ __forceinline__ RowGeo(const GridDesc& g) : PlaneGeo<R, NX, 2 * TB, kThreads>(g) {
    this->ny = 2 * TB;
    this->npair = TB;
    this->gpair = g.ny / 2;
  }
};

template <typename R, int NX, int TB, int MODE>
__global__ void __launch_bounds__(kThreads)
    rowpass_kernel(const GridDesc g, const PlaneArgs<R> a) {
  using C = typename CplxOf<R>::type;
  extern __shared__ __align__(16) unsigned char smraw[];
  const RowGeo<R, NX, TB> G(g);
  C* sm = reinterpret_cast<C*>(smraw);
  C* twx = sm + TB * G.pp;
  for (int i = threadIdx.x; i < G.nx; i += blockDim.x) twx[i] = static_cast<const C*>(a.twx)[i];
  const int nb = (g.ny / 2) / TB;   // TB divides ny / 2
  const int z = blockIdx.x / nb, blk = blockIdx.x - z * nb, s = blockIdx.y;
  const int t0 = blk * TB;
  const long long plane_pts = (long long)G.nx * g.ny;
  const long long real_off = (long long)s * g.n_points + (long long)z * plane_pts;
  const long long fac_off = (long long)z * plane_pts;
  C* specp = static_cast<C*>(a.spec) + ((long long)s * g.nz + z) * (long long)g.ny * G.nxh;
  const int rowlen = 2 * G.nxh;
  __syncthreads();

  if constexpr (MODE == PLANE_FWD_REAL) {
    const C* src = reinterpret_cast<const C*>(a.in_real + real_off) + t0;
    const C* f = a.f_in ? reinterpret_cast<const C*>(a.f_in + fac_off) + t0 : nullptr;
    xA_fwd_global(G, sm, src, f, twx);
    __syncthreads();
  } else {
    // rows y = 2(t0+t) + h of the y-inverted intermediate -> row pair t
    for (int idx = threadIdx.x; idx < TB * rowlen; idx += blockDim.x) {
      const int t = idx / rowlen, rem = idx - t * rowlen;
      sm[t * G.pp + rem] = specp[(long long)(2 * t0) * G.nxh + idx];
    }
    __syncthreads();
    xB_inv_merge(G, sm, twx);
    __syncthreads();
    if constexpr (MODE == PLANE_MERGED) {
      EpiMerged<R> epi{reinterpret_cast<const C*>(a.f_mid + fac_off) + t0, G.gpair, G.ax.r1};
      xA_inv_then(G, sm, twx, epi);
      __syncthreads();
    } else if constexpr (MODE == PLANE_COMBINE) {
      if constexpr (sizeof(R) == 4) {
        EpiCombinePair<R> epi{reinterpret_cast<const C*>(a.f_out + fac_off) + t0,
                              reinterpret_cast<float4*>(a.acc + real_off) + t0,
                              a.phi_out ? reinterpret_cast<C*>(a.phi_out + real_off) + t0 : nullptr,
                              (float)a.coef, a.acc_init, G.gpair, G.ax.r1};
        xA_inv_then(G, sm, twx, epi);
      } else {
        EpiCombine<R> epi{reinterpret_cast<const C*>(a.f_out + fac_off) + t0,
                          reinterpret_cast<double2*>(a.acc + real_off) + t0,
                          a.phi_out ? reinterpret_cast<C*>(a.phi_out + real_off) + t0 : nullptr,
                          a.coef, a.acc_init, G.gpair, G.ax.r1};
        xA_inv_then(G, sm, twx, epi);
      }
      return;
    } else if constexpr (MODE == PLANE_HPSI) {
      EpiHpsi<R> epi{reinterpret_cast<const C*>(a.in_real + real_off) + t0,
                     reinterpret_cast<const double2*>(a.V + fac_off) + t0,
                     reinterpret_cast<double2*>(a.acc + real_off) + t0,
                     a.V_r ? reinterpret_cast<const C*>(a.V_r + fac_off) + t0 : nullptr,
                     a.phi_out ? reinterpret_cast<C*>(a.phi_out + real_off) + t0 : nullptr,
                     G.gpair, G.ax.r1};
      xA_inv_then(G, sm, twx, epi);
      return;
    } else {
      return;   // PLANE_TERM is not used with split passes
    }
  }
  xB_fwd_split(G, sm, twx);
  __syncthreads();
  for (int idx = threadIdx.x; idx < TB * rowlen; idx += blockDim.x) {
    const int t = idx / rowlen, rem = idx - t * rowlen;
    specp[(long long)(2 * t0) * G.nxh + idx] = sm[t * G.pp + rem];
  }
}

// Column pass: the y transform of a block of kx columns of one plane (same
// slab structure as the pencil pass, along y).
template <int R1, typename C, int NT>
__device__ __forceinline__ void col_fwdB_store_r(nt_tag<NT>, const C* sm, C* __restrict__ base,
                                                 long long rstride, int w, int pw, int r2,
                                                 const KinFac<decltype(C{}.x)>& kin, int kx0) {
  for_tasks<NT>(pw, r2, [&](int t, int b) {
    if (t >= w) return;
    C v[R1];
#pragma unroll
    for (int i = 0; i < R1; ++i) v[i] = sm[(i + R1 * b) * pw + t];
    Dft<R1, -1, C>::run(v);
    if (kin.fx) {
#pragma unroll
      for (int k1 = 0; k1 < R1; ++k1) v[k1] = cscale(v[k1], kin_factor(kin, kx0 + t, b + r2 * k1));
    }
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) base[(b + r2 * k1) * rstride + t] = v[k1];
  });
}
template <int R1, typename C, int NT>
__device__ __forceinline__ void col_invB_load_r(nt_tag<NT>, C* sm, const C* __restrict__ base,
                                                const C* tw, long long rstride, int w, int pw,
                                                int r2) {
  for_tasks<NT>(pw, r2, [&](int t, int b) {
    if (t >= w) return;
    C v[R1];
#pragma unroll
    for (int i = 0; i < R1; ++i) v[i] = base[(b + r2 * i) * rstride + t];
    Dft<R1, 1, C>::run(v);
    if (R1 > 1) {
#pragma unroll
      for (int i = 1; i < R1; ++i) v[i] = cmulc(v[i], tw[i * b]);
    }
#pragma unroll
    for (int i = 0; i < R1; ++i) sm[(i + R1 * b) * pw + t] = v[i];
  });
}

template <typename R, int NY, int W, int DIR>
__global__ void __launch_bounds__(launch_threads(task_threads(W)))
    colpass_kernel(const GridDesc g, void* spec, const void* twy_g, int pw_rt,
                   const KinFac<R> kin) {
  constexpr int NT = task_threads(W);
  using C = typename CplxOf<R>::type;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  const AxisT<NY> ay(g.ny, g.ry1, g.ry2);
  const int ny = NY ? NY : g.ny;
  const int pw = W ? W : pw_rt;
  C* twy = sm + ny * pw;
  for (int i = threadIdx.x; i < ny; i += blockDim.x) twy[i] = static_cast<const C*>(twy_g)[i];
  const long long plane = blockIdx.y;
  const int kx0 = blockIdx.x * pw;
  const int w = min(pw, g.nxh - kx0);
  C* base = static_cast<C*>(spec) + plane * (long long)ny * g.nxh + kx0;
  __syncthreads();
  if constexpr (DIR < 0) {
    ITP_WITH_RADIX(ay.r2, pencil_fwdA_r, nt_tag<NT>(), sm, base, twy, (long long)g.nxh, w, pw,
                   ay.r1)
    __syncthreads();
    ITP_WITH_RADIX(ay.r1, col_fwdB_store_r, nt_tag<NT>(), sm, base, (long long)g.nxh, w, pw,
                   ay.r2, kin, kx0)
  } else {
    ITP_WITH_RADIX(ay.r1, col_invB_load_r, nt_tag<NT>(), sm, base, twy, (long long)g.nxh, w, pw,
                   ay.r2)
    __syncthreads();
    ITP_WITH_RADIX(ay.r2, pencil_invA_r, nt_tag<NT>(), sm, base, (long long)g.nxh, w, pw, ay.r1)
  }
}

// ----------------------------------------------------------------------------
// Pencil pass.  Slab element (z, column t) at shared position z * W + t.
template <typename R, int NZ, int W, int MODE>
__device__ __forceinline__ void pencil_body(const GridDesc& g, const PencilArgs<R>& a, int bx,
                                            int s) {
  constexpr int NT = task_threads(W);
  using C = typename CplxOf<R>::type;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  const AxisT<NZ> az(g.nz, g.rz1, g.rz2);
  const int nz = NZ ? NZ : g.nz;
  const int pw = W ? W : g.pencil_w;        // slab pitch = block width
  C* twz = sm + nz * pw;
  for (int i = threadIdx.x; i < nz; i += blockDim.x) twz[i] = static_cast<const C*>(a.twz)[i];
  const int ky = bx % g.ny, chunk = bx / g.ny;
  const int kx0 = chunk * pw;
  const int w = min(pw, g.nxh - kx0);
  const long long zstride = (long long)g.ny * g.nxh;
  C* base = static_cast<C*>(a.spec) + (long long)s * g.n_half + (long long)ky * g.nxh + kx0;
  const R fy = a.ky_tab[ky];
  __syncthreads();

  ITP_WITH_RADIX(az.r2, pencil_fwdA_r, nt_tag<NT>(), sm, base, twz, zstride, w, pw, az.r1)
  __syncthreads();
  ITP_WITH_RADIX(az.r1, pencil_mid_r, nt_tag<NT>(), sm, twz, a.kx_tab, a.kz_tab, fy, a.scale, w,
                 pw, az.r2, kx0, mode_tag<MODE>())
  __syncthreads();
  ITP_WITH_RADIX(az.r2, pencil_invA_r, nt_tag<NT>(), sm, base, zstride, w, pw, az.r1)
}

template <typename R, int NZ, int W, int MODE>
__global__ void __launch_bounds__(launch_threads(task_threads(W)),
                                  min_blocks(pencil_smem_ct(NZ, W, sizeof(R)),
                                             pencil_min_ctas(NZ, sizeof(R))))
    pencil_kernel(const GridDesc g, const PencilArgs<R> a) {
  pencil_body<R, NZ, W, MODE>(g, a, blockIdx.x, blockIdx.y);
}

// Grouped pencil pass (see plane_group_kernel).
template <typename R, int NZ, int W, int MODE>
__global__ void __launch_bounds__(launch_threads(task_threads(W)),
                                  min_blocks(pencil_smem_ct(NZ, W, sizeof(R)),
                                             pencil_min_ctas(NZ, sizeof(R))))
    pencil_group_kernel(const GridDesc g, const PencilArgs<R>* __restrict__ args,
                        const int2* __restrict__ rows) {
  const int2 r = rows[blockIdx.y];
  pencil_body<R, NZ, W, MODE>(g, args[r.x], blockIdx.x, r.y);
}

// ----------------------------------------------------------------------------
template <typename R>
__global__ void term_tables_kernel(const GridDesc g, const double* __restrict__ V, double tau_i,
                                   double lx, double ly, double lz, R* f_half, R* f_full,
                                   R* kx, R* ky, R* kz, int kinetic_only) {
  const long long N = g.n_points;
  const double two_pi = 6.283185307179586476925286766559;
  if (!kinetic_only) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N;
         p += (long long)gridDim.x * blockDim.x) {
      const double v = V[p];
      f_half[p] = (R)exp(-0.5 * tau_i * v);
      if (f_full) f_full[p] = (R)exp(-tau_i * v);
    }
  }
  if (blockIdx.x == 0) {
    const double invN = 1.0 / (double)N;
    for (int j = threadIdx.x; j < g.nxh; j += blockDim.x) {
      const double k = two_pi * j / lx;
      kx[j] = kinetic_only ? (R)(0.5 * k * k) : (R)exp(-0.5 * tau_i * k * k);
    }
    for (int j = threadIdx.x; j < g.ny; j += blockDim.x) {
      const int jj = j <= g.ny / 2 ? j : j - g.ny;
      const double k = two_pi * jj / ly;
      ky[j] = kinetic_only ? (R)(0.5 * k * k) : (R)exp(-0.5 * tau_i * k * k);
    }
    for (int j = threadIdx.x; j < g.nz; j += blockDim.x) {
      const int jj = j <= g.nz / 2 ? j : j - g.nz;
      const double k = two_pi * jj / lz;
      kz[j] = kinetic_only ? (R)(0.5 * k * k) : (R)(exp(-0.5 * tau_i * k * k) * invN);
    }
  }
}

// phi[s][z][:] = sum_i term_i[s][z][:] in FP64, rounded to FP32; term_i is
// stored with the half-spectrum plane pitch (in floats).
// term_sum_kernel sums with two_sum_acc (error-free TwoSum, defined with the
// epilogues): the result is the exact sum of the FP32 contributions up to its
// final rounding.  On this GPU the FP64 pipe runs at a small fraction of the
// FP32 rate, and a plain FP64 sum with its conversions costs an order of
// magnitude more.

__device__ __forceinline__ void term_sum_body(const TermSumArgs& a, long long pl) {
  // pl = plane (state, z); x-blocks stride over the plane's float4s
  const int nvec = a.plane_pts >> 2;
  const float4* src[kMaxTermsK];
#pragma unroll
  for (int i = 0; i < kMaxTermsK; ++i)
    src[i] = reinterpret_cast<const float4*>(a.term[i < a.k ? i : 0] + pl * a.plane_pitch);
  float4* dst = reinterpret_cast<float4*>(a.phi_out + pl * a.plane_pts);
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nvec; v += gridDim.x * blockDim.x) {
    float s[4] = {0.f, 0.f, 0.f, 0.f}, e[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int i = 0; i < kMaxTermsK; ++i) {
      if (i < a.k) {
        const float4 x = __ldg(src[i] + v);
        two_sum_acc(s[0], e[0], x.x);
        two_sum_acc(s[1], e[1], x.y);
        two_sum_acc(s[2], e[2], x.z);
        two_sum_acc(s[3], e[3], x.w);
      }
    }
    dst[v] = make_float4(s[0] + e[0], s[1] + e[1], s[2] + e[2], s[3] + e[3]);
  }
}

__global__ void term_sum_kernel(const TermSumArgs a) { term_sum_body(a, blockIdx.y); }

// Grouped term sum: row y is state rows[y].y of problem rows[y].x, z-plane
// blockIdx.z.
__global__ void term_sum_group_kernel(const TermSumArgs* __restrict__ args,
                                      const int2* __restrict__ rows) {
  const int2 r = rows[blockIdx.y];
  const TermSumArgs& a = args[r.x];
  term_sum_body(a, (long long)r.y * a.nz + blockIdx.z);
}

// dst[p][c][r] = src[p][r][c] for nplanes planes of rows x cols.
template <typename TS, typename TD>
__global__ void transpose_planes_kernel(const TS* __restrict__ src, TD* __restrict__ dst,
                                        long long nplanes, int rows, int cols) {
  __shared__ TS tile[32][33];
  const long long p = blockIdx.z;
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  const TS* s = src + p * rows * cols;
  TD* d = dst + p * rows * cols;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    if (r < rows && c < cols) tile[i][threadIdx.x] = s[(long long)r * cols + c];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int c = c0 + i, r = r0 + threadIdx.x;
    if (r < rows && c < cols) d[(long long)c * rows + r] = (TD)tile[threadIdx.x][i];
  }
}

template <typename K>
cudaError_t set_smem(K kernel, size_t bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename R, int NX, int NY>
cudaError_t plane_dispatch(const GridDesc& g, const PlaneArgs<R>& a, size_t smem, cudaStream_t st) {
  dim3 grid(g.nz, a.m);
  const int nthr = kThreads;
  cudaError_t e;
  switch (a.mode) {
#define ITP_PLANE_CASE(M)                                                   \
  case M:                                                                   \
    e = set_smem(plane_kernel<R, NX, NY, M>, smem);                         \
    if (e != cudaSuccess) return e;                                         \
    plane_kernel<R, NX, NY, M><<<grid, nthr, smem, st>>>(g, a);             \
    break;
    ITP_PLANE_CASE(PLANE_FWD_REAL)
    ITP_PLANE_CASE(PLANE_MERGED)
    ITP_PLANE_CASE(PLANE_COMBINE)
    ITP_PLANE_CASE(PLANE_HPSI)
    ITP_PLANE_CASE(PLANE_TERM)
#undef ITP_PLANE_CASE
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename R, int NZ, int W>
cudaError_t pencil_dispatch(const GridDesc& g, const PencilArgs<R>& a, size_t smem,
                            cudaStream_t st) {
  const int chunks = (g.nxh + g.pencil_w - 1) / g.pencil_w;
  dim3 grid(g.ny * chunks, a.m);
  const int nthr = launch_threads(task_threads(W));
  cudaError_t e;
  if (a.mode == PENCIL_PROPAGATE) {
    e = set_smem(pencil_kernel<R, NZ, W, PENCIL_PROPAGATE>, smem);
    if (e != cudaSuccess) return e;
    pencil_kernel<R, NZ, W, PENCIL_PROPAGATE><<<grid, nthr, smem, st>>>(g, a);
  } else {
    e = set_smem(pencil_kernel<R, NZ, W, PENCIL_KINETIC>, smem);
    if (e != cudaSuccess) return e;
    pencil_kernel<R, NZ, W, PENCIL_KINETIC><<<grid, nthr, smem, st>>>(g, a);
  }
  return cudaGetLastError();
}

}  // namespace

template <typename R, int NX, int TB>
cudaError_t rowpass_dispatch(const GridDesc& g, const PlaneArgs<R>& a, cudaStream_t st) {
  const size_t smem = ((size_t)TB * g.pp + g.nx) * 2 * sizeof(R);
  dim3 grid(g.nz * ((g.ny / 2) / TB), a.m);
  cudaError_t e;
  switch (a.mode) {
#define ITP_ROW_CASE(M)                                                     \
  case M:                                                                   \
    e = set_smem(rowpass_kernel<R, NX, TB, M>, smem);                       \
    if (e != cudaSuccess) return e;                                         \
    rowpass_kernel<R, NX, TB, M><<<grid, kThreads, smem, st>>>(g, a);       \
    break;
    ITP_ROW_CASE(PLANE_FWD_REAL)
    ITP_ROW_CASE(PLANE_MERGED)
    ITP_ROW_CASE(PLANE_COMBINE)
    ITP_ROW_CASE(PLANE_HPSI)
#undef ITP_ROW_CASE
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename R>
cudaError_t rowpass_launch(const GridDesc& g, const PlaneArgs<R>& a, cudaStream_t st) {
  const int tb = g.row_tb[sizeof(R) == 4 ? 0 : 1];
  if (g.nx == 256 && g.pp == row_pitch(256) && tb == (sizeof(R) == 4 ? 32 : 16)) {
    if constexpr (sizeof(R) == 4) return rowpass_dispatch<R, 256, 32>(g, a, st);
    else return rowpass_dispatch<R, 256, 16>(g, a, st);
  }
  if (tb == 32) return rowpass_dispatch<R, 0, 32>(g, a, st);
  if (tb == 16) return rowpass_dispatch<R, 0, 16>(g, a, st);
  if (tb == 8) return rowpass_dispatch<R, 0, 8>(g, a, st);
  return cudaErrorInvalidValue;
}

template <typename R, int NY, int W, int DIR>
cudaError_t colpass_one(const GridDesc& g, void* spec, const void* twy, int m,
                        const KinFac<R>& kin, cudaStream_t st) {
  const int cw = g.col_w[sizeof(R) == 4 ? 0 : 1];
  const size_t smem = ((size_t)g.ny * cw + g.ny) * 2 * sizeof(R);
  cudaError_t e = set_smem(colpass_kernel<R, NY, W, DIR>, smem);
  if (e != cudaSuccess) return e;
  dim3 grid((g.nxh + cw - 1) / cw, (unsigned)((long long)m * g.nz));
  colpass_kernel<R, NY, W, DIR><<<grid, launch_threads(task_threads(W)), smem, st>>>(
      g, spec, twy, cw, kin);
  return cudaGetLastError();
}

template <typename R, int DIR>
cudaError_t colpass_launch(const GridDesc& g, void* spec, const void* twy, int m,
                           const KinFac<R>& kin, cudaStream_t st) {
  if (g.ny == 256 && g.col_w[sizeof(R) == 4 ? 0 : 1] == (sizeof(R) == 4 ? 33 : 17)) {
    if constexpr (sizeof(R) == 4) return colpass_one<R, 256, 33, DIR>(g, spec, twy, m, kin, st);
    else return colpass_one<R, 256, 17, DIR>(g, spec, twy, m, kin, st);
  }
  return colpass_one<R, 0, 0, DIR>(g, spec, twy, m, kin, st);
}

template <typename R>
cudaError_t launch_plane(const GridDesc& g, const PlaneArgs<R>& a, cudaStream_t st, int* nlaunch) {
  if (nlaunch) *nlaunch = 1;
  // FP32 H psi passes write FP32 (potential and output in R)
  if (a.mode == PLANE_HPSI && sizeof(R) == 4 && (!a.V_r || !a.phi_out))
    return cudaErrorInvalidValue;
  if (g.split_planes[sizeof(R) == 4 ? 0 : 1] == 3) {
    // 256 x 256 FP32 planes on four-CTA clusters
    if constexpr (sizeof(R) == 4) {
      if (g.nx != 256 || g.ny != 256) return cudaErrorInvalidValue;
      const size_t smem = ((size_t)32 * row_pitch(256) + 576) * sizeof(float2);
      dim3 grid(4 * g.nz, a.m);
      cudaError_t e;
      switch (a.mode) {
#define ITP_C4_CASE(M)                                                      \
  case M:                                                                   \
    e = set_smem(plane_c4_kernel<M>, smem);                                 \
    if (e != cudaSuccess) return e;                                         \
    plane_c4_kernel<M><<<grid, kC4Threads, smem, st>>>(g, a);               \
    break;
        ITP_C4_CASE(PLANE_FWD_REAL)
        ITP_C4_CASE(PLANE_MERGED)
        ITP_C4_CASE(PLANE_COMBINE)
        ITP_C4_CASE(PLANE_HPSI)
        ITP_C4_CASE(PLANE_TERM)
#undef ITP_C4_CASE
        default:
          return cudaErrorInvalidValue;
      }
      return cudaGetLastError();
    } else {
      return cudaErrorInvalidValue;
    }
  }
  if (g.split_planes[sizeof(R) == 4 ? 0 : 1] == 2) {
    // 256 x 256 FP32 planes on two-CTA clusters
    if constexpr (sizeof(R) == 4) {
      if (g.nx != 256 || g.ny != 256) return cudaErrorInvalidValue;
      const size_t smem = ((size_t)64 * row_pitch(256) + 512) * sizeof(float2);
      dim3 grid(2 * g.nz, a.m);
      cudaError_t e;
      switch (a.mode) {
#define ITP_C2_CASE(M)                                                      \
  case M:                                                                   \
    e = set_smem(plane_c2_kernel<M>, smem);                                 \
    if (e != cudaSuccess) return e;                                         \
    plane_c2_kernel<M><<<grid, kC2Threads, smem, st>>>(g, a);               \
    break;
        ITP_C2_CASE(PLANE_FWD_REAL)
        ITP_C2_CASE(PLANE_MERGED)
        ITP_C2_CASE(PLANE_COMBINE)
        ITP_C2_CASE(PLANE_HPSI)
        ITP_C2_CASE(PLANE_TERM)
#undef ITP_C2_CASE
        default:
          return cudaErrorInvalidValue;
      }
      return cudaGetLastError();
    } else {
      return cudaErrorInvalidValue;
    }
  }
  if (g.split_planes[sizeof(R) == 4 ? 0 : 1]) {
    // planes too large for one CTA: column passes for y, row passes for x
    cudaError_t e = cudaSuccess;
    int n = 0;
    if (a.mode != PLANE_FWD_REAL) {
      e = colpass_launch<R, 1>(g, a.spec, a.twy, a.m, KinFac<R>{}, st);
      ++n;
      if (e != cudaSuccess) return e;
    }
    e = rowpass_launch<R>(g, a, st);
    ++n;
    if (e != cudaSuccess) return e;
    if (a.mode == PLANE_FWD_REAL || a.mode == PLANE_MERGED) {
      e = colpass_launch<R, -1>(g, a.spec, a.twy, a.m, a.kin, st);
      ++n;
    }
    if (nlaunch) *nlaunch = n;
    return e;
  }
  const size_t smem = plane_smem_bytes(g, sizeof(R));
  if (g.nx == g.ny && g.pp == row_pitch(g.nx)) {
    switch (g.nx) {
      case 32: return plane_dispatch<R, 32, 32>(g, a, smem, st);
      case 48: return plane_dispatch<R, 48, 48>(g, a, smem, st);
      case 64: return plane_dispatch<R, 64, 64>(g, a, smem, st);
      case 96: return plane_dispatch<R, 96, 96>(g, a, smem, st);
      case 128: return plane_dispatch<R, 128, 128>(g, a, smem, st);
      default: break;
    }
  }
  return plane_dispatch<R, 0, 0>(g, a, smem, st);
}

template <typename R>
cudaError_t launch_pencil(const GridDesc& g, const PencilArgs<R>& a, cudaStream_t st) {
  if (g.pencil_w == 0) {
    if constexpr (sizeof(R) == 4) {
      return launch_pencil_tm(g, a, st);
    } else {
      // the FP64 passes of a mixed handle: the default slab width
      GridDesc g2 = g;
      const size_t full = (size_t)g.nz * g.nxh * 2 * sizeof(R), budget = 72 * 1024;
      const int chunks = (int)((full + budget - 1) / budget);
      g2.pencil_w = g2.pencil_pitch = (g.nxh + chunks - 1) / chunks;
      return launch_pencil(g2, a, st);
    }
  }
  const size_t smem = pencil_smem_bytes(g, sizeof(R));
  switch (g.nz * 1000 + g.pencil_w) {
    case 32 * 1000 + 17: return pencil_dispatch<R, 32, 17>(g, a, smem, st);
    case 48 * 1000 + 25: return pencil_dispatch<R, 48, 25>(g, a, smem, st);
    case 64 * 1000 + 33: return pencil_dispatch<R, 64, 33>(g, a, smem, st);
    case 96 * 1000 + 49: return pencil_dispatch<R, 96, 49>(g, a, smem, st);
    case 96 * 1000 + 25: return pencil_dispatch<R, 96, 25>(g, a, smem, st);
    case 128 * 1000 + 65: return pencil_dispatch<R, 128, 65>(g, a, smem, st);
    case 128 * 1000 + 33: return pencil_dispatch<R, 128, 33>(g, a, smem, st);
    case 256 * 1000 + 33: return pencil_dispatch<R, 256, 33>(g, a, smem, st);
    default: break;
  }
  return pencil_dispatch<R, 0, 0>(g, a, smem, st);
}

template <typename R>
cudaError_t launch_term_tables(const GridDesc& g, const double* V, double tau_i, double lx,
                               double ly, double lz, R* f_half, R* f_full, R* kx, R* ky, R* kz,
                               cudaStream_t st) {
  term_tables_kernel<R><<<4 * 152, 256, 0, st>>>(g, V, tau_i, lx, ly, lz, f_half, f_full, kx, ky,
                                                 kz, 0);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_kinetic_tables(const GridDesc& g, double lx, double ly, double lz, R* kx,
                                  R* ky, R* kz, cudaStream_t st) {
  term_tables_kernel<R><<<1, 256, 0, st>>>(g, nullptr, 0.0, lx, ly, lz, nullptr, nullptr, kx, ky,
                                           kz, 1);
  return cudaGetLastError();
}

template <typename TS, typename TD>
cudaError_t launch_transpose_planes(const TS* src, TD* dst, long long nplanes, int rows,
                                    int cols, cudaStream_t st) {
  dim3 block(32, 8);
  dim3 grid((cols + 31) / 32, (rows + 31) / 32, (unsigned)nplanes);
  transpose_planes_kernel<TS, TD><<<grid, block, 0, st>>>(src, dst, nplanes, rows, cols);
  return cudaGetLastError();
}

// ---- grouped launches (batches of problems with the same grid) -------------
template <typename R, int NX, int NY>
cudaError_t plane_group_dispatch(const GridDesc& g, int mode, const PlaneArgs<R>* args,
                                 const int2* rows, int nrows, size_t smem, cudaStream_t st) {
  dim3 grid(g.nz, nrows);
  cudaError_t e;
  switch (mode) {
#define ITP_PLANE_GROUP_CASE(M)                                             \
  case M:                                                                   \
    e = set_smem(plane_group_kernel<R, NX, NY, M>, smem);                   \
    if (e != cudaSuccess) return e;                                         \
    plane_group_kernel<R, NX, NY, M><<<grid, kThreads, smem, st>>>(g, args, rows); \
    break;
    ITP_PLANE_GROUP_CASE(PLANE_FWD_REAL)
    ITP_PLANE_GROUP_CASE(PLANE_MERGED)
    ITP_PLANE_GROUP_CASE(PLANE_COMBINE)
    ITP_PLANE_GROUP_CASE(PLANE_HPSI)
    ITP_PLANE_GROUP_CASE(PLANE_TERM)
#undef ITP_PLANE_GROUP_CASE
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_plane_group(const GridDesc& g, int mode, const PlaneArgs<R>* args,
                               const int2* rows, int nrows, cudaStream_t st) {
  if (g.split_planes[sizeof(R) == 4 ? 0 : 1]) return cudaErrorInvalidValue;   // whole planes only
  const size_t smem = plane_smem_bytes(g, sizeof(R));
  if (g.nx == g.ny && g.pp == row_pitch(g.nx)) {
    switch (g.nx) {
      case 32: return plane_group_dispatch<R, 32, 32>(g, mode, args, rows, nrows, smem, st);
      case 48: return plane_group_dispatch<R, 48, 48>(g, mode, args, rows, nrows, smem, st);
      case 64: return plane_group_dispatch<R, 64, 64>(g, mode, args, rows, nrows, smem, st);
      case 96: return plane_group_dispatch<R, 96, 96>(g, mode, args, rows, nrows, smem, st);
      case 128: return plane_group_dispatch<R, 128, 128>(g, mode, args, rows, nrows, smem, st);
      default: break;
    }
  }
  return plane_group_dispatch<R, 0, 0>(g, mode, args, rows, nrows, smem, st);
}

template <typename R, int NZ, int W>
cudaError_t pencil_group_dispatch(const GridDesc& g, int mode, const PencilArgs<R>* args,
                                  const int2* rows, int nrows, size_t smem, cudaStream_t st) {
  const int chunks = (g.nxh + g.pencil_w - 1) / g.pencil_w;
  dim3 grid(g.ny * chunks, nrows);
  const int nthr = launch_threads(task_threads(W));
  cudaError_t e;
  if (mode == PENCIL_PROPAGATE) {
    e = set_smem(pencil_group_kernel<R, NZ, W, PENCIL_PROPAGATE>, smem);
    if (e != cudaSuccess) return e;
    pencil_group_kernel<R, NZ, W, PENCIL_PROPAGATE><<<grid, nthr, smem, st>>>(g, args, rows);
  } else {
    e = set_smem(pencil_group_kernel<R, NZ, W, PENCIL_KINETIC>, smem);
    if (e != cudaSuccess) return e;
    pencil_group_kernel<R, NZ, W, PENCIL_KINETIC><<<grid, nthr, smem, st>>>(g, args, rows);
  }
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_pencil_group(const GridDesc& g, int mode, const PencilArgs<R>* args,
                                const int2* rows, int nrows, cudaStream_t st) {
  const size_t smem = pencil_smem_bytes(g, sizeof(R));
  if (g.pencil_w < 1) return cudaErrorInvalidValue;
  switch (g.nz * 1000 + g.pencil_w) {
    case 32 * 1000 + 17: return pencil_group_dispatch<R, 32, 17>(g, mode, args, rows, nrows, smem, st);
    case 48 * 1000 + 25: return pencil_group_dispatch<R, 48, 25>(g, mode, args, rows, nrows, smem, st);
    case 64 * 1000 + 33: return pencil_group_dispatch<R, 64, 33>(g, mode, args, rows, nrows, smem, st);
    case 96 * 1000 + 49: return pencil_group_dispatch<R, 96, 49>(g, mode, args, rows, nrows, smem, st);
    case 96 * 1000 + 25: return pencil_group_dispatch<R, 96, 25>(g, mode, args, rows, nrows, smem, st);
    case 128 * 1000 + 65: return pencil_group_dispatch<R, 128, 65>(g, mode, args, rows, nrows, smem, st);
    case 128 * 1000 + 33: return pencil_group_dispatch<R, 128, 33>(g, mode, args, rows, nrows, smem, st);
    default: break;
  }
  return pencil_group_dispatch<R, 0, 0>(g, mode, args, rows, nrows, smem, st);
}

}  // namespace itp
