// Plane and pencil passes of the 3D real FFT with the split-operator factors
// fused in (T_2 of Eq. (so) applied as point-wise multiplies around one
// complete FFT; Sec. I).
//
// Data layout in HBM:
//   real states      [m][nz][ny][nx]        (x fastest)
//   half spectrum    [m][nz][ny][nx/2+1]    complex, natural frequency order
//   FP64 accumulator [m][nz][ny][nx]
//
// Plane pass: one CTA per (state, z plane).  The plane is staged in shared
// memory as ny/2 row pairs; row pair r holds the two real rows 2r, 2r+1 as
// one complex row (re = row 2r, im = row 2r+1) of length nx, so the real
// transform along x is one complex FFT per row pair followed by the
// even/odd split.  After the split, row pair r holds the two half-spectrum
// rows A (row 2r) and B (row 2r+1) back to back.  The complex FFT along y
// then runs down the nx/2+1 columns.
//
// Pencil pass: one CTA per (state, ky, block of kx columns).  The xz slab is
// staged in shared memory; the forward FFT along z, the kinetic factor
// exp(-tau |k|^2 / 2) / N and the inverse FFT along z all happen there.
#include "fft_common.cuh"
#include "itp_kernels.cuh"

namespace itp {

namespace {

constexpr int kThreads = 256;

struct RowAddr {   // x rows: transform t = row pair, element e = x
  int pp;
  __device__ __forceinline__ int operator()(int t, int e) const { return t * pp + e; }
};
struct ColAddr {   // y columns: transform t = kx, element e = y (position)
  int pp, nxh;
  __device__ __forceinline__ int operator()(int t, int e) const {
    return (e >> 1) * pp + (e & 1) * nxh + t;
  }
};
struct SlabAddr {  // z columns of a pencil slab: transform t = kx column, element e = z
  int pitch;
  __device__ __forceinline__ int operator()(int t, int e) const { return e * pitch + t; }
};

template <typename R> struct Vec2Of;
template <> struct Vec2Of<float> { using type = float2; };
template <> struct Vec2Of<double> { using type = double2; };

// Real transform along x, forward: split each row pair's spectrum Z of the
// packed row (a + i b) into A = FFT(a), B = FFT(b), k = 0..nx/2.
// One warp per row pair; Z is read in digit-swapped order.
template <typename C>
__device__ __forceinline__ void x_split(C* sm, int npair, int pp, int nx, int nxh, const Axis ax) {
  using Rl = decltype(sm[0].x);
  constexpr int MAXQ = 5;   // (nx/2 + 1) <= 32 * MAXQ  for nx <= 256
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int half = nx >> 1;
  for (int r = warp; r < npair; r += nw) {
    C* row = sm + r * pp;
    C zp[MAXQ], zm[MAXQ];
#pragma unroll
    for (int q = 0; q < MAXQ; ++q) {
      const int k = lane + 32 * q;
      if (k <= half) {
        zp[q] = row[spec_pos(ax, k)];
        zm[q] = row[spec_pos(ax, k == 0 ? 0 : nx - k)];
      }
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < MAXQ; ++q) {
      const int k = lane + 32 * q;
      if (k <= half) {
        // A = (Z[k] + conj(Z[-k])) / 2,  B = (Z[k] - conj(Z[-k])) / (2i)
        C A, B;
        A.x = (Rl)0.5 * (zp[q].x + zm[q].x);
        A.y = (Rl)0.5 * (zp[q].y - zm[q].y);
        B.x = (Rl)0.5 * (zp[q].y + zm[q].y);
        B.y = (Rl)0.5 * (zm[q].x - zp[q].x);
        row[k] = A;
        row[nxh + k] = B;
      }
    }
    __syncwarp();
  }
}

// Inverse of x_split: build Z = A + iB over all nx frequencies (Hermitian
// extension; the imaginary parts of the self-conjugate bins k = 0, nx/2 are
// dropped, as a complex-to-real transform does) in digit-swapped order.
template <typename C>
__device__ __forceinline__ void x_merge(C* sm, int npair, int pp, int nx, int nxh, const Axis ax) {
  constexpr int MAXQ = 5;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int half = nx >> 1;
  for (int r = warp; r < npair; r += nw) {
    C* row = sm + r * pp;
    C av[MAXQ], bv[MAXQ];
#pragma unroll
    for (int q = 0; q < MAXQ; ++q) {
      const int k = lane + 32 * q;
      if (k <= half) {
        av[q] = row[k];
        bv[q] = row[nxh + k];
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
        row[spec_pos(ax, k)] = Z;
        if (k > 0 && k < half) {
          C Zm;
          Zm.x = A.x + B.y;
          Zm.y = B.x - A.y;
          row[spec_pos(ax, nx - k)] = Zm;
        }
      }
    }
    __syncwarp();
  }
}

template <typename R, int MODE>
__global__ void __launch_bounds__(kThreads) plane_kernel(const GridDesc g, const PlaneArgs<R> a) {
  using C = typename CplxOf<R>::type;
  using V2 = typename Vec2Of<R>::type;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);

  const int z = blockIdx.x, s = blockIdx.y;
  const int nx = g.nx, ny = g.ny, nxh = g.nxh, pp = g.pp;
  const int npair = ny >> 1, hx = nx >> 1;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const long long N = g.n_points;
  const long long plane_off = (long long)z * ny * nx;
  const long long spec_off = ((long long)s * g.nz + z) * (long long)ny * nxh;
  const Axis axx{nx, g.rx1, g.rx2}, axy{ny, g.ry1, g.ry2};
  const C* twx = static_cast<const C*>(a.twx);
  const C* twy = static_cast<const C*>(a.twy);
  const RowAddr rows{pp};
  const ColAddr cols{pp, nxh};

  if constexpr (MODE == PLANE_FWD_REAL) {
    const R* src = a.in_real + (long long)s * N + plane_off;
    const R* f = a.f_in ? a.f_in + plane_off : nullptr;
    for (int idx = tid; idx < npair * hx; idx += nthr) {
      const int r = idx / hx, x = 2 * (idx - r * hx);
      V2 va = *reinterpret_cast<const V2*>(src + (2 * r) * nx + x);
      V2 vb = *reinterpret_cast<const V2*>(src + (2 * r + 1) * nx + x);
      if (f) {
        const V2 fa = __ldg(reinterpret_cast<const V2*>(f + (2 * r) * nx + x));
        const V2 fb = __ldg(reinterpret_cast<const V2*>(f + (2 * r + 1) * nx + x));
        va.x *= fa.x; va.y *= fa.y; vb.x *= fb.x; vb.y *= fb.y;
      }
      C c0, c1;
      c0.x = va.x; c0.y = vb.x;
      c1.x = va.y; c1.y = vb.y;
      sm[r * pp + x] = c0;
      sm[r * pp + x + 1] = c1;
    }
    __syncthreads();
  } else {
    const C* src = static_cast<const C*>(a.spec) + spec_off;
    for (int idx = tid; idx < ny * nxh; idx += nthr) {
      const int ky = idx / nxh, kx = idx - ky * nxh;
      sm[cols(kx, spec_pos(axy, ky))] = src[idx];
    }
    __syncthreads();
    fft_inverse(sm, cols, nxh, axy, twy);
    x_merge(sm, npair, pp, nx, nxh, axx);
    __syncthreads();
    fft_inverse(sm, rows, npair, axx, twx);

    if constexpr (MODE == PLANE_COMBINE) {
      double* acc = a.acc + (long long)s * N + plane_off;
      const R* f = a.f_out + plane_off;
      const double c = a.coef;
      for (int idx = tid; idx < npair * hx; idx += nthr) {
        const int r = idx / hx, x = 2 * (idx - r * hx);
        const C v0 = sm[r * pp + x], v1 = sm[r * pp + x + 1];
        const V2 fa = __ldg(reinterpret_cast<const V2*>(f + (2 * r) * nx + x));
        const V2 fb = __ldg(reinterpret_cast<const V2*>(f + (2 * r + 1) * nx + x));
        double2* pa = reinterpret_cast<double2*>(acc + (2 * r) * nx + x);
        double2* pb = reinterpret_cast<double2*>(acc + (2 * r + 1) * nx + x);
        double2 ua, ub;
        ua.x = c * (double)(v0.x * fa.x); ua.y = c * (double)(v1.x * fa.y);
        ub.x = c * (double)(v0.y * fb.x); ub.y = c * (double)(v1.y * fb.y);
        if (!a.acc_init) {
          const double2 oa = *pa, ob = *pb;
          ua.x += oa.x; ua.y += oa.y; ub.x += ob.x; ub.y += ob.y;
        }
        *pa = ua;
        *pb = ub;
      }
      return;
    } else if constexpr (MODE == PLANE_HPSI) {
      double* out = a.acc + (long long)s * N + plane_off;
      const R* psi = a.in_real + (long long)s * N + plane_off;
      const double* V = a.V + plane_off;
      for (int idx = tid; idx < npair * hx; idx += nthr) {
        const int r = idx / hx, x = 2 * (idx - r * hx);
        const C v0 = sm[r * pp + x], v1 = sm[r * pp + x + 1];
        const V2 qa = *reinterpret_cast<const V2*>(psi + (2 * r) * nx + x);
        const V2 qb = *reinterpret_cast<const V2*>(psi + (2 * r + 1) * nx + x);
        const double2 Va = __ldg(reinterpret_cast<const double2*>(V + (2 * r) * nx + x));
        const double2 Vb = __ldg(reinterpret_cast<const double2*>(V + (2 * r + 1) * nx + x));
        double2 ha, hb;
        ha.x = (double)v0.x + Va.x * (double)qa.x;
        ha.y = (double)v1.x + Va.y * (double)qa.y;
        hb.x = (double)v0.y + Vb.x * (double)qb.x;
        hb.y = (double)v1.y + Vb.y * (double)qb.y;
        *reinterpret_cast<double2*>(out + (2 * r) * nx + x) = ha;
        *reinterpret_cast<double2*>(out + (2 * r + 1) * nx + x) = hb;
      }
      return;
    } else {
      // PLANE_MERGED: the two adjacent half steps exp(-tau_i V/2) merge into
      // one exp(-tau_i V) between the inverse and the next forward FFT.
      const R* f = a.f_mid + plane_off;
      for (int idx = tid; idx < npair * nx; idx += nthr) {
        const int r = idx / nx, x = idx - r * nx;
        C v = sm[r * pp + x];
        v.x *= __ldg(f + (2 * r) * nx + x);
        v.y *= __ldg(f + (2 * r + 1) * nx + x);
        sm[r * pp + x] = v;
      }
      __syncthreads();
    }
  }

  if constexpr (MODE == PLANE_FWD_REAL || MODE == PLANE_MERGED) {
    fft_forward(sm, rows, npair, axx, twx);
    x_split(sm, npair, pp, nx, nxh, axx);
    __syncthreads();
    fft_forward(sm, cols, nxh, axy, twy);
    C* dst = static_cast<C*>(a.spec) + spec_off;
    for (int idx = tid; idx < ny * nxh; idx += nthr) {
      const int ky = idx / nxh, kx = idx - ky * nxh;
      dst[idx] = sm[cols(kx, spec_pos(axy, ky))];
    }
  }
}

template <typename R, int MODE>
__global__ void __launch_bounds__(kThreads) pencil_kernel(const GridDesc g, const PencilArgs<R> a) {
  using C = typename CplxOf<R>::type;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  const int s = blockIdx.y;
  const int ky = blockIdx.x % g.ny, chunk = blockIdx.x / g.ny;
  const int kx0 = chunk * g.pencil_w;
  const int w = min(g.pencil_w, g.nxh - kx0);
  const int nz = g.nz, pz = g.pencil_pitch;
  const long long zstride = (long long)g.ny * g.nxh;
  const int tid = threadIdx.x, nthr = blockDim.x;
  C* base = static_cast<C*>(a.spec) + (long long)s * g.n_half + (long long)ky * g.nxh + kx0;
  const Axis axz{nz, g.rz1, g.rz2};
  const C* twz = static_cast<const C*>(a.twz);
  const SlabAddr slab{pz};

  for (int idx = tid; idx < nz * w; idx += nthr) {
    const int zz = idx / w, j = idx - zz * w;
    sm[zz * pz + j] = base[zz * zstride + j];
  }
  __syncthreads();
  fft_forward(sm, slab, w, axz, twz);
  const R fy = a.ky_tab[ky];
  for (int idx = tid; idx < nz * w; idx += nthr) {
    const int p = idx / w, j = idx - p * w;
    const int kz = spec_freq(axz, p);
    R f;
    if constexpr (MODE == PENCIL_PROPAGATE) {
      f = __ldg(&a.kx_tab[kx0 + j]) * fy * __ldg(&a.kz_tab[kz]);
    } else {
      f = (__ldg(&a.kx_tab[kx0 + j]) + fy + __ldg(&a.kz_tab[kz])) * a.scale;
    }
    C v = sm[p * pz + j];
    v.x *= f;
    v.y *= f;
    sm[p * pz + j] = v;
  }
  __syncthreads();
  fft_inverse(sm, slab, w, axz, twz);
  for (int idx = tid; idx < nz * w; idx += nthr) {
    const int zz = idx / w, j = idx - zz * w;
    base[zz * zstride + j] = sm[zz * pz + j];
  }
}

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

template <typename K>
cudaError_t set_smem(K kernel, size_t bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

size_t plane_smem_bytes(const GridDesc& g, int real_bytes) {
  return (size_t)(g.ny / 2) * g.pp * 2 * real_bytes;
}
size_t pencil_smem_bytes(const GridDesc& g, int real_bytes) {
  return (size_t)g.nz * g.pencil_pitch * 2 * real_bytes;
}

template <typename R>
cudaError_t launch_plane(const GridDesc& g, const PlaneArgs<R>& a, cudaStream_t st) {
  const size_t smem = plane_smem_bytes(g, sizeof(R));
  dim3 grid(g.nz, a.m);
  cudaError_t e = cudaSuccess;
  switch (a.mode) {
#define ITP_PLANE_CASE(M)                                                   \
  case M:                                                                   \
    e = set_smem(plane_kernel<R, M>, smem);                                 \
    if (e != cudaSuccess) return e;                                         \
    plane_kernel<R, M><<<grid, kThreads, smem, st>>>(g, a);                 \
    break;
    ITP_PLANE_CASE(PLANE_FWD_REAL)
    ITP_PLANE_CASE(PLANE_MERGED)
    ITP_PLANE_CASE(PLANE_COMBINE)
    ITP_PLANE_CASE(PLANE_HPSI)
#undef ITP_PLANE_CASE
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_pencil(const GridDesc& g, const PencilArgs<R>& a, cudaStream_t st) {
  const size_t smem = pencil_smem_bytes(g, sizeof(R));
  const int chunks = (g.nxh + g.pencil_w - 1) / g.pencil_w;
  dim3 grid(g.ny * chunks, a.m);
  cudaError_t e;
  if (a.mode == PENCIL_PROPAGATE) {
    e = set_smem(pencil_kernel<R, PENCIL_PROPAGATE>, smem);
    if (e != cudaSuccess) return e;
    pencil_kernel<R, PENCIL_PROPAGATE><<<grid, kThreads, smem, st>>>(g, a);
  } else {
    e = set_smem(pencil_kernel<R, PENCIL_KINETIC>, smem);
    if (e != cudaSuccess) return e;
    pencil_kernel<R, PENCIL_KINETIC><<<grid, kThreads, smem, st>>>(g, a);
  }
  return cudaGetLastError();
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

template cudaError_t launch_plane<float>(const GridDesc&, const PlaneArgs<float>&, cudaStream_t);
template cudaError_t launch_plane<double>(const GridDesc&, const PlaneArgs<double>&, cudaStream_t);
template cudaError_t launch_pencil<float>(const GridDesc&, const PencilArgs<float>&, cudaStream_t);
template cudaError_t launch_pencil<double>(const GridDesc&, const PencilArgs<double>&, cudaStream_t);
template cudaError_t launch_term_tables<float>(const GridDesc&, const double*, double, double,
                                               double, double, float*, float*, float*, float*,
                                               float*, cudaStream_t);
template cudaError_t launch_term_tables<double>(const GridDesc&, const double*, double, double,
                                                double, double, double*, double*, double*,
                                                double*, double*, cudaStream_t);
template cudaError_t launch_kinetic_tables<float>(const GridDesc&, double, double, double, float*,
                                                  float*, float*, cudaStream_t);
template cudaError_t launch_kinetic_tables<double>(const GridDesc&, double, double, double,
                                                   double*, double*, double*, cudaStream_t);

}  // namespace itp
