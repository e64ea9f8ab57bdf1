// Register codelets and shared-memory stages of the mixed-radix FFTs used by
// the plane and pencil passes.
//
// A transform of length L = r1 * r2 (r1, r2 in {1,2,3,4,6,8,12,16}) held in
// shared memory is done in two in-place stages (Cooley-Tukey, n = n1 + r1*n2,
// k = k2 + r2*k1):
//   forward  A: for each n1, a size-r2 DFT over n2 (stride r1), then the
//               twiddle w_L^{n1*k2};  B: for each k2, a size-r1 DFT over n1
//               (contiguous).  Position a + r1*b then holds X[b + r2*a]
//               ("digit-swapped" order).
//   inverse B': for each b, a size-r1 inverse DFT over the contiguous block,
//               then the twiddle w_L^{-n1*b};  A': for each n1, a size-r2
//               inverse DFT over stride r1.  Input in digit-swapped order,
//               output in natural order.
// Every task reads and writes the same positions, so a stage needs one
// barrier before it and none inside.  No normalisation is applied.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace itp {

template <typename R> struct CplxOf;
template <> struct CplxOf<float> { using type = float2; };
template <> struct CplxOf<double> { using type = double2; };

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  C r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
// a * conj(b)
template <typename C> __device__ __forceinline__ C cmulc(C a, C b) {
  C r; r.x = a.x * b.x + a.y * b.y; r.y = a.y * b.x - a.x * b.y; return r;
}
// FP32 complex values use the packed two-lane FP32 instructions of sm_100+
// (one instruction updates re and im): add, multiply and fused multiply-add
// on float2.  Each lane rounds as the scalar instruction does.
template <> __device__ __forceinline__ float2 cadd<float2>(float2 a, float2 b) {
  return __fadd2_rn(a, b);
}
template <> __device__ __forceinline__ float2 csub<float2>(float2 a, float2 b) {
  return __fadd2_rn(a, make_float2(-b.x, -b.y));
}
template <> __device__ __forceinline__ float2 cmul<float2>(float2 a, float2 b) {
  // (a.x b.x, a.x b.y) + (a.y (-b.y), a.y b.x)
  return __ffma2_rn(make_float2(a.y, a.y), make_float2(-b.y, b.x),
                    __fmul2_rn(make_float2(a.x, a.x), b));
}
template <> __device__ __forceinline__ float2 cmulc<float2>(float2 a, float2 b) {
  // (a.x b.x, -a.x b.y) + (a.y b.y, a.y b.x)
  return __ffma2_rn(make_float2(a.y, a.y), make_float2(b.y, b.x),
                    __fmul2_rn(make_float2(a.x, a.x), make_float2(b.x, -b.y)));
}
// multiply by i*s, s = +-1
template <int S, typename C> __device__ __forceinline__ C cmul_i(C a) {
  C r; if (S > 0) { r.x = -a.y; r.y = a.x; } else { r.x = a.y; r.y = -a.x; } return r;
}

// cos(2*pi*t/48) for the multiples of 2*pi/48 the codelets need (angles that
// are multiples of pi/8 or pi/6); exact constants from trigonometry.
__host__ __device__ constexpr double cos_q24(int t) {  // cos(pi*t/24), 0 <= t <= 12
  return t == 0 ? 1.0
       : t == 3 ? 0.92387953251128675613   // cos(pi/8)
       : t == 4 ? 0.86602540378443864676   // cos(pi/6) = sqrt(3)/2
       : t == 6 ? 0.70710678118654752440   // cos(pi/4) = sqrt(1/2)
       : t == 8 ? 0.5                      // cos(pi/3)
       : t == 9 ? 0.38268343236508977173   // cos(3pi/8)
       : t == 12 ? 0.0
       : 2.0;                              // never used
}
__host__ __device__ constexpr double cos48(int t) {
  return (t = ((t % 48) + 48) % 48, t = (t > 24 ? 48 - t : t),
          t > 12 ? -cos_q24(24 - t) : cos_q24(t));
}
__host__ __device__ constexpr double sin48(int t) { return cos48(12 - t); }

// a * exp(DIR * 2*pi*i * m / R) with compile-time m, R (48 % R == 0).
template <int DIR, int M, int R, typename C>
__device__ __forceinline__ C twc(C a) {
  constexpr int t = ((M % R) * (48 / R)) % 48;
  constexpr double c = cos48(t);
  constexpr double s = DIR * sin48(t);
  if constexpr (t == 0) {
    return a;
  } else if constexpr (t == 12 || t == 36) {
    return (s > 0) ? cmul_i<1>(a) : cmul_i<-1>(a);
  } else if constexpr (t == 24) {
    C r; r.x = -a.x; r.y = -a.y; return r;
  } else {
    using Rl = decltype(a.x);
    C w; w.x = (Rl)c; w.y = (Rl)s;
    return cmul(a, w);
  }
}

// ---------------------------------------------------------------------------
// Small DFTs in registers, natural order in and out.  DIR = -1 forward,
// +1 inverse (unnormalised).
template <int R, int DIR, typename C> struct Dft;

template <int DIR, typename C> struct Dft<1, DIR, C> {
  static __device__ __forceinline__ void run(C*) {}
};
template <int DIR, typename C> struct Dft<2, DIR, C> {
  static __device__ __forceinline__ void run(C* a) {
    C t = a[0]; a[0] = cadd(t, a[1]); a[1] = csub(t, a[1]);
  }
};
template <int DIR, typename C> struct Dft<3, DIR, C> {
  static __device__ __forceinline__ void run(C* a) {
    using Rl = decltype(a[0].x);
    const Rl h = (Rl)0.86602540378443864676;  // sin(2pi/3)
    C s = cadd(a[1], a[2]);
    C d = csub(a[1], a[2]);
    C m; m.x = a[0].x - (Rl)0.5 * s.x; m.y = a[0].y - (Rl)0.5 * s.y;
    a[0] = cadd(a[0], s);
    // X1 = m + DIR*i*h*d, X2 = m - DIR*i*h*d
    C r; r.x = -DIR * h * d.y; r.y = DIR * h * d.x;
    a[1] = cadd(m, r);
    a[2] = csub(m, r);
  }
};
template <int DIR, typename C> struct Dft<4, DIR, C> {
  static __device__ __forceinline__ void run(C* a) {
    C s02 = cadd(a[0], a[2]), d02 = csub(a[0], a[2]);
    C s13 = cadd(a[1], a[3]), d13 = csub(a[1], a[3]);
    C r = cmul_i<DIR>(d13);   // DIR*i*(a1 - a3)
    a[0] = cadd(s02, s13);
    a[2] = csub(s02, s13);
    a[1] = cadd(d02, r);
    a[3] = csub(d02, r);
  }
};

template <int P, int Q, int DIR, int N1, int K2, typename C>
__device__ __forceinline__ void tw_apply(C* b) {
  if constexpr (N1 < P) {
    if constexpr (K2 < Q) {
      b[N1 * Q + K2] = twc<DIR, N1 * K2, P * Q>(b[N1 * Q + K2]);
      tw_apply<P, Q, DIR, N1, K2 + 1>(b);
    } else {
      tw_apply<P, Q, DIR, N1 + 1, 1>(b);
    }
  }
}

// Composite R = P*Q in registers: n = n1 + P*n2, k = k2 + Q*k1.
template <int P, int Q, int DIR, typename C>
__device__ __forceinline__ void dft_pq(C* a) {
  C b[P * Q];
#pragma unroll
  for (int n1 = 0; n1 < P; ++n1) {
    C t[Q];
#pragma unroll
    for (int n2 = 0; n2 < Q; ++n2) t[n2] = a[n1 + P * n2];
    Dft<Q, DIR, C>::run(t);
#pragma unroll
    for (int k2 = 0; k2 < Q; ++k2) b[n1 * Q + k2] = t[k2];
  }
  // twiddles w_R^{n1*k2}, each a compile-time constant
  tw_apply<P, Q, DIR, 1, 1>(b);
#pragma unroll
  for (int k2 = 0; k2 < Q; ++k2) {
    C t[P];
#pragma unroll
    for (int n1 = 0; n1 < P; ++n1) t[n1] = b[n1 * Q + k2];
    Dft<P, DIR, C>::run(t);
#pragma unroll
    for (int k1 = 0; k1 < P; ++k1) a[k2 + Q * k1] = t[k1];
  }
}
template <int DIR, typename C> struct Dft<6, DIR, C> {
  static __device__ __forceinline__ void run(C* a) { dft_pq<2, 3, DIR, C>(a); }
};
template <int DIR, typename C> struct Dft<8, DIR, C> {
  static __device__ __forceinline__ void run(C* a) { dft_pq<2, 4, DIR, C>(a); }
};
template <int DIR, typename C> struct Dft<12, DIR, C> {
  static __device__ __forceinline__ void run(C* a) { dft_pq<4, 3, DIR, C>(a); }
};
template <int DIR, typename C> struct Dft<16, DIR, C> {
  static __device__ __forceinline__ void run(C* a) { dft_pq<4, 4, DIR, C>(a); }
};

// ---------------------------------------------------------------------------
// Length and factorisation of one axis transform.
struct Axis {
  int L, r1, r2;
};

// Shared-memory stages.  `addr(t, e)` gives the position of element e of
// transform t.  Tasks are numbered with the transform index fastest so that
// neighbouring lanes touch neighbouring transforms (conflict-free when the
// transforms are adjacent columns or rows with an odd pitch).
//
// tw: the L roots exp(-2*pi*i*m/L), m = 0..L-1.
template <int R2, int DIR, typename C, typename Addr>
__device__ __forceinline__ void stage_a_r(C* sm, const Addr& addr, int ntr, const Axis ax,
                                          const C* __restrict__ tw, int tid, int nthr) {
  const int tasks = ntr * ax.r1;
  for (int task = tid; task < tasks; task += nthr) {
    const int t = task % ntr, n1 = task / ntr;
    C a[R2];
#pragma unroll
    for (int j = 0; j < R2; ++j) a[j] = sm[addr(t, n1 + ax.r1 * j)];
    Dft<R2, DIR, C>::run(a);
    if (DIR < 0 && ax.r1 > 1) {
#pragma unroll
      for (int j = 1; j < R2; ++j) a[j] = cmul(a[j], __ldg(&tw[n1 * j]));
    }
#pragma unroll
    for (int j = 0; j < R2; ++j) sm[addr(t, n1 + ax.r1 * j)] = a[j];
  }
}

template <int R1, int DIR, typename C, typename Addr>
__device__ __forceinline__ void stage_b_r(C* sm, const Addr& addr, int ntr, const Axis ax,
                                          const C* __restrict__ tw, int tid, int nthr) {
  const int tasks = ntr * ax.r2;
  for (int task = tid; task < tasks; task += nthr) {
    const int t = task % ntr, b = task / ntr;
    C a[R1];
#pragma unroll
    for (int i = 0; i < R1; ++i) a[i] = sm[addr(t, i + R1 * b)];
    Dft<R1, DIR, C>::run(a);
    if (DIR > 0) {
#pragma unroll
      for (int i = 1; i < R1; ++i) a[i] = cmulc(a[i], __ldg(&tw[i * b]));
    }
#pragma unroll
    for (int i = 0; i < R1; ++i) sm[addr(t, i + R1 * b)] = a[i];
  }
}

#define ITP_RADIX_SWITCH(r, CALL)                  \
  switch (r) {                                     \
    case 2: CALL(2); break;                        \
    case 3: CALL(3); break;                        \
    case 4: CALL(4); break;                        \
    case 6: CALL(6); break;                        \
    case 8: CALL(8); break;                        \
    case 12: CALL(12); break;                      \
    case 16: CALL(16); break;                      \
    default: break;                                \
  }

// Stage A (forward: DIR=-1, twiddle after; inverse A': DIR=+1, no twiddle).
template <int DIR, typename C, typename Addr>
__device__ __forceinline__ void stage_a(C* sm, const Addr& addr, int ntr, const Axis ax,
                                        const C* __restrict__ tw, int tid, int nthr) {
#define ITP_CALL_A(R) stage_a_r<R, DIR>(sm, addr, ntr, ax, tw, tid, nthr)
  ITP_RADIX_SWITCH(ax.r2, ITP_CALL_A)
#undef ITP_CALL_A
}
// Stage B (forward: DIR=-1, no twiddle; inverse B': DIR=+1, twiddle after).
template <int DIR, typename C, typename Addr>
__device__ __forceinline__ void stage_b(C* sm, const Addr& addr, int ntr, const Axis ax,
                                        const C* __restrict__ tw, int tid, int nthr) {
  if (ax.r1 == 1) return;
#define ITP_CALL_B(R) stage_b_r<R, DIR>(sm, addr, ntr, ax, tw, tid, nthr)
  ITP_RADIX_SWITCH(ax.r1, ITP_CALL_B)
#undef ITP_CALL_B
}

// Forward transform (natural -> digit-swapped), barriers included.
template <typename C, typename Addr>
__device__ __forceinline__ void fft_forward(C* sm, const Addr& addr, int ntr, const Axis ax,
                                            const C* __restrict__ tw) {
  stage_a<-1>(sm, addr, ntr, ax, tw, threadIdx.x, blockDim.x);
  __syncthreads();
  if (ax.r1 > 1) {
    stage_b<-1>(sm, addr, ntr, ax, tw, threadIdx.x, blockDim.x);
    __syncthreads();
  }
}
// Inverse transform (digit-swapped -> natural), barriers included.
template <typename C, typename Addr>
__device__ __forceinline__ void fft_inverse(C* sm, const Addr& addr, int ntr, const Axis ax,
                                            const C* __restrict__ tw) {
  if (ax.r1 > 1) {
    stage_b<1>(sm, addr, ntr, ax, tw, threadIdx.x, blockDim.x);
    __syncthreads();
  }
  stage_a<1>(sm, addr, ntr, ax, tw, threadIdx.x, blockDim.x);
  __syncthreads();
}

// Position in shared memory of frequency k after a forward transform.
__device__ __forceinline__ int spec_pos(const Axis& ax, int k) {
  return (k / ax.r2) + ax.r1 * (k % ax.r2);
}
// Frequency held at position p after a forward transform.
__device__ __forceinline__ int spec_freq(const Axis& ax, int p) {
  return (p / ax.r1) + ax.r2 * (p % ax.r1);
}

}  // namespace itp
