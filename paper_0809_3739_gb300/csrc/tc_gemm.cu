// Tensor-core (tcgen05, TF32) contractions of the mixed-precision path:
//   gram:   P_c = X_c Y_c^T over a chunk c of grid points   (overlap S of
//           Eq. (4), subspace matrix of the Ritz step)
//   apply:  Y = M X over all points                         (psi = L^{-1} phi
//           of Eq. (4), rotation onto Ritz vectors)
// with X, Y the state blocks [m][N] (m <= 128) and M an m x m FP64 matrix.
//
// Precision: every operand is split into TF32 hi + lo parts (round to
// nearest) by the warps that stage it into shared memory, and each product
// is hi*hi + hi*lo + lo*hi ("3xTF32"), which keeps FP32 accuracy; the
// tensor core accumulates in FP32 in TMEM.  Gram partial sums per chunk are
// written in FP64 and reduced in FP64.
//
// Shared-memory operand layout: K-major, no swizzle, 8-row x 16-byte core
// matrices; core matrix (r/8, k/4) of a tile with KC four-element K chunks
// lives at ((r/8)*KC + k/4)*128 bytes, row r%8 at +16*(r%8).  The smem
// descriptor's leading byte offset (next core matrix along K) is 128 and its
// stride byte offset (next 8-row group) is KC*128.
//
// Every wait on an mbarrier is bounded; on expiry the kernel records
// ITP status bit 4 and carries on, so no launch can hang.
#include <cuda_runtime.h>
#include <stdint.h>

#include "itp_kernels.cuh"

namespace itp {

namespace {

constexpr int kTcThreads = 256;
constexpr unsigned long long kWaitLimitNs = 2000000000ull;   // 2 s per wait at most
constexpr int kStatusTimeout = 4;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n"
      " .reg .pred p;\n"
      " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait for the phase with the given parity to complete: gives up
// after kWaitLimitNs, records the timeout in the status word and returns.
__device__ __forceinline__ void mbar_wait(uint64_t* bar, uint32_t parity, int* status) {
  if (mbar_try_wait(bar, parity)) return;
  const unsigned long long t0 = global_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (global_ns() - t0 > kWaitLimitNs) {
      atomicOr(status, kStatusTimeout);
      return;
    }
  }
}

__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// TMEM allocation by one full warp; the base address lands in *dst.
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(dst)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}

// Shared-memory matrix descriptor: K-major, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;   // descriptor version of this architecture
  return d;                 // base offset 0, layout type 0 (no swizzle)
}

// Instruction descriptor of kind::tf32: D FP32, A and B TF32, both K-major.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n"
      " .reg .pred p;\n"
      " setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n"
      "}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

// 32 lanes x 32 consecutive 32-bit TMEM columns into registers.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// x -> (hi, lo) with hi = TF32(x) and lo = TF32(x - hi), round to nearest.
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hi) : "f"(x));
  const float r = x - __uint_as_float(hi);
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(lo) : "f"(r));
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c,
                                             uint32_t d) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c),
               "r"(d)
               : "memory");
}

template <typename T> __device__ __forceinline__ float ldf(const T* p) { return (float)__ldg(p); }

// Four consecutive values as floats (16-byte aligned for float, 32 for double).
__device__ __forceinline__ void ld4(const float* p, float (&v)[4]) {
  const float4 q = __ldg(reinterpret_cast<const float4*>(p));
  v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void ld4(const double* p, float (&v)[4]) {
  const double2 a = __ldg(reinterpret_cast<const double2*>(p));
  const double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
  v[0] = (float)a.x; v[1] = (float)a.y; v[2] = (float)b.x; v[3] = (float)b.y;
}

// ---------------------------------------------------------------------------
// Gram partial sums.  Tile = 128 rows x 32 points; two pipeline stages.
constexpr int kGramKT = 32;                          // points per tile
constexpr int kGramKC = kGramKT / 4;                 // 4-element K chunks
constexpr int kTileBytes = 128 * kGramKT * 4;        // 16 KB per operand part

// Stage one operand tile of rows [0,128) x points [p0, p0+32) as hi/lo TF32.
template <typename T>
__device__ __forceinline__ void stage_rows(const T* __restrict__ X, int m, long long N,
                                           long long p0, long long p_end, uint32_t hi_base,
                                           uint32_t lo_base) {
  // 1024 groups of (row, 4 points); lanes 0..7 of a group of 8 take rows
  // r%8 = 0..7 so the 16-byte shared stores are conflict-free.
#pragma unroll
  for (int q = 0; q < 1024 / kTcThreads; ++q) {
    const int L = threadIdx.x + kTcThreads * q;
    const int r = (L >> 6) * 8 + (L & 7);
    const int k4 = (L >> 3) & 7;
    const long long p = p0 + 4 * k4;
    float v[4] = {0.f, 0.f, 0.f, 0.f};
    if (r < m) {
      const T* src = X + (long long)r * N + p;
      if (p + 3 < p_end) {
        ld4(src, v);
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (p + e < p_end) v[e] = ldf(src + e);
      }
    }
    uint32_t h[4], l[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) split_tf32(v[e], h[e], l[e]);
    const uint32_t off = (uint32_t)(((r >> 3) * kGramKC + k4) * 128 + (r & 7) * 16);
    st_shared_v4(hi_base + off, h[0], h[1], h[2], h[3]);
    st_shared_v4(lo_base + off, l[0], l[1], l[2], l[3]);
  }
}

template <typename TA, typename TB>
__global__ void __launch_bounds__(kTcThreads, 1)
    tc_gram_kernel(const TA* __restrict__ A, const TB* __restrict__ B, int m, long long N,
                   long long chunk, double* __restrict__ partial, int* status) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  const bool same = (const void*)A == (const void*)B;
  // stage s: A_hi, A_lo, B_hi, B_lo (B parts unused when A == B)
  unsigned char* base = smraw;
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ uint32_t tmem_base;
  const uint32_t sbase = smem_u32(base);
  auto part = [&](int s, int which) { return sbase + (uint32_t)((s * 4 + which) * kTileBytes); };

  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_barrier_init();
  }
  if (threadIdx.x < 32) tmem_alloc(&tmem_base, 128);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;

  const long long p_begin = (long long)blockIdx.x * chunk;
  const long long p_end = min(N, p_begin + chunk);
  const int ntiles = p_end > p_begin ? (int)((p_end - p_begin + kGramKT - 1) / kGramKT) : 0;
  constexpr uint32_t idesc = idesc_tf32(128, 128);
  const uint32_t sbo = kGramKC * 128;

  for (int t = 0; t < ntiles; ++t) {
    const int s = t & 1;
    if (t >= 2) mbar_wait(&bar[s], (uint32_t)(((t - 2) >> 1) & 1), status);
    const long long p0 = p_begin + (long long)t * kGramKT;
    stage_rows(A, m, N, p0, p_end, part(s, 0), part(s, 1));
    if (!same) stage_rows(B, m, N, p0, p_end, part(s, 2), part(s, 3));
    fence_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
      tc_fence_after();
      const uint32_t ahi = part(s, 0), alo = part(s, 1);
      const uint32_t bhi = same ? ahi : part(s, 2), blo = same ? alo : part(s, 3);
#pragma unroll
      for (int ks = 0; ks < kGramKT / 8; ++ks) {
        const uint32_t koff = ks * 256;   // 8 TF32 = two core matrices along K
        const uint64_t dah = smem_desc(ahi + koff, 128, sbo);
        const uint64_t dal = smem_desc(alo + koff, 128, sbo);
        const uint64_t dbh = smem_desc(bhi + koff, 128, sbo);
        const uint64_t dbl = smem_desc(blo + koff, 128, sbo);
        mma_tf32(tmem, dah, dbh, idesc, (t > 0 || ks > 0) ? 1u : 0u);
        mma_tf32(tmem, dah, dbl, idesc, 1u);
        mma_tf32(tmem, dal, dbh, idesc, 1u);
      }
      mma_commit(&bar[s]);
    }
  }
  double* out = partial + (long long)blockIdx.x * m * m;
  if (ntiles > 0) {
    const int tl = ntiles - 1;
    mbar_wait(&bar[tl & 1], (uint32_t)((tl >> 1) & 1), status);
    tc_fence_after();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // warp w reads TMEM lane quadrant w % 4; warps 4.. take the upper column halves
    const int quad = warp & 3, chalf = warp >> 2;
    const int i = quad * 32 + lane;
#pragma unroll
    for (int cc = 0; cc < 2; ++cc) {
      const int c = chalf * 2 + cc;
      uint32_t r[32];
      tmem_ld32(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(c * 32), r);
      if (i < m) {
#pragma unroll
        for (int q = 0; q < 32; ++q) {
          const int j = c * 32 + q;
          if (j < m) out[(long long)i * m + j] = (double)__uint_as_float(r[q]);
        }
      }
    }
  } else {
    for (int e = threadIdx.x; e < m * m; e += kTcThreads) out[e] = 0.0;
  }
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x < 32) {
    tc_fence_after();
    tmem_dealloc(tmem, 128);
  }
}

// ---------------------------------------------------------------------------
// Y = M X.  A = M (128 x 128, staged once), B = tiles of 32 points x 128
// states (two stages), D = 128 states x 32 points in one of two TMEM slots.
constexpr int kApplyNT = 32;                          // points per tile
constexpr int kMBytes = 128 * 128 * 4;                // one part of M
constexpr int kXTileBytes = kApplyNT * 128 * 4;       // one part of an X tile

template <typename TX>
__device__ __forceinline__ void stage_points(const TX* __restrict__ X, int m, long long N,
                                             long long p0, uint32_t hi_base, uint32_t lo_base) {
  // 256 groups of (4 points, 4 states): four 16-byte loads along the point
  // axis (one per state row), a 4x4 register transpose, four 16-byte shared
  // stores (one per point, its 4 states = one core-matrix row).
  for (int L = threadIdx.x; L < 256; L += kTcThreads) {
    const int n4 = L & 7, k4 = L >> 3;   // k4 in 0..31
    const long long p = p0 + 4 * n4;
    float v[4][4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int k = 4 * k4 + e;
#pragma unroll
      for (int q = 0; q < 4; ++q) v[e][q] = 0.f;
      if (k < m) {
        const TX* src = X + (long long)k * N + p;
        if (p + 3 < N) {
          ld4(src, v[e]);
        } else {
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (p + q < N) v[e][q] = ldf(src + q);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int n = 4 * n4 + q;
      uint32_t h[4], l[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) split_tf32(v[e][q], h[e], l[e]);
      const uint32_t off = (uint32_t)(((n >> 3) * 32 + k4) * 128 + (n & 7) * 16);
      st_shared_v4(hi_base + off, h[0], h[1], h[2], h[3]);
      st_shared_v4(lo_base + off, l[0], l[1], l[2], l[3]);
    }
  }
}

// Epilogue of one finished tile: TMEM -> shared (warps 0..3, one lane
// quadrant each) -> coalesced 16-byte global stores by all threads.
template <typename TY>
__device__ __forceinline__ void apply_epilogue(uint32_t tmem_col, float* stage, int m,
                                               TY* __restrict__ Y, long long N, long long p0) {
  constexpr int NT = 32;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp < 4) {
    uint32_t r[32];
    tmem_ld32(tmem_col + ((uint32_t)(warp * 32) << 16), r);
    float* row = stage + (warp * 32 + lane) * (NT + 4);
#pragma unroll
    for (int q = 0; q < NT; q += 4)
      *reinterpret_cast<float4*>(row + q) =
          make_float4(__uint_as_float(r[q]), __uint_as_float(r[q + 1]),
                      __uint_as_float(r[q + 2]), __uint_as_float(r[q + 3]));
  }
  tc_fence_before();
  __syncthreads();
  // 128 rows x 8 float4 per row
  for (int L = threadIdx.x; L < 128 * (NT / 4); L += kTcThreads) {
    const int i = L >> 3, c4 = L & 7;
    if (i >= m) continue;
    const long long p = p0 + 4 * c4;
    const float4 v = *reinterpret_cast<const float4*>(stage + i * (NT + 4) + 4 * c4);
    TY* dst = Y + (long long)i * N + p;
    if (p + 3 < N) {
      *reinterpret_cast<float4*>(dst) = v;
    } else {
      const float w[4] = {v.x, v.y, v.z, v.w};
      for (int q = 0; q < 4; ++q)
        if (p + q < N) dst[q] = w[q];
    }
  }
}

template <typename TX, typename TY>
__global__ void __launch_bounds__(kTcThreads, 1)
    tc_apply_kernel(const double* __restrict__ Mg, int m, const TX* __restrict__ X,
                    TY* __restrict__ Y, long long N, int* status) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ uint32_t tmem_base;
  const uint32_t sbase = smem_u32(smraw);
  const uint32_t m_hi = sbase, m_lo = sbase + kMBytes;
  auto xpart = [&](int s, int which) {
    return sbase + 2u * kMBytes + (uint32_t)((s * 2 + which) * kXTileBytes);
  };
  float* ostage = reinterpret_cast<float*>(smraw + 2 * kMBytes + 4 * kXTileBytes);

  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_barrier_init();
  }
  if (threadIdx.x < 32) tmem_alloc(&tmem_base, 64);
  // M -> hi/lo, K-major: row i (output state), K = k (input state)
  for (int L = threadIdx.x; L < 128 * 32; L += kTcThreads) {
    const int i = (L >> 8) * 8 + (L & 7);
    const int k4 = (L >> 3) & 31;
    float v[4] = {0.f, 0.f, 0.f, 0.f};
    if (i < m) {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int k = 4 * k4 + e;
        if (k < m) v[e] = (float)Mg[i * m + k];
      }
    }
    // M = hi + lo, both TF32 parts of the FP32-rounded matrix
    uint32_t h[4], l[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) split_tf32(v[e], h[e], l[e]);
    const uint32_t off = (uint32_t)(((i >> 3) * 32 + k4) * 128 + (i & 7) * 16);
    st_shared_v4(m_hi + off, h[0], h[1], h[2], h[3]);
    st_shared_v4(m_lo + off, l[0], l[1], l[2], l[3]);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  constexpr uint32_t idesc = idesc_tf32(128, kApplyNT);
  const uint32_t sbo = 32 * 128;   // K = 128 -> 32 core matrices per 8-row group

  const long long ntiles = (N + kApplyNT - 1) / kApplyNT;
  int local = 0;
  long long prev_tile = -1;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++local) {
    const int s = local & 1;
    if (local >= 2) mbar_wait(&bar[s], (uint32_t)(((local - 2) >> 1) & 1), status);
    stage_points(X, m, N, tile * kApplyNT, xpart(s, 0), xpart(s, 1));
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0) {
      tc_fence_after();
      const uint32_t d = tmem + (uint32_t)(s * kApplyNT);
#pragma unroll
      for (int ks = 0; ks < 16; ++ks) {
        const uint32_t koff = ks * 256;
        const uint64_t dah = smem_desc(m_hi + koff, 128, sbo);
        const uint64_t dal = smem_desc(m_lo + koff, 128, sbo);
        const uint64_t dbh = smem_desc(xpart(s, 0) + koff, 128, sbo);
        const uint64_t dbl = smem_desc(xpart(s, 1) + koff, 128, sbo);
        mma_tf32(d, dah, dbh, idesc, ks > 0 ? 1u : 0u);
        mma_tf32(d, dah, dbl, idesc, 1u);
        mma_tf32(d, dal, dbh, idesc, 1u);
      }
      mma_commit(&bar[s]);
    }
    // epilogue of the previous tile (its MMAs ran while this tile staged)
    if (prev_tile >= 0) {
      const int ps = (local - 1) & 1;
      mbar_wait(&bar[ps], (uint32_t)(((local - 1) >> 1) & 1), status);
      tc_fence_after();
      apply_epilogue(tmem + (uint32_t)(ps * kApplyNT), ostage, m, Y, N, prev_tile * kApplyNT);
    }
    prev_tile = tile;
  }
  if (prev_tile >= 0) {
    const int ps = (local - 1) & 1;
    mbar_wait(&bar[ps], (uint32_t)(((local - 1) >> 1) & 1), status);
    tc_fence_after();
    apply_epilogue(tmem + (uint32_t)(ps * kApplyNT), ostage, m, Y, N, prev_tile * kApplyNT);
  }
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x < 32) {
    tc_fence_after();
    tmem_dealloc(tmem, 64);
  }
}

}  // namespace

template <typename TA, typename TB>
cudaError_t launch_tc_gram(const TA* A, const TB* B, int m, long long n_points, int n_chunks,
                           double* partial, int* status, cudaStream_t st) {
  if (m > 128 || m < 1) return cudaErrorInvalidValue;
  long long chunk = (n_points + n_chunks - 1) / n_chunks;
  chunk = (chunk + kGramKT - 1) / kGramKT * kGramKT;
  const size_t smem = 2 * 4 * (size_t)kTileBytes;   // 128 KB
  cudaError_t e = cudaFuncSetAttribute(tc_gram_kernel<TA, TB>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  tc_gram_kernel<TA, TB><<<n_chunks, kTcThreads, smem, st>>>(A, B, m, n_points, chunk, partial,
                                                             status);
  return cudaGetLastError();
}

template <typename TX, typename TY>
cudaError_t launch_tc_apply(const double* M, int m, const TX* X, TY* Y, long long n_points,
                            int* status, cudaStream_t st) {
  if (m > 128 || m < 1) return cudaErrorInvalidValue;
  // M hi/lo 128 KB, two X stages 64 KB, output staging 18 KB
  const size_t smem = 2 * (size_t)kMBytes + 4 * (size_t)kXTileBytes + 128 * (kApplyNT + 4) * 4;
  cudaError_t e = cudaFuncSetAttribute(tc_apply_kernel<TX, TY>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long ntiles = (n_points + kApplyNT - 1) / kApplyNT;
  const int blocks = (int)(ntiles < sms ? ntiles : sms);
  tc_apply_kernel<TX, TY><<<blocks, kTcThreads, smem, st>>>(M, m, X, Y, n_points, status);
  return cudaGetLastError();
}

template cudaError_t launch_tc_gram<float, float>(const float*, const float*, int, long long, int,
                                                  double*, int*, cudaStream_t);
template cudaError_t launch_tc_gram<float, double>(const float*, const double*, int, long long,
                                                   int, double*, int*, cudaStream_t);
template cudaError_t launch_tc_apply<float, float>(const double*, int, const float*, float*,
                                                   long long, int*, cudaStream_t);

}  // namespace itp
