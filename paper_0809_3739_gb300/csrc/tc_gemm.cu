// Tensor-core (tcgen05, TF32) contractions of the mixed-precision path:
//   gram:   P_c = X_c Y_c^T over a chunk c of grid points   (overlap S of
//           Eq. (4), subspace matrix of the Ritz step)
//   apply:  Y = M X over all points                         (psi = L^{-1} phi
//           of Eq. (4), rotation onto Ritz vectors)
// with X, Y the state blocks [m][N] (m <= 256) and M an m x m FP64 matrix.
// One MMA tile covers 128 states; m > 128 is cut into 128-row blocks: the
// Gram into blocks (bi, bj) of the result (one CTA column per block), the
// update into block products Y[bi] (=|+=) M[bi][bk] X[bk], one launch each.
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
// Every wait on an mbarrier is bounded by one deadline per launch, taken at
// kernel start.  When a wait expires, the CTA agrees on it at its next block
// barrier (__syncthreads_or), issues no further copy or MMA, waits a short
// bounded time for the copies and MMAs it has already issued, frees its
// TMEM, leaves its outputs unwritten and records ITP status bit 4; the host
// reports ITP_ERR_TIMEOUT.  A launch therefore ends within the deadline plus
// the drain limit.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include <mutex>

#include "itp_kernels.cuh"
#include "tcgen05.cuh"

namespace itp {

namespace {

constexpr int kTcThreads = 256;
constexpr unsigned long long kLaunchLimitNs = 2000000000ull;  // 2 s per launch at most
constexpr int kStatusTimeout = 4;

// ---------------------------------------------------------------------------
// Gram partial sums.  Tile = 128 rows x 32 points; two pipeline stages.
constexpr int kGramKT = 32;                          // points per tile
constexpr int kGramKC = kGramKT / 4;                 // 4-element K chunks
constexpr int kTileBytes = 128 * kGramKT * 4;        // 16 KB per operand part

// The tensor core's FP32 accumulation in TMEM is not round-to-nearest: summed
// over a chunk of ~10^5 points (thousands of accumulating MMAs) the diagonal
// of S came out low by ~1e-3 relative.  So every tile gets a fresh TMEM
// accumulator (two, alternating), and the threads add each finished tile
// into FP32 registers, where rounding is to nearest: 64 entries per thread.
//
// Raw tiles (128 state rows x 32 points, FP32) arrive by one 2D TMA load
// per operand into a ring of RAW stages, 128-byte swizzled: 16-byte chunk c
// of row r sits at chunk position c ^ (r % 8), so the converters' column
// reads are free of bank conflicts.  Rows beyond m and points beyond N are
// zero-filled by the TMA.  All warps convert a raw tile into the hi/lo
// canonical layout of one of two MMA stages; one thread issues the MMAs.
constexpr int kRawBytes = 128 * kGramKT * 4;        // 16 KB per operand

// Result blocks of one Gram launch: block b = blockIdx.y covers rows
// [128 bi, +128) of A against rows [128 bj, +128) of B, (bi, bj) packed as
// bi * 256 + bj; mirror: also write the block transposed.
struct TcBlocks {
  int n;
  int ij[4];
};

template <bool SAME>
__global__ void __launch_bounds__(kTcThreads, 1)
    tc_gram_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   int m, long long N, long long chunk, double* __restrict__ partial,
                   int* status, unsigned long long expire_ns, const TcBlocks blocks,
                   int mirror) {
  constexpr int NOPS = SAME ? 1 : 2;                // operands per tile
  constexpr int RAW = SAME ? 4 : 3;                 // raw ring depth
  extern __shared__ __align__(1024) unsigned char smraw[];
  __shared__ __align__(8) uint64_t full[RAW];
  __shared__ __align__(8) uint64_t mma_done[2];
  __shared__ uint32_t tmem_base;
  const uint32_t sbase = (smem_u32(smraw) + 1023u) & ~1023u;   // 1 KB for the swizzle
  unsigned char* sgen = smraw + (sbase - smem_u32(smraw));
  auto canon = [&](int c, int op, int part) {   // part 0 = hi, 1 = lo
    return sbase + (uint32_t)(((c * NOPS + op) * 2 + part) * kTileBytes);
  };
  const uint32_t raw_off = (uint32_t)(2 * NOPS * 2 * kTileBytes);
  auto raw = [&](int r, int op) { return sbase + raw_off + (uint32_t)((r * NOPS + op) * kRawBytes); };

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // one deadline for the whole launch (expire_ns != 0: the test hook's short limit)
  const unsigned long long deadline = global_ns() + (expire_ns ? expire_ns : kLaunchLimitNs);
  if (threadIdx.x == 0) {
    for (int r = 0; r < RAW; ++r) mbar_init(&full[r], 1);
    mbar_init(&mma_done[0], 1);
    mbar_init(&mma_done[1], 1);
    fence_barrier_init();
  }
  if (warp == 0) tmem_alloc(&tmem_base, 256);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  // Test hook: before any copy or MMA is issued, wait on a phase that nothing
  // completes (no copy has been issued on full[0] yet); it expires after
  // expire_ns and the CTA takes the abort path with nothing in flight.
  bool ok = expire_ns ? mbar_wait(&full[0], 0u, deadline) : true;

  // warp w reads TMEM lane quadrant w % 4; warps 4.. take the upper column halves
  const int quad = warp & 3, chalf = warp >> 2;
  float acc[64];
#pragma unroll
  for (int q = 0; q < 64; ++q) acc[q] = 0.f;
  auto drain = [&](int c) {   // all threads: acc += accumulator c
#pragma unroll
    for (int cc = 0; cc < 2; ++cc) {
      uint32_t rr[32];
      tmem_ld32(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(c * 128 + (chalf * 2 + cc) * 32),
                rr);
#pragma unroll
      for (int q = 0; q < 32; ++q) acc[cc * 32 + q] += __uint_as_float(rr[q]);
    }
  };

  const long long p_begin = (long long)blockIdx.x * chunk;
  const long long p_end = min(N, p_begin + chunk);
  const int ntiles = p_end > p_begin ? (int)((p_end - p_begin + kGramKT - 1) / kGramKT) : 0;

  const int bi = blocks.ij[blockIdx.y] >> 8, bj = blocks.ij[blockIdx.y] & 255;
  auto issue = [&](int t, int r) {   // one thread
    const int x = (int)(p_begin + (long long)t * kGramKT);
    mbar_arrive_expect_tx(&full[r], (uint32_t)(NOPS * kRawBytes));
    tma_load_2d(raw(r, 0), &tmA, x, 128 * bi, &full[r]);
    if (!SAME) tma_load_2d(raw(r, 1), &tmB, x, 128 * bj, &full[r]);
  };
  // tiles [0, issued) have their copies issued, [0, committed) their MMAs
  int issued = 0, committed = 0, t_stop = 0;
  bool aborted = __syncthreads_or(!ok) != 0;
  if (!aborted) {
    issued = RAW < ntiles ? RAW : ntiles;
    if (threadIdx.x == 0)
      for (int t = 0; t < issued; ++t) issue(t, t);
  }

  constexpr uint32_t idesc = idesc_tf32(128, 128);
  const uint32_t sbo = kGramKC * 128;
  for (int t = 0; t < ntiles && !aborted; ++t) {
    const int r = t % RAW, c = t & 1;
    ok = mbar_wait(&full[r], (uint32_t)((t / RAW) & 1), deadline);
    if (t >= 2) {   // tile t-2 is done: its stage and accumulator are free
      if (ok) ok = mbar_wait(&mma_done[c], (uint32_t)(((t - 2) >> 1) & 1), deadline);
      // TMEM loads are warp-collective: the warp drains only if all its lanes saw the MMA end
      if (__all_sync(0xffffffffu, ok)) {
        tc_fence_after();
        drain(c);
      }
    }
#pragma unroll
    for (int op = 0; op < NOPS; ++op) {
      const unsigned char* rp = sgen + raw_off + (r * NOPS + op) * kRawBytes;
#pragma unroll
      for (int q = 0; q < 1024 / kTcThreads; ++q) {
        const int L = threadIdx.x + kTcThreads * q;
        const int row = (L >> 6) * 8 + (L & 7);
        const int k4 = (L >> 3) & 7;
        const float4 x =
            *reinterpret_cast<const float4*>(rp + row * 128 + ((k4 ^ (row & 7)) << 4));
        uint32_t h[4], l[4];
        split_tf32(x.x, h[0], l[0]);
        split_tf32(x.y, h[1], l[1]);
        split_tf32(x.z, h[2], l[2]);
        split_tf32(x.w, h[3], l[3]);
        const uint32_t off = (uint32_t)(((row >> 3) * kGramKC + k4) * 128 + (row & 7) * 16);
        st_shared_v4(canon(c, op, 0) + off, h[0], h[1], h[2], h[3]);
        st_shared_v4(canon(c, op, 1) + off, l[0], l[1], l[2], l[3]);
      }
    }
    fence_async_smem();
    tc_fence_before();
    if (__syncthreads_or(!ok)) {   // a wait expired somewhere in the CTA
      aborted = true;
      t_stop = t;
      break;
    }
    committed = t + 1;
    if (t + RAW < ntiles) issued = t + RAW + 1;
    if (threadIdx.x == 0) {
      tc_fence_after();
      const uint32_t ahi = canon(c, 0, 0), alo = canon(c, 0, 1);
      const uint32_t bhi = canon(c, NOPS - 1, 0), blo = canon(c, NOPS - 1, 1);
#pragma unroll
      for (int ks = 0; ks < kGramKT / 8; ++ks) {
        const uint32_t koff = ks * 256;   // 8 TF32 = two core matrices along K
        const uint64_t dah = smem_desc(ahi + koff, 128, sbo);
        const uint64_t dal = smem_desc(alo + koff, 128, sbo);
        const uint64_t dbh = smem_desc(bhi + koff, 128, sbo);
        const uint64_t dbl = smem_desc(blo + koff, 128, sbo);
        const uint32_t d = tmem + (uint32_t)(c * 128);
        mma_tf32(d, dah, dbh, idesc, ks > 0 ? 1u : 0u);
        mma_tf32(d, dah, dbl, idesc, 1u);
        mma_tf32(d, dal, dbh, idesc, 1u);
      }
      mma_commit(&mma_done[c]);
      // raw slot r was consumed by every thread before the barrier above
      if (t + RAW < ntiles) issue(t + RAW, r);
    }
  }
  if (!aborted) {
    // the last two tiles are not drained yet
    ok = true;
    for (int tl = ntiles >= 2 ? ntiles - 2 : 0; tl < ntiles; ++tl) {
      if (ok) ok = mbar_wait(&mma_done[tl & 1], (uint32_t)((tl >> 1) & 1), deadline);
      if (__all_sync(0xffffffffu, ok)) {
        tc_fence_after();
        drain(tl & 1);
      }
    }
    if (__syncthreads_or(!ok)) {
      aborted = true;
      t_stop = ntiles;
    }
  }
  if (aborted) {
    // wait (bounded) for what is still in flight: the copies of tiles
    // [t_stop, issued) and the MMAs of the last two committed tiles
    if (threadIdx.x == 0) {
      atomicOr(status, kStatusTimeout);
      for (int t = t_stop; t < issued; ++t) drain_wait(&full[t % RAW], (uint32_t)((t / RAW) & 1));
      for (int t = committed >= 2 ? committed - 2 : 0; t < committed; ++t)
        drain_wait(&mma_done[t & 1], (uint32_t)((t >> 1) & 1));
    }
  } else {
    double* out = partial + (long long)blockIdx.x * m * m;
    const int i = 128 * bi + quad * 32 + lane;
    if (i < m) {
#pragma unroll
      for (int q = 0; q < 64; ++q) {
        const int j = 128 * bj + chalf * 64 + q;
        if (j < m) {
          out[(long long)i * m + j] = (double)acc[q];
          if (mirror) out[(long long)j * m + i] = (double)acc[q];
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, 256);
  }
}

// Driver entry point for tensor-map encoding (no link-time libcuda).
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// Tensor map of an m x N row-major FP32 block, box 32 points x 128 rows,
// 128-byte swizzle, out-of-range elements read as zero.
bool make_rows_map(CUtensorMap* tm, const float* X, int m, long long N) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)N, (cuuint64_t)m};
  cuuint64_t strides[1] = {(cuuint64_t)N * sizeof(float)};
  cuuint32_t box[2] = {(cuuint32_t)kGramKT, 128u};
  cuuint32_t estr[2] = {1u, 1u};
  return fn(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(X), dims, strides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// ---------------------------------------------------------------------------
// Y = M X.  A = M (128 x 128, staged once), B = tiles of 32 points x 128
// states (two stages), D = 128 states x 32 points in one of two TMEM slots.
constexpr int kApplyNT = 32;                          // points per tile
constexpr int kMBytes = 128 * 128 * 4;                // one part of M
constexpr int kXTileBytes = kApplyNT * 128 * 4;       // one part of an X tile

// Thread L of the CTA owns points n = n4 + 8q (q < 4) of the tile for the
// states k = 4 k4 + e (e < 4), n4 = L & 7, k4 = L >> 3: sixteen scalar loads
// (the 8 lanes of a k4 group read 32 consecutive bytes of a state row per
// load), held in registers; then, per point, one 16-byte shared store of
// its 4 states = row n & 7 = n4 of core matrix (n >> 3, k4).  The 8 lanes
// of a quarter-warp write the 8 rows of one core matrix, so the stores are
// free of bank conflicts.  Loading is split from storing so that the next
// tile's loads are in flight while the current tile is multiplied and
// written back.
static_assert(kTcThreads == 256, "one (4 points, 4 states) group per thread");
template <typename TX>
__device__ __forceinline__ void load_points(const TX* __restrict__ X, int m, long long N,
                                            long long p0, float (&v)[4][4]) {
  // X points at the block's first state row; m = its rows
  const int L = threadIdx.x;
  const int n4 = L & 7, k4 = L >> 3;   // k4 in 0..31
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int k = 4 * k4 + e;
    const TX* src = X + (long long)k * N + p0 + n4;
#pragma unroll
    for (int q = 0; q < 4; ++q)
      v[e][q] = (k < m && p0 + n4 + 8 * q < N) ? ldf(src + 8 * q) : 0.f;
  }
}
__device__ __forceinline__ void store_points(const float (&v)[4][4], uint32_t hi_base,
                                             uint32_t lo_base) {
  const int L = threadIdx.x;
  const int n4 = L & 7, k4 = L >> 3;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) split_tf32(v[e][q], h[e], l[e]);
    const uint32_t off = (uint32_t)((q * 32 + k4) * 128 + n4 * 16);
    st_shared_v4(hi_base + off, h[0], h[1], h[2], h[3]);
    st_shared_v4(lo_base + off, l[0], l[1], l[2], l[3]);
  }
}

// Epilogue of one finished tile: TMEM -> shared (warps 0..3, one lane
// quadrant each) -> coalesced 16-byte global stores by all threads.  ok:
// this thread saw the tile's MMAs complete; if any thread of the CTA did
// not, nothing is stored and false is returned (CTA-uniform).
template <typename TY>
__device__ __forceinline__ bool apply_epilogue(uint32_t tmem_col, float* stage, int m,
                                               TY* __restrict__ Y, long long N, long long p0,
                                               bool ok, int add) {
  constexpr int NT = 32;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // TMEM loads are warp-collective: a warp loads only if all its lanes saw the MMAs end
  if (warp < 4 && __all_sync(0xffffffffu, ok)) {
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
  if (__syncthreads_or(!ok)) return false;
  // 128 rows x 8 float4 per row
  for (int L = threadIdx.x; L < 128 * (NT / 4); L += kTcThreads) {
    const int i = L >> 3, c4 = L & 7;
    if (i >= m) continue;
    const long long p = p0 + 4 * c4;
    float4 v = *reinterpret_cast<const float4*>(stage + i * (NT + 4) + 4 * c4);
    TY* dst = Y + (long long)i * N + p;
    if (p + 3 < N) {
      if (add) {
        const float4 o = *reinterpret_cast<const float4*>(dst);
        v.x += o.x; v.y += o.y; v.z += o.z; v.w += o.w;
      }
      *reinterpret_cast<float4*>(dst) = v;
    } else {
      const float w[4] = {v.x, v.y, v.z, v.w};
      for (int q = 0; q < 4; ++q)
        if (p + q < N) dst[q] = add ? dst[q] + w[q] : w[q];
    }
  }
  return true;
}

// One block product Y[r0 + i] (=|+=) sum_k M[r0 + i][k0 + k] X[k0 + k],
// i < nr, k < nk (both <= 128): Mg is the full m x m matrix (row pitch m),
// X and Y already point at rows k0 and r0; add: the product is added to Y.
template <typename TX, typename TY>
__global__ void __launch_bounds__(kTcThreads, 1)
    tc_apply_kernel(const double* __restrict__ Mg, int m, int r0, int nr, int k0, int nk,
                    int add, const TX* __restrict__ X, TY* __restrict__ Y, long long N,
                    int* status, unsigned long long expire_ns) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ uint32_t tmem_base;
  const uint32_t sbase = smem_u32(smraw);
  const uint32_t m_hi = sbase, m_lo = sbase + kMBytes;
  auto xpart = [&](int s, int which) {
    return sbase + 2u * kMBytes + (uint32_t)((s * 2 + which) * kXTileBytes);
  };
  float* ostage = reinterpret_cast<float*>(smraw + 2 * kMBytes + 4 * kXTileBytes);
  // one deadline for the whole launch (expire_ns != 0: the test hook's short limit)
  const unsigned long long deadline = global_ns() + (expire_ns ? expire_ns : kLaunchLimitNs);

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
    if (i < nr) {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int k = 4 * k4 + e;
        if (k < nk) v[e] = (float)Mg[(long long)(r0 + i) * m + k0 + k];
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
  // bit s: an MMA commit on bar[s] not yet seen complete; its phase parity
  uint32_t pending = 0u, pend_parity = 0u;
  // Test hook: before any MMA is issued, wait on a phase that nothing
  // completes (no commit has been made on bar[0] yet); it expires after
  // expire_ns and the CTA takes the abort path with nothing in flight.
  bool ok = expire_ns ? mbar_wait(&bar[0], 0u, deadline) : true;
  bool aborted = __syncthreads_or(!ok) != 0;
  float cur[4][4], nxt[4][4];
  if ((long long)blockIdx.x < ntiles && !aborted)
    load_points(X, nk, N, (long long)blockIdx.x * kApplyNT, cur);
  for (long long tile = blockIdx.x; tile < ntiles && !aborted; tile += gridDim.x, ++local) {
    const int s = local & 1;
    ok = true;
    if (local >= 2) {
      ok = mbar_wait(&bar[s], (uint32_t)(((local - 2) >> 1) & 1), deadline);
      pending &= ~(1u << s);   // settled: complete, or drained below
    }
    store_points(cur, xpart(s, 0), xpart(s, 1));
    const long long next = tile + gridDim.x;
    if (next < ntiles) load_points(X, nk, N, next * kApplyNT, nxt);   // in flight meanwhile
    fence_async_smem();
    tc_fence_before();
    if (__syncthreads_or(!ok)) {   // a wait expired somewhere in the CTA
      pending |= 1u << s;          // tile local-2's MMAs may still run
      aborted = true;
      break;
    }
    // epilogue of the previous tile (its MMAs ran while this tile staged),
    // then this tile's MMAs: issued before the epilogue, they kept the
    // issuing thread's warp, and with it the epilogue's block barrier, waiting
    if (prev_tile >= 0) {
      const int ps = (local - 1) & 1;
      ok = mbar_wait(&bar[ps], (uint32_t)(((local - 1) >> 1) & 1), deadline);
      tc_fence_after();
      if (!apply_epilogue(tmem + (uint32_t)(ps * kApplyNT), ostage, nr, Y, N,
                          prev_tile * kApplyNT, ok, add)) {
        aborted = true;
        break;
      }
      pending &= ~(1u << ps);
    }
    pending |= 1u << s;
    pend_parity = (pend_parity & ~(1u << s)) | ((uint32_t)((local >> 1) & 1) << s);
    if (threadIdx.x == 0) {
      tc_fence_after();
      const uint32_t d = tmem + (uint32_t)(s * kApplyNT);
      // descriptors of the k-slices: the start-address field (bits 0-13,
      // address / 16) advances by 256 / 16 per slice of 8 K values
      const uint64_t ah = smem_desc(m_hi, 128, sbo), al = smem_desc(m_lo, 128, sbo);
      const uint64_t bh = smem_desc(xpart(s, 0), 128, sbo), bl = smem_desc(xpart(s, 1), 128, sbo);
#pragma unroll
      for (int ks = 0; ks < 16; ++ks) {
        const uint64_t step = (uint64_t)(ks * 16);
        mma_tf32(d, ah + step, bh + step, idesc, ks > 0 ? 1u : 0u);
        mma_tf32(d, ah + step, bl + step, idesc, 1u);
        mma_tf32(d, al + step, bh + step, idesc, 1u);
      }
      mma_commit(&bar[s]);
    }
    prev_tile = tile;
#pragma unroll
    for (int e = 0; e < 4; ++e)
#pragma unroll
      for (int q = 0; q < 4; ++q) cur[e][q] = nxt[e][q];
  }
  if (prev_tile >= 0 && !aborted) {
    const int ps = (local - 1) & 1;
    ok = mbar_wait(&bar[ps], (uint32_t)(((local - 1) >> 1) & 1), deadline);
    tc_fence_after();
    if (apply_epilogue(tmem + (uint32_t)(ps * kApplyNT), ostage, nr, Y, N, prev_tile * kApplyNT,
                       ok, add))
      pending &= ~(1u << ps);
    else
      aborted = true;
  }
  if (aborted && threadIdx.x == 0) {
    // wait (bounded) for the MMAs still in flight before TMEM is freed
    atomicOr(status, kStatusTimeout);
    for (int b = 0; b < 2; ++b)
      if ((pending >> b) & 1u) drain_wait(&bar[b], (pend_parity >> b) & 1u);
  }
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x < 32) {
    tc_fence_after();
    tmem_dealloc(tmem, 64);
  }
}

}  // namespace

cudaError_t launch_tc_gram(const float* A, const float* B, int m, long long n_points,
                           int n_chunks, double* partial, int* status, cudaStream_t st,
                           unsigned long long expire_ns) {
  if (m > 256 || m < 1 || (n_points % 8) || n_points >= (1LL << 31)) return cudaErrorInvalidValue;
  if ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B)) & 15)
    return cudaErrorInvalidValue;
  long long chunk = (n_points + n_chunks - 1) / n_chunks;
  chunk = (chunk + kGramKT - 1) / kGramKT * kGramKT;
  const bool same = A == B;
  CUtensorMap tmA, tmB;
  if (!make_rows_map(&tmA, A, m, n_points) || !make_rows_map(&tmB, B, m, n_points))
    return cudaErrorNotSupported;
  // 128 x 128 result blocks: A A^T takes the diagonal blocks with one operand
  // per tile and the lower off-diagonal ones (mirrored) with two; A B^T
  // takes every block with two operands
  const int nb = (m + 127) / 128;
  TcBlocks diag{}, pair{};
  for (int bi = 0; bi < nb; ++bi)
    for (int bj = 0; bj < nb; ++bj) {
      if (same && bi == bj) diag.ij[diag.n++] = bi * 256 + bj;
      else if (!same || bj < bi) pair.ij[pair.n++] = bi * 256 + bj;
    }
  cudaError_t e;
  if (diag.n) {
    const size_t smem = (size_t)2 * 1 * 2 * kTileBytes + (size_t)4 * 1 * kRawBytes + 1024;
    e = cudaFuncSetAttribute(tc_gram_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    tc_gram_kernel<true><<<dim3(n_chunks, diag.n), kTcThreads, smem, st>>>(
        tmA, tmB, m, n_points, chunk, partial, status, expire_ns, diag, 0);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (pair.n) {
    const size_t smem = (size_t)2 * 2 * 2 * kTileBytes + (size_t)3 * 2 * kRawBytes + 1024;
    e = cudaFuncSetAttribute(tc_gram_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    tc_gram_kernel<false><<<dim3(n_chunks, pair.n), kTcThreads, smem, st>>>(
        tmA, tmB, m, n_points, chunk, partial, status, expire_ns, pair, same ? 1 : 0);
  }
  return cudaGetLastError();
}

template <typename TX, typename TY>
cudaError_t launch_tc_apply(const double* M, int m, const TX* X, TY* Y, long long n_points,
                            int* status, cudaStream_t st, unsigned long long expire_ns,
                            int lower) {
  if (m > 256 || m < 1) return cudaErrorInvalidValue;
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
  // Y[bi] = sum_bk M[bi][bk] X[bk] (bk <= bi when M is lower triangular),
  // in stream order: the first block product sets Y[bi], the others add
  for (int r0 = 0; r0 < m; r0 += 128) {
    const int nr = m - r0 < 128 ? m - r0 : 128;
    for (int k0 = 0; k0 < m && (!lower || k0 <= r0); k0 += 128) {
      const int nk = m - k0 < 128 ? m - k0 : 128;
      tc_apply_kernel<TX, TY><<<blocks, kTcThreads, smem, st>>>(
          M, m, r0, nr, k0, nk, k0 > 0, X + (long long)k0 * n_points,
          Y + (long long)r0 * n_points, n_points, status, expire_ns);
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

template cudaError_t launch_tc_apply<float, float>(const double*, int, const float*, float*,
                                                   long long, int*, cudaStream_t,
                                                   unsigned long long, int);

}  // namespace itp
