// FFT passes with one whole transform per thread, the thread's working set
// held in tensor memory (TMEM).
//
// TMEM is the 256 KB per-SM store that the tcgen05 tensor-core instructions
// use for accumulators.  Read and written with tcgen05.ld / tcgen05.st it
// behaves as a private array per thread (thread i of a warp reaches TMEM lane
// 32 * (warp % 4) + i, every column of the CTA's allocation), on a data path
// of its own: neither the shared-memory pipe nor the L1 sees these accesses.
// A 128-point complex transform (1 KB in FP32) then runs inside one thread:
// each stage reads its inputs from TMEM into registers, does a small DFT
// there, and writes the outputs back, with no data exchange between
// threads and no barriers.  The passes of fft_passes.cuh instead hand every
// stage's outputs to other threads through shared memory.
//
// Pencil pass (the z transform of Eq. (so)'s kinetic factor): thread c owns
// column c of the flattened (state, ky, kx) index space, i.e. the 128 values
// spec[s][z][ky][kx], z = 0..127.  Forward transform, kinetic factor,
// inverse transform, in place.  With n = n1 + 8 n2 and k = k2 + 16 k1:
//   forward  stage 1 (per n1): Y(n1,k2) = w128^{n1 k2} DFT16_{n2}[x(n1 + 8 n2)](k2)
//            stage 2 (per k2): X(k2 + 16 k1) = DFT8_{n1}[Y(n1,k2)](k1)
//   factor   X(k) *= f(k)
//   inverse  stage 1 (per k2): Z(k2,a) = w128^{-a k2} IDFT8_{k1}[X(k2 + 16 k1)](a)
//            stage 2 (per a):  x(a + 8 b) = IDFT16_{k2}[Z(k2,a)](b)
// (w128 = exp(-2 pi i/128); IDFT unnormalised; the factor carries 1/N).
// Forward stage 2, the factor and inverse stage 1 touch the same eight
// values, so they run back to back in registers.  TMEM layout per thread:
// complex value (j, i) at columns 2 (8 j + i), 2 (8 j + i) + 1 with j = k2 and
// i = n1 or a; the k2 groups are contiguous (one 16-column load or store),
// the n1 / a groups are 16 columns apart (16 two-column accesses).
#pragma once
#include "fft_common.cuh"
#include "itp_kernels.cuh"
#include "tcgen05.cuh"

namespace itp {
namespace {

__device__ __forceinline__ float2 cscale2(float2 a, float s) {
  return __fmul2_rn(a, make_float2(s, s));
}

// ---- TMEM access (32x32b shape: thread i of the warp <-> lane base + i) ------
// The loads and stores only issue the access.  tcgen05.ld writes its
// destination registers, and tcgen05.st may read its source registers, after
// the instruction has issued, until the matching tcgen05.wait; so the wait
// helpers take those registers as in-out operands: a loaded value cannot be
// used, and a stored register cannot be reused, before the wait.
__device__ __forceinline__ void tm_ld_x16(uint32_t ta, uint32_t (&r)[16]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
               : "r"(ta)
               : "memory");
}
__device__ __forceinline__ void tm_st_x16(uint32_t ta, const uint32_t (&r)[16]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};"
               ::"r"(ta), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
               : "memory");
}
// 16 two-column accesses 16 columns apart: columns ta + 16 j, ta + 16 j + 1.
__device__ __forceinline__ void tm_ld_x2s16(uint32_t ta, uint32_t (&r)[32]) {
  asm volatile(
      "{\n .reg .b32 a;\n"
      "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%32];\n"
      "add.u32 a, %32, 16;\n tcgen05.ld.sync.aligned.32x32b.x2.b32 {%2, %3}, [a];\n"
      "add.u32 a, %32, 32;\n tcgen05.ld.sync.aligned.32x32b.x2.b32 {%4, %5}, [a];\n"
      "add.u32 a, %32, 48;\n tcgen05.ld.sync.aligned.32x32b.x2.b32 {%6, %7}, [a];\n"
      "add.u32 a, %32, 64;\n tcgen05.ld.sync.aligned.32x32b.x2.b32 {%8, %9}, [a];\n"
      "add.u32 a, %32, 80;\n tcgen05.ld.sync.aligned.32x32b.x2.b32 {%10, %11}, [a];\n"
      "add.u32 a, %32, 96;\n tcgen05.ld.sync.aligned.32x32b.x2.b32 {%12, %13}, [a];\n"
      "add.u32 a, %32, 112;\n tcgen05.ld.sync.aligned.32x32b.x2.b32 {%14, %15}, [a];\n"
      "add.u32 a, %32, 128;\n tcgen05.ld.sync.aligned.32x32b.x2.b32 {%16, %17}, [a];\n"
      "add.u32 a, %32, 144;\n tcgen05.ld.sync.aligned.32x32b.x2.b32 {%18, %19}, [a];\n"
      "add.u32 a, %32, 160;\n tcgen05.ld.sync.aligned.32x32b.x2.b32 {%20, %21}, [a];\n"
      "add.u32 a, %32, 176;\n tcgen05.ld.sync.aligned.32x32b.x2.b32 {%22, %23}, [a];\n"
      "add.u32 a, %32, 192;\n tcgen05.ld.sync.aligned.32x32b.x2.b32 {%24, %25}, [a];\n"
      "add.u32 a, %32, 208;\n tcgen05.ld.sync.aligned.32x32b.x2.b32 {%26, %27}, [a];\n"
      "add.u32 a, %32, 224;\n tcgen05.ld.sync.aligned.32x32b.x2.b32 {%28, %29}, [a];\n"
      "add.u32 a, %32, 240;\n tcgen05.ld.sync.aligned.32x32b.x2.b32 {%30, %31}, [a];\n"
      "}"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(ta)
      : "memory");
}
__device__ __forceinline__ void tm_st_x2s16(uint32_t ta, const uint32_t (&r)[32]) {
  asm volatile(
      "{\n .reg .b32 a;\n"
      "tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%1, %2};\n"
      "add.u32 a, %0, 16;\n tcgen05.st.sync.aligned.32x32b.x2.b32 [a], {%3, %4};\n"
      "add.u32 a, %0, 32;\n tcgen05.st.sync.aligned.32x32b.x2.b32 [a], {%5, %6};\n"
      "add.u32 a, %0, 48;\n tcgen05.st.sync.aligned.32x32b.x2.b32 [a], {%7, %8};\n"
      "add.u32 a, %0, 64;\n tcgen05.st.sync.aligned.32x32b.x2.b32 [a], {%9, %10};\n"
      "add.u32 a, %0, 80;\n tcgen05.st.sync.aligned.32x32b.x2.b32 [a], {%11, %12};\n"
      "add.u32 a, %0, 96;\n tcgen05.st.sync.aligned.32x32b.x2.b32 [a], {%13, %14};\n"
      "add.u32 a, %0, 112;\n tcgen05.st.sync.aligned.32x32b.x2.b32 [a], {%15, %16};\n"
      "add.u32 a, %0, 128;\n tcgen05.st.sync.aligned.32x32b.x2.b32 [a], {%17, %18};\n"
      "add.u32 a, %0, 144;\n tcgen05.st.sync.aligned.32x32b.x2.b32 [a], {%19, %20};\n"
      "add.u32 a, %0, 160;\n tcgen05.st.sync.aligned.32x32b.x2.b32 [a], {%21, %22};\n"
      "add.u32 a, %0, 176;\n tcgen05.st.sync.aligned.32x32b.x2.b32 [a], {%23, %24};\n"
      "add.u32 a, %0, 192;\n tcgen05.st.sync.aligned.32x32b.x2.b32 [a], {%25, %26};\n"
      "add.u32 a, %0, 208;\n tcgen05.st.sync.aligned.32x32b.x2.b32 [a], {%27, %28};\n"
      "add.u32 a, %0, 224;\n tcgen05.st.sync.aligned.32x32b.x2.b32 [a], {%29, %30};\n"
      "add.u32 a, %0, 240;\n tcgen05.st.sync.aligned.32x32b.x2.b32 [a], {%31, %32};\n"
      "}" ::"r"(ta), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
      : "memory");
}
template <int N>
__device__ __forceinline__ void tm_wait_ld(uint32_t (&r)[N]);
template <>
__device__ __forceinline__ void tm_wait_ld<16>(uint32_t (&r)[16]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;" : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]) : : "memory");
}
template <>
__device__ __forceinline__ void tm_wait_ld<32>(uint32_t (&r)[32]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;" : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31]) : : "memory");
}
template <int N>
__device__ __forceinline__ void tm_wait_st(uint32_t (&r)[N]);
template <>
__device__ __forceinline__ void tm_wait_st<16>(uint32_t (&r)[16]) {
  asm volatile("tcgen05.wait::st.sync.aligned;" : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]) : : "memory");
}
template <>
__device__ __forceinline__ void tm_wait_st<32>(uint32_t (&r)[32]) {
  asm volatile("tcgen05.wait::st.sync.aligned;" : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31]) : : "memory");
}
template <int N>
__device__ __forceinline__ void pack(const float2 (&v)[N], uint32_t (&r)[2 * N]) {
#pragma unroll
  for (int i = 0; i < N; ++i) {
    r[2 * i] = __float_as_uint(v[i].x);
    r[2 * i + 1] = __float_as_uint(v[i].y);
  }
}
template <int N>
__device__ __forceinline__ void unpack(const uint32_t (&r)[2 * N], float2 (&v)[N]) {
#pragma unroll
  for (int i = 0; i < N; ++i) v[i] = make_float2(__uint_as_float(r[2 * i]), __uint_as_float(r[2 * i + 1]));
}

// ---- pencil pass, nz = 128, FP32 ----------------------------------------------
constexpr int kTmThreads = 128;   // 4 warps: every TMEM lane once
constexpr int kTmCols = 256;      // TMEM columns per CTA: 128 complex per thread
constexpr int kTmPadSmem = 100 * 1024;   // per CTA: at most two CTAs per SM

// The 16 values z = n1 + 8 n2 (n2 = 0..15) of a column.
__device__ __forceinline__ void pencil_batch(const float2* col, long long zs, int n1,
                                             float2 (&v)[16]) {
  const float2* p = col + (long long)n1 * zs;
#pragma unroll
  for (int n2 = 0; n2 < 16; ++n2) v[n2] = p[(long long)(8 * n2) * zs];
}

// The column of flattened index c (clamped to the last one; `active` says
// whether c was in range) and its kx, ky factors.
struct PencilCol {
  float2* col;
  bool active;
  float fx, fy;
};
__device__ __forceinline__ PencilCol pencil_col(const GridDesc& g, const PencilArgs<float>& a,
                                                long long c, long long total) {
  PencilCol r;
  r.active = c < total;
  if (!r.active) c = total - 1;
  const long long cps = (long long)g.ny * g.nxh;
  const long long s = c / cps;
  const int q = (int)(c - s * cps);
  const int ky = q / g.nxh, kx = q - ky * g.nxh;
  r.col = static_cast<float2*>(a.spec) + s * g.n_half + q;
  r.fx = __ldg(&a.kx_tab[kx]);
  r.fy = __ldg(&a.ky_tab[ky]);
  return r;
}

constexpr int kTmPrefetch = 2;   // stage-1 input batches in flight per thread

// Forward stage 1 of batch n1: DFT16, twiddles w128^{n1 k2}, to TMEM.
__device__ __forceinline__ void pencil_stage1(float2 (&v)[16], int n1, const float2* tw,
                                              uint32_t tm) {
  Dft<16, -1, float2>::run(v);
#pragma unroll
  for (int k2 = 1; k2 < 16; ++k2) v[k2] = cmul(v[k2], tw[(n1 * k2) & 127]);
  uint32_t sr[32];
  pack<16>(v, sr);
  tm_st_x2s16(tm + 2 * n1, sr);
  tm_wait_st<32>(sr);
}

// Persistent: CTA b takes the 128-column tiles b, b + gridDim.x, ...  Threads
// past the last column compute on a valid column and store nothing (every
// thread of a warp must take part in the TMEM accesses).  The stage loops
// are not unrolled (the twiddles come from a table in shared memory), which
// keeps the kernel small enough for the instruction cache.  Global loads
// run ahead of the arithmetic: stage 1 loads batch n1 + 2 while it
// transforms batch n1, and the next tile's first two batches are loaded
// before the current tile's last stage.  (Waiting for each TMEM access one
// step later, after the next step's arithmetic, measured slower: the extra
// registers cost more than the hidden latency gained.)
template <int MODE>
__global__ void __launch_bounds__(kTmThreads, 2)
    pencil128_tm_kernel(const GridDesc g, const PencilArgs<float> a) {
  __shared__ uint32_t tbase;
  __shared__ float kz_s[128];    // kinetic factor along z
  __shared__ float2 tw_s[128];   // exp(-2 pi i m / 128)
  const int warp = threadIdx.x >> 5;
  kz_s[threadIdx.x] = a.kz_tab[threadIdx.x];
  tw_s[threadIdx.x] = static_cast<const float2*>(a.twz)[threadIdx.x];
  if (warp == 0) tmem_alloc(&tbase, kTmCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tm = tbase + ((uint32_t)(32 * warp) << 16);
  const long long zs = (long long)g.ny * g.nxh;
  const long long total = (long long)a.m * zs;
  const long long ntiles = (total + kTmThreads - 1) / kTmThreads;
  long long tile = blockIdx.x;
  PencilCol cur = pencil_col(g, a, tile * kTmThreads + threadIdx.x, total);
  float2 pf[kTmPrefetch][16];
#pragma unroll
  for (int b = 0; b < kTmPrefetch; ++b) pencil_batch(cur.col, zs, b, pf[b]);
  for (; tile < ntiles; tile += gridDim.x) {
    // forward stage 1, kTmPrefetch batches per iteration
#pragma unroll 1
    for (int n1 = 0; n1 < 8; n1 += kTmPrefetch) {
#pragma unroll
      for (int b = 0; b < kTmPrefetch; ++b) {
        float2 v[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = pf[b][i];
        if (n1 + b + kTmPrefetch < 8) pencil_batch(cur.col, zs, n1 + b + kTmPrefetch, pf[b]);
        pencil_stage1(v, n1 + b, tw_s, tm);
      }
    }
    // forward stage 2, factor, inverse stage 1
    const float fxy = cur.fx * cur.fy;
#pragma unroll 1
    for (int k2 = 0; k2 < 16; ++k2) {
      uint32_t r[16];
      tm_ld_x16(tm + 16 * k2, r);
      tm_wait_ld<16>(r);
      float2 u[8];
      unpack<8>(r, u);
      Dft<8, -1, float2>::run(u);
#pragma unroll
      for (int k1 = 0; k1 < 8; ++k1) {
        const float fz = kz_s[k2 + 16 * k1];
        float f;
        if constexpr (MODE == PENCIL_PROPAGATE) f = fxy * fz;
        else f = (cur.fx + cur.fy + fz) * a.scale;
        u[k1] = cscale2(u[k1], f);
      }
      Dft<8, 1, float2>::run(u);
#pragma unroll
      for (int aa = 1; aa < 8; ++aa) u[aa] = cmulc(u[aa], tw_s[(aa * k2) & 127]);
      pack<8>(u, r);
      tm_st_x16(tm + 16 * k2, r);
      tm_wait_st<16>(r);
    }
    // the next tile's first batches (a valid column in any case)
    const PencilCol nxt = pencil_col(g, a, (tile + gridDim.x) * kTmThreads + threadIdx.x, total);
#pragma unroll
    for (int b = 0; b < kTmPrefetch; ++b) pencil_batch(nxt.col, zs, b, pf[b]);
    // inverse stage 2
#pragma unroll 1
    for (int aa = 0; aa < 8; ++aa) {
      uint32_t r[32];
      tm_ld_x2s16(tm + 2 * aa, r);
      tm_wait_ld<32>(r);
      float2 w[16];
      unpack<16>(r, w);
      Dft<16, 1, float2>::run(w);
      if (cur.active) {
        float2* p = cur.col + (long long)aa * zs;
#pragma unroll
        for (int b = 0; b < 16; ++b) p[(long long)(8 * b) * zs] = w[b];
      }
    }
    cur = nxt;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tbase, kTmCols);
}

}  // namespace
}  // namespace itp
