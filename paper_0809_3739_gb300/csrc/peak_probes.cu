// Measured arithmetic rates of this GPU, the denominators of the ALU and
// tensor rooflines of the library's kernels (itp_peak_probe, include/itp.h):
//   FFMA   FP32 fused multiply-add, one value per instruction
//   FFMA2  the packed two-lane FP32 FMA of sm_100+ (the FFT codelets use it)
//   DFMA   FP64 fused multiply-add (the plain FP64 path's arithmetic)
//   TF32   tcgen05.mma kind::tf32, M = 128, N = 256, K = 8, FP32 accumulation
//          in TMEM (the overlap and update kernels' instruction)
// Each probe keeps every SM busy with long chains of independent operations
// and is timed with CUDA events on the caller's stream; no clock or other
// GPU setting is touched.  The FMA chains keep their values bounded
// (x <- x * a + b with |a| < 1), the MMA operands are finite.
#include <cuda_runtime.h>

#include "itp.h"
#include "tcgen05.cuh"

namespace itp {
namespace {

constexpr int kChains = 8;           // independent FMA chains per thread
constexpr int kFmaThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kFmaThreads) fma_probe_kernel(int iters, T a, T b, T* sink) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == (T)12345.678) sink[threadIdx.x] = s;   // keeps the chains alive
}

__global__ void __launch_bounds__(kFmaThreads) ffma2_probe_kernel(int iters, float a, float b,
                                                                  float* sink) {
  float2 x[kChains];
  const float2 av = make_float2(a, a), bv = make_float2(b, b);
#pragma unroll
  for (int c = 0; c < kChains; ++c)
    x[c] = make_float2((threadIdx.x + c) * 1e-3f, (threadIdx.x + 2 * c) * 1e-3f);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = __ffma2_rn(x[c], av, bv);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c].x + x[c].y;
  if (s == 12345.678f) sink[threadIdx.x] = s;
}

// One CTA per SM; one thread issues `iters` rounds of four K = 8 MMAs
// (128 x 256 x 32 per round) into one TMEM accumulator, then waits (bounded)
// for their completion.  A: 128 x 32 and B: 256 x 32 TF32 values in the
// canonical K-major layout (core matrices of 8 rows x 16 bytes).
constexpr int kMmaN = 256;
constexpr int kMmaK = 32;
constexpr int kMmaKC = kMmaK / 4;
__global__ void __launch_bounds__(128, 1) mma_probe_kernel(int iters, int* status) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  __shared__ __align__(8) uint64_t done;
  __shared__ uint32_t tmem_base;
  const uint32_t sa = smem_u32(smraw), sb = sa + 128 * kMmaK * 4;
  // finite operands: small values of both signs
  uint32_t* w = reinterpret_cast<uint32_t*>(smraw);
  for (int e = threadIdx.x; e < (128 + kMmaN) * kMmaK; e += blockDim.x)
    w[e] = __float_as_uint(((e * 37) % 17 - 8) * 0.0625f);
  if (threadIdx.x == 0) {
    mbar_init(&done, 1);
    fence_barrier_init();
  }
  if (threadIdx.x < 32) tmem_alloc(&tmem_base, kMmaN);
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  bool ok = true;
  if (threadIdx.x == 0) {
    constexpr uint32_t idesc = idesc_tf32(128, kMmaN);
    const uint32_t sbo = kMmaKC * 128;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int ks = 0; ks < kMmaK / 8; ++ks) {
        const uint64_t da = smem_desc(sa + ks * 256, 128, sbo);
        const uint64_t db = smem_desc(sb + ks * 256, 128, sbo);
        mma_tf32(tmem, da, db, idesc, (it | ks) ? 1u : 0u);
      }
    }
    mma_commit(&done);
    // every MMA signals `done` on completion; 10 s covers any sane iters
    ok = mbar_wait(&done, 0u, global_ns() + 10000000000ull);
    if (!ok) {
      atomicOr(status, 4);
      drain_wait(&done, 0u);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x < 32) {
    tc_fence_after();
    tmem_dealloc(tmem, kMmaN);
  }
}

}  // namespace
}  // namespace itp

using namespace itp;

extern "C" int itp_peak_probe(int kind, void* cuda_stream, double* tflops, double* ms_out) {
  if (!tflops || kind < ITP_PROBE_FFMA || kind > ITP_PROBE_TF32_MMA) return ITP_ERR_ARG;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return ITP_ERR_CUDA;
  void* sink = nullptr;
  int* status = nullptr;
  if (cudaMalloc(&sink, kFmaThreads * sizeof(double)) != cudaSuccess) return ITP_ERR_OOM;
  if (cudaMalloc(&status, sizeof(int)) != cudaSuccess) {
    cudaFree(sink);
    return ITP_ERR_OOM;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = ITP_OK;
  if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    rc = ITP_ERR_CUDA;
  // work per launch: ~50-100 ms at the expected rates
  const int blocks_fma = sms * 8;
  const int iters_fma = kind == ITP_PROBE_DFMA ? 20000 : 400000;
  const int iters_mma = 200000;
  const size_t smem_mma = (size_t)(128 + kMmaN) * kMmaK * 4;
  double flops = 0.0;
  if (kind == ITP_PROBE_TF32_MMA) {
    flops = (double)sms * iters_mma * 2.0 * 128 * kMmaN * kMmaK;
    if (rc == ITP_OK && cudaFuncSetAttribute(mma_probe_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem_mma) != cudaSuccess)
      rc = ITP_ERR_CUDA;
  } else {
    flops = (double)blocks_fma * kFmaThreads * iters_fma * kChains * 2.0 *
            (kind == ITP_PROBE_FFMA2 ? 2.0 : 1.0);
  }
  float best = 1e30f;
  for (int rep = 0; rep < 4 && rc == ITP_OK; ++rep) {   // the first launch warms up
    cudaEventRecord(e0, st);
    switch (kind) {
      case ITP_PROBE_FFMA:
        fma_probe_kernel<float><<<blocks_fma, kFmaThreads, 0, st>>>(iters_fma, 0.999f, 1e-4f,
                                                                    (float*)sink);
        break;
      case ITP_PROBE_FFMA2:
        ffma2_probe_kernel<<<blocks_fma, kFmaThreads, 0, st>>>(iters_fma, 0.999f, 1e-4f,
                                                               (float*)sink);
        break;
      case ITP_PROBE_DFMA:
        fma_probe_kernel<double><<<blocks_fma, kFmaThreads, 0, st>>>(iters_fma, 0.999, 1e-4,
                                                                     (double*)sink);
        break;
      default:
        mma_probe_kernel<<<sms, 128, smem_mma, st>>>(iters_mma, status);
        break;
    }
    cudaEventRecord(e1, st);
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
      rc = ITP_ERR_CUDA;
      break;
    }
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    if (rep > 0 && t < best) best = t;
  }
  int h_status = 0;
  if (rc == ITP_OK && cudaMemcpy(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost) !=
                          cudaSuccess)
    rc = ITP_ERR_CUDA;
  if (rc == ITP_OK && (h_status & 4)) rc = ITP_ERR_TIMEOUT;
  if (rc == ITP_OK) {
    *tflops = flops / (best * 1e-3) / 1e12;
    if (ms_out) *ms_out = best;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(sink);
  cudaFree(status);
  return rc;
}
