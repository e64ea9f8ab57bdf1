// itp_orthonormalize_noalloc: the FP64 orthonormalisation (overlap, Cholesky,
// psi = L^{-1} phi) on caller-owned device buffers, for callers that cannot
// allocate device memory.
//
// Its scratch space -- the per-chunk partial overlap sums, the overlap
// matrix, its inverse Cholesky factor and a status word -- lives in one
// file-scope __device__ array, so a call allocates nothing.  The array is
// part of the library image: every GPU that loads libitp holds it
// (kNoallocBytes) until the process exits.
#include <cuda_runtime.h>

#include <stdint.h>

#include <mutex>

#include "itp.h"
#include "itp_kernels.cuh"

namespace {

constexpr int kNoallocMaxM = 128;                // states per call at most
constexpr int kNoallocChunks = 32;               // partial sums of the overlap
constexpr size_t kPartialDoubles = (size_t)kNoallocChunks * kNoallocMaxM * kNoallocMaxM;
constexpr size_t kMatDoubles = (size_t)kNoallocMaxM * kNoallocMaxM;
// partials (4 MiB) | S (128 KiB) | L^{-1} (128 KiB) | status (256 B)
constexpr size_t kNoallocBytes = (kPartialDoubles + 2 * kMatDoubles) * sizeof(double) + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
void* g_noalloc_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up
// once per device (cudaGetSymbolAddress, with that device current).
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" int itp_orthonormalize_noalloc(const double* phi_device, double* psi_device, int m,
                                          long long n_points, double dV, void* cuda_stream) {
  if (!phi_device || !psi_device || m < 1 || m > kNoallocMaxM || n_points < 1 ||
      n_points > (1LL << 48) || !(dV > 0))
    return ITP_ERR_ARG;
  // psi = L^{-1} phi is written while other CTAs still read phi: the two
  // byte ranges must be disjoint, not merely start at different addresses
  const uintptr_t bytes = (uintptr_t)m * (uintptr_t)n_points * sizeof(double);
  const uintptr_t a0 = reinterpret_cast<uintptr_t>(phi_device);
  const uintptr_t b0 = reinterpret_cast<uintptr_t>(psi_device);
  if (a0 < b0 + bytes && b0 < a0 + bytes) return ITP_ERR_ARG;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  void* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return ITP_ERR_CUDA;
  double* partial = static_cast<double*>(base);
  double* S = partial + kPartialDoubles;
  double* Minv = S + kMatDoubles;
  int* status = reinterpret_cast<int*>(Minv + kMatDoubles);
  // the array keeps the last call's contents: the status word must start at 0
  if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) return ITP_ERR_CUDA;
  using namespace itp;
  if (launch_gram_partial<double, double, double>(phi_device, phi_device, m, n_points,
                                                  kNoallocChunks, partial, st) != cudaSuccess ||
      launch_gram_reduce(partial, kNoallocChunks, m, dV, 1, S, st) != cudaSuccess ||
      launch_cholesky_inverse(S, m, Minv, status, st) != cudaSuccess ||
      launch_apply_matrix<double, double>(Minv, m, 1, phi_device, psi_device, n_points, st) !=
          cudaSuccess)
    return ITP_ERR_CUDA;
  int h_status = 0;
  if (cudaMemcpyAsync(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return ITP_ERR_CUDA;
  return (h_status & 1) ? ITP_ERR_NOT_PD : ITP_OK;
}
