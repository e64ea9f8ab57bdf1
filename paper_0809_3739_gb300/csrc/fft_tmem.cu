// Instantiation unit of the thread-per-transform FFT passes (fft_tmem.cuh).
#include "fft_tmem.cuh"

namespace itp {

cudaError_t launch_pencil_tm(const GridDesc& g, const PencilArgs<float>& a, cudaStream_t st) {
  if (g.nz != 128) return cudaErrorInvalidValue;
  const long long total = (long long)a.m * g.ny * g.nxh;
  if (total <= 0) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const long long ntiles = (total + kTmThreads - 1) / kTmThreads;
  const int grid = (int)(ntiles < 2LL * sms ? ntiles : 2LL * sms);
  // Unused dynamic shared memory caps residency at two CTAs per SM, the two
  // that the SM's 512 TMEM columns hold: a third would wait in tcgen05.alloc.
  auto kern = a.mode == PENCIL_PROPAGATE ? pencil128_tm_kernel<PENCIL_PROPAGATE>
                                         : pencil128_tm_kernel<PENCIL_KINETIC>;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kTmPadSmem);
  if (e != cudaSuccess) return e;
  kern<<<grid, kTmThreads, kTmPadSmem, st>>>(g, a);
  return cudaGetLastError();
}

}  // namespace itp
