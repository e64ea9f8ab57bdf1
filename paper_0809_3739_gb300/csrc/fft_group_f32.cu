// Instantiation unit of the FFT passes (fft_passes.cuh): the grouped
// FP32 plane and pencil passes of batches.  The passes are split over
// several translation units only so that nvcc compiles them in parallel.
#include "fft_passes.cuh"

namespace itp {

template cudaError_t launch_plane_group<float>(const GridDesc&, int, const PlaneArgs<float>*,
                                              const int2*, int, cudaStream_t);
template cudaError_t launch_pencil_group<float>(const GridDesc&, int, const PencilArgs<float>*,
                                               const int2*, int, cudaStream_t);

}  // namespace itp
