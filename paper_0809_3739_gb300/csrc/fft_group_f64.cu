// Instantiation unit of the FFT passes (fft_passes.cuh): the grouped
// FP64 plane and pencil passes of batches.  The passes are split over
// several translation units only so that nvcc compiles them in parallel.
#include "fft_passes.cuh"

namespace itp {

template cudaError_t launch_plane_group<double>(const GridDesc&, int, const PlaneArgs<double>*,
                                              const int2*, int, cudaStream_t);
template cudaError_t launch_pencil_group<double>(const GridDesc&, int, const PencilArgs<double>*,
                                               const int2*, int, cudaStream_t);

}  // namespace itp
