// Instantiation unit of the FFT passes (fft_passes.cuh): the FP32 plane passes (whole planes, row and
// column passes, cluster planes).
// The passes are split over several translation units only so that nvcc
// compiles them in parallel.
#include "fft_passes.cuh"

namespace itp {

template cudaError_t launch_plane<float>(const GridDesc&, const PlaneArgs<float>&, cudaStream_t,
                                         int*);

}  // namespace itp
