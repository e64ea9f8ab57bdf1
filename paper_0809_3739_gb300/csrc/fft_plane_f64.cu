// Instantiation unit of the FFT passes (fft_passes.cuh): the FP64 plane passes (whole planes, row and
// column passes).
// The passes are split over several translation units only so that nvcc
// compiles them in parallel.
#include "fft_passes.cuh"

namespace itp {

template cudaError_t launch_plane<double>(const GridDesc&, const PlaneArgs<double>&, cudaStream_t,
                                          int*);

}  // namespace itp
