// Instantiation unit of the FFT passes (fft_passes.cuh): the pencil passes (the z transform with the
// kinetic factor).
// The passes are split over several translation units only so that nvcc
// compiles them in parallel.
#include "fft_passes.cuh"

namespace itp {

template cudaError_t launch_pencil<float>(const GridDesc&, const PencilArgs<float>&, cudaStream_t);
template cudaError_t launch_pencil<double>(const GridDesc&, const PencilArgs<double>&, cudaStream_t);

}  // namespace itp
