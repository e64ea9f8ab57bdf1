// Instantiation unit of the FFT passes (fft_passes.cuh): the term sum, the
// factor tables, the layout transposes and the shared-memory sizes.  The
// passes are split over several translation units only so that nvcc
// compiles them in parallel.
#include "fft_passes.cuh"

namespace itp {

int plane_row_pitch(int nx) { return row_pitch(nx); }

size_t plane_smem_bytes(const GridDesc& g, int real_bytes) {
  return ((size_t)(g.ny / 2) * g.pp + g.nx + g.ny) * 2 * real_bytes;
}
size_t pencil_smem_bytes(const GridDesc& g, int real_bytes) {
  return ((size_t)g.nz * g.pencil_w + g.nz) * 2 * real_bytes;
}

cudaError_t launch_term_sum(const TermSumArgs& a, cudaStream_t st) {
  if (a.k < 1 || a.k > kMaxTermsK || (a.plane_pts & 3) || (a.plane_pitch & 3))
    return cudaErrorInvalidValue;
  const int nvec = a.plane_pts / 4;
  dim3 grid((nvec + 255) / 256 < 8 ? (nvec + 255) / 256 : 8, (unsigned)((long long)a.m * a.nz));
  term_sum_kernel<<<grid, 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_term_sum_group(const TermSumArgs* args, const int2* rows, int nrows, int nz,
                                  int plane_pts, cudaStream_t st) {
  if ((plane_pts & 3) || nrows < 1 || nrows > 65535 || nz < 1 || nz > 65535)
    return cudaErrorInvalidValue;
  const int nvec = plane_pts / 4;
  dim3 grid((nvec + 255) / 256 < 8 ? (nvec + 255) / 256 : 8, (unsigned)nrows, (unsigned)nz);
  term_sum_group_kernel<<<grid, 256, 0, st>>>(args, rows);
  return cudaGetLastError();
}

template cudaError_t launch_term_tables<float>(const GridDesc&, const double*, double, double,
                                               double, double, float*, float*, float*, float*,
                                               float*, cudaStream_t);
template cudaError_t launch_term_tables<double>(const GridDesc&, const double*, double, double,
                                                double, double, double*, double*, double*,
                                                double*, double*, cudaStream_t);
template cudaError_t launch_kinetic_tables<float>(const GridDesc&, double, double, double, float*,
                                                  float*, float*, cudaStream_t);
template cudaError_t launch_kinetic_tables<double>(const GridDesc&, double, double, double,
                                                   double*, double*, double*, cudaStream_t);
template cudaError_t launch_transpose_planes<double, double>(const double*, double*, long long,
                                                             int, int, cudaStream_t);
template cudaError_t launch_transpose_planes<double, float>(const double*, float*, long long, int,
                                                            int, cudaStream_t);
template cudaError_t launch_transpose_planes<float, double>(const float*, double*, long long, int,
                                                            int, cudaStream_t);

}  // namespace itp
