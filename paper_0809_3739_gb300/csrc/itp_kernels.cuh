// Internal launch interface between the C-ABI layer (itp_api.cu) and the
// device kernels (fft_passes.cuh, dense.cu, tc_gemm.cu).  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

namespace itp {

// Grid geometry and FFT plans shared by all passes of one handle.
struct GridDesc {
  int nx, ny, nz, nxh;       // nxh = nx/2 + 1
  int rx1, rx2, ry1, ry2, rz1, rz2;
  long long n_points;        // nx*ny*nz
  long long n_half;          // nz*ny*nxh (complex)
  int pp;                    // shared-memory pitch of a row pair (complex, odd)
  int pencil_w;              // kx columns per pencil CTA; 0: one thread per
                             // column, in TMEM (nz = 128, FP32)
  int pencil_pitch;          // shared-memory pitch of a pencil z-row (complex)
  // planes too large for one CTA run as row + column passes; per precision
  // (index 0: FP32, 1: FP64)
  int split_planes[2];
  int row_tb[2];             // row pairs per row-pass CTA
  int col_w[2];              // kx columns per column-pass CTA
};

// Pass kinds.
enum PlaneMode {
  PLANE_FWD_REAL = 0,   // real state * f_in -> half spectrum
  PLANE_MERGED = 1,     // half spectrum -> inverse -> * f_mid -> forward -> half spectrum
  PLANE_COMBINE = 2,    // half spectrum -> inverse -> * f_out -> acc (=|+=) c * u   (FP64 acc)
  PLANE_HPSI = 3,       // half spectrum -> inverse -> acc = u + V * psi            (FP64 acc)
  PLANE_TERM = 4,       // half spectrum -> inverse -> c * f_out * u over the plane itself
};

enum PencilMode {
  PENCIL_PROPAGATE = 0,  // * exp(-tau_i |k|^2 / 2) / N
  PENCIL_KINETIC = 1,    // * (|k|^2 / 2) / N
};

// Kinetic factor applied to the half spectrum at the end of a forward plane
// pass when the grid is planar (nz = 1, no pencil pass): as the pencil pass
// would, fx[kx] * fy[ky] * fz[0] (mode 0, propagation) or
// (fx[kx] + fy[ky] + fz[0]) * scale (mode 1, |k|^2/2 for H psi).  fx == null:
// none.
template <typename R>
struct KinFac {
  const R* fx = nullptr;
  const R* fy = nullptr;
  const R* fz = nullptr;
  int mode = 0;
  R scale = 0;
};

// Arguments of one plane pass over `m` states.  R is float or double.
template <typename R>
struct PlaneArgs {
  int mode;
  int m;                     // states
  const R* in_real;          // [m][N] real states (PLANE_FWD_REAL), also psi for PLANE_HPSI
  void* spec;                // [m][nz][ny][nxh] complex R (in and/or out)
  const R* f_in;             // [N] factor applied to the loaded real state (nullable)
  const R* f_mid;            // [N] factor between inverse and forward (PLANE_MERGED)
  const R* f_out;            // [N] factor applied before combining (PLANE_COMBINE)
  double* acc;               // [m][N] FP64 accumulator / H psi output
  R* phi_out;                // PLANE_COMBINE: if set, the finished sum acc + c*u is
                             // written here in precision R instead of back to acc
  double coef;               // c_i of the term
  int acc_init;              // 1: acc = c*u, 0: acc += c*u
  const double* V;           // [N] potential (PLANE_HPSI)
  const R* V_r;              // [N] potential in R (PLANE_HPSI with phi_out: output in R)
  const void* twx;           // nx roots (complex R)
  const void* twy;           // ny roots
  KinFac<R> kin;             // planar grids: kinetic factor after the forward pass
};

template <typename R>
struct PencilArgs {
  int mode;
  int m;
  void* spec;                // [m][nz][ny][nxh] complex R, in place
  const R* kx_tab;           // [nxh]  exp(-tau kx^2/2) or kx^2/2
  const R* ky_tab;           // [ny]
  const R* kz_tab;           // [nz]   (includes 1/N for PENCIL_PROPAGATE)
  R scale;                   // 1/N for PENCIL_KINETIC
  const void* twz;           // nz roots
};

// phi = sum_i term_i, exact up to the final rounding to FP32 (error-free
// TwoSum accumulation; mixed path): term_i holds the FP32 contribution
// c_i * f_i * u_i of term i, stored plane by plane with the half-spectrum
// plane pitch (floats); phi is [m][N].
constexpr int kMaxTermsK = 6;
struct TermSumArgs {
  int m, k, nz, plane_pts;
  long long plane_pitch;
  const float* term[kMaxTermsK];
  float* phi_out;
};
cudaError_t launch_term_sum(const TermSumArgs& a, cudaStream_t st);

size_t plane_smem_bytes(const GridDesc& g, int real_bytes);
int plane_row_pitch(int nx);   // odd pitch (complex) of a row pair in shared memory
size_t pencil_smem_bytes(const GridDesc& g, int real_bytes);

// Grouped launches over several problems with the same grid and launch
// shapes (batches): args[p] are problem p's arguments (device memory),
// rows[y] = (problem, state) of CTA row y, nrows (<= 65535) rows in all;
// the term sum takes the z planes as a third grid dimension.  Whole-plane
// passes only.
template <typename R>
cudaError_t launch_plane_group(const GridDesc& g, int mode, const PlaneArgs<R>* args,
                               const int2* rows, int nrows, cudaStream_t st);
template <typename R>
cudaError_t launch_pencil_group(const GridDesc& g, int mode, const PencilArgs<R>* args,
                                const int2* rows, int nrows, cudaStream_t st);
cudaError_t launch_term_sum_group(const TermSumArgs* args, const int2* rows, int nrows, int nz,
                                  int plane_pts, cudaStream_t st);

// One plane pass (*nlaunch receives the number of kernels: 1, or 2-3 when
// the planes are split into row and column passes).
template <typename R>
cudaError_t launch_plane(const GridDesc& g, const PlaneArgs<R>& a, cudaStream_t st,
                         int* nlaunch = nullptr);
template <typename R>
cudaError_t launch_pencil(const GridDesc& g, const PencilArgs<R>& a, cudaStream_t st);
// The pencil pass with one thread per z column and the column held in TMEM
// (nz = 128, FP32; GridDesc::pencil_w = 0 selects it in launch_pencil).
cudaError_t launch_pencil_tm(const GridDesc& g, const PencilArgs<float>& a, cudaStream_t st);

// Factor tables of one term, tau_i = tau / i:
//   f_half = exp(-tau_i V / 2), f_full = exp(-tau_i V)   ([N] each, precision R)
//   kx/ky/kz propagation tables (kz includes 1/N).
template <typename R>
cudaError_t launch_term_tables(const GridDesc& g, const double* V, double tau_i, double lx,
                               double ly, double lz, R* f_half, R* f_full, R* kx, R* ky, R* kz,
                               cudaStream_t st);
// Kinetic tables kx^2/2, ky^2/2, kz^2/2.
template <typename R>
cudaError_t launch_kinetic_tables(const GridDesc& g, double lx, double ly, double lz, R* kx,
                                  R* ky, R* kz, cudaStream_t st);

// dst[p][c][r] = src[p][r][c] over nplanes planes of rows x cols (converts
// the element type).  Moves states between the user layout [z][y][x] and
// the internal per-plane transposed layout [z][x][y].
template <typename TS, typename TD>
cudaError_t launch_transpose_planes(const TS* src, TD* dst, long long nplanes, int rows,
                                    int cols, cudaStream_t st);

// ---- dense part (dense.cu) ----
// Partial Gram sums: P[c][i][j] = sum_{p in chunk c} A[i][p] * B[j][p],
// multiplied in precision TC (FP32 products are summed in FP32 over runs of
// 256 points and those runs in FP64).
template <typename TA, typename TB, typename TC>
cudaError_t launch_gram_partial(const TA* A, const TB* B, int m, long long n_points,
                                int n_chunks, double* partial, cudaStream_t st);
// G = scale * sum_c P[c] (fixed order), symmetrised if sym.
cudaError_t launch_gram_reduce(const double* partial, int n_chunks, int m, double scale,
                               int sym, double* G, cudaStream_t st);
// Cholesky S = L L^T of an SPD m x m matrix and M = L^{-1} (lower).
// status[0] set to 1 if a pivot is not positive (S not positive definite).
cudaError_t launch_cholesky_inverse(const double* S, int m, double* Minv, int* status,
                                    cudaStream_t st);
// Symmetric eigen-decomposition (parallel cyclic Jacobi): E ascending,
// Rt = U^T so that Rt * Psi rotates the states onto the eigenvectors.
// work: m*m doubles.  status[0] |= 2 if the sweeps did not converge.
cudaError_t launch_jacobi_eigh(const double* H, int m, double* E, double* Rt, double* work,
                               int* status, cudaStream_t st);
// Eigenvalues only (ascending) of the symmetric m x m matrix H: Householder
// tridiagonalisation into work = (d[m], e[m]), then bisection into E.
cudaError_t launch_tridiag(const double* H, int m, double* work, cudaStream_t st);
cudaError_t launch_bisect(const double* work, int m, double* E, cudaStream_t st);
// out_j = dV sum_p (A[j][p] - c_j B[j][p])^2 over N points (N a multiple of
// 4), c_j = exp(scale E_j) (mode 1) or E_j (mode 0); partial: m * chunks
// doubles of scratch.  The residuals R^E (mode 1) and R^H (mode 0).
template <typename T>
cudaError_t launch_residual_norms(const T* A, const T* B, const double* E, double scale,
                                  int mode, int m, long long N, double dV, int chunks,
                                  double* partial, double* out, cudaStream_t st);
// out = a X + b Y elementwise (out may alias X).
template <typename R>
cudaError_t launch_axpby(double a, const R* X, double b, const R* Y, R* out, long long n,
                         cudaStream_t st);
// E[j] = H[j][j]
cudaError_t launch_diag(const double* H, int m, double* E, cudaStream_t st);
// Y = M * X over all points: Y[i][p] = sum_k M[i][k] X[k][p]   (M lower
// triangular if lower != 0), computed in the precision of TY.  X and Y must
// not overlap.
template <typename TX, typename TY>
cudaError_t launch_apply_matrix(const double* M, int m, int lower, const TX* X, TY* Y,
                                long long n_points, cudaStream_t st);
// Tensor-core (tcgen05 TF32, 3xTF32 split) versions, m <= 256; status gets
// bit 4 if a bounded mbarrier wait expired (the kernel then leaves its
// output unwritten).  expire_ns != 0 is the failure-detection test hook:
// every CTA first waits, with that limit and before issuing any copy or
// MMA, on an mbarrier phase that nothing completes.
// Gram: FP32 operands (16-byte aligned, n_points % 8 == 0) streamed in by
// bulk copies; A == B computes A A^T with one operand tile per step.
cudaError_t launch_tc_gram(const float* A, const float* B, int m, long long n_points,
                           int n_chunks, double* partial, int* status, cudaStream_t st,
                           unsigned long long expire_ns = 0);
// Apply: lower != 0 skips the blocks of M above the diagonal (zero for the
// inverse Cholesky factor); with m > 128 the launch walks 128-row blocks.
template <typename TX, typename TY>
cudaError_t launch_tc_apply(const double* M, int m, const TX* X, TY* Y, long long n_points,
                            int* status, cudaStream_t st, unsigned long long expire_ns = 0,
                            int lower = 0);
// Precision conversion of whole state blocks.
template <typename TS, typename TD>
cudaError_t launch_convert(const TS* src, TD* dst, long long count, cudaStream_t st);

}  // namespace itp
