/*
 * itp.h -- C ABI of the GB300 multi-product imaginary-time propagation
 * library (libitp.so).
 *
 * Method: Chin, Janecek, Krotscheck, "Any order imaginary time propagation
 * method for solving the Schroedinger equation".  The lowest n eigenstates
 * of H = -(1/2) nabla^2 + V (Eq. 2, Hartree units, hbar = m = 1) on a
 * periodic 3D grid are found by repeating
 *     phi_j = T_2k(tau) psi_j            for every state        (Eq. 3)
 *     psi   = orthonormalised phi                                (Eq. 4)
 * with the order-2k multi-product propagator (Eqs. mcomp, coef)
 *     T_2k(tau) = sum_{i=1..k} c_i T_2(tau/i)^i,
 *     c_i = prod_{j != i} i^2 / (i^2 - j^2),
 *     T_2(tau) = exp(-tau V/2) exp(-tau T) exp(-tau V/2)         (Eq. so).
 * tau > 0 is the imaginary time step (the paper's eps = -tau).
 *
 * Conventions shared by every entry point:
 *  - Grid: nx*ny*nz points, each edge even and a product of two factors
 *    from {1,2,3,4,6,8,12,16} (2..256 points); box [-L/2, L/2) per axis,
 *    x_i = -L/2 + i*L/n; periodic.  Point index (z*ny + y)*nx + x.
 *    nz = 1 makes the problem two-dimensional (the paper's second case, a
 *    square array of quantum dots, Sec. III): the z transform is the
 *    identity and k_z = 0; with lz = 1 the volume element is dx*dy.
 *  - States: a block of m = n_states + n_guard real states, row-major
 *    [m][nz][ny][nx] doubles on the host.  Guard states are propagated and
 *    orthonormalised like the others; they speed up the convergence of the
 *    highest wanted states and are reported after them.
 *  - Normalisation: sum_r psi(r)^2 dV = 1, dV = (lx/nx)(ly/ny)(lz/nz).
 *  - Ownership: the library owns all device memory of a handle.  Host arrays
 *    passed in are copied during the call and may be reused on return.
 *  - Streams: all device work of a handle is issued on the CUDA stream given
 *    at creation (or on a stream the handle creates), in call order.  Calls that
 *    return host data (itp_energies, itp_get_states, itp_polish,
 *    itp_synchronize) synchronise that stream; the others do not.
 *  - Errors: every int-returning call returns ITP_OK (0) or an ITP_ERR_*
 *    code; itp_last_error() gives a one-line description of the most recent
 *    failure on the handle.  A failed call leaves the states unspecified but
 *    the handle usable (except after ITP_ERR_CUDA from a sticky device
 *    error).
 *  - A handle may be used by one host thread at a time.
 */
#ifndef ITP_H_
#define ITP_H_

#ifdef __cplusplus
extern "C" {
#endif

#define ITP_OK 0
#define ITP_ERR_ARG 1      /* bad argument or unsupported size             */
#define ITP_ERR_CUDA 2     /* a CUDA runtime call or kernel launch failed  */
#define ITP_ERR_NOT_PD 3   /* overlap matrix not positive definite (Eq. 4) */
#define ITP_ERR_TIMEOUT 4  /* a bounded device-side wait expired           */
#define ITP_ERR_OOM 5      /* device memory allocation failed              */
#define ITP_ERR_STATE 6    /* call out of order (e.g. no potential set)    */
#define ITP_ERR_NOCONV 7   /* subspace eigen-decomposition did not converge */

typedef enum {
  ITP_FP64 = 0,  /* every step in FP64                                      */
  ITP_MIXED = 1  /* FP32 FFT passes, FP64 combination / Cholesky / energies */
} itp_precision;

#define ITP_RITZ 1         /* itp_energies: Ritz values, states rotated onto Ritz vectors */
#define ITP_RITZ_VALUES 2  /* itp_energies: Ritz values only, states left as they are   */
#define ITP_EVAL_FP64 8    /* itp_energies, mixed precision: evaluate in FP64 (below)    */

typedef struct itp_grid* itp_handle;

/* Create a handle for one problem.
 *   out          receives the handle (NULL on failure)
 *   nx, ny, nz   grid points per axis (see conventions)
 *   lx, ly, lz   box lengths (bohr), > 0
 *   n_states     wanted states n >= 1; n_guard >= 0 extra guard states;
 *                m = n + n_guard <= 256 (the n x n work runs in blocks of
 *                128 states: m > 128 costs up to four times the m <= 128
 *                overlap and three times the update per block of states)
 *   precision    ITP_FP64 or ITP_MIXED
 *   cuda_stream  cudaStream_t to issue work on (NULL: default stream)
 * Allocates all device memory for the states, the half-spectrum workspace
 * and the FP64 accumulator.  Returns ITP_ERR_ARG / ITP_ERR_OOM /
 * ITP_ERR_CUDA on failure. */
int itp_create_grid(itp_handle* out, int nx, int ny, int nz, double lx, double ly, double lz,
                    int n_states, int n_guard, int precision, void* cuda_stream);

/* Release every resource of the handle (NULL is a no-op). */
void itp_destroy(itp_handle h);

/* Copy the potential V(r) (Hartree), host [nz][ny][nx] doubles.  Must be
 * called before itp_propagate / itp_energies. */
int itp_set_potential(itp_handle h, const double* V_host);

/* Copy m = n_states + n_guard states, host [m][nz][ny][nx] doubles.  They
 * need not be orthonormal.  ITP_MIXED rounds them to FP32. */
int itp_set_states(itp_handle h, const double* psi_host);

/* Same, from device memory (FP64, [m][N], on the handle's device; read on
 * the handle's stream). */
int itp_set_states_device(itp_handle h, const double* psi_device);

/* Copy the current m states to host [m][nz][ny][nx] doubles (synchronises). */
int itp_get_states(itp_handle h, double* psi_host);

/* Eq. (3): phi_j = T_2k(tau) psi_j for all m states, order = 2k with
 * 2 <= order <= 12 even, tau > 0.  The result is held in the FP64
 * accumulator until itp_orthonormalize.  Sec. II, Eqs. (so), (mcomp),
 * (coef): per term i the plane and pencil passes apply
 * exp(-tau V/2i), then (FFT, exp(-tau|k|^2/2i), inverse FFT, exp(-tau V/i))
 * i-1 times, then (FFT, kinetic, inverse FFT, exp(-tau V/2i)), and add
 * c_i times the result; negative c_i subtract (end of Sec. II). */
int itp_propagate(itp_handle h, int order, double tau);

/* Copy the result of the last itp_propagate, phi_j = T_2k(tau) psi_j, to host
 * [m][nz][ny][nx] doubles (synchronises).  ITP_ERR_STATE if no propagated
 * block is pending (itp_orthonormalize consumes it). */
int itp_get_phi(itp_handle h, double* phi_host);

/* Eq. (4): S = Phi Phi^T dV, S = L L^T (FP64 Cholesky), psi = L^{-1} phi.
 * A non-positive pivot is recorded on the device and reported as
 * ITP_ERR_NOT_PD by the next synchronising call (itp_energies,
 * itp_get_states, itp_synchronize). */
int itp_orthonormalize(itp_handle h);

/* Energies of the (orthonormal) current states, FP64 (Eq. 2):
 *   flags == 0: E_host[j], j < m, receives (psi_j|H|psi_j) dV.
 *   ITP_RITZ: the eigenvalues (ascending) of the subspace matrix
 *     (psi_i|H|psi_j) dV, and the states are rotated onto its eigenvectors
 *     (the subspace step of Sec. III; parallel cyclic Jacobi).
 *   ITP_RITZ_VALUES: the same eigenvalues (Householder tridiagonalisation and
 *     bisection), states unchanged.  The span of the states, and with it the
 *     Ritz values of every later iteration, does not depend on the basis
 *     (Eq. 4 keeps the span), so the rotation only matters when individual
 *     Ritz vectors are read out: iterate with ITP_RITZ_VALUES and finish with
 *     one ITP_RITZ.
 *   ITP_EVAL_FP64 (with 0, ITP_RITZ or ITP_RITZ_VALUES): the final energy
 *     evaluation of the mixed path in FP64 -- the FP32 states are rounded up
 *     to FP64, orthonormalised again in FP64 (Eq. 4: FP64 overlap, Cholesky
 *     and update; the span does not change) and the energies computed in
 *     FP64.  No propagation step is taken.  The states stay FP64 until the
 *     next itp_propagate / itp_step, which continues in FP32.  Converged
 *     FP32 states carry an FP32 rounding error of ~1e-7 in each component;
 *     FP64 Ritz values of them are accurate to its square, while FP32 energy
 *     evaluation is accurate only to ~1e-7 relative.  On ITP_FP64 handles
 *     the flag changes nothing.
 *   E_host may be NULL.  Synchronises; returns a pending ITP_ERR_NOT_PD /
 *   ITP_ERR_NOCONV; ITP_ERR_ARG for unknown flags. */
int itp_energies(itp_handle h, double* E_host, int flags);

/* One whole step -- itp_propagate(order, tau), itp_orthonormalize,
 * itp_energies(flags) -- replayed from a CUDA graph.  The first call for a
 * given (order, tau, flags, precision lane) captures the step's kernels and
 * the copy of the energies into a graph on the handle's stream; later calls
 * launch the graph (one launch instead of ~60).  flags: 0 or
 * ITP_RITZ_VALUES (ITP_RITZ moves the states between buffers and is not
 * captured).  Synchronises; E_host (nullable) receives the m energies.
 * Per-kernel profiling (itp_profile) does not see graph replays. */
int itp_step(itp_handle h, int order, double tau, int flags, double* E_host);

/* One whole step between host buffers: the result of
 *     itp_set_states(psi_in_host); itp_step(order, tau, flags, E_host);
 *     itp_get_states(psi_out_host)
 * (the same kernels on the same values, so bit for bit the same states and
 * energies), with the copies overlapped with the device work.  The states
 * move in 4 chunks of whole states (fewer if m < 4) on a second stream of the
 * library's own: chunk c is copied in while chunk c-1 is propagated (Eq. 3
 * acts on each state alone); after the orthonormalisation (Eq. 4, which
 * needs every state) the result goes out chunk by chunk while the energies
 * are computed.
 *   psi_in_host   [m][nz][ny][nx] doubles, read (not necessarily orthonormal)
 *   psi_out_host  [m][nz][ny][nx] doubles, written: the orthonormalised
 *                 states after the step; may be psi_in_host itself
 *   E_host        (nullable) the m energies, as itp_step
 * flags: 0 or ITP_RITZ_VALUES.  Page-locked host buffers (cudaHostAlloc or
 * cudaHostRegister) are needed for the copies to overlap; pageable ones
 * give the same results with the copies serialised.  The first call
 * allocates an FP64 staging block of m x N doubles and the copy stream.
 * Work already queued on the handle's stream runs first.  Synchronises;
 * neither buffer is touched after the call returns, also on failure.  Runs
 * kernel by kernel (not from a graph); itp_profile sees every launch. */
int itp_step_host(itp_handle h, int order, double tau, int flags, const double* psi_in_host,
                  double* psi_out_host, double* E_host);

/* Mixed precision only: switch the states to FP64 and iterate FP64 steps
 * (propagate, orthonormalise, Ritz values) until
 * max_{j<n_states} |E_j - E_j(previous)| < tol or max_steps steps, then
 * rotate the states onto the Ritz vectors (one ITP_RITZ evaluation).
 * steps_out (nullable) receives the number of steps, E_host (nullable) the
 * m final energies.  Later itp_propagate calls continue in FP32. */
int itp_polish(itp_handle h, int order, double tau, double tol, int max_steps, int* steps_out,
               double* E_host);

/* Eq. (sixp), the Romberg-type sixth-order propagator that the paper sets
 * against the multi-product expansion:
 *     phi_j = -T_4(tau) psi_j / 15 + 16 T_4(tau/2)^2 psi_j / 15,
 * T_4 the order-4 multi-product expansion (Eq. four).  It costs 9 complete
 * FFT pairs per state where the multi-product T_6 costs 6.  With T_4 a sum
 * of products (not time-symmetric) it cancels the tau^5 term only: its
 * local error is tau^6, one order short of the multi-product T_6.  Same
 * contract as itp_propagate (the propagated block is then orthonormalised
 * by itp_orthonormalize); needs one extra state block of device memory,
 * allocated at the first call. */
int itp_propagate_romberg6(itp_handle h, double tau);

/* The adaptive iteration of Sec. III.  The states are orthonormalised and
 * their energies E_j = (psi_j|H|psi_j) dV taken; then, at a fixed time step
 * (first tau0), steps repeat: propagate the states not yet converged, take
 * their variance with respect to the evolution operator
 *     R^E_j = sum_r |T_2k(tau) psi_j - exp(-tau E_j) psi_j|^2 dV,
 * orthonormalise all states (Eq. 4) and take the energies again.  A state
 * counts as converged at this tau once R^E_j < gamma tau^2 / 10 (R^E is
 * about tau^2 times R^H for small tau); the leading converged states are no
 * longer propagated (they precede the others in the Cholesky order, so the
 * orthonormalisation keeps them).  When the n_states wanted states have
 * converged, or after max_steps steps, the variance with respect to H
 *     R^H_j = sum_r |H psi_j - E_j psi_j|^2 dV
 * is taken: if R^H_j < gamma for every wanted state the iteration ends,
 * else tau *= reduce (0 < reduce < 1; the paper uses 0.5, and 0.9 for its
 * figures) and the steps repeat from the current states.  At the end the
 * states are rotated onto the Ritz vectors.
 *   levels_out   (nullable) number of time steps used
 *   level_stats  (nullable) [max_levels][3] doubles: tau, steps at that
 *                tau, propagated state-steps at that tau
 *   RH_host      (nullable) the m values R^H_j of the last basis
 *   E_host       (nullable) the m Ritz values at the end
 * Runs in the handle's precision (ITP_MIXED: FP32 passes, whose rounding,
 * amplified by the kinetic energy of the grid's highest modes, sets a floor
 * near 1e-8 for R^H at a 0.5 bohr spacing; ITP_FP64: FP64).  Synchronises.  Returns
 * ITP_OK, or ITP_ERR_NOCONV (outputs filled) if R^H stayed above gamma for
 * max_levels time steps. */
int itp_solve_adaptive(itp_handle h, int order, double tau0, double reduce, double gamma,
                       int max_steps, int max_levels, int* levels_out, double* level_stats,
                       double* RH_host, double* E_host);

/* Wait for the handle's stream; returns a pending device status. */
int itp_synchronize(itp_handle h);

/* Failure-detection test hook (no counterpart in the paper).  Every wait of
 * the tensor-core kernels of the mixed path (overlap, update, subspace
 * matrix) on an mbarrier is bounded by one deadline per launch (2 s); when a
 * wait expires, the kernel stops issuing copies and MMAs, waits at most
 * 0.1 s for the ones already issued, frees its tensor memory, leaves its
 * output unwritten and records the timeout, which the next synchronising
 * call returns as ITP_ERR_TIMEOUT (the states are then unspecified; the
 * handle stays usable).  This call makes that path run on demand: each of
 * the handle's next `launches` tensor-core kernel launches made outside a
 * CUDA-graph capture first waits, before issuing any copy or MMA, on an
 * mbarrier phase that nothing completes, with a 2 ms limit instead of 2 s.
 * 0 switches it off.  ITP_FP64 handles launch no tensor-core kernels.
 * Returns ITP_OK or ITP_ERR_ARG (launches < 0). */
int itp_test_expire_waits(itp_handle h, int launches);

/* One-line description of the last error on the handle ("" if none); with
 * h == NULL, the reason the calling thread's last itp_create_grid failed
 * (a failed create returns no handle). */
const char* itp_last_error(itp_handle h);

/* Number of device kernels the handle has launched so far. */
long long itp_kernel_launches(itp_handle h);

/* Kernel kinds for per-kernel timing. */
#define ITP_KERNEL_PLANE_FWD 0        /* real state -> half spectrum (plane pass)    */
#define ITP_KERNEL_PLANE_MERGED 1     /* inverse, exp(-tau V/i), forward (plane pass) */
#define ITP_KERNEL_PLANE_COMBINE 2    /* inverse, exp(-tau V/2i), FP64 c_i sum        */
#define ITP_KERNEL_PLANE_HPSI 3       /* inverse, + V psi (H psi for the energies)    */
#define ITP_KERNEL_PENCIL 4           /* z FFT, exp(-tau|k|^2/2i), inverse z FFT      */
#define ITP_KERNEL_PENCIL_KINETIC 5   /* z FFT, |k|^2/2, inverse z FFT                */
#define ITP_KERNEL_GRAM 6             /* overlap / subspace Gram partial sums         */
#define ITP_KERNEL_GRAM_REDUCE 7
#define ITP_KERNEL_CHOLESKY 8
#define ITP_KERNEL_EIGH 9
#define ITP_KERNEL_APPLY 10           /* n x n matrix applied to the state block      */
#define ITP_KERNEL_OTHER 11           /* tables, conversions, diagonal                */
#define ITP_KERNEL_KINDS 12

/* Per-kernel timing: with enable != 0 every later launch is bracketed by
 * CUDA events on the handle's stream (a few microseconds of overhead per
 * launch); calling it again clears the record.  Synchronises. */
int itp_profile(itp_handle h, int enable);

/* Launch count and summed device time (ms) of one ITP_KERNEL_* kind since
 * the last itp_profile call.  Synchronises. */
int itp_profile_read(itp_handle h, int kind, long long* launches, double* total_ms);

/* ---- Launch shapes and the autotuner ----------------------------------------
 * The paper fixes the arithmetic, not how it is cut into GPU work.  A handle
 * carries four launch-shape choices for its main precision lane (FP32 for
 * ITP_MIXED, FP64 for ITP_FP64), as an int[ITP_TUNING_LEN]:
 *   [ITP_TUNE_PENCIL_W]  kx columns per pencil-pass CTA, 1..nx/2+1 (and the
 *                        FP64 pencil slab, nz*(w+1) complex doubles, within
 *                        one CTA's 227 KB of shared memory); 0: one thread
 *                        per z column with the column held in tensor memory
 *                        (nz = 128, FP32 lane only; the FP64 pencils of a
 *                        mixed handle then take the default width)
 *   [ITP_TUNE_SPLIT]     plane-pass form: 0: one CTA per plane for the x
 *                        and y transforms (only where the plane fits one
 *                        CTA); 1: row passes (x) and column passes (y), three
 *                        HBM round trips; 2 or 3: a cluster of two or four
 *                        CTAs per plane exchanging rows through distributed
 *                        shared memory, one round trip (256 x 256 planes,
 *                        FP32 lane only)
 *   [ITP_TUNE_ROW_TB]    row pairs per row-pass CTA with ITP_TUNE_SPLIT = 1
 *                        (0 otherwise):
 *                        8, 16, or 32 (32: FP32 with nx = 256 only); it
 *                        divides ny/2
 *   [ITP_TUNE_GRAM]      CTAs (partial sums) of the overlap kernel,
 *                        1..2 x the SM count
 * Results depend on the shapes only through rounding. */
#define ITP_TUNE_PENCIL_W 0
#define ITP_TUNE_SPLIT 1
#define ITP_TUNE_ROW_TB 2
#define ITP_TUNE_GRAM 3
#define ITP_TUNING_LEN 4

/* Current launch shapes of the handle's main lane. */
int itp_get_tuning(itp_handle h, int* tuning);

/* Set the launch shapes (all four); ITP_ERR_ARG if one is not valid for the
 * grid (the handle keeps its previous shapes).  Later steps use them;
 * itp_step recaptures its graph. */
int itp_set_tuning(itp_handle h, const int* tuning);

/* Time the candidate shapes on the handle's own potential and states and
 * keep the fastest: the plane-pass form and the pencil width by timing
 * itp_propagate(order, tau), then the overlap's CTA count by timing its
 * kernel.  The states are not changed (the timed propagations write only
 * the propagated block, which is discarded).  tuning (nullable) receives
 * the chosen shapes, report (nullable) a one-line summary of the candidates
 * and their times (truncated to report_len bytes, NUL-terminated).
 * Synchronises. */
int itp_autotune(itp_handle h, int order, double tau, int* tuning, char* report,
                 int report_len);

/* ---- Batches of independent problems ----------------------------------------
 * Many independent problems of uneven size -- each with its own grid,
 * potential and state count -- advanced together.  The paper treats one
 * problem at a time; a batch takes exactly the per-problem steps of Eqs. 3
 * and 4 (as itp_step), with each problem's step captured as one branch of a
 * single CUDA graph: one graph launch advances every problem, and the GPU
 * runs the branches concurrently, so small problems fill the SMs together. */
typedef struct itp_batch* itp_batch_handle;

/* itp_batch_step flag: mixed-precision problems take this step in FP64 (the
 * polish steps of the mixed path).  Their states move to FP64 and move back
 * at the next step without the flag. */
#define ITP_STEP_FP64 4

/* Create count >= 1 problems.  Problem p has the grid dims[3p..3p+2] =
 * (nx, ny, nz) and box boxes[3p..3p+2] = (lx, ly, lz) (the rules of
 * itp_create_grid apply), n_states[p] >= 1 states and n_guard[p] >= 0 guard
 * states (n_guard NULL: none); precision as itp_create_grid, the same for
 * all.  Each problem gets a stream of its own; the batch's graph is launched
 * on cuda_stream (NULL: a stream the batch creates).  On failure *out is
 * NULL and itp_batch_last_error(NULL) names the problem that failed and
 * why. */
int itp_create_batch(itp_batch_handle* out, int count, const int* dims, const double* boxes,
                     const int* n_states, const int* n_guard, int precision, void* cuda_stream);

/* The handle of problem p (0 <= p < count), owned by the batch: set its
 * potential and states, read its states and energies with the single-problem
 * calls; never pass it to itp_destroy.  NULL for a bad index. */
itp_handle itp_batch_problem(itp_batch_handle b, int p);

/* Number of problems in the batch (0 for NULL). */
int itp_batch_count(itp_batch_handle b);

/* One step of every problem -- itp_propagate(order, tau),
 * itp_orthonormalize and energies with flags 0 or ITP_RITZ_VALUES, plus
 * optionally ITP_STEP_FP64 -- as one CUDA graph launch on the batch's stream.
 * The first call for a given (order, tau, flags) captures the graph; later
 * calls replay it.  Every problem needs its potential and states set.
 * Synchronises.  E_host (nullable) receives all problems' energies back to
 * back: problem p's m_p = n_states[p] + n_guard[p] values start at
 * sum_{q<p} m_q.  Returns ITP_OK or the first problem's error
 * (ITP_ERR_NOT_PD, ITP_ERR_NOCONV, ITP_ERR_TIMEOUT, ...); the message of
 * itp_batch_last_error names the problem. */
int itp_batch_step(itp_batch_handle b, int order, double tau, int flags, double* E_host);

/* Kernels launched by the batch's steps so far (graph nodes counted per
 * replay). */
long long itp_batch_kernel_launches(itp_batch_handle b);

/* How a batch step's graph is built.  grouped != 0 (the default): problems
 * with the same grid, precision lane, launch shapes and pass sequence form a
 * group, and each FFT pass of a step (plane, pencil, exact term sum) is one
 * launch over all the states of the group's problems -- a CTA row looks up
 * its (problem, state) and that problem's arguments in tables the batch
 * keeps in device memory -- while the remaining kernels of each problem
 * (overlap, Cholesky, update, eigenvalues, copies) run as parallel branches
 * between those launches; groups run as parallel branches.  Every CTA
 * computes exactly what the problem's own launch would, so results are the
 * same bit for bit.  Passes without a grouped form run per problem inside
 * the group: plane passes of row + column or cluster planes, and pencils of
 * width 0 (ITP_TUNE_PENCIL_W).  grouped == 0: one branch of ~50 launches
 * per problem.
 * Takes effect at the next itp_batch_step (which captures a new graph).
 * Returns ITP_OK or ITP_ERR_ARG (null batch). */
int itp_batch_set_grouping(itp_batch_handle b, int grouped);

/* Number of groups in the captured grouped graph (0 before the first
 * grouped step, or in the per-problem form). */
int itp_batch_groups(itp_batch_handle b);

/* One-line description of the last error on the batch; with b == NULL, why
 * the calling thread's last itp_create_batch failed. */
const char* itp_batch_last_error(itp_batch_handle b);

/* Free the batch and every problem handle in it. */
void itp_batch_destroy(itp_batch_handle b);

/* Orthonormalise a block of states that already lives in device memory,
 * without allocating any device memory: for callers that cannot call
 * cudaMalloc -- code running inside a memory pool or arena that owns all
 * device memory, a host process under a fixed device-memory budget, or a
 * path that must not allocate between set-up and a deadline.  The paper has
 * no counterpart; this computes the same FP64 orthonormalisation as
 * itp_orthonormalize (S = Phi Phi^T dV = L L^T, psi = L^{-1} phi) on
 * caller-owned buffers.
 *   phi_device  [m][n_points] doubles on the current device (input, not
 *               modified); any point order, the same for every state
 *   psi_device  [m][n_points] doubles (output); its byte range must not
 *               overlap that of phi_device at all (ITP_ERR_ARG)
 *   m           1..128 states; n_points >= 1; dV > 0 the volume element
 *   cuda_stream the stream to run on (NULL: default stream); the call
 *               synchronises it before returning
 * Returns ITP_OK, ITP_ERR_ARG (bad pointer or size, m > 128, overlapping
 * buffers),
 * ITP_ERR_NOT_PD (overlap not positive definite; psi_device then holds no
 * meaningful values) or ITP_ERR_CUDA.
 * Scratch space is a fixed array of about 4.3 MiB inside the library, present
 * on every GPU that loads it until the process exits.  All calls on a device
 * share it: calls whose work overlaps on the GPU (different streams or
 * threads at the same time) race and must be serialised by the caller.  The
 * first call on each device looks up the array's device address (with that
 * device current); make that first call before capturing a stream into a
 * CUDA graph. */
int itp_orthonormalize_noalloc(const double* phi_device, double* psi_device, int m,
                               long long n_points, double dV, void* cuda_stream);

/* ---- Measured arithmetic rates -----------------------------------------------
 * Denominators for the ALU and tensor rooflines of the kernels (the paper has
 * no counterpart).  Runs one probe on the current device: long chains of
 * independent operations on every SM, timed with CUDA events on cuda_stream
 * (NULL: default stream), best of three launches after one warm-up; no clock
 * or other GPU setting is changed, so the rate is the one at whatever clocks
 * the GPU runs (sample them alongside).  *tflops receives the achieved
 * TFLOP/s (an FMA counts 2 flops; an M x N x K MMA 2MNK), *ms_out (nullable)
 * the duration of one launch.  Allocates and frees a few bytes of device
 * memory.  Returns ITP_OK, ITP_ERR_ARG (unknown kind or null tflops),
 * ITP_ERR_OOM, ITP_ERR_CUDA, or ITP_ERR_TIMEOUT (the MMA probe's bounded wait
 * for its tensor-core work expired). */
#define ITP_PROBE_FFMA 0      /* FP32 FMA, one value per instruction            */
#define ITP_PROBE_FFMA2 1     /* packed two-lane FP32 FMA (sm_100+)             */
#define ITP_PROBE_DFMA 2      /* FP64 FMA                                       */
#define ITP_PROBE_TF32_MMA 3  /* tcgen05.mma kind::tf32 128x256x8, FP32 in TMEM */
int itp_peak_probe(int kind, void* cuda_stream, double* tflops, double* ms_out);

#ifdef __cplusplus
}
#endif

#endif /* ITP_H_ */
