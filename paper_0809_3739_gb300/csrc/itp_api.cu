// C ABI of libitp (declared in include/itp.h): handle management and the
// orchestration of the plane / pencil passes and the dense kernels that make
// up one imaginary-time iteration (Eqs. 3 and 4 of the paper).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <functional>
#include <new>
#include <string>
#include <vector>

#include "itp.h"
#include "itp_kernels.cuh"

using namespace itp;

namespace {

constexpr int kMaxStates = 256;   // two 128-state blocks of the n x n work
constexpr int kMaxTerms = 6;   // order <= 12
constexpr int kHostChunks = 4; // state chunks of the host-buffer step (copy/compute overlap)
constexpr size_t kSmemLimit = 227 * 1024;

template <typename R>
struct Lane {
  bool ready = false;
  R* psi = nullptr;          // [m][N]
  R* psi_tmp = nullptr;      // [m][N]
  void* work = nullptr;      // [m][n_half] complex
  void* work_terms[kMaxTerms] = {};  // per-term spectra / contributions (mixed)
  bool fused_ok = true;              // per-term workspaces could be allocated
  R* f_half[kMaxTerms] = {}; // exp(-tau_i V / 2)
  R* f_full[kMaxTerms] = {}; // exp(-tau_i V)      (terms i >= 2)
  R* ktab = nullptr;         // per term: nxh + ny + nz propagation factors
  R* htab = nullptr;         // nxh + ny + nz kinetic values k^2/2
  R* Vr = nullptr;           // [N] potential in precision R (internal layout)
  R* rom = nullptr;          // [m][N] scratch of the Romberg T_6 comparator (on demand)
  void* twx = nullptr;
  void* twy = nullptr;
  void* twz = nullptr;
  int tab_order = 0;
  double tab_tau = 0.0;
};

// One recorded kernel launch of a problem's step (batches, itp_batch_step):
// the FFT passes keep their arguments, so that the same pass of several
// problems with one grid can run as one grouped launch; every other launch
// keeps a closure that issues it on the problem's stream.
struct RecOp {
  enum Kind { kOther = 0, kPlane = 1, kPencil = 2, kTermSum = 3 };
  int kind = kOther;
  int lane = 0;               // 0: FP32 arguments, 1: FP64
  int mode = 0;               // plane or pencil mode
  PlaneArgs<float> p32{};
  PlaneArgs<double> p64{};
  PencilArgs<float> e32{};
  PencilArgs<double> e64{};
  TermSumArgs ts{};
  std::function<cudaError_t()> fn;   // the launch on the problem's stream
};

}  // namespace

struct itp_grid {
  int device = 0;
  GridDesc g{};
  double lx = 0, ly = 0, lz = 0, dV = 0;
  int n = 0, ng = 0, m = 0;
  int precision = ITP_FP64;
  cudaStream_t st = nullptr;
  double* V = nullptr;        // [N], internal layout [z][x][y]
  double* Vstage = nullptr;   // [N], user layout staging
  double* acc = nullptr;      // [m][N] FP64 accumulator / H psi / staging
  Lane<float> f32;
  Lane<double> f64;
  bool cur64 = true;          // which lane holds the states
  bool have_V = false, have_states = false, have_phi = false;
  int n_chunks = 0;           // Gram partial sums (CUDA-core kernels)
  int n_chunks_tc = 0;        // Gram partial sums (tensor-core kernel, one CTA per SM)
  double* partial = nullptr;  // [n_chunks][m][m]
  double* S = nullptr;        // [m][m]
  double* Mx = nullptr;       // [m][m]
  double* Hs = nullptr;       // [m][m]
  double* Wmm = nullptr;      // [m][m]
  double* E_dev = nullptr;    // [m]
  int* status = nullptr;      // device status word
  int* status_host = nullptr; // pinned
  double* E_host_pinned = nullptr;
  double* res_dev = nullptr;  // [2m] residual norms of the adaptive iteration
  long long launches = 0;
  int expire_waits = 0;       // test hook: tensor-core launches left that expire their wait
  std::vector<RecOp>* rec = nullptr;   // recording a step instead of launching it
  std::string err;
  bool own_stream = false;    // created by the library (no stream given)
  // CUDA graph of one step (itp_step): propagate + orthonormalize + energies
  cudaGraphExec_t step_exec = nullptr;
  int step_order = 0, step_flags = -1, step_lane = -1, step_version = 0;
  double step_tau = 0.0;
  bool capturing = false;
  long long step_launches = 0;
  int tune_version = 0;       // bumped when the launch shapes change
  // optional per-kernel event timing (itp_profile)
  bool prof = false;
  struct ProfEvent { int kind; cudaEvent_t start, stop; };
  std::vector<ProfEvent> prof_events;
  size_t prof_used = 0;
  // host-buffer step (itp_step_host): copy stream, FP64 staging block in the
  // user layout, events (per chunk: input copied, output staged; start; end)
  cudaStream_t cst = nullptr;
  double* hstage = nullptr;   // [m][N]
  cudaEvent_t hev[2 * kHostChunks + 2] = {};
};

namespace {

thread_local std::string g_create_error;

int fail(itp_handle h, int code, const char* fmt, ...) {
  if (h) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    h->err = buf;
  }
  return code;
}

#define ITP_CUDA(h, expr)                                                                 \
  do {                                                                                    \
    cudaError_t e_ = (expr);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(h, e_ == cudaErrorMemoryAllocation ? ITP_ERR_OOM : ITP_ERR_CUDA,        \
                  "%s: %s", #expr, cudaGetErrorString(e_));                               \
  } while (0)

// Launch one kernel of the given ITP_KERNEL_* kind, counted and (when
// profiling is on) bracketed by CUDA events on the handle's stream.  While
// the handle records a step (h->rec), the launch is kept as a closure to be
// issued later on the handle's stream instead.
#define ITP_LAUNCH(h, kind, expr)                                                         \
  do {                                                                                    \
    (h)->launches++;                                                                      \
    if ((h)->rec) {                                                                       \
      RecOp op_;                                                                          \
      op_.fn = [=]() -> cudaError_t { return (expr); };                                   \
      (h)->rec->push_back(std::move(op_));                                                \
      break;                                                                              \
    }                                                                                     \
    const long ev_ = prof_begin(h, kind);                                                 \
    cudaError_t e_ = (expr);                                                              \
    prof_end(h, ev_);                                                                     \
    if (e_ != cudaSuccess)                                                                \
      return fail(h, ITP_ERR_CUDA, "%s: %s", #expr, cudaGetErrorString(e_));              \
  } while (0)

// The same for an FFT pass: while recording, the pass function itself keeps
// its arguments (plane_counted, pencil_counted, term_sum_counted).
#define ITP_LAUNCH_PASS(h, kind, expr)                                                    \
  do {                                                                                    \
    (h)->launches++;                                                                      \
    const long ev_ = (h)->rec ? -1 : prof_begin(h, kind);                                 \
    cudaError_t e_ = (expr);                                                              \
    prof_end(h, ev_);                                                                     \
    if (e_ != cudaSuccess)                                                                \
      return fail(h, ITP_ERR_CUDA, "%s: %s", #expr, cudaGetErrorString(e_));              \
  } while (0)

long prof_begin(itp_handle h, int kind) {
  if (!h->prof || h->capturing) return -1;
  if (h->prof_used == h->prof_events.size()) {
    itp_grid::ProfEvent e{kind, nullptr, nullptr};
    if (cudaEventCreate(&e.start) != cudaSuccess || cudaEventCreate(&e.stop) != cudaSuccess)
      return -1;
    h->prof_events.push_back(e);
  }
  itp_grid::ProfEvent& e = h->prof_events[h->prof_used];
  e.kind = kind;
  if (cudaEventRecord(e.start, h->st) != cudaSuccess) return -1;
  return (long)h->prof_used++;
}

void prof_end(itp_handle h, long idx) {
  if (idx >= 0) cudaEventRecord(h->prof_events[idx].stop, h->st);
}

#define ITP_TRY(expr)             \
  do {                            \
    int r_ = (expr);              \
    if (r_ != ITP_OK) return r_;  \
  } while (0)

// Kernels behind one launch_* call of the n x n work, which walks 128-state
// blocks when m > 128: the update Y = M X (lower: M lower triangular) and
// the tensor-core Gram (A A^T: diagonal and off-diagonal blocks apart).
int apply_launches(int m, bool lower) {
  const int nb = (m + 127) / 128;
  return lower ? nb * (nb + 1) / 2 : nb * nb;
}
int tc_gram_launches(int m, bool same) { return same && m > 128 ? 2 : 1; }

// Wait limit for the next tensor-core launch: 0 (the kernels' own launch
// deadline), or the short limit of the failure-detection test hook
// (itp_test_expire_waits), which only applies outside a graph capture.
constexpr unsigned long long kExpireTestNs = 2000000ull;   // 2 ms
unsigned long long tc_expire(itp_handle h) {
  if (h->expire_waits <= 0 || h->capturing) return 0;
  --h->expire_waits;
  return kExpireTestNs;
}

bool split_axis(int L, int* r1, int* r2) {
  static const int rad[] = {2, 3, 4, 6, 8, 12, 16};
  if (L < 2 || L > 256 || (L & 1)) return false;
  if (L <= 16) {
    for (int r : rad)
      if (r == L) { *r1 = 1; *r2 = L; return true; }
  }
  int best = -1;
  for (int a : rad) {
    if (L % a) continue;
    const int b = L / a;
    bool ok = false;
    for (int r : rad) ok |= (r == b);
    if (!ok || b < a) continue;   // r2 >= r1
    if (best < 0 || (b - a) < (L / best - best)) best = a;
  }
  if (best < 0) return false;
  *r1 = best;
  *r2 = L / best;
  return true;
}

// Exact c_i of Eq. (coef) as a reduced fraction, then rounded to double.
double mp_coefficient(int i, int k) {
  long long num = 1, den = 1;
  auto gcd = [](long long a, long long b) {
    a = a < 0 ? -a : a;
    b = b < 0 ? -b : b;
    while (b) { long long t = a % b; a = b; b = t; }
    return a;
  };
  for (int j = 1; j <= k; ++j) {
    if (j == i) continue;
    long long a = (long long)i * i, b = (long long)i * i - (long long)j * j;
    num *= a;
    den *= b;
    const long long gg = gcd(num, den);
    num /= gg;
    den /= gg;
  }
  return (double)num / (double)den;
}

template <typename R>
void roots_table(int L, std::vector<R>& out) {
  out.resize(2 * (size_t)L);
  for (int j = 0; j < L; ++j) {
    double c, s;
    if ((4 * j) % L == 0) {   // quarter turns exactly
      const int q = (4 * j) / L;
      c = (q == 0) ? 1.0 : (q == 2 ? -1.0 : 0.0);
      s = (q == 1) ? -1.0 : (q == 3 ? 1.0 : 0.0);
    } else {
      const double ang = 2.0 * 3.14159265358979323846 * (double)j / (double)L;
      c = std::cos(ang);
      s = -std::sin(ang);
    }
    out[2 * j] = (R)c;
    out[2 * j + 1] = (R)s;
  }
}

template <typename R>
int alloc_lane(itp_handle h, Lane<R>& L) {
  if (L.ready) return ITP_OK;
  const GridDesc& g = h->g;
  const size_t N = (size_t)g.n_points, Nh = (size_t)g.n_half, m = (size_t)h->m;
  ITP_CUDA(h, cudaMalloc(&L.psi, m * N * sizeof(R)));
  ITP_CUDA(h, cudaMalloc(&L.psi_tmp, m * N * sizeof(R)));
  ITP_CUDA(h, cudaMalloc(&L.work, m * Nh * 2 * sizeof(R)));
  for (int i = 0; i < kMaxTerms; ++i) {
    ITP_CUDA(h, cudaMalloc(&L.f_half[i], N * sizeof(R)));
    if (i > 0) ITP_CUDA(h, cudaMalloc(&L.f_full[i], N * sizeof(R)));
  }
  const size_t tl = (size_t)g.nxh + g.ny + g.nz;
  ITP_CUDA(h, cudaMalloc(&L.ktab, kMaxTerms * tl * sizeof(R)));
  ITP_CUDA(h, cudaMalloc(&L.htab, tl * sizeof(R)));
  ITP_CUDA(h, cudaMalloc(&L.Vr, N * sizeof(R)));
  if (h->have_V)
    ITP_LAUNCH(h, ITP_KERNEL_OTHER, (launch_convert<double, R>(h->V, L.Vr, (long long)N, h->st)));
  std::vector<R> tx, ty, tz;
  roots_table<R>(g.nx, tx);
  roots_table<R>(g.ny, ty);
  roots_table<R>(g.nz, tz);
  ITP_CUDA(h, cudaMalloc(&L.twx, tx.size() * sizeof(R)));
  ITP_CUDA(h, cudaMalloc(&L.twy, ty.size() * sizeof(R)));
  ITP_CUDA(h, cudaMalloc(&L.twz, tz.size() * sizeof(R)));
  ITP_CUDA(h, cudaMemcpy(L.twx, tx.data(), tx.size() * sizeof(R), cudaMemcpyHostToDevice));
  ITP_CUDA(h, cudaMemcpy(L.twy, ty.data(), ty.size() * sizeof(R), cudaMemcpyHostToDevice));
  ITP_CUDA(h, cudaMemcpy(L.twz, tz.data(), tz.size() * sizeof(R), cudaMemcpyHostToDevice));
  ITP_LAUNCH(h, ITP_KERNEL_OTHER, launch_kinetic_tables<R>(g, h->lx, h->ly, h->lz, L.htab, L.htab + g.nxh,
                                         L.htab + g.nxh + g.ny, h->st));
  L.tab_order = 0;
  L.ready = true;
  return ITP_OK;
}

template <typename R>
void free_lane(Lane<R>& L) {
  cudaFree(L.psi);
  cudaFree(L.psi_tmp);
  cudaFree(L.work);
  for (int i = 0; i < kMaxTerms; ++i) {
    cudaFree(L.f_half[i]);
    cudaFree(L.f_full[i]);
  }
  for (int i = 1; i < kMaxTerms; ++i) cudaFree(L.work_terms[i]);
  cudaFree(L.ktab);
  cudaFree(L.htab);
  cudaFree(L.Vr);
  cudaFree(L.rom);
  cudaFree(L.twx);
  cudaFree(L.twy);
  cudaFree(L.twz);
  L = Lane<R>();
}

// A plane pass: 1 kernel, or 2-3 kernels on split planes (counted).
template <typename R>
cudaError_t plane_counted(itp_handle h, const PlaneArgs<R>& a) {
  if (h->rec) {
    RecOp op;
    op.kind = RecOp::kPlane;
    op.lane = sizeof(R) == 8;
    op.mode = a.mode;
    if constexpr (sizeof(R) == 4) op.p32 = a;
    else op.p64 = a;
    op.fn = [h, a]() { int n = 1; return launch_plane<R>(h->g, a, h->st, &n); };
    h->rec->push_back(std::move(op));
    return cudaSuccess;
  }
  int n = 1;
  const cudaError_t e = launch_plane<R>(h->g, a, h->st, &n);
  h->launches += n - 1;
  return e;
}

template <typename R>
cudaError_t pencil_counted(itp_handle h, const PencilArgs<R>& a) {
  if (h->rec) {
    RecOp op;
    op.kind = RecOp::kPencil;
    op.lane = sizeof(R) == 8;
    op.mode = a.mode;
    if constexpr (sizeof(R) == 4) op.e32 = a;
    else op.e64 = a;
    op.fn = [h, a]() { return launch_pencil<R>(h->g, a, h->st); };
    h->rec->push_back(std::move(op));
    return cudaSuccess;
  }
  return launch_pencil<R>(h->g, a, h->st);
}

cudaError_t term_sum_counted(itp_handle h, const TermSumArgs& a) {
  if (h->rec) {
    RecOp op;
    op.kind = RecOp::kTermSum;
    op.ts = a;
    op.fn = [h, a]() { return launch_term_sum(a, h->st); };
    h->rec->push_back(std::move(op));
    return cudaSuccess;
  }
  return launch_term_sum(a, h->st);
}

template <typename R>
Lane<R>& lane_of(itp_handle h);
template <>
Lane<float>& lane_of<float>(itp_handle h) { return h->f32; }
template <>
Lane<double>& lane_of<double>(itp_handle h) { return h->f64; }

// Per-term factor tables for (order, tau).
template <typename R>
int prepare_tables(itp_handle h, Lane<R>& L, int k, double tau) {
  if (L.tab_order == 2 * k && L.tab_tau == tau) return ITP_OK;
  const GridDesc& g = h->g;
  const size_t tl = (size_t)g.nxh + g.ny + g.nz;
  for (int i = 1; i <= k; ++i) {
    R* kt = L.ktab + (i - 1) * tl;
    ITP_LAUNCH(h, ITP_KERNEL_OTHER, launch_term_tables<R>(g, h->V, tau / i, h->lx, h->ly, h->lz, L.f_half[i - 1],
                                        i > 1 ? L.f_full[i - 1] : nullptr, kt, kt + g.nxh,
                                        kt + g.nxh + g.ny, h->st));
  }
  L.tab_order = 2 * k;
  L.tab_tau = tau;
  return ITP_OK;
}

// Eq. (3) with the order-2k expansion: acc = sum_i c_i T_2(tau/i)^i psi.
// Per term i: plane-forward with exp(-tau_i V/2), then i pencils with i-1
// merged plane passes (exp(-tau_i V)) between them, then the final inverse
// plane pass with exp(-tau_i V/2) adds c_i u_i (Sec. II).  The mixed path
// keeps every term's spectrum in its own workspace, writes each term's FP32
// contribution c_i f u_i over it, and sums the contributions once in FP64.
template <typename R>
int propagate_lane(itp_handle h, int k, double tau, int s0 = 0, const R* in = nullptr,
                   R* out = nullptr, int s1 = -1) {
  Lane<R>& L = lane_of<R>(h);
  ITP_TRY(prepare_tables<R>(h, L, k, tau));
  const GridDesc& g = h->g;
  const size_t tl = (size_t)g.nxh + g.ny + g.nz;
  bool fused = sizeof(R) == 4 && L.fused_ok && g.split_planes[0] != 1;
  if (fused) {
    L.work_terms[0] = L.work;
    for (int i = 1; i < k && fused; ++i) {
      if (!L.work_terms[i] &&
          cudaMalloc(&L.work_terms[i], (size_t)h->m * g.n_half * 2 * sizeof(R)) != cudaSuccess) {
        cudaGetLastError();   // clear the allocation error; use the per-term path
        L.fused_ok = fused = false;
      }
    }
  }
  // states s0..s1-1 only (s1 < 0: to the last state; the others are kept)
  const int ms = (s1 < 0 ? h->m : s1) - s0;
  const long long so = s0;
  auto at_state = [&](void* w) {
    return static_cast<void*>(static_cast<char*>(w) + so * g.n_half * 2 * sizeof(R));
  };
  TermSumArgs ts{};
  for (int i = 1; i <= k; ++i) {
    void* work = at_state(fused ? L.work_terms[i - 1] : L.work);
    PlaneArgs<R> pa{};
    pa.m = ms;
    pa.in_real = (in ? in : L.psi) + so * g.n_points;
    pa.spec = work;
    pa.twx = L.twx;
    pa.twy = L.twy;
    pa.mode = PLANE_FWD_REAL;
    pa.f_in = L.f_half[i - 1];
    const bool planar = g.nz == 1;   // the kinetic factor ends each forward pass
    if (planar) {
      const R* kt = L.ktab + (i - 1) * tl;
      pa.kin.fx = kt;
      pa.kin.fy = kt + g.nxh;
      pa.kin.fz = kt + g.nxh + g.ny;
      pa.kin.mode = 0;
    }
    ITP_LAUNCH_PASS(h, ITP_KERNEL_PLANE_FWD, plane_counted<R>(h, pa));
    PencilArgs<R> pe{};
    pe.mode = PENCIL_PROPAGATE;
    pe.m = ms;
    pe.spec = work;
    pe.kx_tab = L.ktab + (i - 1) * tl;
    pe.ky_tab = pe.kx_tab + g.nxh;
    pe.kz_tab = pe.ky_tab + g.ny;
    pe.scale = (R)1;
    pe.twz = L.twz;
    for (int j = 1; j <= i; ++j) {
      if (!planar)
        ITP_LAUNCH_PASS(h, pe.mode == PENCIL_PROPAGATE ? ITP_KERNEL_PENCIL
                                                       : ITP_KERNEL_PENCIL_KINETIC,
                        pencil_counted<R>(h, pe));
      if (j < i) {
        PlaneArgs<R> pm = pa;
        pm.mode = PLANE_MERGED;
        pm.f_in = nullptr;
        pm.f_mid = L.f_full[i - 1];
        ITP_LAUNCH_PASS(h, ITP_KERNEL_PLANE_MERGED, plane_counted<R>(h, pm));
      }
    }
    if (fused) {
      // the term's contribution c_i f u_i, in place over its spectrum
      PlaneArgs<R> pt = pa;
      pt.mode = PLANE_TERM;
      pt.f_in = nullptr;
      pt.f_out = L.f_half[i - 1];
      pt.coef = mp_coefficient(i, k);
      ITP_LAUNCH_PASS(h, ITP_KERNEL_PLANE_COMBINE, plane_counted<R>(h, pt));
      ts.term[i - 1] = reinterpret_cast<const float*>(work);
      continue;
    }
    PlaneArgs<R> pc = pa;
    pc.mode = PLANE_COMBINE;
    pc.f_in = nullptr;
    pc.f_out = L.f_half[i - 1];
    pc.acc = (sizeof(R) == 8 && out ? reinterpret_cast<double*>(out) : h->acc) + so * g.n_points;
    pc.coef = mp_coefficient(i, k);
    pc.acc_init = (i == 1);
    // the mixed path keeps the sum in FP64 and rounds the finished phi once
    pc.phi_out = (sizeof(R) == 4 && i == k) ? (out ? out : L.psi_tmp) + so * g.n_points : nullptr;
    ITP_LAUNCH_PASS(h, ITP_KERNEL_PLANE_COMBINE, plane_counted<R>(h, pc));
  }
  if (fused) {
    // phi = sum_i c_i f u_i in FP64 over the FP32 contributions
    ts.m = ms;
    ts.k = k;
    ts.nz = g.nz;
    ts.plane_pts = g.nx * g.ny;
    ts.plane_pitch = 2LL * g.ny * g.nxh;
    ts.phi_out = reinterpret_cast<float*>((out ? out : L.psi_tmp) + so * g.n_points);
    ITP_LAUNCH_PASS(h, ITP_KERNEL_OTHER, term_sum_counted(h, ts));
  }
  return ITP_OK;
}

// Eq. (4): psi = L^{-1} phi, S = phi phi^T dV = L L^T.
template <typename R>
int orthonormalize_lane(itp_handle h);
template <>
int orthonormalize_lane<double>(itp_handle h) {
  Lane<double>& L = h->f64;
  ITP_LAUNCH(h, ITP_KERNEL_GRAM, (launch_gram_partial<double, double, double>(
                                     h->acc, h->acc, h->m, h->g.n_points, h->n_chunks,
                                     h->partial, h->st)));
  ITP_LAUNCH(h, ITP_KERNEL_GRAM_REDUCE,
             launch_gram_reduce(h->partial, h->n_chunks, h->m, h->dV, 1, h->S, h->st));
  ITP_LAUNCH(h, ITP_KERNEL_CHOLESKY, launch_cholesky_inverse(h->S, h->m, h->Mx, h->status, h->st));
  ITP_LAUNCH(h, ITP_KERNEL_APPLY, (launch_apply_matrix<double, double>(
                                      h->Mx, h->m, 1, h->acc, L.psi, h->g.n_points, h->st)));
  h->launches += apply_launches(h->m, true) - 1;
  return ITP_OK;
}
// Mixed path: phi is FP32 (rounded from the FP64 sum) in psi_tmp; S and the
// update run on the tensor cores (3xTF32).
template <>
int orthonormalize_lane<float>(itp_handle h) {
  Lane<float>& L = h->f32;
  ITP_LAUNCH(h, ITP_KERNEL_GRAM, (launch_tc_gram(L.psi_tmp, L.psi_tmp, h->m,
                                                               h->g.n_points, h->n_chunks_tc,
                                                               h->partial, h->status, h->st,
                                                               tc_expire(h))));
  h->launches += tc_gram_launches(h->m, true) - 1;
  ITP_LAUNCH(h, ITP_KERNEL_GRAM_REDUCE,
             launch_gram_reduce(h->partial, h->n_chunks_tc, h->m, h->dV, 1, h->S, h->st));
  ITP_LAUNCH(h, ITP_KERNEL_CHOLESKY, launch_cholesky_inverse(h->S, h->m, h->Mx, h->status, h->st));
  ITP_LAUNCH(h, ITP_KERNEL_APPLY, (launch_tc_apply<float, float>(h->Mx, h->m, L.psi_tmp, L.psi,
                                                                 h->g.n_points, h->status,
                                                                 h->st, tc_expire(h), 1)));
  h->launches += apply_launches(h->m, true) - 1;
  return ITP_OK;
}

// H psi into acc, subspace matrix, optional Ritz rotation; E into E_dev.
template <typename R>
int energies_lane(itp_handle h, int flags) {
  Lane<R>& L = lane_of<R>(h);
  const GridDesc& g = h->g;
  PlaneArgs<R> pa{};
  pa.m = h->m;
  pa.in_real = L.psi;
  pa.spec = L.work;
  pa.twx = L.twx;
  pa.twy = L.twy;
  pa.mode = PLANE_FWD_REAL;
  pa.f_in = nullptr;
  const bool planar = g.nz == 1;   // |k|^2/2 ends the forward pass, no pencil pass
  if (planar) {
    pa.kin.fx = L.htab;
    pa.kin.fy = L.htab + g.nxh;
    pa.kin.fz = L.htab + g.nxh + g.ny;
    pa.kin.mode = 1;
    pa.kin.scale = (R)(1.0 / (double)g.n_points);
  }
  ITP_LAUNCH_PASS(h, ITP_KERNEL_PLANE_FWD, plane_counted<R>(h, pa));
  pa.kin = KinFac<R>{};
  PencilArgs<R> pe{};
  pe.mode = PENCIL_KINETIC;
  pe.m = h->m;
  pe.spec = L.work;
  pe.kx_tab = L.htab;
  pe.ky_tab = L.htab + g.nxh;
  pe.kz_tab = L.htab + g.nxh + g.ny;
  pe.scale = (R)(1.0 / (double)g.n_points);
  pe.twz = L.twz;
  if (!planar)
    ITP_LAUNCH_PASS(h, pe.mode == PENCIL_PROPAGATE ? ITP_KERNEL_PENCIL : ITP_KERNEL_PENCIL_KINETIC,
                    pencil_counted<R>(h, pe));
  PlaneArgs<R> ph = pa;
  ph.mode = PLANE_HPSI;
  ph.acc = h->acc;
  ph.V = h->V;
  if (sizeof(R) == 4) {   // mixed: H psi in FP32 into psi_tmp
    ph.V_r = L.Vr;
    ph.phi_out = L.psi_tmp;
  }
  ITP_LAUNCH_PASS(h, ITP_KERNEL_PLANE_HPSI, plane_counted<R>(h, ph));
  if (sizeof(R) == 4) {
    ITP_LAUNCH(h, ITP_KERNEL_GRAM, (launch_tc_gram(
                                       reinterpret_cast<const float*>(L.psi),
                                       reinterpret_cast<const float*>(L.psi_tmp), h->m,
                                       g.n_points, h->n_chunks_tc, h->partial, h->status,
                                       h->st, tc_expire(h))));
  } else {
    ITP_LAUNCH(h, ITP_KERNEL_GRAM, (launch_gram_partial<double, double, double>(
                                       reinterpret_cast<const double*>(L.psi), h->acc, h->m,
                                       g.n_points, h->n_chunks, h->partial, h->st)));
  }
  const int chunks = sizeof(R) == 4 ? h->n_chunks_tc : h->n_chunks;
  ITP_LAUNCH(h, ITP_KERNEL_GRAM_REDUCE,
             launch_gram_reduce(h->partial, chunks, h->m, h->dV, 1, h->Hs, h->st));
  if (flags & ITP_RITZ) {
    ITP_LAUNCH(h, ITP_KERNEL_EIGH, launch_jacobi_eigh(h->Hs, h->m, h->E_dev, h->Mx, h->Wmm, h->status, h->st));
    if (sizeof(R) == 4) {
      ITP_LAUNCH(h, ITP_KERNEL_APPLY, (launch_tc_apply<float, float>(
                                          h->Mx, h->m, reinterpret_cast<const float*>(L.psi),
                                          reinterpret_cast<float*>(L.psi_tmp), g.n_points,
                                          h->status, h->st, tc_expire(h))));
      h->launches += apply_launches(h->m, false) - 1;
    } else {
      ITP_LAUNCH(h, ITP_KERNEL_APPLY, (launch_apply_matrix<double, double>(
                                          h->Mx, h->m, 0, reinterpret_cast<const double*>(L.psi),
                                          reinterpret_cast<double*>(L.psi_tmp), g.n_points,
                                          h->st)));
      h->launches += apply_launches(h->m, false) - 1;
    }
    R* t = L.psi;
    L.psi = L.psi_tmp;
    L.psi_tmp = t;
  } else if (flags & ITP_RITZ_VALUES) {
    ITP_LAUNCH(h, ITP_KERNEL_EIGH, launch_tridiag(h->Hs, h->m, h->Wmm, h->st));
    ITP_LAUNCH(h, ITP_KERNEL_EIGH, launch_bisect(h->Wmm, h->m, h->E_dev, h->st));
  } else {
    ITP_LAUNCH(h, ITP_KERNEL_OTHER, launch_diag(h->Hs, h->m, h->E_dev, h->st));
  }
  return ITP_OK;
}

// Report and clear a device status word already copied to status_host.
int take_status(itp_handle h) {
  const int s = *h->status_host;
  if (s) {
    ITP_CUDA(h, cudaMemsetAsync(h->status, 0, sizeof(int), h->st));
    // an expired wait left outputs unwritten, so later flags may follow from it
    if (s & 4) return fail(h, ITP_ERR_TIMEOUT, "a bounded tensor-core pipeline wait expired");
    if (s & 1) return fail(h, ITP_ERR_NOT_PD, "overlap matrix is not positive definite");
    if (s & 2) return fail(h, ITP_ERR_NOCONV, "Jacobi eigensolver did not converge");
  }
  return ITP_OK;
}

// Read and clear the device status word (synchronises the stream).
int collect_status(itp_handle h) {
  ITP_CUDA(h, cudaMemcpyAsync(h->status_host, h->status, sizeof(int), cudaMemcpyDeviceToHost,
                              h->st));
  ITP_CUDA(h, cudaStreamSynchronize(h->st));
  return take_status(h);
}

// Make the lane of precision R hold the states (converting if needed).
template <typename R>
int switch_lane(itp_handle h);
template <>
int switch_lane<double>(itp_handle h) {
  if (h->cur64) return ITP_OK;
  ITP_TRY(alloc_lane<double>(h, h->f64));
  ITP_LAUNCH(h, ITP_KERNEL_OTHER, (launch_convert<float, double>(h->f32.psi, h->f64.psi,
                                               (long long)h->m * h->g.n_points, h->st)));
  h->cur64 = true;
  return ITP_OK;
}
template <>
int switch_lane<float>(itp_handle h) {
  if (!h->cur64) return ITP_OK;
  ITP_LAUNCH(h, ITP_KERNEL_OTHER, (launch_convert<double, float>(h->f64.psi, h->f32.psi,
                                               (long long)h->m * h->g.n_points, h->st)));
  h->cur64 = false;
  return ITP_OK;
}

int check_ready(itp_handle h, bool need_states) {
  if (!h) return ITP_ERR_ARG;
  if (!h->have_V) return fail(h, ITP_ERR_STATE, "potential not set");
  if (need_states && !h->have_states) return fail(h, ITP_ERR_STATE, "states not set");
  ITP_CUDA(h, cudaSetDevice(h->device));
  return ITP_OK;
}

int do_energies(itp_handle h, double* E_host, int flags) {
  if (h->cur64) {
    ITP_TRY(energies_lane<double>(h, flags));
  } else {
    ITP_TRY(energies_lane<float>(h, flags));
  }
  ITP_CUDA(h, cudaMemcpyAsync(h->E_host_pinned, h->E_dev, h->m * sizeof(double),
                              cudaMemcpyDeviceToHost, h->st));
  ITP_TRY(collect_status(h));
  if (E_host) memcpy(E_host, h->E_host_pinned, h->m * sizeof(double));
  return ITP_OK;
}

// Device work of one step, stream-ordered, no host synchronisation.
template <typename R>
int step_work(itp_handle h, int k, double tau, int flags) {
  ITP_TRY(propagate_lane<R>(h, k, tau));
  ITP_TRY(orthonormalize_lane<R>(h));
  ITP_TRY(energies_lane<R>(h, flags));
  ITP_CUDA(h, cudaMemcpyAsync(h->E_host_pinned, h->E_dev, h->m * sizeof(double),
                              cudaMemcpyDeviceToHost, h->st));
  ITP_CUDA(h, cudaMemcpyAsync(h->status_host, h->status, sizeof(int), cudaMemcpyDeviceToHost,
                              h->st));
  return ITP_OK;
}

// Everything a step allocates or builds once, done outside any capture.
template <typename R>
int step_resources(itp_handle h, int k, double tau) {
  Lane<R>& L = lane_of<R>(h);
  ITP_TRY(prepare_tables<R>(h, L, k, tau));
  if (sizeof(R) == 4 && L.fused_ok && h->g.split_planes[0] != 1) {
    L.work_terms[0] = L.work;
    for (int i = 1; i < k; ++i) {
      if (!L.work_terms[i] &&
          cudaMalloc(&L.work_terms[i], (size_t)h->m * h->g.n_half * 2 * sizeof(R)) !=
              cudaSuccess) {
        cudaGetLastError();
        L.fused_ok = false;
        break;
      }
    }
  }
  return ITP_OK;
}

// ---- launch shapes --------------------------------------------------------------
// Index of the handle's main lane in the per-precision shape arrays.
int main_lane(itp_handle h) { return h->precision == ITP_MIXED ? 0 : 1; }

void get_tuning(itp_handle h, int* t) {
  const int pi = main_lane(h);
  t[ITP_TUNE_PENCIL_W] = h->g.pencil_w;
  t[ITP_TUNE_SPLIT] = h->g.split_planes[pi];
  t[ITP_TUNE_ROW_TB] = h->g.row_tb[pi];
  t[ITP_TUNE_GRAM] = pi == 0 ? h->n_chunks_tc : h->n_chunks;
}

// Validate and apply; returns ITP_OK or ITP_ERR_ARG with a message.
int set_tuning(itp_handle h, const int* t) {
  GridDesc& g = h->g;
  const int pi = main_lane(h);
  const int rb = pi == 0 ? 4 : 8;
  const int w = t[ITP_TUNE_PENCIL_W], split = t[ITP_TUNE_SPLIT], tb = t[ITP_TUNE_ROW_TB],
            chunks = t[ITP_TUNE_GRAM];
  if (w == 0 && !(pi == 0 && g.nz == 128))
    return fail(h, ITP_ERR_ARG, "pencil width 0 (a column per thread) needs nz = 128 and FP32");
  if (w < 0 || w > g.nxh || ((size_t)g.nz * w + g.nz) * 16 > kSmemLimit)
    return fail(h, ITP_ERR_ARG, "pencil width %d not in 0..%d or too large", w, g.nxh);
  if (split < 0 || split > 3) return fail(h, ITP_ERR_ARG, "plane form must be 0, 1, 2 or 3");
  if (!split && plane_smem_bytes(g, rb) > kSmemLimit)
    return fail(h, ITP_ERR_ARG, "a %dx%d plane does not fit one CTA", g.nx, g.ny);
  if (split >= 2 && !(pi == 0 && g.nx == 256 && g.ny == 256))
    return fail(h, ITP_ERR_ARG, "cluster planes are 256x256 FP32 only");
  if (split == 1 && !(tb == 8 || tb == 16 || tb == 32) )
    return fail(h, ITP_ERR_ARG, "row-pass block %d not 8, 16 or 32", tb);
  if (split == 1 && ((g.ny / 2) % tb != 0 || ((size_t)tb * g.pp + g.nx) * 2 * rb > 96 * 1024 ||
                     (tb == 32 && !(pi == 0 && g.nx == 256))))
    return fail(h, ITP_ERR_ARG, "row-pass block %d does not suit a %dx%d plane", tb, g.nx, g.ny);
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
  if (chunks < 1 || chunks > 2 * sms)
    return fail(h, ITP_ERR_ARG, "Gram CTA count %d not in 1..%d", chunks, 2 * sms);
  g.pencil_w = w;
  g.pencil_pitch = w;
  g.split_planes[pi] = split;
  g.row_tb[pi] = split == 1 ? tb : 0;
  if (split == 1) {
    const size_t budget = 72 * 1024, full = (size_t)g.ny * g.nxh * 2 * rb;
    const int c = (int)((full + budget - 1) / budget);
    g.col_w[pi] = (g.nxh + c - 1) / c;
  }
  if (pi == 0) h->n_chunks_tc = chunks;
  else h->n_chunks = chunks;
  h->tune_version++;
  return ITP_OK;
}

// Device time (ms) of `reps` calls of fn after one untimed call.
template <typename F>
int time_ms(itp_handle h, int reps, float* ms, F&& fn) {
  ITP_TRY(fn());
  cudaEvent_t a = nullptr, b = nullptr;
  ITP_CUDA(h, cudaEventCreate(&a));
  if (cudaEventCreate(&b) != cudaSuccess) {
    cudaEventDestroy(a);
    return fail(h, ITP_ERR_CUDA, "event");
  }
  int rc = ITP_OK;
  cudaEventRecord(a, h->st);
  for (int r = 0; r < reps && rc == ITP_OK; ++r) rc = fn();
  cudaEventRecord(b, h->st);
  if (rc == ITP_OK && cudaEventSynchronize(b) != cudaSuccess)
    rc = fail(h, ITP_ERR_CUDA, "timing");
  float t = 0.f;
  if (rc == ITP_OK) cudaEventElapsedTime(&t, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  *ms = t / reps;
  return rc;
}

template <typename R>
int autotune_lane(itp_handle h, int k, double tau, std::string& rep) {
  ITP_TRY(step_resources<R>(h, k, tau));
  const GridDesc& g = h->g;
  const int pi = main_lane(h);
  const int rb = pi == 0 ? 4 : 8;
  int best[ITP_TUNING_LEN], cur[ITP_TUNING_LEN];
  get_tuning(h, best);
  char buf[96];
  auto prop = [&]() { return propagate_lane<R>(h, k, tau); };
  // 1. plane-pass form: whole planes (where they fit) or row + column passes
  {
    std::vector<std::pair<int, int>> forms;   // (plane form, row block)
    if (plane_smem_bytes(g, rb) <= kSmemLimit) forms.push_back({0, 0});
    if (pi == 0 && g.nx == 256 && g.ny == 256) {
      forms.push_back({2, 0});
      forms.push_back({3, 0});
    }
    for (int tb : {32, 16, 8})
      if ((g.ny / 2) % tb == 0 && ((size_t)tb * g.pp + g.nx) * 2 * rb <= 96 * 1024 &&
          (tb != 32 || (pi == 0 && g.nx == 256)))
        forms.push_back({1, tb});
    float best_ms = 1e30f;
    rep += "planes:";
    for (auto [split, tb] : forms) {
      memcpy(cur, best, sizeof(cur));
      cur[ITP_TUNE_SPLIT] = split;
      cur[ITP_TUNE_ROW_TB] = tb;
      if (set_tuning(h, cur) != ITP_OK) continue;
      float ms = 0.f;
      ITP_TRY(time_ms(h, 2, &ms, prop));
      snprintf(buf, sizeof(buf), " %s=%.3fms",
               split == 1 ? ("split" + std::to_string(tb)).c_str()
                          : (split == 2 ? "cluster2" : (split == 3 ? "cluster4" : "whole")), ms);
      rep += buf;
      if (ms < best_ms) {
        best_ms = ms;
        memcpy(best, cur, sizeof(cur));
      }
    }
    ITP_TRY(set_tuning(h, best));
  }
  // 2. pencil width: nx/2+1 columns cut into 1..4 blocks
  {
    float best_ms = 1e30f;
    int last = -1;
    rep += "; pencil_w:";
    for (int c = 0; c <= 4; ++c) {
      const int w = c == 0 ? 0 : (g.nxh + c - 1) / c;
      if (c == 0 && !(pi == 0 && g.nz == 128)) continue;
      if (w == last) continue;
      last = w;
      memcpy(cur, best, sizeof(cur));
      cur[ITP_TUNE_PENCIL_W] = w;
      if (set_tuning(h, cur) != ITP_OK) continue;
      float ms = 0.f;
      ITP_TRY(time_ms(h, 2, &ms, prop));
      snprintf(buf, sizeof(buf), " %d=%.3fms", w, ms);
      rep += buf;
      if (ms < best_ms) {
        best_ms = ms;
        memcpy(best, cur, sizeof(cur));
      }
    }
    ITP_TRY(set_tuning(h, best));
  }
  // 3. CTAs of the overlap kernel, timed on the propagated block
  {
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
    float best_ms = 1e30f;
    rep += "; gram:";
    for (int chunks : {sms, 2 * sms}) {
      float ms = 0.f;
      auto gram = [&]() -> int {
        cudaError_t e;
        if (pi == 0)
          e = launch_tc_gram(h->f32.psi_tmp, h->f32.psi_tmp, h->m, g.n_points, chunks,
                             h->partial, h->status, h->st);
        else
          e = launch_gram_partial<double, double, double>(h->acc, h->acc, h->m, g.n_points,
                                                          chunks, h->partial, h->st);
        return e == cudaSuccess ? ITP_OK : fail(h, ITP_ERR_CUDA, "gram: %s",
                                                cudaGetErrorString(e));
      };
      ITP_TRY(time_ms(h, 3, &ms, gram));
      snprintf(buf, sizeof(buf), " %d=%.3fms", chunks, ms);
      rep += buf;
      if (ms < best_ms) {
        best_ms = ms;
        best[ITP_TUNE_GRAM] = chunks;
      }
    }
    ITP_TRY(set_tuning(h, best));
  }
  return ITP_OK;
}

// ---- the adaptive iteration of Sec. III -------------------------------------------
// Residual norms of rows s0..m-1: mode 1 R^E (A = T psi, coefficient
// exp(-tau E_j)), mode 0 R^H (A = H psi, coefficient E_j); into out[s0..].
template <typename R>
int residual_rows(itp_handle h, const R* A, const R* B, int mode, double tau, int s0,
                  double* out) {
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
  const int rows = h->m - s0;
  const int chunks = std::max(1, std::min(2 * sms, (2 * sms * h->m) / rows));
  const long long N = h->g.n_points;
  ITP_LAUNCH(h, ITP_KERNEL_OTHER,
             launch_residual_norms<R>(A + (long long)s0 * N, B + (long long)s0 * N,
                                      h->E_dev + s0, -tau, mode, rows, N, h->dV, chunks,
                                      h->partial, out + s0, h->st));
  return ITP_OK;
}

template <typename R>
int solve_adaptive_lane(itp_handle h, int k, double tau0, double reduce, double gamma,
                        int max_steps, int max_levels, int* levels_out, double* stats,
                        double* RH_host, double* E_host, bool* converged) {
  Lane<R>& L = lane_of<R>(h);
  const int m = h->m, n = h->n;
  const long long N = h->g.n_points;
  // the propagated block: FP32 psi_tmp (mixed) or the FP64 accumulator
  R* phi = sizeof(R) == 4 ? L.psi_tmp : reinterpret_cast<R*>(h->acc);
  const size_t row = (size_t)N * sizeof(R);
  if (!h->res_dev) ITP_CUDA(h, cudaMalloc(&h->res_dev, 2 * (size_t)m * sizeof(double)));
  double* RE_dev = h->res_dev;
  double* RH_dev = h->res_dev + m;
  std::vector<double> RE(m), RH(m, 0.0);
  // orthonormalise the initial states and take their energies
  ITP_CUDA(h, cudaMemcpyAsync(phi, L.psi, (size_t)m * row, cudaMemcpyDeviceToDevice, h->st));
  ITP_TRY(orthonormalize_lane<R>(h));
  ITP_TRY(energies_lane<R>(h, 0));
  double tau = tau0;
  int level = 0;
  *converged = false;
  for (; level < max_levels; ++level) {
    int c = 0, steps = 0;
    long long props = 0;
    while (steps < max_steps && c < n) {
      // fixed leading states enter the orthonormalisation as they are
      phi = sizeof(R) == 4 ? L.psi_tmp : reinterpret_cast<R*>(h->acc);
      if (c > 0)
        ITP_CUDA(h, cudaMemcpyAsync(phi, L.psi, (size_t)c * row, cudaMemcpyDeviceToDevice,
                                    h->st));
      ITP_TRY(propagate_lane<R>(h, k, tau, c));
      ITP_TRY(residual_rows<R>(h, phi, L.psi, 1, tau, c, RE_dev));
      ITP_TRY(orthonormalize_lane<R>(h));
      ITP_TRY(energies_lane<R>(h, 0));
      ITP_CUDA(h, cudaMemcpyAsync(RE.data() + c, RE_dev + c, (size_t)(m - c) * sizeof(double),
                                  cudaMemcpyDeviceToHost, h->st));
      ITP_TRY(collect_status(h));
      ++steps;
      props += m - c;
      int j = c;
      while (j < m && RE[j] < 0.1 * gamma * tau * tau) ++j;
      c = j;
    }
    // R^H of the Ritz vectors of the current span (within a nearly
    // degenerate group only the span converges at the rate of the gap to the
    // unwanted states): rotate, then H psi and the Ritz values again
    ITP_TRY(energies_lane<R>(h, ITP_RITZ));
    ITP_TRY(energies_lane<R>(h, 0));
    phi = sizeof(R) == 4 ? L.psi_tmp : reinterpret_cast<R*>(h->acc);   // the rotation swaps buffers
    ITP_TRY(residual_rows<R>(h, phi, L.psi, 0, 0.0, 0, RH_dev));
    ITP_CUDA(h, cudaMemcpyAsync(RH.data(), RH_dev, (size_t)m * sizeof(double),
                                cudaMemcpyDeviceToHost, h->st));
    ITP_TRY(collect_status(h));
    if (stats) {
      stats[3 * level] = tau;
      stats[3 * level + 1] = steps;
      stats[3 * level + 2] = (double)props;
    }
    bool done = true;
    for (int j = 0; j < n; ++j) done = done && RH[j] < gamma;
    if (done) {
      *converged = true;
      ++level;
      break;
    }
    tau *= reduce;
  }
  if (levels_out) *levels_out = level;
  if (RH_host) memcpy(RH_host, RH.data(), (size_t)m * sizeof(double));
  // the states are the Ritz vectors; report the Ritz values
  h->have_phi = false;
  ITP_CUDA(h, cudaMemcpyAsync(h->E_host_pinned, h->E_dev, (size_t)m * sizeof(double),
                              cudaMemcpyDeviceToHost, h->st));
  ITP_TRY(collect_status(h));
  if (E_host) memcpy(E_host, h->E_host_pinned, (size_t)m * sizeof(double));
  return ITP_OK;
}

// ---- Eq. (sixp): the Romberg-type T_6 (a comparator of Eq. mcomp) ----------------
// phi = -T_4(tau) psi / 15 + 16 T_4(tau/2)^2 psi / 15 with T_4 the order-4
// multi-product expansion: three T_4 applications (9 T_2) against six T_2
// for the multi-product T_6.
template <typename R>
int propagate_romberg6_lane(itp_handle h, double tau) {
  Lane<R>& L = lane_of<R>(h);
  const size_t bytes = (size_t)h->m * h->g.n_points * sizeof(R);
  if (!L.rom) ITP_CUDA(h, cudaMalloc(&L.rom, bytes));
  R* out = sizeof(R) == 4 ? L.psi_tmp : reinterpret_cast<R*>(h->acc);
  ITP_TRY(propagate_lane<R>(h, 2, 0.5 * tau, 0, L.psi, L.rom));   // v = T_4(tau/2) psi
  ITP_TRY(propagate_lane<R>(h, 2, 0.5 * tau, 0, L.rom, out));     // w = T_4(tau/2) v
  ITP_TRY(propagate_lane<R>(h, 2, tau, 0, L.psi, L.rom));         // u = T_4(tau) psi
  ITP_LAUNCH(h, ITP_KERNEL_OTHER, launch_axpby<R>(16.0 / 15.0, out, -1.0 / 15.0, L.rom, out,
                                                  (long long)h->m * h->g.n_points, h->st));
  return ITP_OK;
}

// ---- one step between host buffers (itp_step_host) --------------------------------
int host_step_resources(itp_handle h) {
  if (h->cst) return ITP_OK;
  if (!h->hstage)
    ITP_CUDA(h, cudaMalloc(&h->hstage, (size_t)h->m * h->g.n_points * sizeof(double)));
  for (auto& e : h->hev)
    if (!e) ITP_CUDA(h, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  // non-blocking: no implicit ordering against a legacy default stream; the
  // events below order the two streams
  ITP_CUDA(h, cudaStreamCreateWithFlags(&h->cst, cudaStreamNonBlocking));
  return ITP_OK;
}

// The states travel in kHostChunks chunks of whole states.  The copy stream
// brings chunk c in while the handle's stream propagates chunk c-1 (the
// propagation of a state needs no other state); the orthonormalisation
// then needs all of them; the staged result goes out chunk by chunk on the
// copy stream while the energies are computed.  Every kernel is the one
// itp_set_states + itp_step + itp_get_states would run on the same states.
template <typename R>
int step_host_work(itp_handle h, int k, double tau, int flags, const double* in,
                   double* out) {
  Lane<R>& L = lane_of<R>(h);
  const GridDesc& g = h->g;
  const size_t N = g.n_points;
  const int C = std::min(kHostChunks, h->m);
  auto first = [&](int c) { return (int)((long long)c * h->m / C); };
  cudaEvent_t* ev_in = h->hev;
  cudaEvent_t* ev_out = h->hev + kHostChunks;
  cudaEvent_t ev_go = h->hev[2 * kHostChunks], ev_done = h->hev[2 * kHostChunks + 1];
  // the copies start after the work already queued on the handle's stream
  ITP_CUDA(h, cudaEventRecord(ev_go, h->st));
  ITP_CUDA(h, cudaStreamWaitEvent(h->cst, ev_go, 0));
  for (int c = 0; c < C; ++c) {
    const size_t off = (size_t)first(c) * N, cnt = (size_t)(first(c + 1) - first(c)) * N;
    ITP_CUDA(h, cudaMemcpyAsync(h->hstage + off, in + off, cnt * sizeof(double),
                                cudaMemcpyHostToDevice, h->cst));
    ITP_CUDA(h, cudaEventRecord(ev_in[c], h->cst));
  }
  for (int c = 0; c < C; ++c) {
    const int s0 = first(c), s1 = first(c + 1);
    ITP_CUDA(h, cudaStreamWaitEvent(h->st, ev_in[c], 0));
    // user layout [z][y][x] -> internal [z][x][y], rounded to R
    ITP_LAUNCH(h, ITP_KERNEL_OTHER,
               (launch_transpose_planes<double, R>(h->hstage + (size_t)s0 * N,
                                                   L.psi + (size_t)s0 * N,
                                                   (long long)(s1 - s0) * g.nz, g.ny, g.nx,
                                                   h->st)));
    ITP_TRY(propagate_lane<R>(h, k, tau, s0, nullptr, nullptr, s1));
  }
  ITP_TRY(orthonormalize_lane<R>(h));
  for (int c = 0; c < C; ++c) {
    const int s0 = first(c), s1 = first(c + 1);
    ITP_LAUNCH(h, ITP_KERNEL_OTHER,
               (launch_transpose_planes<R, double>(L.psi + (size_t)s0 * N,
                                                   h->hstage + (size_t)s0 * N,
                                                   (long long)(s1 - s0) * g.nz, g.nx, g.ny,
                                                   h->st)));
    ITP_CUDA(h, cudaEventRecord(ev_out[c], h->st));
  }
  ITP_TRY(energies_lane<R>(h, flags));
  ITP_CUDA(h, cudaMemcpyAsync(h->E_host_pinned, h->E_dev, h->m * sizeof(double),
                              cudaMemcpyDeviceToHost, h->st));
  ITP_CUDA(h, cudaMemcpyAsync(h->status_host, h->status, sizeof(int), cudaMemcpyDeviceToHost,
                              h->st));
  for (int c = 0; c < C; ++c) {
    const size_t off = (size_t)first(c) * N, cnt = (size_t)(first(c + 1) - first(c)) * N;
    ITP_CUDA(h, cudaStreamWaitEvent(h->cst, ev_out[c], 0));
    ITP_CUDA(h, cudaMemcpyAsync(out + off, h->hstage + off, cnt * sizeof(double),
                                cudaMemcpyDeviceToHost, h->cst));
  }
  ITP_CUDA(h, cudaEventRecord(ev_done, h->cst));
  ITP_CUDA(h, cudaStreamWaitEvent(h->st, ev_done, 0));
  return ITP_OK;
}

}  // namespace

// A batch of independent problems: one handle (and stream) per problem and
// the CUDA graph of one step of all of them.
struct itp_batch {
  int device = 0;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  std::vector<itp_handle> probs;
  std::vector<int> e_off;   // offset of problem p's energies
  int m_total = 0;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
  cudaGraphExec_t exec = nullptr;
  int order = 0, flags = -1;
  double tau = 0.0;
  std::vector<int> versions;   // problems' launch-shape versions at capture
  long long step_launches = 0, launches = 0;
  std::string err;
  // grouped launches (itp_batch_set_grouping): the argument tables of the
  // captured graph's grouped passes, and the events that fork and join the
  // per-problem branches between them
  bool grouped = true;
  void* tables = nullptr;
  std::vector<cudaEvent_t> evpool;
  int n_groups = 0;
};

namespace {

thread_local std::string g_batch_create_error;

int batch_fail(itp_batch* b, int code, const std::string& msg) {
  if (b) b->err = msg;
  else g_batch_create_error = msg;
  return code;
}

// Record one whole step of a problem (the kernels of itp_step, and the
// copies of its energies and status word) without launching anything.
template <typename R>
int record_step(itp_handle h, int k, double tau, int flags, std::vector<RecOp>* ops) {
  h->rec = ops;
  int rc = propagate_lane<R>(h, k, tau);
  if (rc == ITP_OK) rc = orthonormalize_lane<R>(h);
  if (rc == ITP_OK) rc = energies_lane<R>(h, flags);
  h->rec = nullptr;
  if (rc != ITP_OK) return rc;
  RecOp e, st;
  e.fn = [h]() {
    return cudaMemcpyAsync(h->E_host_pinned, h->E_dev, h->m * sizeof(double),
                           cudaMemcpyDeviceToHost, h->st);
  };
  st.fn = [h]() {
    return cudaMemcpyAsync(h->status_host, h->status, sizeof(int), cudaMemcpyDeviceToHost,
                           h->st);
  };
  ops->push_back(std::move(e));
  ops->push_back(std::move(st));
  return ITP_OK;
}

// A recorded pass that can run as a grouped launch: every FFT pass except
// plane passes on planes too large for one CTA (row + column passes).
bool groupable(const RecOp& op, itp_handle h) {
  return op.kind != RecOp::kOther && !(op.kind == RecOp::kPlane && h->g.split_planes[op.lane]) &&
         !(op.kind == RecOp::kPencil && h->g.pencil_w == 0);
}

// Grid, precision lane and launch shapes of a problem, and the kinds and
// modes of its recorded passes: problems with equal keys can share grouped
// launches pass by pass.
std::string group_key(itp_handle h, const std::vector<RecOp>& ops) {
  const int lane = h->cur64 ? 1 : 0;
  std::string key = std::to_string(h->g.nx) + "x" + std::to_string(h->g.ny) + "x" +
                    std::to_string(h->g.nz) + "|" + std::to_string(lane) + "|" +
                    std::to_string(h->g.pencil_w) + "|" +
                    std::to_string(h->g.split_planes[lane]) + "|";
  for (const RecOp& op : ops) {
    key += (char)('a' + op.kind);
    key += (char)('0' + op.mode);
  }
  return key;
}

// Build the graph of one step of every problem with grouped launches: each
// FFT pass (plane, pencil, exact term sum) of the problems in a group (same
// grid, lane, launch shapes and pass sequence) is one launch over all their
// states; the other kernels (overlap, Cholesky, update, eigenvalues, the
// copies) run between those launches as one branch per problem.  Groups run
// as parallel branches.  The argument tables are copied to the device
// before the capture.
int build_grouped_graph(itp_batch* b, int k, double tau, int eflags, cudaGraph_t* graph_out) {
  const int np = (int)b->probs.size();
  std::vector<std::vector<RecOp>> ops(np);
  for (int p = 0; p < np; ++p) {
    itp_handle h = b->probs[p];
    const int rc = h->cur64 ? record_step<double>(h, k, tau, eflags, &ops[p])
                            : record_step<float>(h, k, tau, eflags, &ops[p]);
    if (rc != ITP_OK)
      return batch_fail(b, rc, "problem " + std::to_string(p) + ": " + h->err);
  }
  std::vector<std::string> keys(np);
  std::vector<std::vector<int>> groups;
  for (int p = 0; p < np; ++p) {
    keys[p] = group_key(b->probs[p], ops[p]);
    bool placed = false;
    for (auto& G : groups)
      if (keys[G[0]] == keys[p]) {
        G.push_back(p);
        placed = true;
        break;
      }
    if (!placed) groups.push_back({p});
  }
  // argument tables: per group and grouped pass, the members' arguments and
  // the (member, state / plane) of every CTA row, 256-byte aligned
  std::vector<unsigned char> host;
  auto put = [&host](const void* src, size_t bytes) {
    const size_t off = (host.size() + 255) & ~(size_t)255;
    host.resize(off + bytes);
    memcpy(host.data() + off, src, bytes);
    return off;
  };
  struct Planned { size_t args, rows; int nrows; };
  std::vector<std::vector<Planned>> plan(groups.size());
  size_t n_events = 1;
  for (size_t gi = 0; gi < groups.size(); ++gi) {
    const std::vector<int>& G = groups[gi];
    const std::vector<RecOp>& o0 = ops[G[0]];
    plan[gi].resize(o0.size(), Planned{0, 0, 0});
    n_events += 1;
    for (size_t t = 0; t < o0.size(); ++t) {
      if (!groupable(o0[t], b->probs[G[0]])) {
        if (t == 0 || groupable(o0[t - 1], b->probs[G[0]])) n_events += G.size();
        continue;
      }
      if (G.size() < 2) continue;
      std::vector<int2> rows;
      std::vector<unsigned char> args;
      for (int q = 0; q < (int)G.size(); ++q) {
        const RecOp& op = ops[G[q]][t];
        int nrow = 0;
        const void* a = nullptr;
        size_t asz = 0;
        if (op.kind == RecOp::kPlane) {
          nrow = op.lane ? op.p64.m : op.p32.m;
          a = op.lane ? (const void*)&op.p64 : (const void*)&op.p32;
          asz = op.lane ? sizeof(op.p64) : sizeof(op.p32);
        } else if (op.kind == RecOp::kPencil) {
          nrow = op.lane ? op.e64.m : op.e32.m;
          a = op.lane ? (const void*)&op.e64 : (const void*)&op.e32;
          asz = op.lane ? sizeof(op.e64) : sizeof(op.e32);
        } else {
          nrow = op.ts.m;
          a = &op.ts;
          asz = sizeof(op.ts);
        }
        for (int r = 0; r < nrow; ++r) rows.push_back(make_int2(q, r));
        const size_t o = args.size();
        args.resize(o + asz);
        memcpy(args.data() + o, a, asz);
      }
      if (rows.size() > 65535)
        return batch_fail(b, ITP_ERR_ARG, "a group has more than 65535 states; "
                                          "use itp_batch_set_grouping(b, 0)");
      Planned pl;
      pl.args = put(args.data(), args.size());
      pl.rows = put(rows.data(), rows.size() * sizeof(int2));
      pl.nrows = (int)rows.size();
      plan[gi][t] = pl;
    }
  }
  if (b->tables) {
    cudaFree(b->tables);
    b->tables = nullptr;
  }
  if (!host.empty()) {
    if (cudaMalloc(&b->tables, host.size()) != cudaSuccess)
      return batch_fail(b, ITP_ERR_OOM, "grouped argument tables");
    if (cudaMemcpy(b->tables, host.data(), host.size(), cudaMemcpyHostToDevice) != cudaSuccess)
      return batch_fail(b, ITP_ERR_CUDA, "grouped argument tables");
  }
  while (b->evpool.size() < n_events) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
      return batch_fail(b, ITP_ERR_CUDA, "events");
    b->evpool.push_back(e);
  }
  unsigned char* dev = static_cast<unsigned char*>(b->tables);
  size_t ev = 0;
  auto next_event = [&]() { return b->evpool[ev++]; };
  if (cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return batch_fail(b, ITP_ERR_CUDA, "begin capture");
  cudaError_t e = cudaSuccess;
  cudaEvent_t fork = next_event();
  e = cudaEventRecord(fork, b->st);
  for (size_t gi = 0; gi < groups.size() && e == cudaSuccess; ++gi) {
    const std::vector<int>& G = groups[gi];
    itp_handle h0 = b->probs[G[0]];
    cudaStream_t gst = h0->st;
    e = cudaStreamWaitEvent(gst, fork, 0);
    const std::vector<RecOp>& o0 = ops[G[0]];
    for (size_t t = 0; t < o0.size() && e == cudaSuccess;) {
      if (groupable(o0[t], h0)) {
        if (G.size() < 2) {
          e = o0[t].fn();
        } else {
          const Planned& pl = plan[gi][t];
          const int2* rows = reinterpret_cast<const int2*>(dev + pl.rows);
          const RecOp& op = o0[t];
          if (op.kind == RecOp::kPlane)
            e = op.lane ? launch_plane_group<double>(
                              h0->g, op.mode, reinterpret_cast<const PlaneArgs<double>*>(dev + pl.args),
                              rows, pl.nrows, gst)
                        : launch_plane_group<float>(
                              h0->g, op.mode, reinterpret_cast<const PlaneArgs<float>*>(dev + pl.args),
                              rows, pl.nrows, gst);
          else if (op.kind == RecOp::kPencil)
            e = op.lane ? launch_pencil_group<double>(
                              h0->g, op.mode, reinterpret_cast<const PencilArgs<double>*>(dev + pl.args),
                              rows, pl.nrows, gst)
                        : launch_pencil_group<float>(
                              h0->g, op.mode, reinterpret_cast<const PencilArgs<float>*>(dev + pl.args),
                              rows, pl.nrows, gst);
          else
            e = launch_term_sum_group(reinterpret_cast<const TermSumArgs*>(dev + pl.args), rows,
                                      pl.nrows, op.ts.nz, op.ts.plane_pts, gst);
        }
        ++t;
        continue;
      }
      // a run of other kernels: one branch per member problem
      size_t t2 = t;
      while (t2 < o0.size() && !groupable(o0[t2], h0)) ++t2;
      cudaEvent_t f = next_event();
      e = cudaEventRecord(f, gst);
      for (size_t q = 0; q < G.size() && e == cudaSuccess; ++q) {
        itp_handle hq = b->probs[G[q]];
        if (q > 0) e = cudaStreamWaitEvent(hq->st, f, 0);
        for (size_t u = t; u < t2 && e == cudaSuccess; ++u) e = ops[G[q]][u].fn();
        if (q > 0 && e == cudaSuccess) {
          cudaEvent_t j = next_event();
          e = cudaEventRecord(j, hq->st);
          if (e == cudaSuccess) e = cudaStreamWaitEvent(gst, j, 0);
        }
      }
      t = t2;
    }
    if (e == cudaSuccess) {
      cudaEvent_t j = next_event();
      e = cudaEventRecord(j, gst);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(b->st, j, 0);
    }
  }
  cudaGraph_t graph = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(b->st, &graph);
  if (e != cudaSuccess || ec != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return batch_fail(b, ITP_ERR_CUDA, std::string("grouped capture: ") +
                                           cudaGetErrorString(e != cudaSuccess ? e : ec));
  }
  b->n_groups = (int)groups.size();
  *graph_out = graph;
  return ITP_OK;
}

// Kernel nodes of a graph (the launches one replay makes).
long long graph_kernels(cudaGraph_t graph) {
  size_t n = 0;
  if (cudaGraphGetNodes(graph, nullptr, &n) != cudaSuccess || n == 0) return 0;
  std::vector<cudaGraphNode_t> nodes(n);
  if (cudaGraphGetNodes(graph, nodes.data(), &n) != cudaSuccess) return 0;
  long long k = 0;
  for (size_t i = 0; i < n; ++i) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
  }
  return k;
}

}  // namespace

extern "C" {

void itp_destroy(itp_handle h);

int itp_create_grid(itp_handle* out, int nx, int ny, int nz, double lx, double ly, double lz,
                    int n_states, int n_guard, int precision, void* cuda_stream) {
  if (!out) return ITP_ERR_ARG;
  *out = nullptr;
  g_create_error.clear();
  itp_handle h = new (std::nothrow) itp_grid();
  if (!h) return ITP_ERR_OOM;
  auto bail = [&](int code) {
    // the message stays readable through itp_last_error(NULL)
    g_create_error = h->err;
    itp_destroy(h);
    return code;
  };
  GridDesc& g = h->g;
  // nz = 1: a 2D problem in the x-y plane (the z transform is the identity)
  const bool planar = nz == 1;
  if (planar) {
    g.rz1 = 1;
    g.rz2 = 1;
  }
  if (!split_axis(nx, &g.rx1, &g.rx2) || !split_axis(ny, &g.ry1, &g.ry2) ||
      (!planar && !split_axis(nz, &g.rz1, &g.rz2)))
    return bail(fail(h, ITP_ERR_ARG, "unsupported grid %dx%dx%d (edges even, 2..256, "
                                     "a product of two of 1,2,3,4,6,8,12,16; nz may be 1)",
                     nx, ny, nz));
  if (!(lx > 0 && ly > 0 && lz > 0))
    return bail(fail(h, ITP_ERR_ARG, "box lengths must be positive"));
  if (n_states < 1 || n_guard < 0 || n_states + n_guard > kMaxStates)
    return bail(fail(h, ITP_ERR_ARG, "need 1 <= n_states and n_states + n_guard <= %d",
                     kMaxStates));
  if (precision != ITP_FP64 && precision != ITP_MIXED)
    return bail(fail(h, ITP_ERR_ARG, "unknown precision %d", precision));
  g.nx = nx;
  g.ny = ny;
  g.nz = nz;
  g.nxh = nx / 2 + 1;
  g.n_points = (long long)nx * ny * nz;
  g.n_half = (long long)nz * ny * g.nxh;
  g.pp = plane_row_pitch(nx);
  const int cbytes = precision == ITP_FP64 ? 16 : 8;
  {
    const size_t budget = 72 * 1024;
    const size_t full = (size_t)nz * g.nxh * cbytes;
    const int chunks = (int)((full + budget - 1) / budget);
    g.pencil_w = (g.nxh + chunks - 1) / chunks;
    g.pencil_pitch = g.pencil_w;
  }
  // planes whose half spectrum does not fit one CTA run as row + column
  // passes: row-pass blocks of tb row pairs, column-pass blocks of cw columns
  for (int pi = 0; pi < 2; ++pi) {
    const int rb = pi == 0 ? 4 : 8;   // bytes per real
    g.split_planes[pi] = plane_smem_bytes(g, rb) > kSmemLimit;
    g.row_tb[pi] = 0;
    g.col_w[pi] = 0;
    if (!g.split_planes[pi]) continue;
    for (int tb : {32, 16, 8}) {
      if ((ny / 2) % tb == 0 && ((size_t)tb * g.pp + nx) * 2 * rb <= 96 * 1024 &&
          (tb != 32 || (pi == 0 && nx == 256))) {
        g.row_tb[pi] = tb;
        break;
      }
    }
    const size_t budget = 72 * 1024, full = (size_t)ny * g.nxh * 2 * rb;
    const int chunks = (int)((full + budget - 1) / budget);
    g.col_w[pi] = (g.nxh + chunks - 1) / chunks;
  }
  const int need = precision == ITP_MIXED ? 2 : 1;
  for (int pi = (precision == ITP_MIXED ? 0 : 1); pi < 2 && need; ++pi)
    if (g.split_planes[pi] && g.row_tb[pi] == 0)
      return bail(fail(h, ITP_ERR_ARG, "no row-pass blocking for a %dx%d plane", nx, ny));
  h->lx = lx;
  h->ly = ly;
  h->lz = lz;
  h->dV = (lx / nx) * (ly / ny) * (lz / nz);
  h->n = n_states;
  h->ng = n_guard;
  h->m = n_states + n_guard;
  h->precision = precision;
  h->st = (cudaStream_t)cuda_stream;
  if (!h->st) {
    // a stream of its own, so that steps can be captured into a CUDA graph
    if (cudaStreamCreateWithFlags(&h->st, cudaStreamNonBlocking) != cudaSuccess)
      return bail(fail(h, ITP_ERR_CUDA, "cannot create a stream"));
    h->own_stream = true;
  }
  if (cudaGetDevice(&h->device) != cudaSuccess)
    return bail(fail(h, ITP_ERR_CUDA, "no CUDA device"));
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
  h->n_chunks = 2 * sms;
  h->n_chunks_tc = sms;
  const size_t N = (size_t)g.n_points, m = (size_t)h->m;
  int rc;
#define ITP_CREATE(expr)           \
  do {                             \
    rc = (expr);                   \
    if (rc != ITP_OK) return bail(rc); \
  } while (0)
  auto cuda = [&](cudaError_t e, const char* what) {
    if (e == cudaSuccess) return ITP_OK;
    return fail(h, e == cudaErrorMemoryAllocation ? ITP_ERR_OOM : ITP_ERR_CUDA, "%s: %s", what,
                cudaGetErrorString(e));
  };
  ITP_CREATE(cuda(cudaMalloc(&h->V, N * sizeof(double)), "V"));
  ITP_CREATE(cuda(cudaMalloc(&h->Vstage, N * sizeof(double)), "V staging"));
  ITP_CREATE(cuda(cudaMalloc(&h->acc, m * N * sizeof(double)), "accumulator"));
  ITP_CREATE(cuda(cudaMalloc(&h->partial, (size_t)h->n_chunks * m * m * sizeof(double)),
                  "partials"));
  ITP_CREATE(cuda(cudaMalloc(&h->S, m * m * sizeof(double)), "S"));
  ITP_CREATE(cuda(cudaMalloc(&h->Mx, m * m * sizeof(double)), "M"));
  ITP_CREATE(cuda(cudaMalloc(&h->Hs, m * m * sizeof(double)), "H_sub"));
  // eigen-decomposition work: U^T, and the Jacobi matrix when it does not
  // fit one CTA's shared memory
  ITP_CREATE(cuda(cudaMalloc(&h->Wmm, (2 * m + 1) * m * sizeof(double)), "work"));
  ITP_CREATE(cuda(cudaMalloc(&h->E_dev, m * sizeof(double)), "E"));
  ITP_CREATE(cuda(cudaMalloc(&h->status, sizeof(int)), "status"));
  ITP_CREATE(cuda(cudaMemset(h->status, 0, sizeof(int)), "status"));
  ITP_CREATE(cuda(cudaMallocHost(&h->status_host, sizeof(int)), "status (host)"));
  ITP_CREATE(cuda(cudaMallocHost(&h->E_host_pinned, m * sizeof(double)), "E (host)"));
  if (precision == ITP_FP64) {
    ITP_CREATE(alloc_lane<double>(h, h->f64));
    h->cur64 = true;
  } else {
    ITP_CREATE(alloc_lane<float>(h, h->f32));
    h->cur64 = false;
  }
  ITP_CREATE(cuda(cudaStreamSynchronize(h->st), "create"));
#undef ITP_CREATE
  *out = h;
  return ITP_OK;
}

void itp_destroy(itp_handle h) {
  if (!h) return;
  cudaSetDevice(h->device);
  if (h->st) cudaStreamSynchronize(h->st);
  else cudaDeviceSynchronize();
  if (h->step_exec) cudaGraphExecDestroy(h->step_exec);
  free_lane(h->f32);
  free_lane(h->f64);
  cudaFree(h->V);
  cudaFree(h->Vstage);
  cudaFree(h->acc);
  cudaFree(h->partial);
  cudaFree(h->S);
  cudaFree(h->Mx);
  cudaFree(h->Hs);
  cudaFree(h->Wmm);
  cudaFree(h->E_dev);
  cudaFree(h->status);
  cudaFreeHost(h->status_host);
  cudaFreeHost(h->E_host_pinned);
  cudaFree(h->res_dev);
  if (h->cst) {
    cudaStreamSynchronize(h->cst);
    cudaStreamDestroy(h->cst);
  }
  cudaFree(h->hstage);
  for (auto& e : h->hev)
    if (e) cudaEventDestroy(e);
  for (auto& e : h->prof_events) {
    cudaEventDestroy(e.start);
    cudaEventDestroy(e.stop);
  }
  if (h->own_stream) cudaStreamDestroy(h->st);
  delete h;
}

int itp_set_potential(itp_handle h, const double* V_host) {
  if (!h || !V_host) return h ? fail(h, ITP_ERR_ARG, "null potential") : ITP_ERR_ARG;
  ITP_CUDA(h, cudaSetDevice(h->device));
  ITP_CUDA(h, cudaMemcpyAsync(h->Vstage, V_host, (size_t)h->g.n_points * sizeof(double),
                              cudaMemcpyHostToDevice, h->st));
  ITP_LAUNCH(h, ITP_KERNEL_OTHER, (launch_transpose_planes<double, double>(
                                      h->Vstage, h->V, h->g.nz, h->g.ny, h->g.nx, h->st)));
  h->f32.tab_order = 0;
  h->f64.tab_order = 0;
  if (h->f32.ready)
    ITP_LAUNCH(h, ITP_KERNEL_OTHER, (launch_convert<double, float>(h->V, h->f32.Vr,
                                                                   h->g.n_points, h->st)));
  if (h->f64.ready)
    ITP_LAUNCH(h, ITP_KERNEL_OTHER, (launch_convert<double, double>(h->V, h->f64.Vr,
                                                                    h->g.n_points, h->st)));
  h->have_V = true;
  return ITP_OK;
}

static int set_states_impl(itp_handle h, const double* src, cudaMemcpyKind kind) {
  ITP_CUDA(h, cudaSetDevice(h->device));
  const size_t count = (size_t)h->m * h->g.n_points;
  const long long planes = (long long)h->m * h->g.nz;
  // user layout [m][z][y][x] -> staging -> internal [m][z][x][y]
  if (h->precision == ITP_FP64) {
    ITP_CUDA(h, cudaMemcpyAsync(h->f64.psi_tmp, src, count * sizeof(double), kind, h->st));
    ITP_LAUNCH(h, ITP_KERNEL_OTHER, (launch_transpose_planes<double, double>(
                                        h->f64.psi_tmp, h->f64.psi, planes, h->g.ny, h->g.nx,
                                        h->st)));
    h->cur64 = true;
  } else {
    ITP_CUDA(h, cudaMemcpyAsync(h->acc, src, count * sizeof(double), kind, h->st));
    ITP_LAUNCH(h, ITP_KERNEL_OTHER, (launch_transpose_planes<double, float>(
                                        h->acc, h->f32.psi, planes, h->g.ny, h->g.nx, h->st)));
    h->cur64 = false;
  }
  h->have_states = true;
  h->have_phi = false;
  return ITP_OK;
}

int itp_set_states(itp_handle h, const double* psi_host) {
  if (!h || !psi_host) return h ? fail(h, ITP_ERR_ARG, "null states") : ITP_ERR_ARG;
  return set_states_impl(h, psi_host, cudaMemcpyHostToDevice);
}

int itp_set_states_device(itp_handle h, const double* psi_device) {
  if (!h || !psi_device) return h ? fail(h, ITP_ERR_ARG, "null states") : ITP_ERR_ARG;
  return set_states_impl(h, psi_device, cudaMemcpyDeviceToDevice);
}

int itp_get_states(itp_handle h, double* psi_host) {
  if (!h || !psi_host) return h ? fail(h, ITP_ERR_ARG, "null output") : ITP_ERR_ARG;
  if (!h->have_states) return fail(h, ITP_ERR_STATE, "states not set");
  ITP_CUDA(h, cudaSetDevice(h->device));
  const size_t count = (size_t)h->m * h->g.n_points;
  const long long planes = (long long)h->m * h->g.nz;
  double* stage;
  if (h->cur64) {
    stage = h->f64.psi_tmp;
    ITP_LAUNCH(h, ITP_KERNEL_OTHER, (launch_transpose_planes<double, double>(
                                        h->f64.psi, stage, planes, h->g.nx, h->g.ny, h->st)));
  } else {
    stage = h->acc;
    h->have_phi = false;
    ITP_LAUNCH(h, ITP_KERNEL_OTHER, (launch_transpose_planes<float, double>(
                                        h->f32.psi, stage, planes, h->g.nx, h->g.ny, h->st)));
  }
  ITP_CUDA(h, cudaMemcpyAsync(psi_host, stage, count * sizeof(double), cudaMemcpyDeviceToHost,
                              h->st));
  return collect_status(h);
}

int itp_get_phi(itp_handle h, double* phi_host) {
  if (!h || !phi_host) return h ? fail(h, ITP_ERR_ARG, "null output") : ITP_ERR_ARG;
  if (!h->have_phi) return fail(h, ITP_ERR_STATE, "no propagated states pending");
  ITP_CUDA(h, cudaSetDevice(h->device));
  const GridDesc& g = h->g;
  const size_t count = (size_t)h->m * g.n_points;
  std::vector<double> tmp(count);
  if (h->cur64) {
    ITP_CUDA(h, cudaMemcpyAsync(tmp.data(), h->acc, count * sizeof(double),
                                cudaMemcpyDeviceToHost, h->st));
    ITP_TRY(collect_status(h));
  } else {
    std::vector<float> t32(count);
    ITP_CUDA(h, cudaMemcpyAsync(t32.data(), h->f32.psi_tmp, count * sizeof(float),
                                cudaMemcpyDeviceToHost, h->st));
    ITP_TRY(collect_status(h));
    for (size_t q = 0; q < count; ++q) tmp[q] = t32[q];
  }
  // internal [m][z][x][y] -> user [m][z][y][x] (diagnostic path, on the host)
  const size_t plane = (size_t)g.nx * g.ny;
  for (size_t p = 0; p < (size_t)h->m * g.nz; ++p) {
    const double* s = tmp.data() + p * plane;
    double* d = phi_host + p * plane;
    for (int x = 0; x < g.nx; ++x)
      for (int y = 0; y < g.ny; ++y) d[(size_t)y * g.nx + x] = s[(size_t)x * g.ny + y];
  }
  return ITP_OK;
}

int itp_propagate(itp_handle h, int order, double tau) {
  ITP_TRY(check_ready(h, true));
  if (order < 2 || order > 2 * kMaxTerms || (order & 1))
    return fail(h, ITP_ERR_ARG, "order must be even, 2..%d (got %d)", 2 * kMaxTerms, order);
  if (!(tau > 0) || !std::isfinite(tau)) return fail(h, ITP_ERR_ARG, "tau must be > 0");
  const int k = order / 2;
  if (h->precision == ITP_MIXED) {
    ITP_TRY(switch_lane<float>(h));
    ITP_TRY(propagate_lane<float>(h, k, tau));
  } else {
    ITP_TRY(propagate_lane<double>(h, k, tau));
  }
  h->have_phi = true;
  return ITP_OK;
}

int itp_orthonormalize(itp_handle h) {
  ITP_TRY(check_ready(h, true));
  if (!h->have_phi) return fail(h, ITP_ERR_STATE, "no propagated states (call itp_propagate)");
  if (h->cur64) {
    ITP_TRY(orthonormalize_lane<double>(h));
  } else {
    ITP_TRY(orthonormalize_lane<float>(h));
  }
  h->have_phi = false;
  return ITP_OK;
}

// ITP_EVAL_FP64: the mixed path's final evaluation in FP64 -- the FP32
// states rounded up to FP64, orthonormalised again in FP64 (Eq. 4), after
// which the energies run on the FP64 lane.  No propagation.
static int eval_fp64(itp_handle h) {
  if (h->cur64) return ITP_OK;
  ITP_TRY(alloc_lane<double>(h, h->f64));
  ITP_LAUNCH(h, ITP_KERNEL_OTHER, (launch_convert<float, double>(
                                      h->f32.psi, h->acc, (long long)h->m * h->g.n_points,
                                      h->st)));
  ITP_TRY(orthonormalize_lane<double>(h));
  h->cur64 = true;
  return ITP_OK;
}

int itp_energies(itp_handle h, double* E_host, int flags) {
  ITP_TRY(check_ready(h, true));
  if (flags & ~(ITP_RITZ | ITP_RITZ_VALUES | ITP_EVAL_FP64))
    return fail(h, ITP_ERR_ARG, "unknown energy flags %d", flags);
  h->have_phi = false;
  if (flags & ITP_EVAL_FP64) ITP_TRY(eval_fp64(h));
  return do_energies(h, E_host, flags & ~ITP_EVAL_FP64);
}

int itp_step(itp_handle h, int order, double tau, int flags, double* E_host) {
  ITP_TRY(check_ready(h, true));
  if (order < 2 || order > 2 * kMaxTerms || (order & 1))
    return fail(h, ITP_ERR_ARG, "order must be even, 2..%d (got %d)", 2 * kMaxTerms, order);
  if (!(tau > 0) || !std::isfinite(tau)) return fail(h, ITP_ERR_ARG, "tau must be > 0");
  if (flags != 0 && flags != ITP_RITZ_VALUES)
    return fail(h, ITP_ERR_ARG, "itp_step takes flags 0 or ITP_RITZ_VALUES");
  const int k = order / 2;
  int lane;
  if (h->precision == ITP_MIXED) {
    ITP_TRY(switch_lane<float>(h));
    ITP_TRY(step_resources<float>(h, k, tau));
    lane = 0;
  } else {
    ITP_TRY(step_resources<double>(h, k, tau));
    lane = 1;
  }
  if (!h->step_exec || h->step_order != order || h->step_tau != tau ||
      h->step_flags != flags || h->step_lane != lane || h->step_version != h->tune_version) {
    if (h->step_exec) {
      cudaGraphExecDestroy(h->step_exec);
      h->step_exec = nullptr;
    }
    ITP_CUDA(h, cudaStreamSynchronize(h->st));
    cudaGraph_t graph = nullptr;
    ITP_CUDA(h, cudaStreamBeginCapture(h->st, cudaStreamCaptureModeThreadLocal));
    h->capturing = true;
    const long long launches0 = h->launches;
    const int rc = lane == 0 ? step_work<float>(h, k, tau, flags)
                             : step_work<double>(h, k, tau, flags);
    h->capturing = false;
    h->step_launches = h->launches - launches0;
    h->launches = launches0;
    const cudaError_t ec = cudaStreamEndCapture(h->st, &graph);
    if (rc != ITP_OK) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    ITP_CUDA(h, ec);
    const cudaError_t ei = cudaGraphInstantiate(&h->step_exec, graph, 0);
    cudaGraphDestroy(graph);
    ITP_CUDA(h, ei);
    h->step_order = order;
    h->step_tau = tau;
    h->step_flags = flags;
    h->step_lane = lane;
    h->step_version = h->tune_version;
  }
  ITP_CUDA(h, cudaGraphLaunch(h->step_exec, h->st));
  h->launches += h->step_launches;
  h->have_phi = false;
  ITP_CUDA(h, cudaStreamSynchronize(h->st));
  ITP_TRY(take_status(h));
  if (E_host) memcpy(E_host, h->E_host_pinned, h->m * sizeof(double));
  return ITP_OK;
}

int itp_step_host(itp_handle h, int order, double tau, int flags, const double* psi_in_host,
                  double* psi_out_host, double* E_host) {
  ITP_TRY(check_ready(h, false));
  if (!psi_in_host || !psi_out_host) return fail(h, ITP_ERR_ARG, "null state buffer");
  if (order < 2 || order > 2 * kMaxTerms || (order & 1))
    return fail(h, ITP_ERR_ARG, "order must be even, 2..%d (got %d)", 2 * kMaxTerms, order);
  if (!(tau > 0) || !std::isfinite(tau)) return fail(h, ITP_ERR_ARG, "tau must be > 0");
  if (flags != 0 && flags != ITP_RITZ_VALUES)
    return fail(h, ITP_ERR_ARG, "itp_step_host takes flags 0 or ITP_RITZ_VALUES");
  const int k = order / 2;
  const bool mixed = h->precision == ITP_MIXED;
  // everything allocated or built once, before the first copy is queued
  if (mixed) {
    ITP_TRY(step_resources<float>(h, k, tau));
  } else {
    ITP_TRY(step_resources<double>(h, k, tau));
  }
  ITP_TRY(host_step_resources(h));
  h->have_states = true;   // the lane's states are being replaced
  h->have_phi = false;
  h->cur64 = !mixed;
  const int rc = mixed ? step_host_work<float>(h, k, tau, flags, psi_in_host, psi_out_host)
                       : step_host_work<double>(h, k, tau, flags, psi_in_host, psi_out_host);
  // nothing may still read or write the caller's buffers when this returns
  const cudaError_t e1 = cudaStreamSynchronize(h->cst);
  const cudaError_t e2 = cudaStreamSynchronize(h->st);
  if (rc != ITP_OK) {
    h->have_states = false;   // partly overwritten
    return rc;
  }
  ITP_CUDA(h, e1);
  ITP_CUDA(h, e2);
  ITP_TRY(take_status(h));
  if (E_host) memcpy(E_host, h->E_host_pinned, h->m * sizeof(double));
  return ITP_OK;
}

int itp_polish(itp_handle h, int order, double tau, double tol, int max_steps, int* steps_out,
               double* E_host) {
  ITP_TRY(check_ready(h, true));
  if (steps_out) *steps_out = 0;
  if (h->precision != ITP_MIXED) return fail(h, ITP_ERR_ARG, "itp_polish needs ITP_MIXED");
  if (order < 2 || order > 2 * kMaxTerms || (order & 1) || !(tau > 0) || !(tol > 0) ||
      max_steps < 1)
    return fail(h, ITP_ERR_ARG, "bad polish arguments");
  ITP_TRY(switch_lane<double>(h));
  std::vector<double> prev(h->m), cur(h->m);
  int step;
  for (step = 1; step <= max_steps; ++step) {
    ITP_TRY(propagate_lane<double>(h, order / 2, tau));
    ITP_TRY(orthonormalize_lane<double>(h));
    ITP_TRY(do_energies(h, cur.data(), ITP_RITZ_VALUES));
    if (step > 1) {
      double d = 0;
      for (int j = 0; j < h->n; ++j) d = std::fmax(d, std::fabs(cur[j] - prev[j]));
      if (d < tol) break;
    }
    prev.swap(cur);
  }
  if (step > max_steps) {
    step = max_steps;
    prev.swap(cur);   // last computed energies are in prev after the final swap
  }
  // leave the states on the Ritz vectors of the converged subspace
  ITP_TRY(do_energies(h, nullptr, ITP_RITZ));
  if (steps_out) *steps_out = step;
  if (E_host) memcpy(E_host, cur.data(), h->m * sizeof(double));
  return ITP_OK;
}

int itp_test_expire_waits(itp_handle h, int launches) {
  if (!h) return ITP_ERR_ARG;
  if (launches < 0) return fail(h, ITP_ERR_ARG, "launch count must be >= 0");
  h->expire_waits = launches;
  return ITP_OK;
}

int itp_synchronize(itp_handle h) {
  if (!h) return ITP_ERR_ARG;
  ITP_CUDA(h, cudaSetDevice(h->device));
  return collect_status(h);
}

const char* itp_last_error(itp_handle h) { return h ? h->err.c_str() : g_create_error.c_str(); }

long long itp_kernel_launches(itp_handle h) { return h ? h->launches : 0; }

int itp_profile(itp_handle h, int enable) {
  if (!h) return ITP_ERR_ARG;
  ITP_CUDA(h, cudaSetDevice(h->device));
  ITP_CUDA(h, cudaStreamSynchronize(h->st));
  h->prof = enable != 0;
  h->prof_used = 0;
  return ITP_OK;
}

int itp_profile_read(itp_handle h, int kind, long long* launches, double* total_ms) {
  if (!h || kind < 0 || kind >= ITP_KERNEL_KINDS) return h ? fail(h, ITP_ERR_ARG, "bad kind")
                                                           : ITP_ERR_ARG;
  ITP_CUDA(h, cudaSetDevice(h->device));
  ITP_CUDA(h, cudaStreamSynchronize(h->st));
  long long n = 0;
  double ms = 0.0;
  for (size_t i = 0; i < h->prof_used; ++i) {
    const itp_grid::ProfEvent& e = h->prof_events[i];
    if (e.kind != kind) continue;
    float t = 0.f;
    ITP_CUDA(h, cudaEventElapsedTime(&t, e.start, e.stop));
    ms += t;
    ++n;
  }
  if (launches) *launches = n;
  if (total_ms) *total_ms = ms;
  return ITP_OK;
}

int itp_get_tuning(itp_handle h, int* tuning) {
  if (!h || !tuning) return h ? fail(h, ITP_ERR_ARG, "null tuning") : ITP_ERR_ARG;
  get_tuning(h, tuning);
  return ITP_OK;
}

int itp_set_tuning(itp_handle h, const int* tuning) {
  if (!h || !tuning) return h ? fail(h, ITP_ERR_ARG, "null tuning") : ITP_ERR_ARG;
  ITP_CUDA(h, cudaSetDevice(h->device));
  ITP_CUDA(h, cudaStreamSynchronize(h->st));
  int old[ITP_TUNING_LEN];
  get_tuning(h, old);
  const int rc = set_tuning(h, tuning);
  if (rc != ITP_OK) set_tuning(h, old);
  return rc;
}

int itp_autotune(itp_handle h, int order, double tau, int* tuning, char* report,
                 int report_len) {
  ITP_TRY(check_ready(h, true));
  if (order < 2 || order > 2 * kMaxTerms || (order & 1))
    return fail(h, ITP_ERR_ARG, "order must be even, 2..%d (got %d)", 2 * kMaxTerms, order);
  if (!(tau > 0) || !std::isfinite(tau)) return fail(h, ITP_ERR_ARG, "tau must be > 0");
  ITP_CUDA(h, cudaStreamSynchronize(h->st));
  const bool had_phi = h->have_phi;
  std::string rep;
  int rc;
  if (h->precision == ITP_MIXED) {
    ITP_TRY(switch_lane<float>(h));
    rc = autotune_lane<float>(h, order / 2, tau, rep);
  } else {
    rc = autotune_lane<double>(h, order / 2, tau, rep);
  }
  // the timed propagations overwrote the propagated block
  h->have_phi = false;
  (void)had_phi;
  if (rc != ITP_OK) return rc;
  ITP_CUDA(h, cudaStreamSynchronize(h->st));
  if (tuning) get_tuning(h, tuning);
  if (report && report_len > 0) {
    const size_t n = std::min(rep.size(), (size_t)report_len - 1);
    memcpy(report, rep.data(), n);
    report[n] = 0;
  }
  return ITP_OK;
}

int itp_propagate_romberg6(itp_handle h, double tau) {
  ITP_TRY(check_ready(h, true));
  if (!(tau > 0) || !std::isfinite(tau)) return fail(h, ITP_ERR_ARG, "tau must be > 0");
  if (h->precision == ITP_MIXED) {
    ITP_TRY(switch_lane<float>(h));
    ITP_TRY(propagate_romberg6_lane<float>(h, tau));
  } else {
    ITP_TRY(propagate_romberg6_lane<double>(h, tau));
  }
  h->have_phi = true;
  return ITP_OK;
}

int itp_solve_adaptive(itp_handle h, int order, double tau0, double reduce, double gamma,
                       int max_steps, int max_levels, int* levels_out, double* level_stats,
                       double* RH_host, double* E_host) {
  ITP_TRY(check_ready(h, true));
  if (order < 2 || order > 2 * kMaxTerms || (order & 1))
    return fail(h, ITP_ERR_ARG, "order must be even, 2..%d (got %d)", 2 * kMaxTerms, order);
  if (!(tau0 > 0) || !std::isfinite(tau0) || !(reduce > 0 && reduce < 1) || !(gamma > 0) ||
      max_steps < 1 || max_levels < 1)
    return fail(h, ITP_ERR_ARG, "bad adaptive-iteration arguments");
  if (levels_out) *levels_out = 0;
  bool converged = false;
  if (h->precision == ITP_MIXED) {
    ITP_TRY(switch_lane<float>(h));
    ITP_TRY(solve_adaptive_lane<float>(h, order / 2, tau0, reduce, gamma, max_steps,
                                       max_levels, levels_out, level_stats, RH_host, E_host,
                                       &converged));
  } else {
    ITP_TRY(solve_adaptive_lane<double>(h, order / 2, tau0, reduce, gamma, max_steps,
                                        max_levels, levels_out, level_stats, RH_host, E_host,
                                        &converged));
  }
  if (!converged)
    return fail(h, ITP_ERR_NOCONV, "R^H above gamma after %d levels", max_levels);
  return ITP_OK;
}

// ---- batches of independent problems --------------------------------------------

void itp_batch_destroy(itp_batch_handle b) {
  if (!b) return;
  cudaSetDevice(b->device);
  if (b->st) cudaStreamSynchronize(b->st);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (itp_handle h : b->probs) itp_destroy(h);
  if (b->fork) cudaEventDestroy(b->fork);
  for (cudaEvent_t e : b->join)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : b->evpool) cudaEventDestroy(e);
  cudaFree(b->tables);
  if (b->own_stream) cudaStreamDestroy(b->st);
  delete b;
}

int itp_create_batch(itp_batch_handle* out, int count, const int* dims, const double* boxes,
                     const int* n_states, const int* n_guard, int precision, void* cuda_stream) {
  if (!out) return ITP_ERR_ARG;
  *out = nullptr;
  g_batch_create_error.clear();
  if (count < 1 || !dims || !boxes || !n_states)
    return batch_fail(nullptr, ITP_ERR_ARG, "need count >= 1 and non-null dims, boxes, n_states");
  itp_batch_handle b = new (std::nothrow) itp_batch();
  if (!b) return ITP_ERR_OOM;
  auto bail = [&](int code, const std::string& msg) {
    itp_batch_destroy(b);
    return batch_fail(nullptr, code, msg);
  };
  if (cudaGetDevice(&b->device) != cudaSuccess) return bail(ITP_ERR_CUDA, "no CUDA device");
  b->st = (cudaStream_t)cuda_stream;
  if (!b->st) {
    if (cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking) != cudaSuccess)
      return bail(ITP_ERR_CUDA, "cannot create a stream");
    b->own_stream = true;
  }
  if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess)
    return bail(ITP_ERR_CUDA, "cannot create an event");
  b->probs.assign(count, nullptr);
  b->join.assign(count, nullptr);
  b->e_off.assign(count, 0);
  for (int p = 0; p < count; ++p) {
    itp_handle h = nullptr;
    const int rc = itp_create_grid(&h, dims[3 * p], dims[3 * p + 1], dims[3 * p + 2],
                                   boxes[3 * p], boxes[3 * p + 1], boxes[3 * p + 2], n_states[p],
                                   n_guard ? n_guard[p] : 0, precision, nullptr);
    if (rc != ITP_OK)
      return bail(rc, "problem " + std::to_string(p) + ": " + itp_last_error(nullptr));
    b->probs[p] = h;
    b->e_off[p] = b->m_total;
    b->m_total += h->m;
    if (cudaEventCreateWithFlags(&b->join[p], cudaEventDisableTiming) != cudaSuccess)
      return bail(ITP_ERR_CUDA, "cannot create an event");
  }
  *out = b;
  return ITP_OK;
}

itp_handle itp_batch_problem(itp_batch_handle b, int p) {
  if (!b || p < 0 || p >= (int)b->probs.size()) return nullptr;
  return b->probs[p];
}

int itp_batch_count(itp_batch_handle b) { return b ? (int)b->probs.size() : 0; }

int itp_batch_step(itp_batch_handle b, int order, double tau, int flags, double* E_host) {
  if (!b) return ITP_ERR_ARG;
  if (order < 2 || order > 2 * kMaxTerms || (order & 1))
    return batch_fail(b, ITP_ERR_ARG, "order must be even, 2.." + std::to_string(2 * kMaxTerms));
  if (!(tau > 0) || !std::isfinite(tau)) return batch_fail(b, ITP_ERR_ARG, "tau must be > 0");
  const int eflags = flags & ~ITP_STEP_FP64;
  if (eflags != 0 && eflags != ITP_RITZ_VALUES)
    return batch_fail(b, ITP_ERR_ARG, "flags: 0 or ITP_RITZ_VALUES, plus ITP_STEP_FP64");
  if (cudaSetDevice(b->device) != cudaSuccess) return batch_fail(b, ITP_ERR_CUDA, "device");
  const int k = order / 2;
  const int np = (int)b->probs.size();
  auto prob_fail = [&](int p, int rc) {
    return batch_fail(b, rc, "problem " + std::to_string(p) + ": " + b->probs[p]->err);
  };
  // per problem, outside any capture: lane, tables and workspaces
  for (int p = 0; p < np; ++p) {
    itp_handle h = b->probs[p];
    int rc = check_ready(h, true);
    if (rc == ITP_OK) {
      if (h->precision == ITP_MIXED && !(flags & ITP_STEP_FP64)) {
        rc = switch_lane<float>(h);
        if (rc == ITP_OK) rc = step_resources<float>(h, k, tau);
      } else {
        if (h->precision == ITP_MIXED) rc = switch_lane<double>(h);
        if (rc == ITP_OK) rc = step_resources<double>(h, k, tau);
      }
    }
    if (rc != ITP_OK) return prob_fail(p, rc);
    // the batch stream must not start the graph before this problem's own work
    if (cudaEventRecord(b->join[p], h->st) != cudaSuccess ||
        cudaStreamWaitEvent(b->st, b->join[p], 0) != cudaSuccess)
      return batch_fail(b, ITP_ERR_CUDA, "stream ordering");
  }
  bool stale = (int)b->versions.size() != np;
  for (int p = 0; p < np && !stale; ++p) stale = b->versions[p] != b->probs[p]->tune_version;
  if (!b->exec || stale || b->order != order || b->tau != tau || b->flags != flags) {
    if (b->exec) {
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
    if (cudaStreamSynchronize(b->st) != cudaSuccess)
      return batch_fail(b, ITP_ERR_CUDA, "synchronise before capture");
    if (b->grouped) {
      std::vector<long long> l0(np);
      for (int p = 0; p < np; ++p) {
        l0[p] = b->probs[p]->launches;
        b->probs[p]->capturing = true;
      }
      cudaGraph_t graph = nullptr;
      const int rcg = build_grouped_graph(b, k, tau, eflags, &graph);
      for (int p = 0; p < np; ++p) {
        b->probs[p]->capturing = false;
        b->probs[p]->launches = l0[p];
      }
      if (rcg != ITP_OK) return rcg;
      const long long nk = graph_kernels(graph);
      const cudaError_t ei = cudaGraphInstantiate(&b->exec, graph, 0);
      cudaGraphDestroy(graph);
      if (ei != cudaSuccess)
        return batch_fail(b, ITP_ERR_CUDA, std::string("instantiate: ") + cudaGetErrorString(ei));
      b->order = order;
      b->tau = tau;
      b->flags = flags;
      b->step_launches = nk;
      b->versions.resize(np);
      for (int p = 0; p < np; ++p) b->versions[p] = b->probs[p]->tune_version;
    }
  }
  if (!b->exec) {
    if (cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return batch_fail(b, ITP_ERR_CUDA, "begin capture");
    cudaEventRecord(b->fork, b->st);
    int rc = ITP_OK, bad = -1;
    long long n = 0;
    for (int p = 0; p < np && rc == ITP_OK; ++p) {
      itp_handle h = b->probs[p];
      // each problem's stream joins the capture as one branch of the graph
      if (cudaStreamWaitEvent(h->st, b->fork, 0) != cudaSuccess) {
        rc = batch_fail(b, ITP_ERR_CUDA, "fork");
        break;
      }
      h->capturing = true;
      const long long l0 = h->launches;
      rc = h->cur64 ? step_work<double>(h, k, tau, eflags) : step_work<float>(h, k, tau, eflags);
      h->capturing = false;
      n += h->launches - l0;
      h->launches = l0;
      if (rc != ITP_OK) {
        bad = p;
        break;
      }
      if (cudaEventRecord(b->join[p], h->st) != cudaSuccess ||
          cudaStreamWaitEvent(b->st, b->join[p], 0) != cudaSuccess)
        rc = batch_fail(b, ITP_ERR_CUDA, "join");
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(b->st, &graph);
    if (rc != ITP_OK) {
      if (graph) cudaGraphDestroy(graph);
      return bad >= 0 ? prob_fail(bad, rc) : rc;
    }
    if (ec != cudaSuccess)
      return batch_fail(b, ITP_ERR_CUDA, std::string("end capture: ") + cudaGetErrorString(ec));
    const cudaError_t ei = cudaGraphInstantiate(&b->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess)
      return batch_fail(b, ITP_ERR_CUDA, std::string("instantiate: ") + cudaGetErrorString(ei));
    b->order = order;
    b->tau = tau;
    b->flags = flags;
    b->step_launches = n;
    b->versions.resize(np);
    for (int p = 0; p < np; ++p) b->versions[p] = b->probs[p]->tune_version;
  }
  if (cudaGraphLaunch(b->exec, b->st) != cudaSuccess)
    return batch_fail(b, ITP_ERR_CUDA, "graph launch");
  b->launches += b->step_launches;
  if (cudaStreamSynchronize(b->st) != cudaSuccess)
    return batch_fail(b, ITP_ERR_CUDA, "graph execution failed");
  int first = ITP_OK;
  for (int p = 0; p < np; ++p) {
    itp_handle h = b->probs[p];
    h->have_phi = false;
    const int stw = *h->status_host;
    if (stw) {
      cudaMemsetAsync(h->status, 0, sizeof(int), h->st);
      int rc = ITP_OK;
      if (stw & 4) rc = fail(h, ITP_ERR_TIMEOUT, "a bounded tensor-core wait expired");
      else if (stw & 1) rc = fail(h, ITP_ERR_NOT_PD, "overlap matrix is not positive definite");
      else if (stw & 2) rc = fail(h, ITP_ERR_NOCONV, "eigensolver did not converge");
      if (rc != ITP_OK && first == ITP_OK) first = prob_fail(p, rc);
    }
    if (E_host) memcpy(E_host + b->e_off[p], h->E_host_pinned, h->m * sizeof(double));
  }
  return first;
}

long long itp_batch_kernel_launches(itp_batch_handle b) { return b ? b->launches : 0; }

int itp_batch_set_grouping(itp_batch_handle b, int grouped) {
  if (!b) return ITP_ERR_ARG;
  if ((grouped != 0) != b->grouped) {
    b->grouped = grouped != 0;
    if (b->exec) {   // the next step captures the graph in the new form
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
  }
  return ITP_OK;
}

int itp_batch_groups(itp_batch_handle b) { return b && b->exec && b->grouped ? b->n_groups : 0; }

const char* itp_batch_last_error(itp_batch_handle b) {
  return b ? b->err.c_str() : g_batch_create_error.c_str();
}

}  // extern "C"
