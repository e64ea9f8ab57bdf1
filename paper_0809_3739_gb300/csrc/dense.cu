// Dense n x n side of one iteration (Eq. 4 and the subspace step of
// Sec. III): Gram sums over the grid, Cholesky + triangular inverse, the
// symmetric eigen-decomposition, and the application of an n x n matrix to
// the block of states.  These are the CUDA-core versions; all small-matrix
// work is FP64.
#include <cooperative_groups.h>
#include <math.h>

#include "itp_kernels.cuh"

namespace cg = cooperative_groups;

namespace itp {

namespace {

constexpr int kMaxM = 256;   // states of the n x n work at most
constexpr int kBlk = 128;    // rows of one state block of the Gram and apply kernels

// ---------------------------------------------------------------------------
// Gram partial sums over chunks of points.  The m x m result is cut into
// 128 x 128 blocks; CTA (chunk c, block b) sums rows [128 bi, +128) of A
// against rows [128 bj, +128) of B, (bi, bj) = block b of the list that
// launch_gram_partial builds (with A == B only bj <= bi, each off-diagonal
// block also written transposed).  512 threads as 16 (tx) x 32 (ty); thread
// owns block rows i = ty + 32*q (q < 4) and cols j = tx + 16*r (r < 8).
// points per shared tile: 32 (FP32) or 16 (FP64), 33 KB of shared tiles;
// FP32 products are summed over runs of 256 points, then in FP64.
template <typename TC> struct GramTile { static constexpr int KT = sizeof(TC) == 4 ? 32 : 16; };
constexpr int kGramRun = 256;

// Block b of the Gram kernels' block list: (bi, bj) packed as bi * 256 + bj.
struct GramBlocks {
  int n;
  int ij[(kMaxM / kBlk) * (kMaxM / kBlk)];
};

template <typename TA, typename TB, typename TC>
__global__ void __launch_bounds__(512) gram_partial_kernel(const TA* __restrict__ A,
                                                           const TB* __restrict__ B, int m,
                                                           long long N, long long chunk,
                                                           double* __restrict__ partial,
                                                           const GramBlocks blocks, int mirror) {
  constexpr int KT = GramTile<TC>::KT;
  constexpr int kFlushTiles = kGramRun / KT;
  __shared__ TC sA[KT][kBlk + 1];
  __shared__ TC sB[KT][kBlk + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int bi = blocks.ij[blockIdx.y] >> 8, bj = blocks.ij[blockIdx.y] & 255;
  const int ia = kBlk * bi, jb = kBlk * bj;   // first row of A and of B
  const long long p_begin = (long long)blockIdx.x * chunk;
  const long long p_end = min(N, p_begin + chunk);
  double accd[4][8];
  TC accf[4][8];
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int r = 0; r < 8; ++r) { accd[q][r] = 0.0; accf[q][r] = (TC)0; }
  int tiles_in_run = 0;
  for (long long p0 = p_begin; p0 < p_end; p0 += KT) {
    // load tiles: element (row i, point p0 + k)
    for (int e = threadIdx.x; e < KT * kBlk; e += blockDim.x) {
      const int i = e / KT, k = e - i * KT;
      const long long p = p0 + k;
      TC va = (TC)0, vb = (TC)0;
      if (p < p_end) {
        if (ia + i < m) va = (TC)A[(long long)(ia + i) * N + p];
        if (jb + i < m) vb = (TC)B[(long long)(jb + i) * N + p];
      }
      sA[k][i] = va;
      sB[k][i] = vb;
    }
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < KT; ++k) {
      TC a[4], b[8];
#pragma unroll
      for (int q = 0; q < 4; ++q) a[q] = sA[k][ty + 32 * q];
#pragma unroll
      for (int r = 0; r < 8; ++r) b[r] = sB[k][tx + 16 * r];
      if constexpr (sizeof(TC) == 8) {
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int r = 0; r < 8; ++r) accd[q][r] = fma((double)a[q], (double)b[r], accd[q][r]);
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int r = 0; r < 8; ++r) accf[q][r] = fma(a[q], b[r], accf[q][r]);
      }
    }
    __syncthreads();
    if (sizeof(TC) == 4 && ++tiles_in_run == kFlushTiles) {
      tiles_in_run = 0;
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int r = 0; r < 8; ++r) { accd[q][r] += (double)accf[q][r]; accf[q][r] = (TC)0; }
    }
  }
  double* out = partial + (long long)blockIdx.x * m * m;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = ia + ty + 32 * q;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int j = jb + tx + 16 * r;
      if (i < m && j < m) {
        const double v = accd[q][r] + (double)accf[q][r];
        out[i * m + j] = v;
        if (mirror && bi != bj) out[j * m + i] = v;
      }
    }
  }
}

__global__ void gram_reduce_kernel(const double* __restrict__ partial, int n_chunks, int m,
                                   double scale, int sym, double* __restrict__ G) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m * m) return;
  const int i = e / m, j = e - i * m;
  double s = 0.0, t = 0.0;
  for (int c = 0; c < n_chunks; ++c) {
    s += partial[(long long)c * m * m + i * m + j];
    if (sym) t += partial[(long long)c * m * m + j * m + i];
  }
  G[e] = sym ? 0.5 * scale * (s + t) : scale * s;
}

// ---------------------------------------------------------------------------
// Cholesky S = L L^T and M = L^{-1} (right-looking, column by column) on a
// cluster of kClus CTAs, for the FP64 rate: an SM retires about two FP64 FMAs per clock, so the O(m^3) work is spread
// over the cluster's SMs.  CTA r owns rows [r*rp, r*rp + rp) of S (lower
// part) and of R = I - sum_j L[:, j] M[j, :], in its shared memory; other
// CTAs read them through distributed shared memory.  Step k (one cluster
// barrier): every CTA reads the pivot S[k][k], column k of the updated S
// (giving column k of L) and row k of R (giving row k of M = L^{-1}), then
// updates its own rows i > k:
//   S[i][j] -= L[i][k] L[j][k]  (k < j <= i),   R[i][j] -= L[i][k] M[k][j]  (j <= k).
// Nothing a step reads remotely (column k of S, row k of R) is written in
// that step, so one barrier per step orders everything.
constexpr int kClus = 8;                      // CTAs per cluster (portable size)
constexpr int kClusThreads = 256;

// Shared memory of the cluster kernels: rp = ceil(m / kClus) rows of pitch
// m + 1 (odd: conflict-free column reads), `mats` such matrices, plus
// `vecs` vectors of m doubles.
__host__ __device__ constexpr size_t clus_smem(int m, int mats, int vecs) {
  return ((size_t)mats * ((m + kClus - 1) / kClus) * (m + 1) + (size_t)vecs * m) *
         sizeof(double);
}

__global__ void __cluster_dims__(kClus, 1, 1) __launch_bounds__(kClusThreads)
    cholesky_inverse_cluster_kernel(const double* __restrict__ S, int m,
                                    double* __restrict__ Minv, int* status) {
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ double csh[];
  __shared__ double s_piv;
  __shared__ int s_bad;
  const int rank = (int)cl.block_rank();
  const int rp = (m + kClus - 1) / kClus;
  const int pitch = m + 1;
  double* A_ = csh;                       // [rp][pitch] own rows of S (lower part)
  double* Rr_ = A_ + (size_t)rp * pitch;  // [rp][pitch] own rows of R
  double* lf = Rr_ + (size_t)rp * pitch;  // [m]
  double* mk = lf + m;                    // [m]
  auto A = [&](int il, int j) -> double& { return A_[il * pitch + j]; };
  auto Rr = [&](int il, int j) -> double& { return Rr_[il * pitch + j]; };
  const int r0 = rank * rp, r1 = max(r0, min(m, r0 + rp));
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NW = kClusThreads / 32;
  if (tid == 0) s_bad = 0;
  for (int q = tid; q < (r1 - r0) * m; q += kClusThreads) {
    const int il = q / m, j = q - il * m;
    A(il, j) = S[(long long)(r0 + il) * m + j];
    Rr(il, j) = (r0 + il == j) ? 1.0 : 0.0;
  }
  cl.sync();
  for (int k = 0; k < m; ++k) {
    const int ok = k / rp;
    if (tid == 0) {
      const double akk = *cl.map_shared_rank(&A(k - ok * rp, k), ok);
      double piv = 1.0;
      if (!(akk > 0.0) || !isfinite(akk)) s_bad = 1;
      else piv = sqrt(akk);
      s_piv = piv;
    }
    __syncthreads();
    const double rpiv = 1.0 / s_piv;
    for (int j = k + 1 + tid; j < m; j += kClusThreads) {
      const int o = j / rp;
      lf[j] = *cl.map_shared_rank(&A(j - o * rp, k), o) * rpiv;
    }
    for (int j = tid; j <= k; j += kClusThreads)
      mk[j] = *cl.map_shared_rank(&Rr(k - ok * rp, j), ok) * rpiv;
    __syncthreads();
    if (rank == ok)
      for (int j = tid; j < m; j += kClusThreads) Minv[(long long)k * m + j] = j <= k ? mk[j] : 0.0;
    // own rows i > k: one warp per row, lanes over columns
    for (int i = max(r0, k + 1) + warp; i < r1; i += NW) {
      const int il = i - r0;
      const double li = lf[i];
      for (int j = lane; j <= i; j += 32) {
        if (j <= k) Rr(il, j) -= li * mk[j];
        else A(il, j) -= li * lf[j];
      }
    }
    cl.sync();
  }
  if (tid == 0 && s_bad) atomicOr(status, 1);
}

// Householder tridiagonalisation (eigenvalues only) on a cluster: CTA r
// owns full rows [r*rp, r*rp + rp) of the symmetric matrix.  Step k takes
// two cluster barriers: after the partial sums of squares of column k
// (giving the reflector, which every CTA forms alike from the same values in
// the same order), and after the partial products p = beta A v and v^T p;
// then each CTA applies A -= v w^T + w v^T to its own rows.
__global__ void __cluster_dims__(kClus, 1, 1) __launch_bounds__(kClusThreads)
    tridiag_cluster_kernel(const double* __restrict__ H, int m, double* __restrict__ d,
                           double* __restrict__ e) {
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ double csh[];
  __shared__ double s_sig[2], s_dot[2];  // partial sums (read by the others)
  __shared__ double s_beta, s_K;
  const int rank = (int)cl.block_rank();
  const int rp = (m + kClus - 1) / kClus;
  const int pitch = m + 1;
  double* A_ = csh;                       // [rp][pitch] own rows
  double* vf = A_ + (size_t)rp * pitch;   // [m]
  double* wf = vf + m;                    // [m]
  double* pl = wf + m;                    // [m] (rp used): own entries of p (read by the others)
  auto A = [&](int il, int j) -> double& { return A_[il * pitch + j]; };
  const int r0 = rank * rp, r1 = max(r0, min(m, r0 + rp));
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NW = kClusThreads / 32;
  for (int q = tid; q < (r1 - r0) * m; q += kClusThreads) {
    const int il = q / m, j = q - il * m, i = r0 + il;
    A(il, j) = 0.5 * (H[(long long)i * m + j] + H[(long long)j * m + i]);
  }
  __syncthreads();
  for (int k = 0; k + 2 < m; ++k) {
    const int n0 = k + 1, b = k & 1;
    if (warp == 0) {
      double sig = 0.0;
      for (int i = max(r0, n0 + 1) + lane; i < r1; i += 32) sig += A(i - r0, k) * A(i - r0, k);
      for (int o = 16; o; o >>= 1) sig += __shfl_xor_sync(0xffffffffu, sig, o);
      if (lane == 0) s_sig[b] = sig;
    }
    if (tid == 0 && k >= r0 && k < r1) d[k] = A(k - r0, k);
    cl.sync();
    if (tid == 0) {
      double sig = 0.0;
      for (int r = 0; r < kClus; ++r) sig += *cl.map_shared_rank(&s_sig[b], r);
      const int o = n0 / rp;
      const double x0 = *cl.map_shared_rank(&A(n0 - o * rp, k), o);
      double alpha = x0, beta = 0.0, v0 = 0.0;
      if (sig != 0.0) {
        const double nrm = sqrt(x0 * x0 + sig);
        alpha = x0 > 0 ? -nrm : nrm;
        v0 = x0 - alpha;
        beta = 2.0 / (v0 * v0 + sig);
      }
      s_beta = beta;
      vf[n0] = v0;
      if (rank == 0) e[k] = alpha;
    }
    for (int j = n0 + 1 + tid; j < m; j += kClusThreads) {
      const int o = j / rp;
      vf[j] = *cl.map_shared_rank(&A(j - o * rp, k), o);
    }
    __syncthreads();
    const double beta = s_beta;
    for (int i = max(r0, n0) + warp; i < r1; i += NW) {
      double acc = 0.0;
      for (int j = n0 + lane; j < m; j += 32) acc += A(i - r0, j) * vf[j];
      for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) pl[i - r0] = beta * acc;
    }
    __syncthreads();
    if (warp == 0) {
      double acc = 0.0;
      for (int i = max(r0, n0) + lane; i < r1; i += 32) acc += vf[i] * pl[i - r0];
      for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) s_dot[b] = acc;
    }
    cl.sync();
    if (tid == 0) {
      double dot = 0.0;
      for (int r = 0; r < kClus; ++r) dot += *cl.map_shared_rank(&s_dot[b], r);
      s_K = 0.5 * beta * dot;
    }
    __syncthreads();
    const double K = s_K;
    for (int j = n0 + tid; j < m; j += kClusThreads) {
      const int o = j / rp;
      wf[j] = *cl.map_shared_rank(&pl[j - o * rp], o) - K * vf[j];
    }
    __syncthreads();
    for (int i = max(r0, n0) + warp; i < r1; i += NW) {
      const int il = i - r0;
      const double vi = vf[i], wi = wf[i];
      for (int j = n0 + lane; j < m; j += 32) A(il, j) -= vi * wf[j] + wi * vf[j];
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (m >= 2 && m - 2 >= r0 && m - 2 < r1) d[m - 2] = A(m - 2 - r0, m - 2);
    if (m >= 2 && m - 1 >= r0 && m - 1 < r1) e[m - 2] = A(m - 1 - r0, m - 2);
    if (m - 1 >= r0 && m - 1 < r1) d[m - 1] = A(m - 1 - r0, m - 1);
  }
  cl.sync();   // no CTA leaves while another may still read its shared memory
}

// ---------------------------------------------------------------------------
// Parallel cyclic Jacobi (round-robin pairing: m/2 disjoint rotations per
// round, m-1 rounds per sweep).  A in shared memory (pitch m+1), U^T in
// global memory (row p of U^T is eigenvector p).
__global__ void __launch_bounds__(1024) jacobi_kernel(const double* __restrict__ H, int m,
                                                      double* __restrict__ E,
                                                      double* __restrict__ Rt,
                                                      double* __restrict__ Ut,
                                                      double* __restrict__ Aglob, int* status) {
  extern __shared__ double sh[];
  const int mm = (m + 1) & ~1;          // even number of players (a dummy if m is odd)
  const int P = m + 1;
  // m x P working matrix: in shared memory, or (Aglob set: too large for
  // one CTA) in global memory, where it stays in L2
  double* A = Aglob ? Aglob : sh;
  double* cs = Aglob ? sh : sh + m * P;  // [mm/2] c, [mm/2] s
  int* pr = reinterpret_cast<int*>(cs + mm);   // [mm/2] p, [mm/2] q
  __shared__ double off_norm, tot_norm;
  __shared__ int done;
  const int tid = threadIdx.x, nthr = blockDim.x;
  for (int e = tid; e < m * m; e += nthr) {
    const int i = e / m, j = e - i * m;
    A[i * P + j] = 0.5 * (H[i * m + j] + H[j * m + i]);
    Ut[e] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  const int npairs = mm / 2;
  int sweep;
  for (sweep = 0; sweep < 40; ++sweep) {
    if (tid == 0) { off_norm = 0.0; tot_norm = 0.0; }
    __syncthreads();
    double lo = 0.0, lt = 0.0;
    for (int e = tid; e < m * m; e += nthr) {
      const int i = e / m, j = e - i * m;
      const double v = A[i * P + j] * A[i * P + j];
      lt += v;
      if (i != j) lo += v;
    }
    atomicAdd(&off_norm, lo);
    atomicAdd(&tot_norm, lt);
    __syncthreads();
    // off-diagonal Frobenius norm <= 1e-13 of the total: eigenvalue errors
    // are then second order in it (~1e-26 |H|^2 / gap)
    if (tid == 0) done = (off_norm <= 1e-26 * tot_norm) || (off_norm == 0.0);
    __syncthreads();
    if (done) break;
    for (int round = 0; round < mm - 1; ++round) {
      for (int t = tid; t < npairs; t += nthr) {
        // players 0..mm-1; player 0 fixed, the others rotate
        const int a = (t == 0) ? 0 : 1 + (t - 1 + round) % (mm - 1);
        const int b = 1 + (mm - 2 - t + round) % (mm - 1);
        int p = min(a, b), q = max(a, b);
        double c = 1.0, s = 0.0;
        if (q < m) {
          const double apq = A[p * P + q];
          if (apq != 0.0) {
            const double app = A[p * P + p], aqq = A[q * P + q];
            const double zeta = (aqq - app) / (2.0 * apq);
            const double tt = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
            c = 1.0 / sqrt(1.0 + tt * tt);
            s = tt * c;
          }
        } else {
          p = q = -1;
        }
        cs[t] = c;
        cs[npairs + t] = s;
        pr[t] = p;
        pr[npairs + t] = q;
      }
      __syncthreads();
      // columns: A <- A J
      for (int e = tid; e < npairs * m; e += nthr) {
        const int t = e / m, r = e - t * m;
        const int p = pr[t], q = pr[npairs + t];
        if (p < 0) continue;
        const double c = cs[t], s = cs[npairs + t];
        const double arp = A[r * P + p], arq = A[r * P + q];
        A[r * P + p] = c * arp - s * arq;
        A[r * P + q] = s * arp + c * arq;
      }
      __syncthreads();
      // rows: A <- J^T A ; and U^T <- J^T U^T (rows p, q)
      for (int e = tid; e < npairs * m; e += nthr) {
        const int t = e / m, r = e - t * m;
        const int p = pr[t], q = pr[npairs + t];
        if (p < 0) continue;
        const double c = cs[t], s = cs[npairs + t];
        const double apr = A[p * P + r], aqr = A[q * P + r];
        A[p * P + r] = c * apr - s * aqr;
        A[q * P + r] = s * apr + c * aqr;
        const double up = Ut[p * m + r], uq = Ut[q * m + r];
        Ut[p * m + r] = c * up - s * uq;
        Ut[q * m + r] = s * up + c * uq;
      }
      __syncthreads();
    }
  }
  if (tid == 0 && sweep >= 40) atomicOr(status, 2);
  __syncthreads();
  // sort eigenvalues ascending (stable by index) and permute the rows of U^T
  for (int i = tid; i < m; i += nthr) {
    const double ei = A[i * P + i];
    int rank = 0;
    for (int j = 0; j < m; ++j) {
      const double ej = A[j * P + j];
      rank += (ej < ei) || (ej == ei && j < i);
    }
    E[rank] = ei;
    for (int r = 0; r < m; ++r) Rt[rank * m + r] = Ut[i * m + r];
  }
}

// ---------------------------------------------------------------------------
// Eigenvalues only: the cluster tridiagonalisation above, then bisection on
// Sturm counts, one CTA of four warps per eigenvalue (128-point
// multisection: seven bits per round, one warp on each of the SM's four
// sub-partitions, whose FP64 units the counts keep busy).
constexpr int kBisWarps = 4;
constexpr int kBisPts = 32 * kBisWarps;   // points per round; the last is hi

// Biased binary exponent of a double (0 for zero and subnormals).
__device__ __forceinline__ int dexp(double v) { return (__double2hiint(v) >> 20) & 0x7ff; }
// v * 2^k by its exponent field (v normal, the result normal).
__device__ __forceinline__ double dscale(double v, int k) {
  return __hiloint2double(__double2hiint(v) + (k << 20), __double2loint(v));
}

// Number of eigenvalues below x of the symmetric tridiagonal with diagonal
// d and squared off-diagonal e2 (e2[i] couples rows i and i+1), scaled so
// that |d_i|, |x| < 1 and e2_i <= 4.  The sign changes of the leading
// principal minors of T - x I,
//   p_0 = 1,  p_1 = d_0 - x,  p_{i+1} = (d_i - x) p_i - e2_{i-1} p_{i-1},
// i.e. the negative pivots p_{i+1}/p_i of its LDL^T factorisation.  No
// division: three FP64 operations per row, the rest on the integer pipe.
//  - A minor that vanishes against the previous one (|p_{i+1}| < 2^-599
//    |p_i|, zero included) becomes -2^-600 p_i: the pivot -2^-600, as a
//    zero pivot of the LDL^T recurrence is replaced by a tiny negative one.
//  - p_i and p_{i-1} are rescaled together by a power of two (exponent
//    arithmetic, exact) whenever |p_i| leaves [2^-256, 2^257).
// With the pivot rule |p_{i-1}| <= 2^600 |p_i|, so |p_{i+1}| < 2^603 |p_i|
// and every value stays a normal double between 2^-860 and 2^860.
__device__ __forceinline__ int sturm_count(const double* __restrict__ d,
                                           const double* __restrict__ e2, int m, double x) {
  double pm = 1.0, p = d[0] - x;
  int ep = dexp(p);
  if (ep < 1023 - 599) {
    p = -0x1p-600;
    ep = 1023 - 600;
  }
  int cnt = __double2hiint(p) < 0;
  if (ep < 1023 - 256) {
    p = dscale(p, 1023 - ep);
    pm = dscale(pm, 1023 - ep);
    ep = 1023;
  }
  for (int i = 1; i < m; ++i) {
    double pn = fma(d[i] - x, p, -(e2[i - 1] * pm));
    int en = dexp(pn);
    if (en < ep - 599) {
      pn = __hiloint2double((__double2hiint(p) ^ (int)0x80000000) - (600 << 20),
                            __double2loint(p));
      en = ep - 600;
    }
    cnt += (__double2hiint(pn) ^ __double2hiint(p)) < 0;
    pm = p;
    p = pn;
    ep = en;
    if ((unsigned)(en - (1023 - 256)) > 512u) {
      p = dscale(p, 1023 - en);
      pm = dscale(pm, 1023 - en);
      ep = 1023;
    }
  }
  return cnt;
}

// One CTA per eigenvalue index j (ascending): the Gershgorin interval of
// the tridiagonal, scaled by a power of two into (-1, 1), narrowed by
// 128-point multisection down to a few ulps.
__global__ void __launch_bounds__(kBisPts) bisect_kernel(const double* __restrict__ dg,
                                                          const double* __restrict__ eg, int m,
                                                          double* __restrict__ E) {
  __shared__ double sd[kMaxM], se2[kMaxM];
  __shared__ double s_lo, s_hi, s_scale;
  __shared__ unsigned s_ball[2][kBisWarps];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (warp == 0) {
    double lo = dg[0], hi = dg[0];
    for (int i = lane; i < m; i += 32) {
      const double r = (i > 0 ? fabs(eg[i - 1]) : 0.0) + (i + 1 < m ? fabs(eg[i]) : 0.0);
      lo = fmin(lo, dg[i] - r);
      hi = fmax(hi, dg[i] + r);
    }
    for (int o = 16; o; o >>= 1) {
      lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if (lane == 0) {
      const double span = fmax(hi - lo, 1e-300);
      lo -= 1e-14 * span + 1e-300;
      hi += 1e-14 * span + 1e-300;
      int k;
      frexp(fmax(fabs(lo), fabs(hi)), &k);   // max |.| = f 2^k, f in [1/2, 1)
      const double g = ldexp(1.0, -k);
      s_scale = g;
      s_lo = lo * g;
      s_hi = hi * g;
    }
  }
  __syncthreads();
  const double g = s_scale;
  for (int i = tid; i < m; i += blockDim.x) {
    sd[i] = dg[i] * g;
    const double ei = i + 1 < m ? eg[i] * g : 0.0;
    se2[i] = ei * ei;
  }
  __syncthreads();
  const int j = blockIdx.x;
  double lo = s_lo, hi = s_hi;
  for (int it = 0; it < 16; ++it) {
    const double width = hi - lo;
    if (width <= 4.0 * 2.220446049250313e-16 * fmax(fabs(lo), fabs(hi)) + 0x1p-70) break;
    // points lo + width (t+1)/128, t < 127; point 127 is hi (count m + 1)
    const double x = lo + width * (double)(tid + 1) / (double)kBisPts;
    const int c = tid < kBisPts - 1 ? sturm_count(sd, se2, m, x) : m + 1;
    const unsigned ball = __ballot_sync(0xffffffffu, c > j);
    if (lane == 0) s_ball[it & 1][warp] = ball;
    __syncthreads();
    // the eigenvalue j lies in the first part whose right end has count > j
    int first = kBisPts - 1;
    for (int w = kBisWarps - 1; w >= 0; --w) {
      const unsigned b = s_ball[it & 1][w];
      if (b) first = 32 * w + __ffs(b) - 1;
    }
    const double nlo = first == 0 ? lo : lo + width * (double)first / (double)kBisPts;
    const double nhi =
        first == kBisPts - 1 ? hi : lo + width * (double)(first + 1) / (double)kBisPts;
    lo = nlo;
    hi = nhi;
  }
  if (tid == 0) E[j] = 0.5 * (lo + hi) / g;
}

__global__ void diag_kernel(const double* __restrict__ H, int m, double* __restrict__ E) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) E[i] = H[i * m + i];
}

// ---------------------------------------------------------------------------
// Residual norms of the adaptive iteration (Sec. III):
//   out_j = dV * sum_p (A[j][p] - c_j B[j][p])^2,
// c_j = exp(scale E_j) (mode 1: R^E with A = T psi, B = psi, scale = -tau) or
// c_j = E_j (mode 0: R^H with A = H psi, B = psi).  Chunks of points per
// CTA, the per-thread sums in the precision of the data, the rest in FP64,
// partial sums combined in a fixed order.
template <typename T> struct Vec4Of;
template <> struct Vec4Of<float> { using type = float4; static constexpr int W = 4; };
template <> struct Vec4Of<double> { using type = double2; static constexpr int W = 2; };

__device__ __forceinline__ float sqdiff_sum(const float4 a, const float4 b, float c) {
  const float d0 = a.x - c * b.x, d1 = a.y - c * b.y, d2 = a.z - c * b.z, d3 = a.w - c * b.w;
  return d0 * d0 + d1 * d1 + d2 * d2 + d3 * d3;
}
__device__ __forceinline__ double sqdiff_sum(const double2 a, const double2 b, double c) {
  const double d0 = a.x - c * b.x, d1 = a.y - c * b.y;
  return d0 * d0 + d1 * d1;
}

template <typename T>
__global__ void __launch_bounds__(256) residual_partial_kernel(
    const T* __restrict__ A, const T* __restrict__ B, const double* __restrict__ E,
    double scale, int mode, long long N, int chunks, double* __restrict__ partial) {
  using V = typename Vec4Of<T>::type;
  constexpr int W = Vec4Of<T>::W;
  const int j = blockIdx.y, c = blockIdx.x;
  const T cj = (T)(mode ? exp(scale * E[j]) : E[j]);
  const long long nv = N / W;
  const long long per = (nv + chunks - 1) / chunks;
  const long long v0 = (long long)c * per, v1 = min(nv, v0 + per);
  const V* a = reinterpret_cast<const V*>(A + (long long)j * N);
  const V* b = reinterpret_cast<const V*>(B + (long long)j * N);
  T acc = 0;
  for (long long v = v0 + threadIdx.x; v < v1; v += blockDim.x) acc += sqdiff_sum(a[v], b[v], cj);
  double s = (double)acc;
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ double ws[8];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
    partial[(long long)j * chunks + c] = t;
  }
}

__global__ void residual_final_kernel(const double* __restrict__ partial, int chunks, int m,
                                      double dV, double* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m) return;
  double t = 0.0;
  for (int c = 0; c < chunks; ++c) t += partial[(long long)j * chunks + c];
  out[j] = t * dV;
}

// ---------------------------------------------------------------------------
// Y[r0 + i] (=|+=) sum_k M[r0 + i][k0 + k] X[k0 + k] for i < nr, k < nk: one
// block of Y = M X (the host walks the blocks of 128 rows).  Persistent CTAs
// over tiles of 32 points; the M block (as TC) stays in shared memory.  512
// threads: tx = point in tile, ty = row group (16 rows).  lower: M[i][k] = 0
// for k > i (global indices).  add: the block's product is added to Y.
constexpr int kApplyPT = 32;

template <typename TX, typename TY, typename TC>
__global__ void __launch_bounds__(512) apply_matrix_kernel(const double* __restrict__ M, int m,
                                                           int lower, const TX* __restrict__ X,
                                                           TY* __restrict__ Y, long long N,
                                                           int r0, int nr, int k0, int nk,
                                                           int add) {
  extern __shared__ __align__(16) unsigned char smraw[];
  TC* sM = reinterpret_cast<TC*>(smraw);            // nr x nk
  TC* sX = sM + nr * nk;                            // nk x kApplyPT
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // ty in 0..15
  for (int e = threadIdx.x; e < nr * nk; e += blockDim.x) {
    const int i = e / nk, k = e - i * nk;
    sM[e] = (TC)M[(long long)(r0 + i) * m + k0 + k];
  }
  const long long ntiles = (N + kApplyPT - 1) / kApplyPT;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long p0 = tile * kApplyPT;
    __syncthreads();
    for (int e = threadIdx.x; e < nk * kApplyPT; e += blockDim.x) {
      const int k = e / kApplyPT, j = e - k * kApplyPT;
      const long long p = p0 + j;
      sX[e] = (p < N) ? (TC)X[(long long)(k0 + k) * N + p] : (TC)0;
    }
    __syncthreads();
    const long long p = p0 + tx;
    for (int i0 = ty; i0 < nr; i0 += 16 * 8) {
      TC acc[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) acc[q] = (TC)0;
      // lower triangular: row r0 + i needs k0 + k <= r0 + i
      const int kmax = lower ? max(0, min(nk, r0 + i0 + 16 * 7 + 1 - k0)) : nk;
      for (int k = 0; k < kmax; ++k) {
        const TC x = sX[k * kApplyPT + tx];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int i = i0 + 16 * q;
          if (i < nr) acc[q] = fma(sM[i * nk + k], x, acc[q]);
        }
      }
      if (p < N) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int i = i0 + 16 * q;
          if (i < nr) {
            TY* y = Y + (long long)(r0 + i) * N + p;
            *y = add ? (TY)((TC)*y + acc[q]) : (TY)acc[q];
          }
        }
      }
    }
  }
}

template <typename TS, typename TD>
__global__ void convert_kernel(const TS* __restrict__ src, TD* __restrict__ dst, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    dst[i] = (TD)src[i];
}

template <typename T> struct ComputeOf;
template <> struct ComputeOf<float> { using type = float; };
template <> struct ComputeOf<double> { using type = double; };

}  // namespace

template <typename TA, typename TB, typename TC>
cudaError_t launch_gram_partial(const TA* A, const TB* B, int m, long long n_points, int n_chunks,
                                double* partial, cudaStream_t st) {
  if (m < 1 || m > kMaxM) return cudaErrorInvalidValue;
  long long chunk = (n_points + n_chunks - 1) / n_chunks;
  chunk = (chunk + kGramRun - 1) / kGramRun * kGramRun;
  // 128 x 128 blocks of the result; A A^T: the lower blocks, mirrored
  const bool same = (const void*)A == (const void*)B;
  const int nb = (m + kBlk - 1) / kBlk;
  GramBlocks blocks{};
  for (int bi = 0; bi < nb; ++bi)
    for (int bj = 0; bj < nb; ++bj)
      if (!same || bj <= bi) blocks.ij[blocks.n++] = bi * 256 + bj;
  gram_partial_kernel<TA, TB, TC><<<dim3(n_chunks, blocks.n), 512, 0, st>>>(
      A, B, m, n_points, chunk, partial, blocks, same ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_gram_reduce(const double* partial, int n_chunks, int m, double scale, int sym,
                               double* G, cudaStream_t st) {
  gram_reduce_kernel<<<(m * m + 255) / 256, 256, 0, st>>>(partial, n_chunks, m, scale, sym, G);
  return cudaGetLastError();
}

cudaError_t launch_cholesky_inverse(const double* S, int m, double* Minv, int* status,
                                    cudaStream_t st) {
  if (m < 1 || m > kMaxM) return cudaErrorInvalidValue;
  const size_t smem = clus_smem(m, 2, 2);
  cudaError_t e = cudaFuncSetAttribute(cholesky_inverse_cluster_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cholesky_inverse_cluster_kernel<<<kClus, kClusThreads, smem, st>>>(S, m, Minv, status);
  return cudaGetLastError();
}

cudaError_t launch_jacobi_eigh(const double* H, int m, double* E, double* Rt, double* work,
                               int* status, cudaStream_t st) {
  if (m < 1 || m > kMaxM) return cudaErrorInvalidValue;
  const int mm = (m + 1) & ~1;
  const size_t amat = (size_t)m * (m + 1) * sizeof(double);
  const size_t rest = (size_t)mm * sizeof(double) + (size_t)mm * sizeof(int);
  // the working matrix goes to global memory (after U^T in work) when it
  // does not fit one CTA's shared memory
  const bool global_a = amat + rest > 227 * 1024;
  const size_t smem = global_a ? rest : amat + rest;
  cudaError_t e = cudaFuncSetAttribute(jacobi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  jacobi_kernel<<<1, 1024, smem, st>>>(H, m, E, Rt, work,
                                       global_a ? work + (size_t)m * m : nullptr, status);
  return cudaGetLastError();
}

cudaError_t launch_tridiag(const double* H, int m, double* work, cudaStream_t st) {
  if (m < 1 || m > kMaxM) return cudaErrorInvalidValue;
  const size_t smem = clus_smem(m, 1, 3);
  cudaError_t e = cudaFuncSetAttribute(tridiag_cluster_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  tridiag_cluster_kernel<<<kClus, kClusThreads, smem, st>>>(H, m, work, work + m);
  return cudaGetLastError();
}

cudaError_t launch_bisect(const double* work, int m, double* E, cudaStream_t st) {
  if (m > kMaxM) return cudaErrorInvalidValue;
  bisect_kernel<<<m, kBisPts, 0, st>>>(work, work + m, m, E);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_residual_norms(const T* A, const T* B, const double* E, double scale,
                                  int mode, int m, long long N, double dV, int chunks,
                                  double* partial, double* out, cudaStream_t st) {
  if (m < 1 || chunks < 1 || (N % Vec4Of<T>::W)) return cudaErrorInvalidValue;
  residual_partial_kernel<T><<<dim3(chunks, m), 256, 0, st>>>(A, B, E, scale, mode, N, chunks,
                                                              partial);
  residual_final_kernel<<<(m + 127) / 128, 128, 0, st>>>(partial, chunks, m, dV, out);
  return cudaGetLastError();
}
template cudaError_t launch_residual_norms<float>(const float*, const float*, const double*,
                                                  double, int, int, long long, double, int,
                                                  double*, double*, cudaStream_t);
template cudaError_t launch_residual_norms<double>(const double*, const double*, const double*,
                                                   double, int, int, long long, double, int,
                                                   double*, double*, cudaStream_t);

template <typename R>
__global__ void axpby_kernel(R a, const R* __restrict__ X, R b, const R* Y, R* out,
                             long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = fma(b, Y[i], a * X[i]);
}

template <typename R>
cudaError_t launch_axpby(double a, const R* X, double b, const R* Y, R* out, long long n,
                         cudaStream_t st) {
  axpby_kernel<R><<<4 * 152, 256, 0, st>>>((R)a, X, (R)b, Y, out, n);
  return cudaGetLastError();
}
template cudaError_t launch_axpby<float>(double, const float*, double, const float*, float*,
                                         long long, cudaStream_t);
template cudaError_t launch_axpby<double>(double, const double*, double, const double*,
                                          double*, long long, cudaStream_t);

cudaError_t launch_diag(const double* H, int m, double* E, cudaStream_t st) {
  diag_kernel<<<(m + 127) / 128, 128, 0, st>>>(H, m, E);
  return cudaGetLastError();
}

template <typename TX, typename TY>
cudaError_t launch_apply_matrix(const double* M, int m, int lower, const TX* X, TY* Y,
                                long long n_points, cudaStream_t st) {
  using TC = typename ComputeOf<TY>::type;
  if (m < 1 || m > kMaxM) return cudaErrorInvalidValue;
  const int bm = m < kBlk ? m : kBlk;   // rows of an M block
  const size_t smem = ((size_t)bm * bm + (size_t)bm * kApplyPT) * sizeof(TC);
  cudaError_t e = cudaFuncSetAttribute(apply_matrix_kernel<TX, TY, TC>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long ntiles = (n_points + kApplyPT - 1) / kApplyPT;
  const long long cap = (long long)sms * (smem > 110000 ? 1 : 2);
  const int blocks = (int)(ntiles < cap ? ntiles : cap);
  // Y block bi = sum over bk of M[bi][bk] X[bk] (bk <= bi when lower), in
  // stream order: the first block product sets Y[bi], the others add to it
  for (int r0 = 0; r0 < m; r0 += kBlk) {
    const int nr = m - r0 < kBlk ? m - r0 : kBlk;
    for (int k0 = 0; k0 < m && (!lower || k0 <= r0 + nr - 1); k0 += kBlk) {
      const int nk = m - k0 < kBlk ? m - k0 : kBlk;
      apply_matrix_kernel<TX, TY, TC><<<blocks, 512, smem, st>>>(M, m, lower, X, Y, n_points,
                                                                 r0, nr, k0, nk, k0 > 0);
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

template <typename TS, typename TD>
cudaError_t launch_convert(const TS* src, TD* dst, long long count, cudaStream_t st) {
  convert_kernel<TS, TD><<<4 * 152, 256, 0, st>>>(src, dst, count);
  return cudaGetLastError();
}

template cudaError_t launch_gram_partial<double, double, double>(const double*, const double*, int,
                                                                 long long, int, double*,
                                                                 cudaStream_t);
template cudaError_t launch_apply_matrix<double, double>(const double*, int, int, const double*,
                                                         double*, long long, cudaStream_t);
template cudaError_t launch_apply_matrix<double, float>(const double*, int, int, const double*,
                                                        float*, long long, cudaStream_t);
template cudaError_t launch_apply_matrix<float, float>(const double*, int, int, const float*,
                                                       float*, long long, cudaStream_t);
template cudaError_t launch_convert<float, double>(const float*, double*, long long, cudaStream_t);
template cudaError_t launch_convert<double, float>(const double*, float*, long long, cudaStream_t);
template cudaError_t launch_convert<double, double>(const double*, double*, long long, cudaStream_t);

}  // namespace itp
