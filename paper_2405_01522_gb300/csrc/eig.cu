// FP64 symmetric eigen-solve of the Tamm-Dancoff matrix on the device (Eq. 7, Sec. 2:
// with B = 0 the problem A X = omega X is Hermitian; only the lowest roots are needed).
//
//   k_tda_assemble    A = diag(eps_a - eps_i) + delta_M K - K_d, symmetrised
//   k_tridiag_cluster Householder reduction A = Q T Q^T on one thread-block cluster with the
//                     matrix in distributed shared memory (n up to ~530); k_tridiag_coop the
//                     cooperative multi-CTA form for larger n; k_tridiagonalise one CTA
//                     (reflectors kept in A in every form)
//   k_multisect       lowest nroots eigenvalues of T by Sturm-count multisection (a warp
//                     per root)
//   k_invit           inverse iteration on T (a warp per root); k_invit_clusters redoes
//                     roots of clusters of close eigenvalues with re-orthogonalisation
//   k_backtransform   x = Q y (a warp per root, reflectors read as rows after
//                     k_reflectors_to_rows)
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <string>

#include "../../include/rsx.h"
#include "api_internal.cuh"
#include "eig.cuh"

namespace rsx {
namespace {

constexpr int kEigThreads = 1024;

__device__ __forceinline__ double block_sum(double v, double* red) {
  // full-block reduction, result broadcast to every thread
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    double t = lane < nw ? red[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) red[32] = t;
  }
  __syncthreads();
  return red[32];
}

__global__ void k_tda_assemble(const double* __restrict__ eo, int no, const double* __restrict__ ev, int nv,
                               const double* __restrict__ K, const double* __restrict__ Kd, double dm,
                               double* __restrict__ A) {
  const int n = no * nv;
  const long long total = (long long)n * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int t = (int)(e / n), s = (int)(e - (long long)t * n);
    const long long et = (long long)s * n + t;
    double v = 0.5 * dm * (K[e] + K[et]);
    if (Kd) v -= 0.5 * (Kd[e] + Kd[et]);
    if (t == s) v += ev[t % nv] - eo[t / nv];
    A[e] = v;
  }
}

// Householder tridiagonalisation of the symmetric n x n matrix A (row-major, full
// storage).  Step k zeroes A[k+2.., k] with H_k = I - tau_k v v^T, v[k+1] = 1; v is
// stored in A[k+1.., k] (below the subdiagonal) and tau_k in tau[k].  Output: d (n),
// e (n - 1) of T.  work: 2 n doubles.
__global__ void __launch_bounds__(kEigThreads) k_tridiagonalise(double* __restrict__ A, int n, double* __restrict__ d,
                                                                double* __restrict__ e, double* __restrict__ tau,
                                                                double* __restrict__ work) {
  __shared__ double red[33];
  __shared__ double sh_alpha, sh_beta, sh_tau, sh_scale;
  double* v = work;       // n
  double* p = work + n;   // n
  for (int k = 0; k + 2 < n; ++k) {
    const int m0 = k + 1;  // first row of the trailing block
    // norm of A[k+2.., k]
    double s = 0.0;
    for (int i = m0 + 1 + threadIdx.x; i < n; i += blockDim.x) {
      const double x = A[(size_t)i * n + k];
      s += x * x;
    }
    const double xnorm2 = block_sum(s, red);
    if (threadIdx.x == 0) {
      const double alpha = A[(size_t)m0 * n + k];
      if (xnorm2 == 0.0) {
        sh_tau = 0.0;
        sh_beta = alpha;
        sh_scale = 0.0;
      } else {
        const double beta = -copysign(sqrt(alpha * alpha + xnorm2), alpha);
        sh_tau = (beta - alpha) / beta;
        sh_scale = 1.0 / (alpha - beta);
        sh_beta = beta;
      }
      sh_alpha = alpha;
    }
    __syncthreads();
    const double tk = sh_tau;
    if (threadIdx.x == 0) {
      e[k] = sh_beta;
      tau[k] = tk;
      d[k] = A[(size_t)k * n + k];
    }
    // v (stored back into the column)
    for (int i = m0 + threadIdx.x; i < n; i += blockDim.x) {
      const double vi = (i == m0) ? 1.0 : A[(size_t)i * n + k] * sh_scale;
      v[i] = vi;
      if (i > m0) A[(size_t)i * n + k] = vi;
    }
    __syncthreads();
    if (tk != 0.0) {
      // p = tau A22 v
      for (int i = m0 + threadIdx.x; i < n; i += blockDim.x) {
        const double* row = A + (size_t)i * n;
        double acc = 0.0;
        for (int j = m0; j < n; ++j) acc += row[j] * v[j];
        p[i] = tk * acc;
      }
      __syncthreads();
      double pv = 0.0;
      for (int i = m0 + threadIdx.x; i < n; i += blockDim.x) pv += p[i] * v[i];
      const double c = 0.5 * tk * block_sum(pv, red);
      for (int i = m0 + threadIdx.x; i < n; i += blockDim.x) p[i] -= c * v[i];   // w
      __syncthreads();
      // A22 -= v w^T + w v^T
      const int m = n - m0;
      for (long long q = threadIdx.x; q < (long long)m * m; q += blockDim.x) {
        const int i = m0 + (int)(q / m), j = m0 + (int)(q - (q / m) * m);
        A[(size_t)i * n + j] -= v[i] * p[j] + p[i] * v[j];
      }
      __syncthreads();
    }
  }
  if (threadIdx.x == 0) {
    if (n >= 2) {
      d[n - 2] = A[(size_t)(n - 2) * n + (n - 2)];
      e[n - 2] = A[(size_t)(n - 1) * n + (n - 2)];
      if (n >= 3) tau[n - 2] = 0.0;
    }
    d[n - 1] = A[(size_t)(n - 1) * n + (n - 1)];
  }
}

// number of eigenvalues of T strictly below x (Sturm sequence of the LDL^T pivots)

// ---------------------------------------------------------------------------------
// Multi-CTA Householder tridiagonalisation (same reflectors and outputs as
// k_tridiagonalise).  Rows are dealt cyclically to the CTAs; per step one grid-wide
// barrier separates (v from the CTA's copy of the current column, p = tau A22 v on own
// rows, p^T v partials) -> (rank-2 update of own rows, their entries of the column after
// next, the next column formed locally).  The kernel is launched cooperatively so that
// all CTAs are resident; the barrier itself is bounded and raises RSX_ETIMEOUT.
constexpr uint32_t kGridWaitLimit = 1u << 24;

struct GridBar {
  unsigned int count;
  volatile unsigned int gen;
  volatile int abort;
};

// wait_limit: spin rounds before a waiting CTA gives up (kGridWaitLimit unless the context
// sets another; 0 makes every CTA but the last arriver give up at once)
__device__ __forceinline__ bool grid_barrier(GridBar* gb, unsigned int nblocks, unsigned int wait_limit) {
  __syncthreads();
  __shared__ int ok_sh;
  if (threadIdx.x == 0) {
    ok_sh = 1;
    const unsigned int g0 = gb->gen;
    __threadfence();
    if (atomicAdd(&gb->count, 1u) == nblocks - 1) {
      gb->count = 0;
      __threadfence();
      atomicAdd((unsigned int*)&gb->gen, 1u);
    } else {
      uint32_t i = 0;
      while (gb->gen == g0) {
        if (gb->abort || ++i > wait_limit) {
          gb->abort = 1;
          ok_sh = 0;
          break;
        }
        // plain spin: the wait is a few microseconds at most
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok_sh != 0;
}

// first row >= r0 owned by CTA c (rows are dealt cyclically and never change owner,
// so a CTA only ever reads matrix rows it wrote itself; vectors shared between CTAs are
// read with __ldcg, which bypasses the non-coherent L1)
__device__ __forceinline__ int first_owned(int r0, int c, int G) { return r0 + ((c - r0) % G + G) % G; }

// precision traits of the reduction and root-finding kernels (F = double, or float for
// the first, FP32 stage of the mixed-precision eigensolver)
template <typename F> struct Prec;
template <> struct Prec<double> {
  static constexpr double eps = 2.220446049250313e-16, tiny = 1e-300, gap = 1e-6;
};
template <> struct Prec<float> {
  static constexpr float eps = 1.1920929e-7f, tiny = 1e-30f, gap = 1e-5f;
};
__device__ __forceinline__ double rsq(double x) { return rsqrt(x); }
__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
// Sturm count: division-free minors recurrence in FP64, the pivot ratio form in FP32
__device__ __forceinline__ int sturm_cnt(const double* d, const double* e2, int n, double x, double) {
  return sturm_count_prod(d, e2, n, x);
}
__device__ __forceinline__ int sturm_cnt(const float* d, const float* e2, int n, float x, float pivmin) {
  return sturm_count_f32(d, e2, n, x, pivmin);
}


// sum of the G per-CTA partials, by the whole CTA (one L2 round trip, shuffle reduction)
template <typename F>
__device__ __forceinline__ F cta_sum_partials(const F* part, unsigned int G, F* red, F* out_sh) {
  F v = F(0);
  for (unsigned int c = threadIdx.x; c < G; c += blockDim.x) v += __ldcg(part + c);
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {   // a shuffle tree, not a serial chain of dependent FP64 adds
    F t = lane < nwarp ? red[lane] : F(0);
    t = warp_sum(t);
    if (lane == 0) *out_sh = t;
  }
  __syncthreads();
  return *out_sh;
}

// scratch layout (Fs): p of even / odd steps [2][n], the next columns as they stood before
// the step's update [2][n], part_pv of even / odd steps [2][1024].  Every CTA keeps the
// current column (below the diagonal) in shared memory and forms the norm, tau and v from
// it; after the step's one grid barrier it knows p, hence w, updates its own rows, writes
// their entries of the column after next (after the update) and forms the next column from
// the replica written one step earlier minus the rank-2 terms.  Double buffers keep a CTA
// one step ahead from overwriting what a slower one still reads.
template <typename F>
__global__ void __launch_bounds__(256) k_tridiag_coop(F* __restrict__ A, int n, F* __restrict__ d,
                                                      F* __restrict__ e, F* __restrict__ tau,
                                                      F* __restrict__ scr, GridBar* gb, int* status,
                                                      unsigned int wait_limit) {
  const unsigned int G = gridDim.x;
  const int cta = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  F* ppb = scr;                 // [2][n]
  F* preg = scr + 2 * n;        // [2][n]
  F* part_pvb = scr + 4 * n;    // [2][1024]
  extern __shared__ __align__(16) unsigned char tri_smem_raw[];   // v, w, current column (3 n values)
  F* tri_smem = reinterpret_cast<F*>(tri_smem_raw);
  F* vs = tri_smem;
  F* ps = tri_smem + n;
  F* col = tri_smem + 2 * n;
  __shared__ F red[8];
  __shared__ F sh_tau, sh_scale, sh_sum;
  bool live = true;

  // column 0 (rows >= 1) straight from A; owners put column 1 (rows >= 2) in preg[1]
  for (int i = 1 + threadIdx.x; i < n; i += blockDim.x) col[i] = A[(size_t)i * n];
  for (int i = first_owned(2, cta, G) + (int)G * threadIdx.x; i < n; i += (int)G * blockDim.x)
    preg[n + i] = A[(size_t)i * n + 1];
  live = grid_barrier(gb, G, wait_limit);

  for (int k = 0; k + 2 < n && live; ++k) {
    const int m0 = k + 1;
    F* pp = ppb + (size_t)(k & 1) * n;
    F* part_pv = part_pvb + (size_t)(k & 1) * 1024;
    // ---- reflector from the column (every CTA computes the same scalars, in the same
    // order, from the same values)
    F s2 = F(0);
    for (int j = m0 + 1 + threadIdx.x; j < n; j += blockDim.x) s2 += col[j] * col[j];
    s2 = warp_sum(s2);
    if (lane == 0) red[warp] = s2;
    __syncthreads();
    if (warp == 0) {
      const F t = warp_sum(lane < nwarp ? red[lane] : F(0));
      if (lane == 0) sh_sum = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      const F xn2 = sh_sum, alpha = col[m0];
      F beta;
      if (xn2 == F(0)) {
        sh_tau = F(0);
        beta = alpha;
        sh_scale = F(0);
      } else {
        // beta = -sign(alpha) |x|, tau = 1 + |alpha| / |x|: one rsqrt, one division
        const F s = alpha * alpha + xn2, rs = rsq(s);
        beta = -copysign(s * rs, alpha);
        sh_tau = F(1) + fabs(alpha) * rs;
        sh_scale = F(1) / (alpha - beta);
      }
      if (cta == 0) {
        e[k] = beta;
        tau[k] = sh_tau;
      }
      if (k % (int)G == cta) d[k] = A[(size_t)k * n + k];
    }
    __syncthreads();
    const F tk = sh_tau, sc = sh_scale;
    // v (every entry), own rows keep theirs in the column for the back-transformation
    for (int j = m0 + threadIdx.x; j < n; j += blockDim.x) vs[j] = (j == m0) ? F(1) : col[j] * sc;
    for (int i = first_owned(m0 + 1, cta, G) + (int)G * threadIdx.x; i < n; i += (int)G * blockDim.x)
      A[(size_t)i * n + k] = col[i] * sc;
    __syncthreads();
    // ---- p_i = tau (A22 v)_i for own rows, partial p^T v
    F pv_part = F(0);
    if (tk != F(0)) {
      int r = 0;
      for (int i = first_owned(m0, cta, G); i < n; i += G, ++r) {
        if (r % nwarp != warp) continue;
        const F* row = A + (size_t)i * n;
        F a0 = F(0), a1 = F(0);   // two chains
        int j = m0 + lane;
        for (; j + 32 < n; j += 64) {
          a0 += row[j] * vs[j];
          a1 += row[j + 32] * vs[j + 32];
        }
        if (j < n) a0 += row[j] * vs[j];
        const F acc = warp_sum(a0 + a1);
        const F pi = tk * acc;
        if (lane == 0) {
          pp[i] = pi;
          pv_part += pi * vs[i];
        }
      }
    }
    if (lane == 0) red[warp] = pv_part;
    __syncthreads();
    if (warp == 0) {
      const F t = warp_sum(lane < nwarp ? red[lane] : F(0));
      if (lane == 0) part_pv[cta] = t;
    }
    if (!(live = grid_barrier(gb, G, wait_limit))) break;
    // ---- w = p - (tau/2)(p^T v) v ; A22 -= v w^T + w v^T on own rows; their entries of
    // column k + 2 after the update; the next column from its replica
    const F* prek = preg + (size_t)((k + 1) & 1) * n;   // column k + 1 before this update
    F* pren = preg + (size_t)(k & 1) * n;               // column k + 2 after it
    const bool need_next = k + 3 < n, need_after = k + 4 < n;
    F cc = F(0);
    if (tk != F(0)) {
      const F pvs = cta_sum_partials(part_pv, G, red, &sh_sum);
      cc = F(0.5) * tk * pvs;
      for (int j = m0 + threadIdx.x; j < n; j += blockDim.x) ps[j] = __ldcg(pp + j) - cc * vs[j];   // w
      __syncthreads();
      int r = 0;
      for (int i = first_owned(m0, cta, G); i < n; i += G, ++r) {
        if (r % nwarp != warp) continue;
        const F vi = vs[i];
        const F wi = ps[i];
        F* row = A + (size_t)i * n;
        for (int j = m0 + lane; j < n; j += 32) row[j] -= vi * ps[j] + wi * vs[j];
        __syncwarp();
        if (lane == 0 && need_after && i >= k + 3) pren[i] = row[k + 2];
      }
      if (need_next) {
        const F vm = vs[m0], wm = ps[m0];   // column m0's own v and w entries (v_m0 = 1)
        for (int j = m0 + 1 + threadIdx.x; j < n; j += blockDim.x)
          col[j] = __ldcg(prek + j) - (vs[j] * wm + ps[j] * vm);
      }
    } else {
      for (int i = first_owned(k + 3, cta, G) + (int)G * threadIdx.x; need_after && i < n;
           i += (int)G * blockDim.x)
        pren[i] = A[(size_t)i * n + k + 2];
      if (need_next)
        for (int j = m0 + 1 + threadIdx.x; j < n; j += blockDim.x) col[j] = __ldcg(prek + j);
    }
    __syncthreads();
  }
  if (cta == 0 && threadIdx.x == 0) {
    if (!live) {
      if (status) atomicMax(status, RSX_ETIMEOUT);
    } else {
      if (n >= 2) {
        d[n - 2] = __ldcg(A + (size_t)(n - 2) * n + (n - 2));
        e[n - 2] = __ldcg(A + (size_t)(n - 1) * n + (n - 2));
        if (n >= 3) tau[n - 2] = F(0);
      }
      d[n - 1] = __ldcg(A + (size_t)(n - 1) * n + (n - 1));
    }
  }
}

// ---------------------------------------------------------------------------------
// Householder tridiagonalisation on one thread-block cluster (same reflectors and outputs
// as k_tridiagonalise).  The matrix lives in the CTAs' shared memory: rows dealt
// cyclically (row i in CTA i % CS, local row i / CS).  Every CTA holds a replica of the
// current column (below the diagonal), from which it forms the norm, tau and v itself, and
// of the next column as it stood before this step's update.  Per step one hardware
// cluster barrier: before it, p = tau A22 v on own rows and each warp's p^T v partial go to
// every CTA; after it, every CTA knows w = p - (tau/2)(p^T v) v, updates its own rows,
// sends their entries of the column after next (before the next step's update), and forms
// the next column itself from its replica minus the rank-2 terms.  p, the partials and
// the pre-update column replicas are double-buffered, so that a CTA one step ahead never
// writes what a slower one still reads.  The rows are copied back to global memory at the
// end (the reflectors below the subdiagonal, for the back-transformation).
constexpr int kClThreads = 512;
namespace cg = cooperative_groups;

// shared-memory values of k_tridiag_cluster (rows unless GROWS, v, p x 2, the current
// column, the pre-update next columns x 2, the p^T v partials of every warp of every CTA x 2)
template <typename F>
inline size_t tridiag_cluster_smem(int n, int CS, bool grows) {
  return ((grows ? 0 : ((size_t)(n + CS - 1) / CS) * n) + 6 * (size_t)n + 2 * (size_t)CS * (kClThreads / 32)) *
         sizeof(F);
}

// GROWS: the owned rows stay in global memory (rows of A, L2-resident) instead of
// distributed shared memory, for n too large for the latter; only p, the columns and the
// partials go through DSMEM.  A CTA only ever touches the rows it owns.
template <typename F, bool GROWS>
__global__ void __launch_bounds__(kClThreads, 1) k_tridiag_cluster(F* __restrict__ A, int n, F* __restrict__ d,
                                                                F* __restrict__ e, F* __restrict__ tau) {
  cg::cluster_group cl = cg::this_cluster();
  const int CS = (int)cl.num_blocks();
  const int me = (int)cl.block_rank();
  const int nloc = (n - me + CS - 1) / CS;          // rows me, me + CS, ...
  const int lda = n;
  extern __shared__ __align__(16) unsigned char cl_smem_raw[];
  F* cl_smem = reinterpret_cast<F*>(cl_smem_raw);
  F* R = cl_smem;                               // [nloc][n] (shared-memory rows)
  F* v = GROWS ? cl_smem : R + (size_t)((n + CS - 1) / CS) * n;   // [n]
  F* pb = v + n;                                // [2][n] p of even / odd steps
  F* col = pb + 2 * n;                          // [n] current column (below the diagonal)
  F* pre = col + n;                             // [2][n] next columns before the step's update
  F* part2 = pre + 2 * n;                       // [2][CS][warps] p^T v partials
  __shared__ F red[kClThreads / 32];
  __shared__ F sh_tau, sh_scale;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = kClThreads / 32;
  auto grow = [&](int li) { return me + li * CS; };
  auto rowp = [&](int li) -> F* { return GROWS ? A + (size_t)grow(li) * lda : R + (size_t)li * n; };
  if (!GROWS) {
    for (size_t q = tid; q < (size_t)nloc * n; q += kClThreads) {
      const int li = (int)(q / n), j = (int)(q - (size_t)li * n);
      R[q] = A[(size_t)grow(li) * lda + j];
    }
  }
  __syncthreads();
  // block-wide sum of one value per thread, result to thread 0 (trees throughout: a
  // dependent FP64 add costs hundreds of cycles on this part)
  auto block_sum0 = [&](F x) {
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) red[warp] = x;
    __syncthreads();
    F t = F(0);
    if (warp == 0) {
      t = lane < nw ? red[lane] : F(0);
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    __syncthreads();
    return t;
  };
  // own rows' entries i >= r0 of column c, sent to every CTA's replica
  auto send_column = [&](int c, int r0, F* dst) {
    for (int q = tid; q < nloc * CS; q += kClThreads) {
      const int li = q / CS, to = q - li * CS;
      const int i = grow(li);
      if (i >= r0) *cl.map_shared_rank(dst + i, to) = rowp(li)[c];
    }
  };
  // replicas of column 0 (rows >= 1) and of column 1 before any update (rows >= 2)
  if (n > 2) send_column(0, 1, col);
  if (n > 3) send_column(1, 2, pre + n);
  cl.sync();
  for (int k = 0; k + 2 < n; ++k) {
    const int m0 = k + 1;
    F* p = pb + (size_t)(k & 1) * n;
    F* part = part2 + (size_t)(k & 1) * CS * nw;
    // norm of the column below the subdiagonal and alpha = A[m0][k], from the replica
    // (one warp: the other warps wait at the barrier below anyway)
    if (warp == 0) {
      F s2 = F(0);
      for (int j = m0 + 1 + lane; j < n; j += 32) s2 += col[j] * col[j];
      for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
      if (lane == 0) {
        const F alpha = col[m0];
        F beta;
        if (s2 == F(0)) {
          sh_tau = F(0);
          beta = alpha;
          sh_scale = F(0);
        } else {
          // beta = -sign(alpha) |x|, tau = (beta - alpha) / beta = 1 + |alpha| / |x|:
          // one reciprocal square root and one division
          const F s = alpha * alpha + s2, rs = rsq(s);
          beta = -copysign(s * rs, alpha);
          sh_tau = F(1) + fabs(alpha) * rs;
          sh_scale = F(1) / (alpha - beta);
        }
        if (me == 0) {
          e[k] = beta;
          tau[k] = sh_tau;
        }
        if (k % CS == me) d[k] = rowp(k / CS)[k];
      }
    }
    __syncthreads();
    const F tk = sh_tau, sc = sh_scale;
    // v (every entry, from the replica); own rows keep theirs as the reflector
    for (int j = m0 + tid; j < n; j += kClThreads) v[j] = (j == m0) ? F(1) : col[j] * sc;
    for (int li = tid; li < nloc; li += kClThreads) {
      const int i = grow(li);
      if (i > m0) rowp(li)[k] = col[i] * sc;
    }
    __syncthreads();
    // p_i = tau (A22 v)_i on own rows, a warp per row, sent to every CTA; each warp's
    // p^T v partial to every CTA's partial array
    F pv = F(0);
    if (tk != F(0)) {
      for (int li = warp; li < nloc; li += nw) {
        const int i = grow(li);
        if (i < m0) continue;
        const F* row = rowp(li);
        F a0 = F(0), a1 = F(0);   // two chains
        int j = m0 + lane;
        for (; j + 32 < n; j += 64) {
          a0 += row[j] * v[j];
          a1 += row[j + 32] * v[j + 32];
        }
        if (j < n) a0 += row[j] * v[j];
        F acc = a0 + a1;
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        const F pi = tk * acc;
        if (lane < CS) *cl.map_shared_rank(p + i, lane) = pi;
        pv += pi * v[i];   // the same in every lane
      }
    }
    if (lane < CS) *cl.map_shared_rank(part + me * nw + warp, lane) = pv;
    cl.sync();
    // w = p - (tau/2)(p^T v) v formed on the fly
    F pvs = F(0);
    for (int q = lane; q < CS * nw; q += 32) pvs += part[q];
    for (int o = 16; o > 0; o >>= 1) pvs += __shfl_xor_sync(0xffffffffu, pvs, o);
    const F cc = F(0.5) * tk * pvs;
    const F* prek = pre + (size_t)((k + 1) & 1) * n;   // column k + 1 before this update
    F* pren = pre + (size_t)(k & 1) * n;               // column k + 2 after it (next step's pre)
    const bool need_next = k + 3 < n, need_after = k + 4 < n;
    // rank-2 update of own rows, then their entries of column k + 2 to every replica
    if (tk != F(0)) {
      for (int li = warp; li < nloc; li += nw) {
        const int i = grow(li);
        if (i < m0) continue;
        const F vi = v[i], wi = p[i] - cc * vi;
        F* row = rowp(li);
        for (int j = m0 + lane; j < n; j += 32) row[j] -= vi * (p[j] - cc * v[j]) + wi * v[j];
        __syncwarp();
        if (need_after && i >= k + 3 && lane < CS) *cl.map_shared_rank(pren + i, lane) = row[k + 2];
      }
    } else {
      for (int li = warp; li < nloc; li += nw) {
        const int i = grow(li);
        if (need_after && i >= k + 3 && lane < CS) *cl.map_shared_rank(pren + i, lane) = rowp(li)[k + 2];
      }
    }
    // the next column (column m0, rows >= m0 + 1), here: its pre-update replica minus the
    // rank-2 terms v_j w_m0 + w_j v_m0
    if (need_next) {
      const F vm = v[m0], wm = p[m0] - cc * vm;   // column m0's own v and w entries (v_m0 = 1)
      for (int j = m0 + 1 + tid; j < n; j += kClThreads) {
        const F vj = v[j];
        col[j] = tk != F(0) ? prek[j] - (vj * wm + (p[j] - cc * vj) * vm) : prek[j];
      }
    }
    __syncthreads();
  }
  // last 2 x 2 block, rows back to global memory
  if (tid == 0) {
    if (n >= 2) {
      if ((n - 2) % CS == me) d[n - 2] = rowp((n - 2) / CS)[n - 2];
      if ((n - 1) % CS == me) e[n - 2] = rowp((n - 1) / CS)[n - 2];
      if (me == 0 && n >= 3) tau[n - 2] = F(0);
    }
    if ((n - 1) % CS == me) d[n - 1] = rowp((n - 1) / CS)[n - 1];
  }
  if (!GROWS) {
    for (size_t q = tid; q < (size_t)nloc * n; q += kClThreads) {
      const int li = (int)(q / n), j = (int)(q - (size_t)li * n);
      A[(size_t)grow(li) * lda + j] = R[q];
    }
  }
  cl.sync();   // no CTA leaves while others may still address its shared memory
}

// Lowest roots of the tridiagonal T (d, e), a warp per root: each round evaluates the
// Sturm count at 32 interior points of [lo, hi] (one per lane) and keeps the sub-interval
// in which the count passes k (FP64 is scarce on this part: 32 points per root and round
// instead of a whole CTA).
template <typename F>
__global__ void __launch_bounds__(32) k_multisect(const F* __restrict__ d, const F* __restrict__ e, int n,
                                                   int nroots, F* __restrict__ w) {
  extern __shared__ __align__(16) unsigned char ms_smem_raw[];   // d (n), e^2 (n)
  F* ms_smem = reinterpret_cast<F*>(ms_smem_raw);
  const int lane = threadIdx.x & 31;
  const int k = blockIdx.x;   // one warp (CTA) per root: spread over SMs, FP64 units are scarce
  if (k >= nroots) return;
  F* ds = ms_smem;
  F* e2 = ms_smem + n;
  for (int i = lane; i < n; i += 32) {
    ds[i] = d[i];
    e2[i] = i < n - 1 ? e[i] * e[i] : F(0);
  }
  __syncwarp();
  F lo = F(1) / Prec<F>::tiny, hi = -F(1) / Prec<F>::tiny, emax = F(0);
  for (int i = lane; i < n; i += 32) {
    const F r = (i > 0 ? fabs(e[i - 1]) : F(0)) + (i < n - 1 ? fabs(e[i]) : F(0));
    lo = fmin(lo, d[i] - r);
    hi = fmax(hi, d[i] + r);
    if (i < n - 1) emax = fmax(emax, fabs(e[i]));
  }
  for (int o = 16; o > 0; o >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    emax = fmax(emax, __shfl_xor_sync(0xffffffffu, emax, o));
  }
  const F scale = fmax(fabs(lo), fabs(hi));
  lo -= F(64) * Prec<F>::eps * scale + Prec<F>::tiny;
  hi += F(64) * Prec<F>::eps * scale + Prec<F>::tiny;
  const F pivmin = F(1.2e-38) * fmax(F(1), emax * emax);
  for (int round = 0; round < 16; ++round) {
    if (!(hi - lo > F(2) * Prec<F>::eps * fmax(fabs(lo), fabs(hi)))) break;
    const F x = lo + (hi - lo) * (F)(lane + 1) / F(33);
    const unsigned above = __ballot_sync(0xffffffffu, sturm_cnt(ds, e2, n, x, pivmin) > k);
    const int f = above ? __ffs(above) - 1 : 32;
    const F nlo = (f == 0) ? lo : lo + (hi - lo) * (F)f / F(33);
    const F nhi = (f == 32) ? hi : lo + (hi - lo) * (F)(f + 1) / F(33);
    lo = nlo;
    hi = nhi;
  }
  if (lane == 0) w[k] = F(0.5) * (lo + hi);
}

// Eigenvectors of T by inverse iteration, a warp per root (3 iterations from a fixed
// start); y: [nroots][n]; scratch: 4 n doubles + n ints per root.
template <typename F>
__global__ void __launch_bounds__(32) k_invit(const F* __restrict__ d, const F* __restrict__ e, int n,
                                               const F* __restrict__ w, int nroots, F* __restrict__ y,
                                               F* __restrict__ scratch) {
  const int lane = threadIdx.x & 31;
  const int k = blockIdx.x;   // one warp (CTA) per root: spread over SMs, FP64 units are scarce
  if (k >= nroots) return;
  F* z = y + (size_t)k * n;
  F* sc = scratch + (size_t)k * 5 * n;
  for (int i = lane; i < n; i += 32) z[i] = F(1) + F(0.001) * (F)((i * 7919 + k * 104729) % 997);
  __syncwarp();
  warp_inverse_iteration<F>(d, e, n, w[k], z, sc, reinterpret_cast<int*>(sc + 4 * n), 3, y, n, 0u);
}

// Roots closer than the cluster gap to an earlier root are recomputed one after another
// (one warp), each orthogonalised inside every iteration against the earlier roots of
// its cluster, so that (nearly) degenerate roots get orthonormal vectors.
template <typename F>
__global__ void k_invit_clusters(const F* __restrict__ d, const F* __restrict__ e, int n,
                                 const F* __restrict__ w, int nroots, F* __restrict__ y,
                                 F* __restrict__ scratch) {
  const int lane = threadIdx.x & 31;
  F s = F(0);
  for (int i = lane; i < n; i += 32) s = fmax(s, fabs(d[i]));
  for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_xor_sync(0xffffffffu, s, o));
  const F gap = Prec<F>::gap * fmax(F(1), s);
  int* piv = reinterpret_cast<int*>(scratch + 4 * n);
  for (int r = 1; r < nroots; ++r) {
    // the roots are ascending: the earlier members of r's cluster are the run j0 .. r - 1
    int j0 = r;
    while (j0 > 0 && fabs(w[r] - w[j0 - 1]) < gap) --j0;
    if (j0 == r) continue;
    F* z = y + (size_t)r * n;
    for (int i = lane; i < n; i += 32) z[i] = F(1) + F(0.001) * (F)((i * 7919 + r * 104729) % 997);
    __syncwarp();
    if (lane == 0) tri_factor_shifted<F>(d, e, n, w[r], scratch, piv);
    __syncwarp();
    for (int it = 0; it < 3; ++it) {
      if (lane == 0) tri_solve_factored<F>(n, z, scratch, piv);
      __syncwarp();
      for (int j = j0; j < r; ++j) {
        const F* zj = y + (size_t)j * n;
        F dot = F(0);
        for (int i = lane; i < n; i += 32) dot += zj[i] * z[i];
        dot = warp_sum(dot);
        for (int i = lane; i < n; i += 32) z[i] -= dot * zj[i];
        __syncwarp();
      }
      F nn = F(0);
      for (int i = lane; i < n; i += 32) nn += z[i] * z[i];
      nn = warp_sum(nn);
      const F inv = nn > F(0) ? F(1) / sqrt(nn) : F(0);
      for (int i = lane; i < n; i += 32) z[i] *= inv;
      __syncwarp();
    }
  }
}

// Reflector vectors moved to rows: A[j][i] = A[i][j] for i > j + 1 (the strict upper
// triangle past the superdiagonal is dead after the reduction), so that the
// back-transformation reads each reflector contiguously.  32 x 32 tiles through shared
// memory.
template <typename F>
__global__ void k_reflectors_to_rows(F* __restrict__ A, int n) {
  __shared__ F tile[32][33];
  const int j0 = blockIdx.x * 32, i0 = blockIdx.y * 32;   // source tile: rows i0.., columns j0..
  if (i0 + 31 < j0 + 2) return;                          // no entry with i > j + 1
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 8 rows per pass
  for (int r = ty; r < 32; r += 8) {
    const int i = i0 + r, j = j0 + tx;
    tile[r][tx] = (i < n && j < n && i > j + 1) ? A[(size_t)i * n + j] : F(0);
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int j = j0 + r, i = i0 + tx;   // destination A[j][i]
    if (i < n && j < n && i > j + 1) A[(size_t)j * n + i] = tile[tx][r];
  }
}

// x_k = H_0 H_1 ... H_{n-3} y_k, one warp (CTA) per root, x in shared memory;
// H_j = I - tau_j v_j v_j^T, v_j[j+1] = 1, v_j[i] = A[j][i] (i > j + 1, rows form)
template <typename F>
__global__ void __launch_bounds__(32) k_backtransform(const F* __restrict__ A, const F* __restrict__ tau,
                                                      int n, const F* __restrict__ y, int nroots,
                                                      F* __restrict__ X) {
  extern __shared__ __align__(16) unsigned char xs_bt_raw[];
  F* xs_bt = reinterpret_cast<F*>(xs_bt_raw);
  const int lane = threadIdx.x & 31;
  const int k = blockIdx.x;
  if (k >= nroots) return;
  F* x = xs_bt;
  for (int i = lane; i < n; i += 32) x[i] = y[(size_t)k * n + i];
  __syncwarp();
  for (int kk = n - 3; kk >= 0; --kk) {
    const F tk = tau[kk];
    if (tk == F(0)) continue;
    const F* v = A + (size_t)kk * n;
    F s = (lane == 0) ? x[kk + 1] : F(0);
    for (int i = kk + 2 + lane; i < n; i += 32) s += v[i] * x[i];
    s = tk * warp_sum(s);
    if (lane == 0) x[kk + 1] -= s;
    for (int i = kk + 2 + lane; i < n; i += 32) x[i] -= s * v[i];
    __syncwarp();
  }
  for (int i = lane; i < n; i += 32) X[(size_t)k * n + i] = x[i];
}

}  // namespace

// workspace after A, d, e, tau: tw (2 n, one-CTA tridiagonalisation), the T-basis vectors
// y (nroots n), inverse-iteration scratch (nroots 5 n), then the cooperative kernel's
// scratch (v, p, partials, alpha, grid barrier)
// scratch after the tridiagonal arrays: 2 n (tridiagonalisation), yv (nroots n), 5 n per root
template <typename F>
static F* y_end(F* tw, int n, int nroots) { return tw + 2 * n + (size_t)nroots * n + 5 * (size_t)nroots * n; }
// coop scratch (v, p, partials, alpha) + the grid barrier, in units of F
template <typename F>
static size_t coop_scratch(int n) { return 4 * (size_t)n + 2048 + 2 + (sizeof(GridBar) + sizeof(F) - 1) / sizeof(F) + 2; }

static size_t tda_work_doubles_fp64(int n, int nroots) {
  return (size_t)n * n + 14 * (size_t)n + 6 * (size_t)nroots * n + 4096;
}

constexpr int kMixedMinN = 96;   // below this the FP64 path is as fast
constexpr int kNewtonSteps = 2;  // FP64 correction steps of the mixed path

size_t tda_work_doubles(int n, int nroots) {
  const size_t fp64 = tda_work_doubles_fp64(n, nroots);
  if (n < kMixedMinN) return fp64;
  const size_t nn = (size_t)n * n, k = nroots;
  // FP32 part (counted in doubles): A32, d / e / tau, coop scratch, roots, vectors of T,
  // inverse-iteration scratch (5 n per root), eigenvectors of A32
  const size_t f32 = (nn + 3 * (size_t)n + coop_scratch<float>(n) + n + nn + 5 * nn + nn + 16) / 2 + 2;
  // FP64 part: Xh (n x n), lambda, Xk / Y / R / D (k x n each), C (n x k), the small
  // Rayleigh-Ritz (G, H, Linv, Yc, Zc, theta) and its eigensolver workspace
  const size_t f64 = nn + n + 5 * k * n + 5 * k * k + 4 * k + tda_work_doubles_fp64((int)k, nroots);
  return std::max(fp64, nn + f32 + f64 + 64);
}

// Householder reduction of the n x n matrix A (F) into d, e, tau: one thread-block cluster
// with the matrix in distributed shared memory when it fits, else the cooperative grid,
// else (F = double only) one CTA.  scr: coop_scratch<F>(n) values; tw: 2 n (one CTA).
template <typename F>
static int tridiagonalise(rsx_ctx* c, F* A, int n, F* d, F* e, F* tau, F* scr, F* tw, cudaStream_t s) {
  int coop = 0, per_sm = 0;
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, c->device);
  cudaFuncSetAttribute(k_tridiag_coop<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(3 * (size_t)n * sizeof(F)));
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tridiag_coop<F>, 256, 3 * (size_t)n * sizeof(F));
  // FP64: 64 CTAs (fewer make each grid barrier cheaper, the FP64 work per step is
  // small); FP32: one per SM (measured at n = 960: 64 -> 24.0 ms, 152 -> 19.8 ms)
  int gcap = sizeof(F) == 4 ? c->nsm : 64;
  if (const char* ev = getenv("RSX_TRIDIAG_CTAS")) gcap = std::max(1, atoi(ev));
  const int G = std::min(std::min(std::min(c->nsm * std::max(per_sm, 0), gcap), std::max(1, n / 2)), 1024);
  // rows in distributed shared memory (16 CTAs, else 8), else the cooperative grid, else
  // one 16-CTA cluster with the rows in global memory (slower than the grid at n ~ 1000,
  // measured), else one CTA.  RSX_TRIDIAG_PATH = cluster, coop, global or cta forces one
  // (tests cover every path with it).
  const char* fp = getenv("RSX_TRIDIAG_PATH");
  const std::string force = fp ? fp : "";
  auto try_cluster = [&](int CS, bool grows) -> int {   // -1: not possible here
    if (n < 64) return -1;
    const size_t smem = tridiag_cluster_smem<F>(n, CS, grows);
    if (smem > (size_t)227 * 1024) return -1;
    auto kern = grows ? k_tridiag_cluster<F, true> : k_tridiag_cluster<F, false>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        (CS > 8 && cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)) {
      cudaGetLastError();
      return -1;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CS);
    cfg.blockDim = dim3(kClThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int ncl = 0;
    if (cudaOccupancyMaxActiveClusters(&ncl, kern, &cfg) != cudaSuccess || ncl < 1) {
      cudaGetLastError();
      return -1;
    }
    return check_cuda(c, cudaLaunchKernelEx(&cfg, kern, A, n, d, e, tau), "cluster tridiagonalisation");
  };
  if (force.empty() || force == "cluster")
    for (int CS : {16, 8}) {
      const int r = try_cluster(CS, false);
      if (r >= 0) return r;
    }
  if (coop && per_sm > 0 && n >= 64 && (force.empty() || force == "coop")) {
    GridBar* gb = reinterpret_cast<GridBar*>(scr + 4 * (size_t)n + 2048 + 2);
    cudaMemsetAsync(gb, 0, sizeof(GridBar), s);
    unsigned int wait_limit = c->wait_limit < 0 ? kGridWaitLimit
                              : (unsigned int)std::min<long long>(c->wait_limit, 0xffffffffLL);
    void* args[] = {(void*)&A, (void*)&n, (void*)&d, (void*)&e, (void*)&tau, (void*)&scr, (void*)&gb,
                    (void*)&c->status, (void*)&wait_limit};
    const size_t smem = 3 * (size_t)n * sizeof(F);
    cudaFuncSetAttribute(k_tridiag_coop<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return check_cuda(c, cudaLaunchCooperativeKernel((const void*)k_tridiag_coop<F>, dim3(G), dim3(256), args, smem, s),
                      "cooperative tridiagonalisation");
  }
  if (force.empty() || force == "global") {
    const int r = try_cluster(16, true);
    if (r >= 0) return r;
  }
  if constexpr (sizeof(F) == 8) {
    k_tridiagonalise<<<1, kEigThreads, 0, s>>>(A, n, d, e, tau, tw);
    return check_cuda(c, cudaGetLastError(), "tridiagonalisation");
  }
  return set_error(c, RSX_EUNSUPPORTED, "no FP32 tridiagonalisation path for this size");
}

// Blocked back-transformation (compact WY form, as in LAPACK's xLARFT / xLARFB): the
// reflectors are taken 32 at a time, H_j0 ... H_j0+m-1 = I - V T V^T with V the block's
// reflector vectors (n x m) and T upper triangular, T[i][i] = tau_i,
// T[0:i][i] = -tau_i T[0:i][0:i] (V[:, 0:i]^T v_i).  k_wy_t builds T of every block (one
// CTA per block, into Tg[block][32][32]); k_backtransform_wy applies the blocks, last
// first, to each root's vector (a warp per root): s = V^T x (a lane per reflector),
// u = T s, x -= V u (lanes over the rows).  The dependent steps per root drop from one
// per reflector to three per block.
constexpr int kWy = 32;

template <typename F>
__global__ void __launch_bounds__(256) k_wy_t(const F* __restrict__ A, const F* __restrict__ tau, int n, int nref,
                                              F* __restrict__ Tg) {
  __shared__ F G[kWy][kWy + 1];
  __shared__ F T[kWy][kWy + 1];
  const int b = blockIdx.x, j0 = b * kWy, m = min(kWy, nref - j0);
  // G[a][c] = v_a^T v_c for a < c (v_a[r] = 0 for r <= ja, 1 at ja + 1, A[ja][r] beyond)
  for (int q = threadIdx.x; q < kWy * kWy; q += blockDim.x) {
    const int a = q / kWy, c = q - a * kWy;
    F g = F(0);
    if (a < c && c < m) {
      const int ja = j0 + a, jc = j0 + c;   // ja < jc: v_c vanishes at and above jc
      const F* va = A + (size_t)ja * n;
      const F* vc = A + (size_t)jc * n;
      g = va[jc + 1];                        // v_c[jc + 1] = 1
      for (int r = jc + 2; r < n; ++r) g += va[r] * vc[r];
    }
    G[a][c] = g;
    T[a][c] = F(0);
  }
  __syncthreads();
  for (int i = 0; i < m; ++i) {
    const F ti = tau[j0 + i];
    // T[a][i] = -tau_i sum_{c < i} T[a][c] G[c][i], a < i (T[0:i][0:i] is final)
    F t = F(0);
    const int a = threadIdx.x;
    if (a < i) {
      for (int c = a; c < i; ++c) t += T[a][c] * G[c][i];
    }
    __syncthreads();
    if (a < i) T[a][i] = -ti * t;
    if (a == i) T[i][i] = ti;
    __syncthreads();
  }
  for (int q = threadIdx.x; q < kWy * kWy; q += blockDim.x) {
    const int a = q / kWy, c = q - a * kWy;
    Tg[(size_t)b * kWy * kWy + q] = T[a][c];
  }
}

template <typename F>
__global__ void __launch_bounds__(32) k_backtransform_wy(const F* __restrict__ A, const F* __restrict__ Tg, int n,
                                                         int nref, const F* __restrict__ y, int nroots,
                                                         F* __restrict__ X) {
  extern __shared__ __align__(16) unsigned char xs_wy_raw[];
  F* x = reinterpret_cast<F*>(xs_wy_raw);
  __shared__ F us[kWy];
  const int lane = threadIdx.x & 31;
  const int k = blockIdx.x;
  if (k >= nroots) return;
  for (int i = lane; i < n; i += 32) x[i] = y[(size_t)k * n + i];
  __syncwarp();
  const int nb = (nref + kWy - 1) / kWy;
  for (int b = nb - 1; b >= 0; --b) {
    const int j0 = b * kWy, m = min(kWy, nref - j0);
    // s_j = v_j^T x, lane j
    F sj = F(0);
    if (lane < m) {
      const int ja = j0 + lane;
      const F* va = A + (size_t)ja * n;
      F s0 = x[ja + 1], s1 = F(0);   // two chains
      int r = ja + 2;
      for (; r + 1 < n; r += 2) {
        s0 += va[r] * x[r];
        s1 += va[r + 1] * x[r + 1];
      }
      if (r < n) s0 += va[r] * x[r];
      sj = s0 + s1;
    }
    // u_i = sum_{j >= i} T[i][j] s_j, lane i
    F ui = F(0);
    const F* Trow = Tg + (size_t)b * kWy * kWy + (size_t)lane * kWy;
    for (int j = 0; j < kWy; ++j) {
      const F sjj = __shfl_sync(0xffffffffu, sj, j);
      if (j >= lane && j < m) ui += Trow[j] * sjj;
    }
    us[lane] = ui;
    __syncwarp();
    // x_r -= sum_j v_j[r] u_j for r > j0 (rows of the block's reflectors)
    for (int r = j0 + 1 + lane; r < n; r += 32) {
      F acc = F(0);
      const int jmax = min(m, r - j0);   // v_j[r] = 0 for r <= j0 + j
      for (int j = 0; j < jmax; ++j) {
        const int ja = j0 + j;
        const F vj = (r == ja + 1) ? F(1) : A[(size_t)ja * n + r];
        acc += vj * us[j];
      }
      x[r] -= acc;
    }
    __syncwarp();
  }
  for (int i = lane; i < n; i += 32) X[(size_t)k * n + i] = x[i];
}

// lowest q eigenpairs of the tridiagonal (d, e) and x = Q y through the reflectors of A
template <typename F>
static void tridiag_eigs(F* A, const F* tau, const F* d, const F* e, int n, int q, F* w, F* yv, F* sc, F* X,
                         cudaStream_t s) {
  cudaFuncSetAttribute(k_multisect<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(2 * (size_t)n * sizeof(F)));
  k_multisect<F><<<q, 32, 2 * (size_t)n * sizeof(F), s>>>(d, e, n, q, w);
  if (!X) return;
  k_invit<F><<<q, 32, 0, s>>>(d, e, n, w, q, yv, sc);
  k_invit_clusters<F><<<1, 32, 0, s>>>(d, e, n, w, q, yv, sc);
  k_reflectors_to_rows<F><<<dim3((n + 31) / 32, (n + 31) / 32), 256, 0, s>>>(A, n);
  const size_t smem = (size_t)n * sizeof(F);
  const int nref = n - 2, nb = (nref + kWy - 1) / kWy;
  if (nref >= kWy && (size_t)nb * kWy * kWy <= 5 * (size_t)n * q) {
    // T of every block in the inverse-iteration scratch (free again here)
    k_wy_t<F><<<nb, 256, 0, s>>>(A, tau, n, nref, sc);
    cudaFuncSetAttribute(k_backtransform_wy<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_backtransform_wy<F><<<q, 32, smem, s>>>(A, sc, n, nref, yv, q, X);
    return;
  }
  cudaFuncSetAttribute(k_backtransform<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_backtransform<F><<<q, 32, smem, s>>>(A, tau, n, yv, q, X);
}

// FP64 form throughout (Householder, multisection, inverse iteration, back-transformation)
static int sym_eig_lowest_fp64(rsx_ctx* c, double* work, int n, int nroots, double* omega, double* X, cudaStream_t s) {
  double* A = work;
  double* d = A + (size_t)n * n;
  double* e = d + n;
  double* tau = e + n;
  double* tw = tau + n;          // 2 n (tridiagonalisation), then 5 n (eigvec scratch needs 4 n + n ints)
  int rc = tridiagonalise<double>(c, A, n, d, e, tau, y_end(tw, n, nroots), tw, s);
  if (rc) return rc;
  tridiag_eigs<double>(A, tau, d, e, n, nroots, omega, tw + 2 * n, tw + 2 * n + (size_t)nroots * n, X, s);
  return check_cuda(c, cudaGetLastError(), "symmetric eigensolve");
}

namespace {
__global__ void k_f64_to_f32(const double* __restrict__ a, size_t n, float* __restrict__ b) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}
__global__ void k_f32_to_f64(const float* __restrict__ a, size_t n, double* __restrict__ b) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    b[i] = (double)a[i];
}
// W = V M (q x n times n x n, row-major): block (32 columns, 8 splits of the inner index),
// grid (column tiles, rows of V); two chains per thread, shared-memory tree over the splits
__global__ void __launch_bounds__(256) k_vm(const double* __restrict__ V, const double* __restrict__ M, int n,
                                            double* __restrict__ W) {
  __shared__ double red[8][33];
  const int tx = threadIdx.x & 31, ks = threadIdx.x >> 5;
  const int i = blockIdx.x * 32 + tx, r = blockIdx.y;
  const double* v = V + (size_t)r * n;
  double a0 = 0.0, a1 = 0.0;
  if (i < n) {
    int j = ks;
    for (; j + 8 < n; j += 16) {
      a0 += v[j] * M[(size_t)j * n + i];
      a1 += v[j + 8] * M[(size_t)(j + 8) * n + i];
    }
    if (j < n) a0 += v[j] * M[(size_t)j * n + i];
  }
  red[ks][tx] = a0 + a1;
  __syncthreads();
  if (ks == 0 && i < n)
    W[(size_t)r * n + i] = ((red[0][tx] + red[1][tx]) + (red[2][tx] + red[3][tx])) +
                           ((red[4][tx] + red[5][tx]) + (red[6][tx] + red[7][tx]));
}
// out[a * nb + b] = sum_i X[a][i] Y[b][i] (length n): a block per output, tree reduction
__global__ void __launch_bounds__(256) k_dots(const double* __restrict__ X, const double* __restrict__ Y, int n, int nb,
                                              double* __restrict__ out) {
  __shared__ double red[8];
  const int a = blockIdx.x / nb, b = blockIdx.x % nb;
  const double* x = X + (size_t)a * n;
  const double* y = Y + (size_t)b * n;
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) acc += x[i] * y[i];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    const double t = warp_sum(threadIdx.x < 8 ? red[threadIdx.x] : 0.0);
    if (threadIdx.x == 0) out[blockIdx.x] = t;
  }
}
// theta_j = <x_j, (A x)_j> / <x_j, x_j>;  R_j = (A x)_j - theta_j x_j   (k x n)
__global__ void k_residuals(const double* __restrict__ Xk, const double* __restrict__ Y, const double* __restrict__ GH,
                            int k, int n, double* __restrict__ theta, double* __restrict__ R) {
  for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < (size_t)k * n; x += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(x / n);
    const double th = GH[2 * j + 1] / GH[2 * j];
    R[x] = Y[x] - th * Xk[x];
    if (x - (size_t)j * n == 0) theta[j] = th;
  }
}
// correction coefficients D[j][i] = -C[i][j] / (lambda_i - theta_j) (zero within gthr of
// theta_j: the root itself and its near-degenerate partners, left to the final
// Rayleigh-Ritz), C[i][j] = <xh_i, r_j>
__global__ void k_newton_coeffs(const double* __restrict__ C, const double* __restrict__ lam,
                                const double* __restrict__ theta, int n, int k, double gthr, double* __restrict__ D) {
  for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < (size_t)k * n; x += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(x / n), i = (int)(x - (size_t)j * n);
    const double dl = lam[i] - theta[j];
    D[x] = fabs(dl) > gthr ? -C[(size_t)i * k + j] / dl : 0.0;
  }
}
__global__ void k_add_inplace(double* __restrict__ a, const double* __restrict__ b, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) a[i] += b[i];
}
// the diagonal of two k x k Gram results interleaved: GH[2 j] = G_jj, GH[2 j + 1] = H_jj
__global__ void k_diag2(const double* __restrict__ G, const double* __restrict__ H, int k, double* __restrict__ GH) {
  const int j = threadIdx.x;
  if (j < k) {
    GH[2 * j] = G[j * k + j];
    GH[2 * j + 1] = H[j * k + j];
  }
}
// G = L L^T (q <= 64, one CTA), Linv = L^-1, C = Linv H Linv^T (H symmetrised)
__global__ void __launch_bounds__(256) k_whiten(const double* __restrict__ G, const double* __restrict__ H, int q,
                                                double* __restrict__ C, double* __restrict__ Linv, int* status) {
  extern __shared__ double wh_smem[];   // L, Li, T: 3 q^2
  double* L = wh_smem;
  double* Li = L + q * q;
  double* T = Li + q * q;
  const int tid = threadIdx.x;
  for (int x = tid; x < q * q; x += 256) {
    const int r = x / q, cc = x - r * q;
    L[x] = 0.5 * (G[r * q + cc] + G[cc * q + r]);
    Li[x] = 0.0;
  }
  __syncthreads();
  for (int j = 0; j < q; ++j) {
    if (tid == 0) {
      double p = L[j * q + j];
      if (!(p > 0.0)) {
        atomicMax(status, RSX_ENOTPD);
        p = 1.0;
      }
      L[j * q + j] = sqrt(p);
    }
    __syncthreads();
    const double rl = 1.0 / L[j * q + j];
    for (int i = j + 1 + tid; i < q; i += 256) L[i * q + j] *= rl;
    __syncthreads();
    const int t = q - j - 1;
    for (int x = tid; x < t * t; x += 256) {
      const int i = j + 1 + x / t, l = j + 1 + x % t;
      if (l <= i) L[i * q + l] -= L[i * q + j] * L[l * q + j];
    }
    __syncthreads();
  }
  if (tid < q) {
    const int cc = tid;
    Li[cc * q + cc] = 1.0 / L[cc * q + cc];
    for (int i = cc + 1; i < q; ++i) {
      double sum = 0.0;
      for (int p = cc; p < i; ++p) sum += L[i * q + p] * Li[p * q + cc];
      Li[i * q + cc] = -sum / L[i * q + i];
    }
  }
  __syncthreads();
  for (int x = tid; x < q * q; x += 256) {   // T = Li H
    const int r = x / q, cc = x - r * q;
    double sum = 0.0;
    for (int p = 0; p <= r; ++p) sum += Li[r * q + p] * 0.5 * (H[p * q + cc] + H[cc * q + p]);
    T[x] = sum;
  }
  __syncthreads();
  for (int x = tid; x < q * q; x += 256) {   // C = T Li^T
    const int r = x / q, cc = x - r * q;
    double sum = 0.0;
    for (int p = 0; p <= cc; ++p) sum += T[r * q + p] * Li[cc * q + p];
    C[x] = sum;
    Linv[x] = Li[x];
  }
}
// Zc[k][r] = sum_s Yc[k][s] Linv[s][r]: the wanted eigenvectors' coefficients over the rows of V
__global__ void k_coeffs(const double* __restrict__ Yc, const double* __restrict__ Linv, int q, int nroots,
                         double* __restrict__ Zc) {
  for (int x = threadIdx.x; x < nroots * q; x += blockDim.x) {
    const int k = x / q, r = x - k * q;
    double sum = 0.0;
    for (int sidx = r; sidx < q; ++sidx) sum += Yc[k * q + sidx] * Linv[sidx * q + r];
    Zc[x] = sum;
  }
}
// X[k][:] = sum_r Zc[k][r] V[r][:]
__global__ void k_expand(const double* __restrict__ Zc, const double* __restrict__ V, int q, int nroots, int n,
                         double* __restrict__ X) {
  for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < (size_t)nroots * n; x += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(x / n), i = (int)(x - (size_t)k * n);
    double sum = 0.0;
    for (int r = 0; r < q; ++r) sum += Zc[k * q + r] * V[(size_t)r * n + i];
    X[x] = sum;
  }
}
unsigned blocks_of(size_t n) { return (unsigned)std::min<size_t>((n + 255) / 256, 4096); }
}  // namespace

// Mixed precision.  The Householder reduction, every root of T, its vector and the
// back-transformation run in FP32 (A32 = A rounded), giving a full approximate
// eigenbasis Xh, lambda of A.  The wanted k vectors are then corrected in FP64 against A
// itself, kNewtonSteps times: r_j = A x_j - theta_j x_j (theta_j the Rayleigh quotient),
// x_j <- x_j - sum_i xh_i <xh_i, r_j> / (lambda_i - theta_j) over the roots i not within
// gthr of theta_j -- the correction equation solved in the approximate eigenbasis, which
// converges quadratically from FP32 accuracy -- and a final FP64 Rayleigh-Ritz on the k
// corrected vectors (G = X X^T, H = X A X^T, H z = theta G z) resolves near-degenerate
// roots and gives the eigenvalues.
static int sym_eig_lowest_mixed(rsx_ctx* c, double* work, int n, int nroots, double* omega, double* X,
                                cudaStream_t s) {
  const int k = nroots;
  const size_t nn = (size_t)n * n;
  double* A = work;                                   // FP64 A, kept
  float* A32 = reinterpret_cast<float*>(A + nn);
  float* d32 = A32 + nn;
  float* e32 = d32 + n;
  float* tau32 = e32 + n;
  float* scr32 = tau32 + n;
  float* w32 = scr32 + coop_scratch<float>(n);
  float* yv32 = w32 + n;                              // n x n, then 5 n per root
  float* sc32 = yv32 + nn;
  float* X32 = sc32 + 5 * nn;
  uintptr_t gp = reinterpret_cast<uintptr_t>(X32 + nn) + 16;
  double* g = reinterpret_cast<double*>((gp + 15) & ~uintptr_t(15));
  double* Xh = g;                                     // n x n
  double* lam = Xh + nn;                              // n
  double* Xk = lam + n;                               // k x n
  double* Y = Xk + (size_t)k * n;
  double* R = Y + (size_t)k * n;
  double* D = R + (size_t)k * n;
  double* Cm = D + (size_t)k * n;                     // n x k
  double* G = Cm + (size_t)k * n;                     // k x k
  double* H = G + (size_t)k * k;
  double* Linv = H + (size_t)k * k;
  double* Yc = Linv + (size_t)k * k;
  double* Zc = Yc + (size_t)k * k;
  double* th = Zc + (size_t)k * k;                    // 2 k (theta, then G / H diagonals)
  double* GH = th + k;
  double* Cw = GH + 2 * k;                            // the small problem: C and its workspace
  k_f64_to_f32<<<blocks_of(nn), 256, 0, s>>>(A, nn, A32);
  int rc = tridiagonalise<float>(c, A32, n, d32, e32, tau32, scr32, nullptr, s);
  if (rc) return rc;
  tridiag_eigs<float>(A32, tau32, d32, e32, n, n, w32, yv32, sc32, X32, s);
  k_f32_to_f64<<<blocks_of(nn), 256, 0, s>>>(X32, nn, Xh);
  k_f32_to_f64<<<blocks_of(n), 256, 0, s>>>(w32, n, lam);
  cudaMemcpyAsync(Xk, Xh, (size_t)k * n * sizeof(double), cudaMemcpyDeviceToDevice, s);
  // near-degeneracy threshold: FP32 can not separate roots closer than a few eps32 |A|
  double gthr = 0.0;
  {
    // |A| from the extreme FP32 roots
    float ends[2];
    cudaMemcpyAsync(&ends[0], w32, sizeof(float), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&ends[1], w32 + n - 1, sizeof(float), cudaMemcpyDeviceToHost, s);
    rc = check_cuda(c, cudaStreamSynchronize(s), "mixed eigensolve (FP32 stage)");
    if (rc) return rc;
    gthr = 1e-5 * std::max(1.0, std::max(std::fabs((double)ends[0]), std::fabs((double)ends[1])));
  }
  const dim3 gvm((n + 31) / 32, k);
  for (int it = 0; it < kNewtonSteps; ++it) {
    k_vm<<<gvm, 256, 0, s>>>(Xk, A, n, Y);                        // Y = Xk A (A symmetric)
    k_dots<<<k * k, 256, 0, s>>>(Xk, Xk, n, k, G);
    k_dots<<<k * k, 256, 0, s>>>(Xk, Y, n, k, H);
    k_diag2<<<1, 64, 0, s>>>(G, H, k, GH);
    k_residuals<<<blocks_of((size_t)k * n), 256, 0, s>>>(Xk, Y, GH, k, n, th, R);
    k_dots<<<n * k, 256, 0, s>>>(Xh, R, n, k, Cm);                 // Cm[i][j] = <xh_i, r_j>
    k_newton_coeffs<<<blocks_of((size_t)k * n), 256, 0, s>>>(Cm, lam, th, n, k, gthr, D);
    k_vm<<<gvm, 256, 0, s>>>(D, Xh, n, R);                         // R = D Xh (the correction)
    k_add_inplace<<<blocks_of((size_t)k * n), 256, 0, s>>>(Xk, R, (size_t)k * n);
  }
  // final Rayleigh-Ritz on the k corrected vectors
  k_vm<<<gvm, 256, 0, s>>>(Xk, A, n, Y);
  k_dots<<<k * k, 256, 0, s>>>(Xk, Xk, n, k, G);
  k_dots<<<k * k, 256, 0, s>>>(Y, Xk, n, k, H);
  const size_t wsm = 3 * (size_t)k * k * sizeof(double);
  cudaFuncSetAttribute(k_whiten, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wsm);
  k_whiten<<<1, 256, wsm, s>>>(G, H, k, Cw, Linv, c->status);
  rc = check_cuda(c, cudaGetLastError(), "mixed eigensolve (FP64 correction)");
  if (rc) return rc;
  rc = sym_eig_lowest_fp64(c, Cw, k, k, omega, Yc, s);
  if (rc) return rc;
  if (X) {
    k_coeffs<<<1, 256, 0, s>>>(Yc, Linv, k, k, Zc);
    k_expand<<<blocks_of((size_t)k * n), 256, 0, s>>>(Zc, Xk, k, k, n, X);
  }
  return check_cuda(c, cudaGetLastError(), "mixed eigensolve");
}

int sym_eig_lowest(rsx_ctx* c, double* work, int n, int nroots, double* omega, double* X, cudaStream_t s) {
  const char* ev = getenv("RSX_EIG_FP64");
  if (n >= kMixedMinN && !(ev && atoi(ev) != 0)) return sym_eig_lowest_mixed(c, work, n, nroots, omega, X, s);
  return sym_eig_lowest_fp64(c, work, n, nroots, omega, X, s);
}

namespace {
// spin-polarised TDA matrix: alpha transitions [0, nta), beta [nta, nta + ntb)
__global__ void k_uhf_assemble(const double* __restrict__ eoa, int noa, const double* __restrict__ eva, int nva,
                               const double* __restrict__ eob, int nob, const double* __restrict__ evb, int nvb,
                               const double* __restrict__ K, const double* __restrict__ Kda,
                               const double* __restrict__ Kdb, double* __restrict__ A) {
  const int nta = noa * nva, ntb = nob * nvb, n = nta + ntb;
  const long long total = (long long)n * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int t = (int)(e / n), u = (int)(e - (long long)t * n);
    double v = 0.5 * (K[e] + K[(long long)u * n + t]);
    if (t < nta && u < nta) {
      if (Kda) v -= 0.5 * (Kda[(long long)t * nta + u] + Kda[(long long)u * nta + t]);
      if (t == u) v += eva[t % nva] - eoa[t / nva];
    } else if (t >= nta && u >= nta) {
      const int tb = t - nta, ub = u - nta;
      if (Kdb) v -= 0.5 * (Kdb[(long long)tb * ntb + ub] + Kdb[(long long)ub * ntb + tb]);
      if (tb == ub) v += evb[tb % nvb] - eob[tb / nvb];
    }
    A[e] = v;
  }
}
}  // namespace

int uhf_tda_solve(rsx_ctx* c, const double* eoa, int noa, const double* eva, int nva, const double* eob, int nob,
                  const double* evb, int nvb, const double* K, const double* Kda, const double* Kdb, int nroots,
                  double* omega, double* X, double* work, cudaStream_t s) {
  const int n = noa * nva + nob * nvb;
  ProfScope ps(c, kKEig, s);
  k_uhf_assemble<<<256, 256, 0, s>>>(eoa, noa, eva, nva, eob, nob, evb, nvb, K, Kda, Kdb, work);
  return sym_eig_lowest(c, work, n, nroots, omega, X, s);
}

int tda_solve(rsx_ctx* c, const double* eo, int no, const double* ev, int nv, const double* K, const double* Kd,
              double dm, int nroots, double* omega, double* X, double* work, cudaStream_t s) {
  const int n = no * nv;
  ProfScope ps(c, kKEig, s);
  k_tda_assemble<<<256, 256, 0, s>>>(eo, no, ev, nv, K, Kd, dm, work);
  return sym_eig_lowest(c, work, n, nroots, omega, X, s);
}

}  // namespace rsx
