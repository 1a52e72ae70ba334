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
// k_tridiagonalise).  Rows are dealt cyclically to the CTAs; per step three grid-wide
// barriers separate (v) -> (p = tau A22 v, p^T v partials) -> (rank-2 update of own rows
// and the next column's norm partials).  The kernel is launched cooperatively so that
// all CTAs are resident; the barrier itself is bounded and raises RSX_ETIMEOUT.
constexpr uint32_t kGridWaitLimit = 1u << 24;

struct GridBar {
  unsigned int count;
  volatile unsigned int gen;
  volatile int abort;
};

__device__ __forceinline__ bool grid_barrier(GridBar* gb, unsigned int nblocks) {
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
        if (gb->abort || ++i > kGridWaitLimit) {
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

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// sum of the G per-CTA partials, by the whole CTA (one L2 round trip, shuffle reduction)
__device__ __forceinline__ double cta_sum_partials(const double* part, unsigned int G, double* red, double* out_sh) {
  double v = 0.0;
  for (unsigned int c = threadIdx.x; c < G; c += blockDim.x) v += __ldcg(part + c);
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {   // a shuffle tree, not a serial chain of dependent FP64 adds
    double t = lane < nwarp ? red[lane] : 0.0;
    t = warp_sum(t);
    if (lane == 0) *out_sh = t;
  }
  __syncthreads();
  return *out_sh;
}

// scratch layout (doubles): v[n], p[n], part_norm[G], part_pv[G], alpha
__global__ void __launch_bounds__(256) k_tridiag_coop(double* __restrict__ A, int n, double* __restrict__ d,
                                                      double* __restrict__ e, double* __restrict__ tau,
                                                      double* __restrict__ scr, GridBar* gb, int* status) {
  const unsigned int G = gridDim.x;
  const int cta = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  double* vv = scr;
  double* pp = scr + n;
  double* part_norm = scr + 2 * n;
  double* part_pv = part_norm + G;
  double* alpha_g = part_pv + G;
  extern __shared__ double tri_smem[];   // local copies of v and p (2 n doubles)
  double* vs = tri_smem;
  double* ps = tri_smem + n;
  __shared__ double red[8];
  __shared__ double sh_tau, sh_beta, sh_scale, sh_sum;
  bool live = true;

  // norm partials of column 0 below the subdiagonal, alpha of column 0
  {
    double s = 0.0;
    for (int i = first_owned(2, cta, G); i < n; i += G)
      if (threadIdx.x == 0) s += A[(size_t)i * n] * A[(size_t)i * n];
    if (threadIdx.x == 0) {
      part_norm[cta] = s;
      if (n > 1 && 1 % (int)G == cta) *alpha_g = A[(size_t)1 * n];
    }
  }
  live = grid_barrier(gb, G);

  for (int k = 0; k + 2 < n && live; ++k) {
    const int m0 = k + 1;
    // ---- reflector (every CTA computes the same scalars)
    const double xn2 = cta_sum_partials(part_norm, G, red, &sh_sum);
    if (threadIdx.x == 0) {
      const double alpha = __ldcg(alpha_g);
      if (xn2 == 0.0) {
        sh_tau = 0.0;
        sh_beta = alpha;
        sh_scale = 0.0;
      } else {
        // beta = -sign(alpha) |x|, tau = 1 + |alpha| / |x|: one rsqrt, one division
        const double s2 = alpha * alpha + xn2, rs = rsqrt(s2);
        const double beta = -copysign(s2 * rs, alpha);
        sh_tau = 1.0 + fabs(alpha) * rs;
        sh_scale = 1.0 / (alpha - beta);
        sh_beta = beta;
      }
      if (cta == 0) {
        e[k] = sh_beta;
        tau[k] = sh_tau;
      }
      if (k % (int)G == cta) d[k] = A[(size_t)k * n + k];
    }
    __syncthreads();
    const double tk = sh_tau, sc = sh_scale;
    // own rows: v_i, stored in the column for the back-transformation
    for (int i = first_owned(m0, cta, G) + (int)G * threadIdx.x; i < n; i += (int)G * blockDim.x) {
      const double vi = (i == m0) ? 1.0 : A[(size_t)i * n + k] * sc;
      vv[i] = vi;
      if (i > m0) A[(size_t)i * n + k] = vi;
    }
    if (!(live = grid_barrier(gb, G))) break;
    // ---- p_i = tau (A22 v)_i for own rows, partial p^T v
    double pv_part = 0.0;
    if (tk != 0.0) {
      for (int j = m0 + threadIdx.x; j < n; j += blockDim.x) vs[j] = __ldcg(vv + j);
      __syncthreads();
      int r = 0;
      for (int i = first_owned(m0, cta, G); i < n; i += G, ++r) {
        if (r % nwarp != warp) continue;
        const double* row = A + (size_t)i * n;
        double a0 = 0.0, a1 = 0.0;   // two chains
        int j = m0 + lane;
        for (; j + 32 < n; j += 64) {
          a0 += row[j] * vs[j];
          a1 += row[j + 32] * vs[j + 32];
        }
        if (j < n) a0 += row[j] * vs[j];
        const double acc = warp_sum(a0 + a1);
        const double pi = tk * acc;
        if (lane == 0) {
          pp[i] = pi;
          pv_part += pi * vs[i];
        }
      }
    }
    if (lane == 0) red[warp] = pv_part;
    __syncthreads();
    if (warp == 0) {
      const double t = warp_sum(lane < nwarp ? red[lane] : 0.0);
      if (lane == 0) part_pv[cta] = t;
    }
    if (!(live = grid_barrier(gb, G))) break;
    // ---- w = p - (tau/2)(p^T v) v ; A22 -= v w^T + w v^T on own rows; next column norm
    double nrm_part = 0.0;
    if (tk != 0.0) {
      const double pvs = cta_sum_partials(part_pv, G, red, &sh_sum);
      const double cc = 0.5 * tk * pvs;
      for (int j = m0 + threadIdx.x; j < n; j += blockDim.x) ps[j] = __ldcg(pp + j) - cc * vs[j];   // w
      __syncthreads();
      int r = 0;
      for (int i = first_owned(m0, cta, G); i < n; i += G, ++r) {
        if (r % nwarp != warp) continue;
        const double vi = vs[i];
        const double wi = ps[i];
        double* row = A + (size_t)i * n;
        for (int j = m0 + lane; j < n; j += 32) row[j] -= vi * ps[j] + wi * vs[j];
        __syncwarp();
        if (lane == 0) {
          const double x = row[m0];   // column k + 1 of row i
          if (i >= m0 + 2) nrm_part += x * x;
          if (i == m0 + 1) *alpha_g = x;
        }
      }
    } else {
      int r = 0;
      for (int i = first_owned(m0, cta, G); i < n; i += G, ++r) {
        if (r % nwarp != warp || lane != 0) continue;
        const double x = A[(size_t)i * n + m0];
        if (i >= m0 + 2) nrm_part += x * x;
        if (i == m0 + 1) *alpha_g = x;
      }
    }
    if (lane == 0) red[warp] = nrm_part;
    __syncthreads();
    if (warp == 0) {
      const double t = warp_sum(lane < nwarp ? red[lane] : 0.0);
      if (lane == 0) part_norm[cta] = t;
    }
    live = grid_barrier(gb, G);
  }
  if (cta == 0 && threadIdx.x == 0) {
    if (!live) {
      if (status) atomicMax(status, RSX_ETIMEOUT);
    } else {
      if (n >= 2) {
        d[n - 2] = __ldcg(A + (size_t)(n - 2) * n + (n - 2));
        e[n - 2] = __ldcg(A + (size_t)(n - 1) * n + (n - 2));
        if (n >= 3) tau[n - 2] = 0.0;
      }
      d[n - 1] = __ldcg(A + (size_t)(n - 1) * n + (n - 1));
    }
  }
}

// ---------------------------------------------------------------------------------
// Householder tridiagonalisation on one thread-block cluster (same reflectors and outputs
// as k_tridiagonalise).  The matrix lives in the CTAs' shared memory: rows dealt
// cyclically (row i in CTA i % CS, local row i / CS); v, p/w and the per-CTA partial sums
// are replicated in every CTA, which writes its own entries into all the others through
// distributed shared memory.  Per step three hardware cluster barriers separate
// (norm partials -> v) -> (p = tau A22 v, p^T v partials) -> (rank-2 update of own rows,
// next column's norm partials).  The rows are copied back to global memory at the end
// (the reflectors below the subdiagonal, for the back-transformation).
constexpr int kClThreads = 512;
namespace cg = cooperative_groups;

__global__ void __launch_bounds__(kClThreads) k_tridiag_cluster(double* __restrict__ A, int n, double* __restrict__ d,
                                                                double* __restrict__ e, double* __restrict__ tau) {
  cg::cluster_group cl = cg::this_cluster();
  const int CS = (int)cl.num_blocks();
  const int me = (int)cl.block_rank();
  const int nloc = (n - me + CS - 1) / CS;          // rows me, me + CS, ...
  const int lda = n;
  extern __shared__ double cl_smem[];
  double* R = cl_smem;                               // [nloc][n]
  double* v = R + (size_t)((n + CS - 1) / CS) * n;   // [n]
  double* p = v + n;                                 // [n] (p, then w)
  double* part = p + n;                              // [CS] norm partials, [CS] p^T v partials, alpha
  double* part2 = part + CS;
  double* alpha_sl = part2 + CS;
  __shared__ double red[kClThreads / 32];
  __shared__ double sh_tau, sh_beta, sh_scale;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = kClThreads / 32;
  auto grow = [&](int li) { return me + li * CS; };
  for (size_t q = tid; q < (size_t)nloc * n; q += kClThreads) {
    const int li = (int)(q / n), j = (int)(q - (size_t)li * n);
    R[q] = A[(size_t)grow(li) * lda + j];
  }
  __syncthreads();
  // block-wide sum of one value per thread, result to thread 0 (trees throughout: a
  // dependent FP64 add costs hundreds of cycles on this part)
  auto block_sum0 = [&](double x) {
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) red[warp] = x;
    __syncthreads();
    double t = 0.0;
    if (warp == 0) {
      t = lane < nw ? red[lane] : 0.0;
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    __syncthreads();
    return t;
  };
  // publish this CTA's partial (and alpha when it owns row m0 + 1) for column c
  auto publish_norm = [&](int c) {
    double s = 0.0;
    for (int li = tid; li < nloc; li += kClThreads) {
      const int i = grow(li);
      if (i >= c + 2) s += R[(size_t)li * n + c] * R[(size_t)li * n + c];
    }
    const double t = block_sum0(s);
    if (tid == 0) red[0] = t;
    __syncthreads();
    const double tot = red[0];
    if (tid < CS) *cl.map_shared_rank(part + me, tid) = tot;
    if ((c + 1) % CS == me && tid >= 32 && tid < 32 + CS)
      *cl.map_shared_rank(alpha_sl, tid - 32) = R[(size_t)((c + 1) / CS) * n + c];
  };
  if (n > 2) publish_norm(0);
  cl.sync();
  for (int k = 0; k + 2 < n; ++k) {
    const int m0 = k + 1;
    if (warp == 0) {
      double xn2 = lane < CS ? part[lane] : 0.0;
      for (int o = 16; o > 0; o >>= 1) xn2 += __shfl_xor_sync(0xffffffffu, xn2, o);
      if (lane == 0) {
        const double alpha = *alpha_sl;
        if (xn2 == 0.0) {
          sh_tau = 0.0;
          sh_beta = alpha;
          sh_scale = 0.0;
        } else {
          // beta = -sign(alpha) |x|, tau = (beta - alpha) / beta = 1 + |alpha| / |x|:
          // one reciprocal square root and one division
          const double s2 = alpha * alpha + xn2, rs = rsqrt(s2);
          const double beta = -copysign(s2 * rs, alpha);
          sh_tau = 1.0 + fabs(alpha) * rs;
          sh_scale = 1.0 / (alpha - beta);
          sh_beta = beta;
        }
        if (me == 0) {
          e[k] = sh_beta;
          tau[k] = sh_tau;
        }
        if (k % CS == me) d[k] = R[(size_t)(k / CS) * n + k];
      }
    }
    __syncthreads();
    const double tk = sh_tau, sc = sh_scale;
    // v on own rows (stored in the column), sent to every CTA
    for (int q = tid; q < nloc * CS; q += kClThreads) {
      const int li = q / CS, dst = q - li * CS;
      const int i = grow(li);
      if (i < m0) continue;
      const double vi = (i == m0) ? 1.0 : R[(size_t)li * n + k] * sc;
      *cl.map_shared_rank(v + i, dst) = vi;
    }
    cl.sync();
    for (int li = tid; li < nloc; li += kClThreads) {
      const int i = grow(li);
      if (i > m0) R[(size_t)li * n + k] = v[i];
    }
    if (tk != 0.0) {
      // p_i = tau (A22 v)_i on own rows, a warp per row; p^T v partial
      double pv = 0.0;
      for (int li = warp; li < nloc; li += nw) {
        const int i = grow(li);
        if (i < m0) continue;
        const double* row = R + (size_t)li * n;
        double a0 = 0.0, a1 = 0.0;   // two chains
        int j = m0 + lane;
        for (; j + 32 < n; j += 64) {
          a0 += row[j] * v[j];
          a1 += row[j + 32] * v[j + 32];
        }
        if (j < n) a0 += row[j] * v[j];
        double acc = a0 + a1;
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        const double pi = tk * acc;
        if (lane < CS) *cl.map_shared_rank(p + i, lane) = pi;
        if (lane == 0) pv += pi * v[i];
      }
      const double t = block_sum0(pv);
      if (tid == 0) red[0] = t;
      __syncthreads();
      if (tid < CS) *cl.map_shared_rank(part2 + me, tid) = red[0];
      cl.sync();
      // w = p - (tau/2)(p^T v) v, rank-2 update of own rows
      double pvs = lane < CS ? part2[lane] : 0.0;   // every warp reduces the CS partials
      for (int o = 16; o > 0; o >>= 1) pvs += __shfl_xor_sync(0xffffffffu, pvs, o);
      const double cc = 0.5 * tk * pvs;
      for (int j = m0 + tid; j < n; j += kClThreads) p[j] -= cc * v[j];
      __syncthreads();
      for (int li = warp; li < nloc; li += nw) {
        const int i = grow(li);
        if (i < m0) continue;
        const double vi = v[i], wi = p[i];
        double* row = R + (size_t)li * n;
        for (int j = m0 + lane; j < n; j += 32) row[j] -= vi * p[j] + wi * v[j];
      }
      __syncthreads();
    } else {
      cl.sync();   // matches the p-broadcast barrier of the other branch (tau is the same everywhere)
    }
    if (m0 + 2 < n) publish_norm(m0);
    cl.sync();
  }
  // last 2 x 2 block, rows back to global memory
  if (tid == 0) {
    if (n >= 2) {
      if ((n - 2) % CS == me) d[n - 2] = R[(size_t)((n - 2) / CS) * n + (n - 2)];
      if ((n - 1) % CS == me) e[n - 2] = R[(size_t)((n - 1) / CS) * n + (n - 2)];
      if (me == 0 && n >= 3) tau[n - 2] = 0.0;
    }
    if ((n - 1) % CS == me) d[n - 1] = R[(size_t)((n - 1) / CS) * n + (n - 1)];
  }
  for (size_t q = tid; q < (size_t)nloc * n; q += kClThreads) {
    const int li = (int)(q / n), j = (int)(q - (size_t)li * n);
    A[(size_t)grow(li) * lda + j] = R[q];
  }
  cl.sync();   // no CTA leaves while others may still address its shared memory
}

// Lowest roots of the tridiagonal T (d, e), a warp per root: each round evaluates the
// Sturm count at 32 interior points of [lo, hi] (one per lane) and keeps the sub-interval
// in which the count passes k (FP64 is scarce on this part: 32 points per root and round
// instead of a whole CTA).
__global__ void __launch_bounds__(32) k_multisect(const double* __restrict__ d, const double* __restrict__ e, int n,
                                                   int nroots, double* __restrict__ w) {
  extern __shared__ double ms_smem[];   // d (n), e^2 (n)
  const int lane = threadIdx.x & 31;
  const int k = blockIdx.x;   // one warp (CTA) per root: spread over SMs, FP64 units are scarce
  if (k >= nroots) return;
  double* ds = ms_smem;
  double* e2 = ms_smem + n;
  for (int i = lane; i < n; i += 32) {
    ds[i] = d[i];
    e2[i] = i < n - 1 ? e[i] * e[i] : 0.0;
  }
  __syncwarp();
  double lo = 1e300, hi = -1e300, emax = 0.0;
  for (int i = lane; i < n; i += 32) {
    const double r = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i < n - 1 ? fabs(e[i]) : 0.0);
    lo = fmin(lo, d[i] - r);
    hi = fmax(hi, d[i] + r);
    if (i < n - 1) emax = fmax(emax, fabs(e[i]));
  }
  for (int o = 16; o > 0; o >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    emax = fmax(emax, __shfl_xor_sync(0xffffffffu, emax, o));
  }
  const double scale = fmax(fabs(lo), fabs(hi));
  lo -= 1e-12 * scale + 1e-300;
  hi += 1e-12 * scale + 1e-300;
  for (int round = 0; round < 16; ++round) {
    if (!(hi - lo > 2.0 * 2.220446049250313e-16 * fmax(fabs(lo), fabs(hi)))) break;
    const double x = lo + (hi - lo) * (double)(lane + 1) / 33.0;
    const unsigned above = __ballot_sync(0xffffffffu, sturm_count_prod(ds, e2, n, x) > k);
    const int f = above ? __ffs(above) - 1 : 32;
    const double nlo = (f == 0) ? lo : lo + (hi - lo) * (double)f / 33.0;
    const double nhi = (f == 32) ? hi : lo + (hi - lo) * (double)(f + 1) / 33.0;
    lo = nlo;
    hi = nhi;
  }
  if (lane == 0) w[k] = 0.5 * (lo + hi);
}

// Eigenvectors of T by inverse iteration, a warp per root (3 iterations from a fixed
// start); y: [nroots][n]; scratch: 4 n doubles + n ints per root.
__global__ void __launch_bounds__(32) k_invit(const double* __restrict__ d, const double* __restrict__ e, int n,
                                               const double* __restrict__ w, int nroots, double* __restrict__ y,
                                               double* __restrict__ scratch) {
  const int lane = threadIdx.x & 31;
  const int k = blockIdx.x;   // one warp (CTA) per root: spread over SMs, FP64 units are scarce
  if (k >= nroots) return;
  double* z = y + (size_t)k * n;
  double* sc = scratch + (size_t)k * 5 * n;
  for (int i = lane; i < n; i += 32) z[i] = 1.0 + 0.001 * (double)((i * 7919 + k * 104729) % 997);
  __syncwarp();
  warp_inverse_iteration(d, e, n, w[k], z, sc, reinterpret_cast<int*>(sc + 4 * n), 3, y, n, 0u);
}

// Roots closer than the cluster gap to an earlier root are recomputed one after another
// (one warp), each orthogonalised inside every iteration against the earlier roots of
// its cluster, so that (nearly) degenerate roots get orthonormal vectors.
__global__ void k_invit_clusters(const double* __restrict__ d, const double* __restrict__ e, int n,
                                 const double* __restrict__ w, int nroots, double* __restrict__ y,
                                 double* __restrict__ scratch) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int i = lane; i < n; i += 32) s = fmax(s, fabs(d[i]));
  for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_xor_sync(0xffffffffu, s, o));
  const double gap = 1e-6 * fmax(1.0, s);
  int* piv = reinterpret_cast<int*>(scratch + 4 * n);
  for (int r = 1; r < nroots; ++r) {
    bool clustered = false;
    for (int j = 0; j < r; ++j) clustered |= fabs(w[r] - w[j]) < gap;
    if (!clustered) continue;
    double* z = y + (size_t)r * n;
    for (int i = lane; i < n; i += 32) z[i] = 1.0 + 0.001 * (double)((i * 7919 + r * 104729) % 997);
    __syncwarp();
    if (lane == 0) tri_factor_shifted(d, e, n, w[r], scratch, piv);
    __syncwarp();
    for (int it = 0; it < 3; ++it) {
      if (lane == 0) tri_solve_factored(n, z, scratch, piv);
      __syncwarp();
      for (int j = 0; j < r; ++j) {
        if (!(fabs(w[r] - w[j]) < gap)) continue;
        const double* zj = y + (size_t)j * n;
        double dot = 0.0;
        for (int i = lane; i < n; i += 32) dot += zj[i] * z[i];
        dot = warp_sum(dot);
        for (int i = lane; i < n; i += 32) z[i] -= dot * zj[i];
        __syncwarp();
      }
      double nn = 0.0;
      for (int i = lane; i < n; i += 32) nn += z[i] * z[i];
      nn = warp_sum(nn);
      const double inv = nn > 0.0 ? 1.0 / sqrt(nn) : 0.0;
      for (int i = lane; i < n; i += 32) z[i] *= inv;
      __syncwarp();
    }
  }
}

// Reflector vectors moved to rows: A[j][i] = A[i][j] for i > j + 1 (the strict upper
// triangle past the superdiagonal is dead after the reduction), so that the
// back-transformation reads each reflector contiguously.  32 x 32 tiles through shared
// memory.
__global__ void k_reflectors_to_rows(double* __restrict__ A, int n) {
  __shared__ double tile[32][33];
  const int j0 = blockIdx.x * 32, i0 = blockIdx.y * 32;   // source tile: rows i0.., columns j0..
  if (i0 + 31 < j0 + 2) return;                          // no entry with i > j + 1
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 8 rows per pass
  for (int r = ty; r < 32; r += 8) {
    const int i = i0 + r, j = j0 + tx;
    tile[r][tx] = (i < n && j < n && i > j + 1) ? A[(size_t)i * n + j] : 0.0;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int j = j0 + r, i = i0 + tx;   // destination A[j][i]
    if (i < n && j < n && i > j + 1) A[(size_t)j * n + i] = tile[tx][r];
  }
}

// x_k = H_0 H_1 ... H_{n-3} y_k, one warp (CTA) per root, x in shared memory;
// H_j = I - tau_j v_j v_j^T, v_j[j+1] = 1, v_j[i] = A[j][i] (i > j + 1, rows form)
__global__ void __launch_bounds__(32) k_backtransform(const double* __restrict__ A, const double* __restrict__ tau,
                                                      int n, const double* __restrict__ y, int nroots,
                                                      double* __restrict__ X) {
  extern __shared__ double xs_bt[];
  const int lane = threadIdx.x & 31;
  const int k = blockIdx.x;
  if (k >= nroots) return;
  double* x = xs_bt;
  for (int i = lane; i < n; i += 32) x[i] = y[(size_t)k * n + i];
  __syncwarp();
  for (int kk = n - 3; kk >= 0; --kk) {
    const double tk = tau[kk];
    if (tk == 0.0) continue;
    const double* v = A + (size_t)kk * n;
    double s = (lane == 0) ? x[kk + 1] : 0.0;
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
static double* y_end(double* tw, int n, int nroots) { return tw + 2 * n + (size_t)nroots * n + 5 * (size_t)nroots * n; }

size_t tda_work_doubles(int n, int nroots) {
  return (size_t)n * n + 14 * (size_t)n + 6 * (size_t)nroots * n + 4096;
}

int sym_eig_lowest(rsx_ctx* c, double* work, int n, int nroots, double* omega, double* X, cudaStream_t s) {
  double* A = work;
  double* d = A + (size_t)n * n;
  double* e = d + n;
  double* tau = e + n;
  double* tw = tau + n;          // 2 n (tridiagonalisation), then 5 n (eigvec scratch needs 4 n + n ints)
  // cooperative multi-CTA reduction when the device supports it, one CTA otherwise
  int coop = 0, per_sm = 0;
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, c->device);
  cudaFuncSetAttribute(k_tridiag_coop, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(2 * (size_t)n * sizeof(double)));
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tridiag_coop, 256, 2 * (size_t)n * sizeof(double));
  // fewer CTAs make each grid barrier cheaper; the FP64 work per step is small
  int gcap = 64;
  if (const char* ev = getenv("RSX_TRIDIAG_CTAS")) gcap = std::max(1, atoi(ev));
  const int G = std::min(std::min(c->nsm * std::max(per_sm, 0), gcap), std::max(1, n / 2));
  // one thread-block cluster with the matrix in distributed shared memory when it fits
  // (16 CTAs, non-portable size, else 8), else the cooperative grid, else one CTA
  bool done = false;
  for (int CS : {16, 8}) {
    if (done || n < 64) break;
    const size_t smem = (((size_t)(n + CS - 1) / CS) * n + 2 * (size_t)n + 2 * CS + 1) * sizeof(double);
    if (smem > (size_t)227 * 1024) continue;
    if (cudaFuncSetAttribute(k_tridiag_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        (CS > 8 && cudaFuncSetAttribute(k_tridiag_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)) {
      cudaGetLastError();
      continue;
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
    if (cudaOccupancyMaxActiveClusters(&ncl, k_tridiag_cluster, &cfg) != cudaSuccess || ncl < 1) {
      cudaGetLastError();
      continue;
    }
    const cudaError_t err = cudaLaunchKernelEx(&cfg, k_tridiag_cluster, A, n, d, e, tau);
    if (err != cudaSuccess) return check_cuda(c, err, "cluster tridiagonalisation");
    done = true;
  }
  if (done) {
  } else if (coop && per_sm > 0 && n >= 64) {
    double* scr = y_end(tw, n, nroots);            // v, p, partials, alpha
    GridBar* gb = reinterpret_cast<GridBar*>(scr + 2 * n + 2 * 1024 + 2);
    cudaMemsetAsync(gb, 0, sizeof(GridBar), s);
    void* args[] = {(void*)&A, (void*)&n, (void*)&d, (void*)&e, (void*)&tau, (void*)&scr, (void*)&gb,
                    (void*)&c->status};
    const size_t smem = 2 * (size_t)n * sizeof(double);
    cudaFuncSetAttribute(k_tridiag_coop, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaError_t err = cudaLaunchCooperativeKernel((const void*)k_tridiag_coop, dim3(G), dim3(256), args, smem, s);
    if (err != cudaSuccess) return check_cuda(c, err, "cooperative tridiagonalisation");
  } else {
    k_tridiagonalise<<<1, kEigThreads, 0, s>>>(A, n, d, e, tau, tw);
  }
  cudaFuncSetAttribute(k_multisect, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(2 * (size_t)n * sizeof(double)));
  k_multisect<<<nroots, 32, 2 * (size_t)n * sizeof(double), s>>>(d, e, n, nroots, omega);
  if (X) {
    double* yv = tw + 2 * n;                       // T-basis vectors
    double* sc = yv + (size_t)nroots * n;          // 5 n per root
    k_invit<<<nroots, 32, 0, s>>>(d, e, n, omega, nroots, yv, sc);
    k_invit_clusters<<<1, 32, 0, s>>>(d, e, n, omega, nroots, yv, sc);
    k_reflectors_to_rows<<<dim3((n + 31) / 32, (n + 31) / 32), 256, 0, s>>>(A, n);
    const size_t smem = (size_t)n * sizeof(double);
    cudaFuncSetAttribute(k_backtransform, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_backtransform<<<nroots, 32, smem, s>>>(A, tau, n, yv, nroots, X);
  }
  return check_cuda(c, cudaGetLastError(), "symmetric eigensolve");
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
