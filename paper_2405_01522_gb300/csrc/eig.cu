// FP64 symmetric eigen-solve of the Tamm-Dancoff matrix on the device (Eq. 7, Sec. 2:
// with B = 0 the problem A X = omega X is Hermitian; only the lowest roots are needed).
//
//   k_tda_assemble    A = diag(eps_a - eps_i) + delta_M K - K_d, symmetrised
//   k_tridiag_coop    Householder reduction A = Q T Q^T, cooperative multi-CTA (reflectors
//                     kept in A); k_tridiagonalise is the one-CTA form for small n
//   k_multisect       lowest nroots eigenvalues of T by Sturm-count multisection
//   k_eigvec          inverse iteration on T (with re-orthogonalisation inside clusters of
//                     close eigenvalues), then x = Q y
#include <cuda_runtime.h>

#include <algorithm>

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
        __nanosleep(64);
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
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < nwarp; ++w) t += red[w];
    *out_sh = t;
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
        const double beta = -copysign(sqrt(alpha * alpha + xn2), alpha);
        sh_tau = (beta - alpha) / beta;
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
        double acc = 0.0;
        for (int j = m0 + lane; j < n; j += 32) acc += row[j] * vs[j];
        acc = warp_sum(acc);
        const double pi = tk * acc;
        if (lane == 0) {
          pp[i] = pi;
          pv_part += pi * vs[i];
        }
      }
    }
    if (lane == 0) red[warp] = pv_part;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < nwarp; ++w) t += red[w];
      part_pv[cta] = t;
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
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < nwarp; ++w) t += red[w];
      part_norm[cta] = t;
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

// Multisection: one CTA per root; each round evaluates the Sturm count at blockDim.x
// interior points of [lo, hi] and keeps the sub-interval where the count passes k.
__global__ void __launch_bounds__(256) k_multisect(const double* __restrict__ d, const double* __restrict__ e, int n,
                                                   double* __restrict__ w) {
  const int k = blockIdx.x;
  __shared__ double lo_sh, hi_sh;
  __shared__ int first_sh;
  if (threadIdx.x == 0) {
    double lo = d[0], hi = d[0];
    for (int i = 0; i < n; ++i) {
      const double r = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i < n - 1 ? fabs(e[i]) : 0.0);
      lo = fmin(lo, d[i] - r);
      hi = fmax(hi, d[i] + r);
    }
    const double scale = fmax(fabs(lo), fabs(hi));
    lo_sh = lo - 1e-12 * scale - 1e-300;
    hi_sh = hi + 1e-12 * scale + 1e-300;
  }
  __syncthreads();
  double emax = 0.0;
  for (int i = 0; i < n - 1; ++i) emax = fmax(emax, fabs(e[i]));
  const double pivmin = fmax(2.2250738585072014e-308, 1e-300 * fmax(1.0, emax * emax));
  const int T = blockDim.x;
  for (int round = 0; round < 12; ++round) {
    const double lo = lo_sh, hi = hi_sh;
    if (!(hi - lo > 2.0 * 2.220446049250313e-16 * fmax(fabs(lo), fabs(hi)))) break;
    const double x = lo + (hi - lo) * (double)(threadIdx.x + 1) / (double)(T + 1);
    const bool above = sturm_count(d, e, n, x, pivmin) > k;
    if (threadIdx.x == 0) first_sh = T;
    __syncthreads();
    if (above) atomicMin(&first_sh, (int)threadIdx.x);
    __syncthreads();
    if (threadIdx.x == 0) {
      const int f = first_sh;
      const double nlo = (f == 0) ? lo : lo + (hi - lo) * (double)f / (double)(T + 1);
      const double nhi = (f == T) ? hi : lo + (hi - lo) * (double)(f + 1) / (double)(T + 1);
      lo_sh = nlo;
      hi_sh = nhi;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) w[k] = 0.5 * (lo_sh + hi_sh);
}

// eigenvectors: one CTA per root, serial tridiagonal solves by thread 0, parallel
// back-transformation.  Roots are processed in ascending order by the launch loop on
// the host (one launch per root) so that a vector can be orthogonalised against the
// previous ones of its cluster.  y: [nroots][n] scratch (T basis); X: [nroots][n] out.
__global__ void __launch_bounds__(kEigThreads) k_eigvec(const double* __restrict__ d, const double* __restrict__ e,
                                                        const double* __restrict__ A, const double* __restrict__ tau,
                                                        int n, const double* __restrict__ w, int k, double* __restrict__ y,
                                                        double* __restrict__ X, double* __restrict__ scratch) {
  __shared__ double red[33];
  double* yk = y + (size_t)k * n;
  double* lu = scratch;  // 5 n doubles: diag, up, up2, low, rhs
  const double lam = w[k];
  double gap_tol = 1e-9;
  {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s = fmax(s, fabs(d[i]));
    gap_tol *= fmax(1.0, s);
  }
  // starting vector
  for (int i = threadIdx.x; i < n; i += blockDim.x) yk[i] = 1.0 + 0.001 * (double)((i * 7919 + k * 104729) % 997);
  __syncthreads();
  for (int iter = 0; iter < 4; ++iter) {
    if (threadIdx.x == 0) {
      // LU with partial pivoting of (T - lam I), solve in place in yk
      double* dg = lu;
      double* u1 = lu + n;
      double* u2 = lu + 2 * n;
      double* lw = lu + 3 * n;
      int* piv = reinterpret_cast<int*>(lu + 4 * n);
      const double eps_shift = 1e-14 * fmax(1.0, fabs(lam));
      for (int i = 0; i < n; ++i) {
        dg[i] = d[i] - lam;
        u1[i] = i < n - 1 ? e[i] : 0.0;
        u2[i] = 0.0;
      }
      for (int i = 0; i < n - 1; ++i) {
        const double sub = e[i];
        if (fabs(dg[i]) >= fabs(sub)) {
          piv[i] = 0;
          if (dg[i] == 0.0) dg[i] = eps_shift;
          const double l = sub / dg[i];
          lw[i] = l;
          dg[i + 1] -= l * u1[i];
        } else {
          piv[i] = 1;
          const double l = dg[i] / sub;
          lw[i] = l;
          // swap rows i and i+1
          const double t0 = dg[i + 1], t1 = (i + 1 < n - 1) ? u1[i + 1] : 0.0;
          dg[i] = sub;
          const double old_u1 = u1[i];
          u1[i] = t0;
          u2[i] = t1;
          dg[i + 1] = old_u1 - l * t0;
          if (i + 1 < n - 1) u1[i + 1] = -l * t1;
        }
      }
      if (dg[n - 1] == 0.0) dg[n - 1] = eps_shift;
      // forward: apply the row swaps and eliminations to the right-hand side
      for (int i = 0; i < n - 1; ++i) {
        if (piv[i]) {
          const double t = yk[i];
          yk[i] = yk[i + 1];
          yk[i + 1] = t - lw[i] * yk[i];
        } else {
          yk[i + 1] -= lw[i] * yk[i];
        }
      }
      // back substitution
      for (int i = n - 1; i >= 0; --i) {
        double s = yk[i];
        if (i + 1 < n) s -= u1[i] * yk[i + 1];
        if (i + 2 < n) s -= u2[i] * yk[i + 2];
        yk[i] = s / dg[i];
      }
    }
    __syncthreads();
    // orthogonalise against earlier roots of the same cluster, then normalise
    for (int j = 0; j < k; ++j) {
      if (fabs(w[j] - lam) > gap_tol * 1e3) continue;
      const double* yj = y + (size_t)j * n;
      double s = 0.0;
      for (int i = threadIdx.x; i < n; i += blockDim.x) s += yj[i] * yk[i];
      s = block_sum(s, red);
      for (int i = threadIdx.x; i < n; i += blockDim.x) yk[i] -= s * yj[i];
      __syncthreads();
    }
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += yk[i] * yk[i];
    s = block_sum(s, red);
    const double inv = 1.0 / sqrt(s);
    for (int i = threadIdx.x; i < n; i += blockDim.x) yk[i] *= inv;
    __syncthreads();
  }
  // x = H_0 H_1 ... H_{n-3} y ; H_k = I - tau_k v_k v_k^T, v_k[k+1] = 1, v_k[i] = A[i][k] (i > k+1)
  double* x = X + (size_t)k * n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] = yk[i];
  __syncthreads();
  for (int kk = n - 3; kk >= 0; --kk) {
    const double tk = tau[kk];
    if (tk == 0.0) continue;
    double s = 0.0;
    for (int i = kk + 1 + threadIdx.x; i < n; i += blockDim.x) {
      const double vi = (i == kk + 1) ? 1.0 : A[(size_t)i * n + kk];
      s += vi * x[i];
    }
    s = tk * block_sum(s, red);
    for (int i = kk + 1 + threadIdx.x; i < n; i += blockDim.x) {
      const double vi = (i == kk + 1) ? 1.0 : A[(size_t)i * n + kk];
      x[i] -= s * vi;
    }
    __syncthreads();
  }
}

}  // namespace

// start of the scratch that follows the eigenvector area (see tda_solve's layout)
static double* y_end(double* tw, int n, int nroots) { return tw + 2 * n + (size_t)nroots * n + 5 * (size_t)n; }

size_t tda_work_doubles(int n, int nroots) {
  return (size_t)n * n + 14 * (size_t)n + (size_t)nroots * n + 4096;
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
  const int G = std::min(std::min(c->nsm * std::max(per_sm, 0), 128), std::max(1, n / 2));
  if (coop && per_sm > 0 && n >= 64) {
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
  k_multisect<<<nroots, 256, 0, s>>>(d, e, n, omega);
  if (X) {
    // eigvec scratch: 5 n doubles after the T-basis vectors
    double* yv = tw + 2 * n;
    double* sc = yv + (size_t)nroots * n;
    for (int k = 0; k < nroots; ++k) k_eigvec<<<1, kEigThreads, 0, s>>>(d, e, A, tau, n, omega, k, yv, X, sc);
  }
  return check_cuda(c, cudaGetLastError(), "symmetric eigensolve");
}

int tda_solve(rsx_ctx* c, const double* eo, int no, const double* ev, int nv, const double* K, const double* Kd,
              double dm, int nroots, double* omega, double* X, double* work, cudaStream_t s) {
  const int n = no * nv;
  ProfScope ps(c, kKEig, s);
  k_tda_assemble<<<256, 256, 0, s>>>(eo, no, ev, nv, K, Kd, dm, work);
  return sym_eig_lowest(c, work, n, nroots, omega, X, s);
}

}  // namespace rsx
