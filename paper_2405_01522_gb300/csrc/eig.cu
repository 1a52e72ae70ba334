// FP64 symmetric eigen-solve of the Tamm-Dancoff matrix on the device (Eq. 7, Sec. 2:
// with B = 0 the problem A X = omega X is Hermitian; only the lowest roots are needed).
//
//   k_tda_assemble    A = diag(eps_a - eps_i) + delta_M K - K_d, symmetrised
//   k_tridiagonalise  Householder reduction A = Q T Q^T (one CTA; reflectors kept in A)
//   k_bisect          lowest nroots eigenvalues of T by Sturm-count bisection
//   k_eigvec          inverse iteration on T (with re-orthogonalisation inside clusters of
//                     close eigenvalues), then x = Q y
#include <cuda_runtime.h>

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
__device__ int sturm_count(const double* d, const double* e, int n, double x, double pivmin) {
  int cnt = 0;
  double q = d[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  if (q < 0) ++cnt;
  for (int i = 1; i < n; ++i) {
    q = d[i] - x - e[i - 1] * e[i - 1] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    if (q < 0) ++cnt;
  }
  return cnt;
}

// eigenvalue k (0-based, ascending) of T per thread, by bisection to full precision
__global__ void k_bisect(const double* __restrict__ d, const double* __restrict__ e, int n, int nroots,
                         double* __restrict__ w) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nroots) return;
  double lo = d[0], hi = d[0], emax = 0.0;
  for (int i = 0; i < n; ++i) {
    const double r = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i < n - 1 ? fabs(e[i]) : 0.0);
    lo = fmin(lo, d[i] - r);
    hi = fmax(hi, d[i] + r);
    if (i < n - 1) emax = fmax(emax, fabs(e[i]));
  }
  const double scale = fmax(fabs(lo), fabs(hi));
  const double pivmin = fmax(2.2250738585072014e-308, 1e-300 * fmax(1.0, emax * emax));
  lo -= 1e-12 * scale + 1e-300;
  hi += 1e-12 * scale + 1e-300;
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (sturm_count(d, e, n, mid, pivmin) > k)
      hi = mid;
    else
      lo = mid;
  }
  w[k] = 0.5 * (lo + hi);
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

size_t tda_work_doubles(int n, int nroots) { return (size_t)n * n + 10 * (size_t)n + (size_t)nroots * n + 8; }

int tda_solve(rsx_ctx* c, const double* eo, int no, const double* ev, int nv, const double* K, const double* Kd,
              double dm, int nroots, double* omega, double* X, double* work, cudaStream_t s) {
  const int n = no * nv;
  double* A = work;
  double* d = A + (size_t)n * n;
  double* e = d + n;
  double* tau = e + n;
  double* tw = tau + n;          // 2 n (tridiagonalisation), then 5 n (eigvec scratch needs 4 n + n ints)
  double* y = tw + 2 * n;        // nroots * n  (eigvec T-basis vectors)
  (void)y;
  ProfScope ps(c, kKEig, s);
  k_tda_assemble<<<256, 256, 0, s>>>(eo, no, ev, nv, K, Kd, dm, A);
  k_tridiagonalise<<<1, kEigThreads, 0, s>>>(A, n, d, e, tau, tw);
  k_bisect<<<(nroots + 127) / 128, 128, 0, s>>>(d, e, n, nroots, omega);
  if (X) {
    // eigvec scratch: 5 n doubles after the T-basis vectors
    double* yv = tw + 2 * n;
    double* sc = yv + (size_t)nroots * n;
    for (int k = 0; k < nroots; ++k) k_eigvec<<<1, kEigThreads, 0, s>>>(d, e, A, tau, n, omega, k, yv, X, sc);
  }
  return check_cuda(c, cudaGetLastError(), "tda eigensolve");
}

}  // namespace rsx
