// Absorption spectrum and full (non-Tamm-Dancoff) TDHF on the device (FP64 results).
//
//   rsx_casida_dipoles     <i|r_d|a> = h^3 sum_r phi_i r_d phi_a (the single-particle
//                          matrix elements of Eq. 8), three weighted Gram products
//   rsx_casida_oscillator  d_k = sum_t X[k][t] <t|r|> (Eq. 8), f_k = 2/3 omega_k |d_k|^2
//                          (Eq. 9, atomic units)
//   rsx_strength_function  S(w) = sum_k f_k L(w - omega_k) (Eq. 10), Lorentzian of
//                          half-width gamma
//   rsx_casida_solve_full  Eq. 3 for real orbitals in the half-size symmetric form:
//                          A - B = L L^T (blocked Cholesky), M = L^T (A + B) L,
//                          M z = omega^2 z (Householder + multisection + inverse
//                          iteration, eig.cu), X + Y = omega^{-1/2} L z.  B is the RHF
//                          form delta_M (ia|bj) - (ib|aj) = delta_M K[ia,jb] - K[ib,ja].
#include <cuda_runtime.h>

#include <cmath>

#include "../../include/rsx.h"
#include "api_internal.cuh"
#include "dense.cuh"
#include "eig.cuh"

using namespace rsx;

namespace {

constexpr int kChB = 32;   // Cholesky block

// pos[d][v] = (coordinate d of grid point v): ((x - nx/2) h, (y - ny/2) h, (z - nz/2) h)
template <typename R>
__global__ void k_positions(int nz, int ny, int nx, double h, R* __restrict__ pos) {
  const size_t N = (size_t)nz * ny * nx;
  for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < N; v += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(v % nx), y = (int)((v / nx) % ny), z = (int)(v / ((size_t)nx * ny));
    pos[v] = (R)((x - 0.5 * nx) * h);
    pos[N + v] = (R)((y - 0.5 * ny) * h);
    pos[2 * N + v] = (R)((z - 0.5 * nz) * h);
  }
}

// one warp per root: d = sum_t X[k][t] dip[:, t], f_k = 2/3 omega_k |d|^2
__global__ void k_oscillator(const double* __restrict__ omega, const double* __restrict__ X, int nroots, int nt,
                             const double* __restrict__ dip, double* __restrict__ f) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= nroots) return;
  double d0 = 0.0, d1 = 0.0, d2 = 0.0;
  for (int t = lane; t < nt; t += 32) {
    const double x = X[(size_t)warp * nt + t];
    d0 += x * dip[t];
    d1 += x * dip[nt + t];
    d2 += x * dip[2 * nt + t];
  }
  for (int o = 16; o > 0; o >>= 1) {
    d0 += __shfl_xor_sync(0xffffffffu, d0, o);
    d1 += __shfl_xor_sync(0xffffffffu, d1, o);
    d2 += __shfl_xor_sync(0xffffffffu, d2, o);
  }
  if (lane == 0) f[warp] = (2.0 / 3.0) * omega[warp] * (d0 * d0 + d1 * d1 + d2 * d2);
}

__global__ void k_strength(const double* __restrict__ omega, const double* __restrict__ f, int nroots, double gamma,
                           const double* __restrict__ grid, int ngrid, double* __restrict__ S) {
  const double inv_pi = 0.31830988618379067154;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < ngrid; j += gridDim.x * blockDim.x) {
    const double w = grid[j];
    double s = 0.0;
    for (int k = 0; k < nroots; ++k) {
      const double x = w - omega[k];
      s += f[k] * gamma * inv_pi / (x * x + gamma * gamma);
    }
    S[j] = s;
  }
}

// AmB = A - B, ApB = A + B (n x n), A = diag(de) + dm K - Kd, B = dm K - Kx,
// Kx[ia, jb] = K[ib, ja]; both symmetrised
__global__ void k_tdhf_assemble(const double* __restrict__ eo, int no, const double* __restrict__ ev, int nv,
                                const double* __restrict__ K, const double* __restrict__ Kd, double dm,
                                double* __restrict__ AmB, double* __restrict__ ApB) {
  const int n = no * nv;
  const long long total = (long long)n * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int t = (int)(e / n), s = (int)(e - (long long)t * n);
    const int i = t / nv, a = t - i * nv, j = s / nv, b = s - j * nv;
    const long long et = (long long)s * n + t;
    const double k = 0.5 * (K[e] + K[et]);
    const long long x1 = (long long)(i * nv + b) * n + (j * nv + a), x2 = (long long)(j * nv + a) * n + (i * nv + b);
    const double kx = 0.5 * (K[x1] + K[x2]);
    const double kd = Kd ? 0.5 * (Kd[e] + Kd[et]) : 0.0;
    const double diag = (t == s) ? ev[a] - eo[i] : 0.0;
    const double A = diag + dm * k - kd;
    const double B = dm * k - kx;
    AmB[e] = A - B;
    ApB[e] = A + B;
  }
}

// Cholesky step jb (one CTA): factor the diagonal block and solve the panel below it.
// Rows below: L[i][jb + c] = (A[i][jb + c] - sum_{p<c} L[i][jb+p] L11[c][p]) / L11[c][c].
__global__ void __launch_bounds__(256) k_potrf_panel(double* __restrict__ L, int n, int jb, int* status) {
  __shared__ double D[kChB][kChB + 1];
  const int b = min(kChB, n - jb);
  for (int q = threadIdx.x; q < b * b; q += blockDim.x) {
    const int r = q / b, c = q - r * b;
    D[r][c] = L[(size_t)(jb + r) * n + jb + c];
  }
  __syncthreads();
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  for (int j = 0; j < b; ++j) {
    if (threadIdx.x == 0) {
      double d = D[j][j];
      for (int p = 0; p < j; ++p) d -= D[j][p] * D[j][p];
      if (!(d > 0.0)) {
        bad = 1;
        d = 1.0;
      }
      D[j][j] = sqrt(d);
    }
    __syncthreads();
    for (int i = j + 1 + threadIdx.x; i < b; i += blockDim.x) {
      double s = D[i][j];
      for (int p = 0; p < j; ++p) s -= D[i][p] * D[j][p];
      D[i][j] = s / D[j][j];
    }
    __syncthreads();
  }
  for (int q = threadIdx.x; q < b * b; q += blockDim.x) {
    const int r = q / b, c = q - r * b;
    L[(size_t)(jb + r) * n + jb + c] = c <= r ? D[r][c] : 0.0;
  }
  for (int i = jb + b + threadIdx.x; i < n; i += blockDim.x) {
    double x[kChB];
    double* row = L + (size_t)i * n + jb;
    for (int c = 0; c < b; ++c) {
      double s = row[c];
      for (int p = 0; p < c; ++p) s -= x[p] * D[c][p];
      x[c] = s / D[c][c];
    }
    for (int c = 0; c < b; ++c) row[c] = x[c];
  }
  if (threadIdx.x == 0 && bad && status) atomicMax(status, RSX_ENOTPD);
}

// trailing update of the lower triangle: L[i][j] -= sum_p L[i][jb+p] L[j][jb+p], i >= j >= jb + b
__global__ void __launch_bounds__(256) k_chol_trailing(double* __restrict__ L, int n, int jb) {
  const int b = min(kChB, n - jb);
  const int t0 = jb + b;
  const int nb = (n - t0 + 31) / 32;
  // lower-triangle tile index -> (I, J), J <= I
  int I = 0, rem = blockIdx.x;
  while (rem > I) {
    rem -= I + 1;
    ++I;
  }
  const int J = rem;
  if (I >= nb) return;
  __shared__ double Pi[32][kChB + 1], Pj[32][kChB + 1];
  const int i0 = t0 + 32 * I, j0 = t0 + 32 * J;
  for (int q = threadIdx.x; q < 32 * b; q += blockDim.x) {
    const int r = q / b, c = q - r * b;
    Pi[r][c] = (i0 + r < n) ? L[(size_t)(i0 + r) * n + jb + c] : 0.0;
    Pj[r][c] = (j0 + r < n) ? L[(size_t)(j0 + r) * n + jb + c] : 0.0;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < 32 * 32; q += blockDim.x) {
    const int r = q >> 5, c = q & 31;
    const int i = i0 + r, j = j0 + c;
    if (i >= n || j >= n || j > i) continue;
    double s = 0.0;
    for (int p = 0; p < b; ++p) s += Pi[r][p] * Pj[c][p];
    L[(size_t)i * n + j] -= s;
  }
}

__global__ void k_zero_upper(double* __restrict__ L, int n) {
  const long long total = (long long)n * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e / n), c = (int)(e - (long long)r * n);
    if (c > r) L[e] = 0.0;
  }
}

// C = op(A) B (n x n, FP64, 32 x 32 tiles): op(A) = A (ta = 0) or A^T (ta = 1)
__global__ void __launch_bounds__(256) k_gemm_f64(const double* __restrict__ A, const double* __restrict__ B, int n,
                                                  int ta, double* __restrict__ C) {
  __shared__ double As[32][33], Bs[32][33];
  const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 8 rows of 4 outputs each
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int k0 = 0; k0 < n; k0 += 32) {
    for (int q = threadIdx.x; q < 1024; q += 256) {
      const int r = q >> 5, c = q & 31;
      const int gi = i0 + r, gk = k0 + c;
      double a = 0.0;
      if (gi < n && gk < n) a = ta ? A[(size_t)gk * n + gi] : A[(size_t)gi * n + gk];
      As[r][c] = a;
      const int bk = k0 + r, bj = j0 + c;
      Bs[r][c] = (bk < n && bj < n) ? B[(size_t)bk * n + bj] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < 32; ++k) {
      const double bv = Bs[k][tx];
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[u] += As[ty + 8 * u][k] * bv;
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int i = i0 + ty + 8 * u, j = j0 + tx;
    if (i < n && j < n) C[(size_t)i * n + j] = acc[u];
  }
}

// XpY[k][i] = omega_k^{-1/2} sum_{p <= i} L[i][p] Z[k][p]; omega <- sqrt(omega^2)
__global__ void k_tdhf_vectors(const double* __restrict__ L, int n, const double* __restrict__ Z, int nroots,
                               const double* __restrict__ w2, double* __restrict__ XpY) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nroots * n; q += gridDim.x * blockDim.x) {
    const int k = q / n, i = q - k * n;
    double s = 0.0;
    for (int p = 0; p <= i; ++p) s += L[(size_t)i * n + p] * Z[(size_t)k * n + p];
    XpY[q] = s / sqrt(sqrt(fmax(w2[k], 0.0)));
  }
}

__global__ void k_sqrt_roots(const double* __restrict__ w2, int nroots, double* __restrict__ omega, int* status) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < nroots) {
    const double v = w2[k];
    if (!(v > 0.0) && status) atomicMax(status, RSX_ENOTPD);
    omega[k] = sqrt(fmax(v, 0.0));
  }
}

template <typename R>
int dipoles(rsx_ctx* c, const void* po, int no, const void* pv, int nv, double* dip, cudaStream_t s) {
  const size_t N = c->g.N();
  const bool fresh = c->pos == nullptr;
  int rc = grow(c, &c->pos, &c->pos_bytes, 3 * N * sizeof(R), "positions");
  if (rc) return rc;
  if (fresh) k_positions<R><<<1024, 256, 0, s>>>(c->g.nz, c->g.ny, c->g.nx, c->h, (R*)c->pos);
  const int nblk = 2 * c->nsm;
  rc = grow(c, (void**)&c->dsm, &c->dsm_bytes, sizeof(double) * ((size_t)nblk * 4096 + 3 * 4096), "small FP64");
  if (rc) return rc;
  for (int d = 0; d < 3; ++d) {
    rc = check_cuda(c, launch_gram<R>((const R*)po, no, (const R*)pv, nv, N, c->dsm, nblk, s, (const R*)c->pos + d * N),
                    "dipole gram");
    if (!rc)
      rc = check_cuda(c, launch_gram_reduce<R>(c->dsm, nblk, no, nv, c->h * c->h * c->h, false, dip + (size_t)d * no * nv,
                                               (R*)nullptr, s, nv),
                      "dipole reduce");
    if (rc) return rc;
  }
  return RSX_OK;
}

}  // namespace

extern "C" {

int rsx_casida_dipoles(rsx_ctx* c, const void* phi_occ, int nocc, const void* phi_virt, int nvirt, double* dip,
                       void* stream) {
  rsx::NvtxRange nvtx_range("rsx_casida_dipoles");
  if (!c) return RSX_EINVAL;
  if (!phi_occ || !phi_virt || !dip || nocc < 1 || nvirt < 1 || nocc * nvirt > 4096)
    return set_error(c, RSX_EINVAL, "casida_dipoles: bad arguments (nocc * nvirt <= 4096)");
  if (cudaSetDevice(c->device) != cudaSuccess) return check_cuda(c, cudaGetLastError(), "cudaSetDevice");
  cudaStream_t s = (cudaStream_t)stream;
  return c->precision == RSX_FP32 ? dipoles<float>(c, phi_occ, nocc, phi_virt, nvirt, dip, s)
                                  : dipoles<double>(c, phi_occ, nocc, phi_virt, nvirt, dip, s);
}

int rsx_casida_oscillator(rsx_ctx* c, const double* omega, const double* X, int nroots, int nt, const double* dip,
                          double* f, void* stream) {
  rsx::NvtxRange nvtx_range("rsx_casida_oscillator");
  if (!c) return RSX_EINVAL;
  if (!omega || !X || !dip || !f || nroots < 1 || nt < 1) return set_error(c, RSX_EINVAL, "oscillator: bad arguments");
  if (cudaSetDevice(c->device) != cudaSuccess) return check_cuda(c, cudaGetLastError(), "cudaSetDevice");
  k_oscillator<<<(nroots * 32 + 255) / 256, 256, 0, (cudaStream_t)stream>>>(omega, X, nroots, nt, dip, f);
  return check_cuda(c, cudaGetLastError(), "oscillator");
}

int rsx_strength_function(rsx_ctx* c, const double* omega, const double* f, int nroots, double gamma,
                          const double* grid, int ngrid, double* S, void* stream) {
  rsx::NvtxRange nvtx_range("rsx_strength_function");
  if (!c) return RSX_EINVAL;
  if (!omega || !f || !grid || !S || nroots < 1 || ngrid < 1 || !(gamma > 0.0))
    return set_error(c, RSX_EINVAL, "strength_function: bad arguments");
  if (cudaSetDevice(c->device) != cudaSuccess) return check_cuda(c, cudaGetLastError(), "cudaSetDevice");
  k_strength<<<(ngrid + 255) / 256, 256, 0, (cudaStream_t)stream>>>(omega, f, nroots, gamma, grid, ngrid, S);
  return check_cuda(c, cudaGetLastError(), "strength function");
}

int rsx_casida_solve_full(rsx_ctx* c, const double* eps_occ, int nocc, const double* eps_virt, int nvirt,
                          const double* K, const double* Kd, double delta_M, int nroots, double* omega, double* XpY,
                          void* stream) {
  rsx::NvtxRange nvtx_range("rsx_casida_solve_full");
  if (!c) return RSX_EINVAL;
  const int n = nocc * nvirt;
  if (!eps_occ || !eps_virt || !K || !omega || nocc < 1 || nvirt < 1 || n > 4096 || nroots < 1 || nroots > n)
    return set_error(c, RSX_EINVAL, "casida_solve_full: bad arguments");
  if (cudaSetDevice(c->device) != cudaSuccess) return check_cuda(c, cudaGetLastError(), "cudaSetDevice");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t nn = (size_t)n * n;
  // workspace: L (A - B, then its factor), P (A + B), T, eigen workspace (M first), Z, w2
  const size_t ew = tda_work_doubles(n, nroots);
  int rc = grow(c, &c->tdhf_work, &c->tdhf_work_bytes, (3 * nn + ew + (size_t)nroots * n + nroots) * sizeof(double),
                "full TDHF");
  if (rc) return rc;
  double* L = (double*)c->tdhf_work;
  double* P = L + nn;
  double* T = P + nn;
  double* E = T + nn;                 // eigen workspace; M in its first n^2 doubles
  double* Z = E + ew;
  double* w2 = Z + (size_t)nroots * n;
  ProfScope ps(c, kKEig, s);
  k_tdhf_assemble<<<256, 256, 0, s>>>(eps_occ, nocc, eps_virt, nvirt, K, Kd, delta_M, L, P);
  for (int jb = 0; jb < n; jb += kChB) {
    k_potrf_panel<<<1, 256, 0, s>>>(L, n, jb, c->status);
    const int t0 = jb + std::min(kChB, n - jb);
    if (t0 < n) {
      const int nb = (n - t0 + 31) / 32;
      k_chol_trailing<<<nb * (nb + 1) / 2, 256, 0, s>>>(L, n, jb);
    }
  }
  k_zero_upper<<<256, 256, 0, s>>>(L, n);
  const dim3 g((n + 31) / 32, (n + 31) / 32);
  k_gemm_f64<<<g, 256, 0, s>>>(P, L, n, 0, T);    // T = (A + B) L
  k_gemm_f64<<<g, 256, 0, s>>>(L, T, n, 1, E);    // M = L^T T
  rc = sym_eig_lowest(c, E, n, nroots, w2, XpY ? Z : nullptr, s);
  if (rc) return rc;
  k_sqrt_roots<<<(nroots + 63) / 64, 64, 0, s>>>(w2, nroots, omega, c->status);
  if (XpY) k_tdhf_vectors<<<(nroots * n + 255) / 256, 256, 0, s>>>(L, n, Z, nroots, w2, XpY);
  return check_cuda(c, cudaGetLastError(), "full TDHF");
}

}  // extern "C"
