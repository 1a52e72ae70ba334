// Plain block eigensolver for H = -1/2 Lap + V (fourth-order finite differences, zero
// boundary values) with the kinetic-energy preconditioner, optionally widened by the
// learned preconditioner's directions.  The paper's own eigensolvers are conjugate
// gradients and preconditioned Lanczos (Sec. 3.1); this block preconditioned
// steepest-descent / Rayleigh-Ritz solver is the project's plain method.
//
// One step, k bands, basis B = [Psi | W_plain (| W_learned)], m = 2k or 3k:
//   R = H Psi - Psi diag(theta)              (k_residual)
//   T_i = theta_i - <psi_i, V psi_i>          (orbital kinetic energy, weighted Gram)
//   W_plain = (K + T)^-1 R by damped Jacobi   (k_ke_jacobi, K = -1/2 Lap)
//   W_learned = s net(R / s, V c)             (convnet.cu, s = |R_i|)
//   normalise the W blocks, H W               (k_ham_apply)
//   S = <B, B>, Hs = <B, H B> (FP64 Gram), then in one CTA (FP64): S = L L^T,
//   C = L^-1 Hs L^-T, Jacobi eigen-solve, Q = L^-T Y[:, :k]   (k_rayleigh_ritz)
//   Psi <- Q^T B, H Psi <- Q^T H B            (k_combine, in place)
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <vector>

#include "../../include/rsx.h"
#include "api_internal.cuh"
#include "dense.cuh"

using namespace rsx;

namespace {

constexpr int kMaxBasis = 64;

// out = -1/2 Lap_FD4 f + V f  (or only the kinetic part when V is null; plus shift T_i f
// when shift is not null).  f, out: [nb][n^3].
__global__ void k_ham_apply(const float* __restrict__ f, int nb, int n, float inv12h2, const float* __restrict__ V,
                            const double* __restrict__ shift, float* __restrict__ out) {
  const size_t N = (size_t)n * n * n;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < (size_t)nb * N;
       i += (size_t)gridDim.x * blockDim.x) {
    const size_t b = i / N, v = i - b * N;
    const int x = (int)(v % n), y = (int)((v / n) % n), z = (int)(v / ((size_t)n * n));
    const float* fb = f + b * N;
    const float c = fb[v];
    float lap = -90.f * c;   // -30 per axis
    // x
    lap += 16.f * ((x > 0 ? fb[v - 1] : 0.f) + (x < n - 1 ? fb[v + 1] : 0.f));
    lap -= (x > 1 ? fb[v - 2] : 0.f) + (x < n - 2 ? fb[v + 2] : 0.f);
    const size_t sy = n, sz = (size_t)n * n;
    lap += 16.f * ((y > 0 ? fb[v - sy] : 0.f) + (y < n - 1 ? fb[v + sy] : 0.f));
    lap -= (y > 1 ? fb[v - 2 * sy] : 0.f) + (y < n - 2 ? fb[v + 2 * sy] : 0.f);
    lap += 16.f * ((z > 0 ? fb[v - sz] : 0.f) + (z < n - 1 ? fb[v + sz] : 0.f));
    lap -= (z > 1 ? fb[v - 2 * sz] : 0.f) + (z < n - 2 ? fb[v + 2 * sz] : 0.f);
    float r = -0.5f * lap * inv12h2;
    if (V) r += V[v] * c;
    if (shift) r += (float)shift[b] * c;
    out[i] = r;
  }
}

// R_i = HPsi_i - theta_i Psi_i
__global__ void k_residual(const float* __restrict__ psi, const float* __restrict__ hpsi, const double* __restrict__ th,
                           int k, size_t N, float* __restrict__ R) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < (size_t)k * N; i += (size_t)gridDim.x * blockDim.x) {
    const size_t b = i / N;
    R[i] = hpsi[i] - (float)th[b] * psi[i];
  }
}

// one damped-Jacobi sweep for (K + T) x = r:  x_out = x_in + omega (r - (K + T) x_in) / d,
// d = 3.75 / h^2 + T; with x_in null the sweep starts from x0 = r / d.
__global__ void k_ke_jacobi(const float* __restrict__ r, const float* __restrict__ xin, const float* __restrict__ axin,
                            const double* __restrict__ T, int nb, size_t N, float d0, float omega,
                            float* __restrict__ xout) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < (size_t)nb * N;
       i += (size_t)gridDim.x * blockDim.x) {
    const size_t b = i / N;
    const float d = d0 + (float)T[b];
    xout[i] = xin ? xin[i] + omega * (r[i] - axin[i]) / d : r[i] / d;
  }
}

// T_i = max(theta_i - <psi_i, V psi_i>, 0): the orbital's kinetic energy
__global__ void k_kinetic(const double* __restrict__ th, const double* __restrict__ vdiag, int k, double* __restrict__ T) {
  const int i = threadIdx.x;
  if (i < k) T[i] = fmax(th[i] - vdiag[i], 0.0);
}

// diag[i] = G[i][i] of a k x k matrix
__global__ void k_diag(const double* __restrict__ G, int k, double* __restrict__ diag) {
  const int i = threadIdx.x;
  if (i < k) diag[i] = G[i * k + i];
}

// rows of X scaled by 1/sqrt(g[i]) (g: squared norms); zero rows stay zero
__global__ void k_normalise_rows(float* __restrict__ X, const double* __restrict__ g, int nb, size_t N) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < (size_t)nb * N;
       i += (size_t)gridDim.x * blockDim.x) {
    const size_t b = i / N;
    const double s = g[b];
    X[i] = s > 0.0 ? (float)(X[i] / sqrt(s)) : 0.f;
  }
}

// net input [k][2][N]: channel 0 = R_i / |R_i|, channel 1 = V * vscale
__global__ void k_net_input(const float* __restrict__ R, const double* __restrict__ g, const float* __restrict__ V,
                            float vscale, int k, size_t N, float* __restrict__ x) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < (size_t)k * N; i += (size_t)gridDim.x * blockDim.x) {
    const size_t b = i / N, v = i - b * N;
    const double s = g[b];
    x[(2 * b) * N + v] = s > 0.0 ? (float)(R[i] / sqrt(s)) : 0.f;
    x[(2 * b + 1) * N + v] = V[v] * vscale;
  }
}

// Rayleigh-Ritz in one CTA (FP64): S = L L^T (with a tiny diagonal shift for safety),
// C = L^-1 Hs L^-T, eigen-decomposition of C by parallel cyclic Jacobi (round-robin
// pairing, m/2 rotations per round), ascending sort, Q = L^-T Y[:, :k].
// Outputs: theta[k]; qt[k][m] (float, rows = new orbitals' coefficients).
__global__ void __launch_bounds__(256) k_rayleigh_ritz(const double* __restrict__ Sg, const double* __restrict__ Hg,
                                                       int m, int k, double* __restrict__ theta, float* __restrict__ qt,
                                                       int* status) {
  extern __shared__ double rr_smem[];   // 4 m x m matrices (dynamic shared memory)
  double* S = rr_smem;
  double* L = S + m * m;
  double* C = L + m * m;
  double* V = C + m * m;
  __shared__ double cs[kMaxBasis / 2], sn[kMaxBasis / 2];
  __shared__ int pp[kMaxBasis / 2], qq[kMaxBasis / 2];
  __shared__ double ev[kMaxBasis];
  __shared__ int ord[kMaxBasis];
  double tr = 0.0;
  for (int i = 0; i < m; ++i) tr += Sg[i * m + i];
  for (int i = threadIdx.x; i < m * m; i += blockDim.x) {
    const int r = i / m, c = i - r * m;
    S[i] = 0.5 * (Sg[r * m + c] + Sg[c * m + r]) + (r == c ? 1e-13 * tr / m : 0.0);
    C[i] = 0.5 * (Hg[r * m + c] + Hg[c * m + r]);
  }
  __syncthreads();
  // S = L L^T ; S <- L^{-1}
  const bool ok = chol_linv_block(S, L, m);
  // C <- L^-1 C L^-T  (V as scratch)
  for (int i = threadIdx.x; i < m * m; i += blockDim.x) {
    const int r = i / m, c = i - r * m;
    double s = 0.0;
    for (int j = 0; j <= r; ++j) s += S[r * m + j] * C[j * m + c];
    V[i] = s;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < m * m; i += blockDim.x) {
    const int r = i / m, c = i - r * m;
    double s = 0.0;
    for (int j = 0; j <= c; ++j) s += V[r * m + j] * S[c * m + j];
    C[i] = s;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < m * m; i += blockDim.x) V[i] = (i / m == i % m) ? 1.0 : 0.0;
  __syncthreads();
  // parallel cyclic Jacobi
  const int half = m / 2;
  for (int sweep = 0; sweep < 30; ++sweep) {
    double off = 0.0, dia = 0.0;
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) (i == j ? dia : off) += C[i * m + j] * C[i * m + j];
    if (off <= 1e-30 * dia) break;
    for (int round = 0; round < m - 1; ++round) {
      if (threadIdx.x < half) {
        const int i = threadIdx.x;
        auto pos = [&](int j) { return j == 0 ? 0 : 1 + ((j - 1 + round) % (m - 1)); };
        int p = pos(i), q = pos(m - 1 - i);
        if (p > q) { const int t = p; p = q; q = t; }
        pp[i] = p;
        qq[i] = q;
        const double apq = C[p * m + q];
        double c = 1.0, s = 0.0;
        if (fabs(apq) > 1e-300) {
          const double th = (C[q * m + q] - C[p * m + p]) / (2.0 * apq);
          const double t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
          c = 1.0 / sqrt(t * t + 1.0);
          s = t * c;
        }
        cs[i] = c;
        sn[i] = s;
      }
      __syncthreads();
      // columns: C <- C J, V <- V J
      for (int idx = threadIdx.x; idx < half * m; idx += blockDim.x) {
        const int i = idx / m, r = idx - i * m;
        const int p = pp[i], q = qq[i];
        const double c = cs[i], s = sn[i];
        const double cp = C[r * m + p], cq = C[r * m + q];
        C[r * m + p] = c * cp - s * cq;
        C[r * m + q] = s * cp + c * cq;
        const double vp = V[r * m + p], vq = V[r * m + q];
        V[r * m + p] = c * vp - s * vq;
        V[r * m + q] = s * vp + c * vq;
      }
      __syncthreads();
      // rows: C <- J^T C
      for (int idx = threadIdx.x; idx < half * m; idx += blockDim.x) {
        const int i = idx / m, col = idx - i * m;
        const int p = pp[i], q = qq[i];
        const double c = cs[i], s = sn[i];
        const double rp = C[p * m + col], rq = C[q * m + col];
        C[p * m + col] = c * rp - s * rq;
        C[q * m + col] = s * rp + c * rq;
      }
      __syncthreads();
    }
  }
  if (threadIdx.x == 0) {
    for (int i = 0; i < m; ++i) {
      ev[i] = C[i * m + i];
      ord[i] = i;
    }
    for (int i = 0; i < m; ++i)
      for (int j = i + 1; j < m; ++j)
        if (ev[ord[j]] < ev[ord[i]]) {
          const int t = ord[i];
          ord[i] = ord[j];
          ord[j] = t;
        }
  }
  __syncthreads();
  // Q = L^-T Y: qt[o][r] = sum_j Linv[j][r] V[j][ord[o]]
  for (int idx = threadIdx.x; idx < k * m; idx += blockDim.x) {
    const int o = idx / m, r = idx - o * m;
    double s = 0.0;
    for (int j = r; j < m; ++j) s += S[j * m + r] * V[j * m + ord[o]];
    qt[idx] = (float)s;
  }
  if (threadIdx.x < k) theta[threadIdx.x] = ev[ord[threadIdx.x]];
  if (threadIdx.x == 0 && !ok && status) atomicMax(status, RSX_ENOTPD);
}

size_t blocks_for(size_t n) { return std::min<size_t>((n + 255) / 256, 4096); }

}  // namespace

struct rsx_eig {
  rsx_ctx* ctx = nullptr;        // owns the Gram / combine workspace
  int n = 0, k = 0;
  double h = 0.0;
  const float* V = nullptr;      // caller's potential (device)
  float vscale = 1.f;
  float* B = nullptr;            // [3k][N] basis: Psi | W_plain | W_learned
  float* HB = nullptr;           // [3k][N]
  float* R = nullptr;            // [k][N] residual of the last step
  float* tmp = nullptr;          // [2k][N] Jacobi scratch / net input
  float* xnet = nullptr;         // [k][2][N]
  double* sm = nullptr;          // small FP64: theta, T, gram outputs, S, Hs
  float* qt = nullptr;           // [k][3k]
  bool started = false;
  char err[256] = {0};
};

namespace {

int efail(rsx_eig* e, int code, const char* msg) {
  snprintf(e->err, sizeof(e->err), "%s", msg);
  return code;
}

int ecuda(rsx_eig* e, cudaError_t c, const char* what) {
  if (c == cudaSuccess) return RSX_OK;
  snprintf(e->err, sizeof(e->err), "%s: %s", what, cudaGetErrorString(c));
  return RSX_ECUDA;
}

// out[a * ldo + b] = h^3 <X_a, Y_b w>
int gram(rsx_eig* e, const float* X, int na, const float* Y, int nb, const float* w, double* out, cudaStream_t s) {
  rsx_ctx* c = e->ctx;
  const int nblk = 2 * c->nsm;
  const size_t N = (size_t)e->n * e->n * e->n;
  int rc = grow(c, (void**)&c->dsm, &c->dsm_bytes, sizeof(double) * ((size_t)nblk * 4096 + 3 * 4096), "small FP64");
  if (rc) return rc;
  rc = check_cuda(c, launch_gram<float>(X, na, Y, nb, N, c->dsm, nblk, s, w), "gram");
  if (rc) return rc;
  return check_cuda(c, launch_gram_reduce<float>(c->dsm, nblk, na, nb, e->h * e->h * e->h, false, out, (float*)nullptr, s),
                    "gram reduce");
}

int ham(rsx_eig* e, const float* f, int nb, float* out, const double* shift, const float* V, cudaStream_t s) {
  const size_t N = (size_t)e->n * e->n * e->n;
  k_ham_apply<<<(unsigned)blocks_for(nb * N), 256, 0, s>>>(f, nb, e->n, (float)(1.0 / (12.0 * e->h * e->h)), V, shift,
                                                           out);
  return ecuda(e, cudaGetLastError(), "hamiltonian");
}

// Rayleigh-Ritz over the first m rows of B / HB, update Psi and HPsi in place
int rr_update(rsx_eig* e, int m, cudaStream_t s) {
  const int k = e->k;
  const size_t N = (size_t)e->n * e->n * e->n;
  double* S = e->sm + 256;
  double* Hs = S + kMaxBasis * kMaxBasis;
  double* theta = e->sm;
  int rc = gram(e, e->B, m, e->B, m, nullptr, S, s);
  if (!rc) rc = gram(e, e->B, m, e->HB, m, nullptr, Hs, s);
  if (rc) return rc;
  const size_t smem = 4 * (size_t)m * m * sizeof(double);
  cudaFuncSetAttribute(k_rayleigh_ritz, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_rayleigh_ritz<<<1, 256, smem, s>>>(S, Hs, m, k, theta, e->qt, e->ctx->status);
  rc = ecuda(e, cudaGetLastError(), "rayleigh-ritz");
  if (rc) return rc;
  rc = check_cuda(e->ctx, launch_combine<float>(e->qt, k, m, e->B, N, e->B, 4 * e->ctx->nsm, s), "psi update");
  if (!rc) rc = check_cuda(e->ctx, launch_combine<float>(e->qt, k, m, e->HB, N, e->HB, 4 * e->ctx->nsm, s), "hpsi update");
  return rc;
}

}  // namespace

extern "C" {

int rsx_eig_create(rsx_eig** out, int n, double h, const float* V, float vscale, int nband, int device) {
  if (!out) return RSX_EINVAL;
  *out = nullptr;
  if (n < 8 || !(h > 0.0) || !V || nband < 1 || 3 * nband > kMaxBasis) return RSX_EINVAL;
  rsx_eig* e = new rsx_eig();
  // a context on the same grid provides the Gram / combine workspace (any supported edge
  // for the tables is irrelevant here; use the smallest box)
  int rc = rsx_create(&e->ctx, 16, 16, 16, h, RSX_FP32, device);
  if (rc) {
    delete e;
    return rc;
  }
  e->n = n;
  e->k = nband;
  e->h = h;
  e->V = V;
  e->vscale = vscale;
  const size_t N = (size_t)n * n * n;
  if (cudaMalloc(&e->B, 3 * nband * N * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&e->HB, 3 * nband * N * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&e->R, nband * N * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&e->tmp, 2 * nband * N * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&e->xnet, 2 * nband * N * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&e->sm, (256 + 2 * kMaxBasis * kMaxBasis) * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&e->qt, kMaxBasis * kMaxBasis * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    rsx_eig_destroy(e);
    return RSX_ENOMEM;
  }
  *out = e;
  return RSX_OK;
}

// Load starting orbitals psi0 [k][N] (any linearly independent set); Rayleigh-Ritz on them.
int rsx_eig_init(rsx_eig* e, const float* psi0, void* stream) {
  if (!e || !psi0) return RSX_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t N = (size_t)e->n * e->n * e->n;
  int rc = ecuda(e, cudaMemcpyAsync(e->B, psi0, e->k * N * sizeof(float), cudaMemcpyDeviceToDevice, s), "init copy");
  if (!rc) rc = ham(e, e->B, e->k, e->HB, nullptr, e->V, s);
  if (!rc) rc = rr_update(e, e->k, s);
  e->started = rc == RSX_OK;
  return rc;
}

// One step; net may be NULL (plain).  theta_host[k] receives the new Ritz values; the
// residual used in this step is kept (rsx_eig_residual).  Synchronises the stream.
int rsx_eig_step(rsx_eig* e, rsx_net* net, int jacobi_sweeps, double* theta_host, void* stream) {
  if (!e || !e->started || jacobi_sweeps < 0) return RSX_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const int k = e->k;
  const size_t N = (size_t)e->n * e->n * e->n;
  double* theta = e->sm;
  double* T = e->sm + 64;
  double* diag = e->sm + 128;
  double* G = e->sm + 256;          // Gram scratch (the Rayleigh-Ritz S matrix reuses it later)
  float* psi = e->B;
  float* hpsi = e->HB;
  float* wp = e->B + k * N;
  // residual
  k_residual<<<(unsigned)blocks_for(k * N), 256, 0, s>>>(psi, hpsi, theta, k, N, e->R);
  // kinetic energies T_i = theta_i - <psi_i, V psi_i>
  int rc = gram(e, psi, k, psi, k, e->V, G, s);
  if (rc) return rc;
  k_diag<<<1, 64, 0, s>>>(G, k, diag);
  k_kinetic<<<1, 64, 0, s>>>(theta, diag, k, T);
  rc = ecuda(e, cudaGetLastError(), "kinetic");
  if (rc) return rc;
  // plain preconditioner: damped Jacobi sweeps on (K + T) x = R
  const float d0 = (float)(3.75 / (e->h * e->h));
  const float omega = 2.f / 3.f;
  float* x = wp;
  float* ax = e->tmp;
  k_ke_jacobi<<<(unsigned)blocks_for(k * N), 256, 0, s>>>(e->R, nullptr, nullptr, T, k, N, d0, omega, x);
  for (int sw = 0; sw < jacobi_sweeps; ++sw) {
    rc = ham(e, x, k, ax, T, nullptr, s);
    if (rc) return rc;
    k_ke_jacobi<<<(unsigned)blocks_for(k * N), 256, 0, s>>>(e->R, x, ax, T, k, N, d0, omega, e->tmp + k * N);
    rc = ecuda(e, cudaMemcpyAsync(x, e->tmp + k * N, k * N * sizeof(float), cudaMemcpyDeviceToDevice, s), "jacobi copy");
    if (rc) return rc;
  }
  int m = 2 * k;
  // learned directions
  if (net) {
    rc = gram(e, e->R, k, e->R, k, nullptr, G, s);
    if (rc) return rc;
    k_diag<<<1, 64, 0, s>>>(G, k, diag);
    k_net_input<<<(unsigned)blocks_for(k * N), 256, 0, s>>>(e->R, diag, e->V, e->vscale, k, N, e->xnet);
    float* wl = e->B + 2 * k * N;
    rc = rsx_net_forward(net, e->xnet, k, e->n, e->n, e->n, wl, s);
    if (rc) return efail(e, rc, "learned preconditioner forward failed");
    m = 3 * k;
  }
  // normalise the W blocks, apply H to them
  rc = gram(e, wp, m - k, wp, m - k, nullptr, G, s);
  if (rc) return rc;
  k_diag<<<1, 64, 0, s>>>(G, m - k, diag);
  k_normalise_rows<<<(unsigned)blocks_for((m - k) * N), 256, 0, s>>>(wp, diag, m - k, N);
  rc = ham(e, wp, m - k, e->HB + k * N, nullptr, e->V, s);
  if (rc) return rc;
  rc = rr_update(e, m, s);
  if (rc) return rc;
  if (theta_host) rc = ecuda(e, cudaMemcpyAsync(theta_host, theta, k * sizeof(double), cudaMemcpyDeviceToHost, s), "theta");
  if (!rc) rc = ecuda(e, cudaStreamSynchronize(s), "step sync");
  return rc;
}

int rsx_eig_orbitals(rsx_eig* e, float* psi_out, void* stream) {
  if (!e || !psi_out) return RSX_EINVAL;
  const size_t N = (size_t)e->n * e->n * e->n;
  return ecuda(e, cudaMemcpyAsync(psi_out, e->B, e->k * N * sizeof(float), cudaMemcpyDeviceToDevice, (cudaStream_t)stream),
               "orbitals");
}

int rsx_eig_residual(rsx_eig* e, float* r_out, void* stream) {
  if (!e || !r_out) return RSX_EINVAL;
  const size_t N = (size_t)e->n * e->n * e->n;
  return ecuda(e, cudaMemcpyAsync(r_out, e->R, e->k * N * sizeof(float), cudaMemcpyDeviceToDevice, (cudaStream_t)stream),
               "residual");
}

const char* rsx_eig_last_error(const rsx_eig* e) { return e ? e->err : "null eigensolver"; }

int rsx_eig_destroy(rsx_eig* e) {
  if (!e) return RSX_OK;
  void* bufs[] = {e->B, e->HB, e->R, e->tmp, e->xnet, e->sm, e->qt};
  for (void* p : bufs)
    if (p) cudaFree(p);
  rsx_destroy(e->ctx);
  delete e;
  return RSX_OK;
}

}  // extern "C"
