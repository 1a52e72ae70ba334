// Declarations of the small dense kernels (dense.cu).
#pragma once
#include "rsx_internal.cuh"

namespace rsx {

// Kernel spectrum table T[kx][ky][kz] = scale * ghat(k), k_i in [0, M_i/2]; cos_* hold
// cos(2 pi j / M_i), j < M_i; buf0/buf1 are FP64 scratch of (M_z/2+1)(M_y/2+1)(M_x/2+1).
cudaError_t launch_ghat(const Geom& g, double h, double scale, const double* cos_z, const double* cos_y,
                        const double* cos_x, double* buf0, double* buf1, void* table, bool fp64,
                        cudaStream_t s);
// FP32 kernel table in pass 2's lane order, (Mx/2+1)(My/2+1) Mz floats (k_vhat_lanes)
cudaError_t launch_vhat_lanes(const Geom& g, const float* table, float* out, cudaStream_t s);
// the kernel table in the 8-lane y/z kernel's order [kx][|ky|][s][j][k2], kz = (s + 8 j) + 2 Az k2
cudaError_t launch_vhat_lanes8(const Geom& g, const float* table, float* out, cudaStream_t s);
// part[blk][a][b] = partial sums of X_a(r) Y_b(r) w(r) (w may be null); na * nb <= 4096.
// A kernel that gives up a bounded wait writes NaN partials and raises RSX_ETIMEOUT in *status.
template <typename R>
cudaError_t launch_gram(const R* X, int na, const R* Y, int nb, size_t N, double* part, int nblk,
                        cudaStream_t s, const R* w = nullptr, int* status = nullptr);
// out[a * ldo + b] (or out[b * ldo + a] when transpose) = scale * sum of the partials
template <typename R>
cudaError_t launch_gram_reduce(const double* part, int nblk, int na, int nb, double scale, bool transpose,
                               double* out, R* out_r, cudaStream_t s, int ldo = 0);
cudaError_t launch_chol_linv(double* M, int k, double* Linv, float* linv_f, double* linv_d, int* status,
                             cudaStream_t s);
template <typename R>
cudaError_t launch_combine(const R* C, int no, int ni, const R* X, size_t N, R* out, int nblk,
                           cudaStream_t s);
template <typename R>
cudaError_t launch_pair_products(const R* A, int na, const R* B, int nb, size_t N, R* rho, cudaStream_t s);

// Block-wide FP64 Cholesky of B (k x k, shared memory, = -M symmetrised) into L (lower,
// shared memory) and L^{-1} written over B.  Returns true if every pivot was > 0
// (on failure the pivots are replaced by 1 so the arithmetic stays finite).
__device__ __forceinline__ bool chol_linv_block(double* B, double* L, int k) {
  __shared__ int bad_sh;
  if (threadIdx.x == 0) bad_sh = 0;
  for (int i = threadIdx.x; i < k * k; i += blockDim.x) L[i] = 0.0;
  __syncthreads();
  for (int j = 0; j < k; ++j) {
    if (threadIdx.x == 0) {
      double d = B[j * k + j];
      for (int p = 0; p < j; ++p) d -= L[j * k + p] * L[j * k + p];
      if (!(d > 0.0)) {
        bad_sh = 1;
        d = 1.0;
      }
      L[j * k + j] = sqrt(d);
    }
    __syncthreads();
    for (int i = j + 1 + threadIdx.x; i < k; i += blockDim.x) {
      double s = B[i * k + j];
      for (int p = 0; p < j; ++p) s -= L[i * k + p] * L[j * k + p];
      L[i * k + j] = s / L[j * k + j];
    }
    __syncthreads();
  }
  for (int c = threadIdx.x; c < k; c += blockDim.x) {
    for (int i = 0; i < k; ++i) {
      if (i < c) {
        B[i * k + c] = 0.0;
        continue;
      }
      double s = (i == c) ? 1.0 : 0.0;
      for (int p = c; p < i; ++p) s -= L[i * k + p] * B[p * k + c];
      B[i * k + c] = s / L[i * k + i];
    }
  }
  __syncthreads();
  return bad_sh == 0;
}

}  // namespace rsx
