// Small dense kernels around the pair solves: the kernel spectrum table, Gram
// reductions <X_a, Y_b>, the FP64 Cholesky of -M with L^{-1}, and the
// small-matrix application out_o = sum_i C[o][i] X_i used by ACE (Sec. 3.1, Eqs. 11-13).
#include "dense.cuh"

namespace rsx {

// ---------------------------------------------------------------------------------
// Kernel spectrum.  ghat(k) = sum_d g(d) exp(-2 pi i k.d / M) over the periodic offsets
// d of the padded grid, g(d) = 1/(h|d|), g(0) = C0/h.  g is even in every coordinate,
// so ghat is a product of three cosine sums over d_i in [0, M_i/2] with weights 1 at
// d_i = 0 and d_i = M_i/2 and 2 otherwise.  FP64 throughout; the final table holds
// ghat * scale (scale = h^3 / N_pad) as T[kx][ky][kz] for k_i in [0, M_i/2].

__global__ void k_ghat_init(double* buf, int hz, int hy, int hx, double h, double c0) {
  const size_t n = (size_t)hz * hy * hx;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int dx = (int)(i % hx);
    const int dy = (int)((i / hx) % hy);
    const int dz = (int)(i / ((size_t)hx * hy));
    const double r2 = (double)dx * dx + (double)dy * dy + (double)dz * dz;
    buf[i] = (r2 == 0.0) ? c0 / h : 1.0 / (h * sqrt(r2));
  }
}

// out[i0][i1][k] = sum_d w(d) cos(2 pi k d / M) in[i0][i1][d], then the result is
// stored rotated as out[k][i0][i1] so that three calls transform all three axes.
__global__ void k_cos_axis(const double* __restrict__ in, double* __restrict__ out, int h0, int h1, int h2,
                           int M, const double* __restrict__ cosM) {
  const size_t n = (size_t)h0 * h1 * h2;
  for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
    const int i1 = (int)(o % h1);
    const int i0 = (int)((o / h1) % h0);
    const int k = (int)(o / ((size_t)h0 * h1));
    const double* row = in + ((size_t)i0 * h1 + i1) * h2;
    double s = 0.0;
    for (int d = 0; d < h2; ++d) {
      const double w = (d == 0 || 2 * d == M) ? 1.0 : 2.0;
      s += w * cosM[((long long)k * d) % M] * row[d];
    }
    out[o] = s;
  }
}

// in[kz][ky][kx] -> out[kx][ky][kz]
__global__ void k_cos_axis_permute(const double* __restrict__ in, double* __restrict__ out, int hz, int hy,
                                   int hx) {
  const size_t n = (size_t)hz * hy * hx;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int kx = (int)(i % hx);
    const int ky = (int)((i / hx) % hy);
    const int kz = (int)(i / ((size_t)hx * hy));
    out[((size_t)kx * hy + ky) * hz + kz] = in[i];
  }
}

template <typename R>
__global__ void k_scale_cast(const double* __restrict__ in, R* __restrict__ out, size_t n, double scale) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = (R)(in[i] * scale);
}

// ---------------------------------------------------------------------------------
// Gram partials: part[blk][a][b] = sum over this block's points of X[a][r] Y[b][r].
// Chunks of kGramChunk points are staged in shared memory; each thread owns up to 16
// outputs; per-chunk sums in R, accumulated across chunks in FP64.
constexpr int kGramChunk = 128;
constexpr int kGramThreads = 256;

// (w, when not null, multiplies Y point-wise: sum X_a Y_b w)
template <typename R>
__global__ void __launch_bounds__(kGramThreads) k_gram(const R* __restrict__ X, int na, const R* __restrict__ Y,
                                                       int nb, const R* __restrict__ w, size_t N,
                                                       double* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* xs = reinterpret_cast<R*>(smem_raw);
  R* ys = xs + (size_t)na * (kGramChunk + 1);
  const int nout = na * nb;
  double acc[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) acc[k] = 0.0;
  const size_t nchunk = (N + kGramChunk - 1) / kGramChunk;
  for (size_t c = blockIdx.x; c < nchunk; c += gridDim.x) {
    const size_t r0 = c * kGramChunk;
    const int len = (int)min((size_t)kGramChunk, N - r0);
    __syncthreads();
    for (int i = threadIdx.x; i < na * kGramChunk; i += kGramThreads) {
      const int a = i / kGramChunk, j = i - a * kGramChunk;
      xs[a * (kGramChunk + 1) + j] = j < len ? X[(size_t)a * N + r0 + j] : R(0);
    }
    for (int i = threadIdx.x; i < nb * kGramChunk; i += kGramThreads) {
      const int b = i / kGramChunk, j = i - b * kGramChunk;
      ys[b * (kGramChunk + 1) + j] = j < len ? (w ? Y[(size_t)b * N + r0 + j] * w[r0 + j] : Y[(size_t)b * N + r0 + j]) : R(0);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const int o = threadIdx.x + k * kGramThreads;
      if (o < nout) {
        const int a = o / nb, b = o - a * nb;
        const R* xa = xs + a * (kGramChunk + 1);
        const R* yb = ys + b * (kGramChunk + 1);
        R s = R(0);
#pragma unroll 8
        for (int j = 0; j < kGramChunk; ++j) s += xa[j] * yb[j];
        acc[k] += (double)s;
      }
    }
  }
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const int o = threadIdx.x + k * kGramThreads;
    if (o < nout) part[(size_t)blockIdx.x * nout + o] = acc[k];
  }
}

// out[a][b] (or out[b][a] when transpose) = scale * sum_blk part[blk][a][b]; optional
// R copy with the same layout.
// (ldo: row stride of out / out_r; 0 means na or nb as implied by transpose)
template <typename R>
__global__ void k_gram_reduce(const double* __restrict__ part, int nblk, int na, int nb, double scale,
                              int transpose, double* __restrict__ out, R* __restrict__ out_r, int ldo) {
  const int nout = na * nb;
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < nout; o += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < nblk; ++k) s += part[(size_t)k * nout + o];
    s *= scale;
    const int a = o / nb, b = o - a * nb;
    const size_t d = transpose ? (size_t)b * (ldo ? ldo : na) + a : (size_t)a * (ldo ? ldo : nb) + b;
    if (out) out[d] = s;
    if (out_r) out_r[d] = (R)s;
  }
}

// ---------------------------------------------------------------------------------
// ACE factorisation (one CTA, FP64): Ms = (M + M^T)/2 written back to M; -Ms = L L^T;
// Linv = L^{-1}.  A pivot <= 0 (or NaN) sets *status = 4 and fills Linv with NaN.
__global__ void k_chol_linv(double* __restrict__ M, int k, double* __restrict__ Linv_out, float* linv_f,
                            double* linv_d, int* status) {
  extern __shared__ double sm[];
  double* B = sm;            // k*k
  double* L = sm + k * k;    // k*k
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  for (int i = threadIdx.x; i < k * k; i += blockDim.x) {
    const int r = i / k, c = i - r * k;
    const double s = 0.5 * (M[r * k + c] + M[c * k + r]);
    B[i] = -s;
    L[i] = 0.0;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < k * k; i += blockDim.x) M[i] = -B[i];
  for (int j = 0; j < k; ++j) {
    if (threadIdx.x == 0) {
      double d = B[j * k + j];
      for (int p = 0; p < j; ++p) d -= L[j * k + p] * L[j * k + p];
      if (!(d > 0.0)) {
        bad = 1;
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
  // forward substitution, one column of the inverse per thread
  for (int c = threadIdx.x; c < k; c += blockDim.x) {
    for (int i = 0; i < k; ++i) {
      double s = (i == c) ? 1.0 : 0.0;
      if (i < c) {
        B[i * k + c] = 0.0;
        continue;
      }
      for (int p = c; p < i; ++p) s -= L[i * k + p] * B[p * k + c];
      B[i * k + c] = s / L[i * k + i];
    }
  }
  __syncthreads();
  const double nan = __longlong_as_double(0x7ff8000000000000LL);
  for (int i = threadIdx.x; i < k * k; i += blockDim.x) {
    const double v = bad ? nan : B[i];
    if (Linv_out) Linv_out[i] = v;
    if (linv_f) linv_f[i] = (float)v;
    if (linv_d) linv_d[i] = v;
  }
  if (threadIdx.x == 0 && bad && status) atomicMax(status, 4);
}

// ---------------------------------------------------------------------------------
// out[o][r] = sum_i C[o][i] X[i][r] for o < no, i < ni.  A block stages X[0..ni)[256
// points] in shared memory; each thread owns one point.  In place (out == X) is safe
// because every block reads its whole chunk before writing it.
constexpr int kCombPts = 256;

template <typename R>
__global__ void __launch_bounds__(kCombPts) k_combine(const R* __restrict__ C, int no, int ni, const R* X,
                                                      size_t N, R* out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* cs = reinterpret_cast<R*>(smem_raw);  // no*ni
  R* xs = cs + no * ni;                    // ni * kCombPts
  for (int i = threadIdx.x; i < no * ni; i += kCombPts) cs[i] = C[i];
  const size_t nchunk = (N + kCombPts - 1) / kCombPts;
  for (size_t c = blockIdx.x; c < nchunk; c += gridDim.x) {
    const size_t r = c * kCombPts + threadIdx.x;
    __syncthreads();
    for (int i = 0; i < ni; ++i) xs[i * kCombPts + threadIdx.x] = r < N ? X[(size_t)i * N + r] : R(0);
    __syncthreads();
    if (r < N) {
      for (int o = 0; o < no; ++o) {
        R s = R(0);
        const R* co = cs + o * ni;
        for (int i = 0; i < ni; ++i) s += co[i] * xs[i * kCombPts + threadIdx.x];
        out[(size_t)o * N + r] = s;
      }
    }
  }
}

// rho[a * nb + b][r] = A[a][r] * B[b][r]
template <typename R>
__global__ void k_pair_products(const R* __restrict__ A, int na, const R* __restrict__ B, int nb, size_t N,
                                R* __restrict__ rho) {
  const size_t total = (size_t)na * nb * N;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const size_t q = i / N, r = i - q * N;
    const size_t a = q / nb, b = q - a * nb;
    rho[i] = A[a * N + r] * B[b * N + r];
  }
}

// ---------------------------------------------------------------------------------
// host launchers

cudaError_t launch_ghat(const Geom& g, double h, double scale, const double* cos_z, const double* cos_y,
                        const double* cos_x, double* buf0, double* buf1, void* table, bool fp64,
                        cudaStream_t s) {
  const int hz = g.Mz / 2 + 1, hy = g.My / 2 + 1, hx = g.Mx / 2 + 1;
  const size_t n = (size_t)hz * hy * hx;
  const int blocks = 1024, threads = 256;
  const double c0 = 3.0 * log(2.0 + sqrt(3.0)) - 0.5 * 3.14159265358979323846;
  k_ghat_init<<<blocks, threads, 0, s>>>(buf0, hz, hy, hx, h, c0);            // [dz][dy][dx]
  k_cos_axis<<<blocks, threads, 0, s>>>(buf0, buf1, hz, hy, hx, g.Mx, cos_x);  // [kx][dz][dy]
  k_cos_axis<<<blocks, threads, 0, s>>>(buf1, buf0, hx, hz, hy, g.My, cos_y);  // [ky][kx][dz]
  k_cos_axis<<<blocks, threads, 0, s>>>(buf0, buf1, hy, hx, hz, g.Mz, cos_z);  // [kz][ky][kx]
  // reorder [kz][ky][kx] -> T[kx][ky][kz] while scaling
  k_cos_axis_permute<<<blocks, threads, 0, s>>>(buf1, buf0, hz, hy, hx);
  if (fp64)
    k_scale_cast<double><<<blocks, threads, 0, s>>>(buf0, (double*)table, n, scale);
  else
    k_scale_cast<float><<<blocks, threads, 0, s>>>(buf0, (float*)table, n, scale);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_gram(const R* X, int na, const R* Y, int nb, size_t N, double* part, int nblk,
                        cudaStream_t s, const R* w) {
  if (na * nb > 16 * kGramThreads) return cudaErrorInvalidValue;
  const size_t smem = sizeof(R) * (size_t)(na + nb) * (kGramChunk + 1);
  cudaError_t e = cudaFuncSetAttribute(k_gram<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_gram<R><<<nblk, kGramThreads, smem, s>>>(X, na, Y, nb, w, N, part);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_gram_reduce(const double* part, int nblk, int na, int nb, double scale, bool transpose,
                               double* out, R* out_r, cudaStream_t s, int ldo) {
  k_gram_reduce<R><<<(na * nb + 255) / 256, 256, 0, s>>>(part, nblk, na, nb, scale, transpose ? 1 : 0, out,
                                                          out_r, ldo);
  return cudaGetLastError();
}

cudaError_t launch_chol_linv(double* M, int k, double* Linv, float* linv_f, double* linv_d, int* status,
                             cudaStream_t s) {
  const size_t smem = sizeof(double) * 2 * (size_t)k * k;
  cudaError_t e = cudaFuncSetAttribute(k_chol_linv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_chol_linv<<<1, 256, smem, s>>>(M, k, Linv, linv_f, linv_d, status);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_combine(const R* C, int no, int ni, const R* X, size_t N, R* out, int nblk,
                           cudaStream_t s) {
  const size_t smem = sizeof(R) * ((size_t)no * ni + (size_t)ni * kCombPts);
  cudaError_t e = cudaFuncSetAttribute(k_combine<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_combine<R><<<nblk, kCombPts, smem, s>>>(C, no, ni, X, N, out);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_pair_products(const R* A, int na, const R* B, int nb, size_t N, R* rho, cudaStream_t s) {
  k_pair_products<R><<<2048, 256, 0, s>>>(A, na, B, nb, N, rho);
  return cudaGetLastError();
}

#define RSX_INST(R)                                                                                        \
  template cudaError_t launch_gram<R>(const R*, int, const R*, int, size_t, double*, int, cudaStream_t,   \
                                      const R*);                                                          \
  template cudaError_t launch_gram_reduce<R>(const double*, int, int, int, double, bool, double*, R*,      \
                                             cudaStream_t, int);                                          \
  template cudaError_t launch_combine<R>(const R*, int, int, const R*, size_t, R*, int, cudaStream_t);     \
  template cudaError_t launch_pair_products<R>(const R*, int, const R*, int, size_t, R*, cudaStream_t);
RSX_INST(float)
RSX_INST(double)
#undef RSX_INST

}  // namespace rsx
