// Small dense kernels around the pair solves: the kernel spectrum table, Gram
// reductions <X_a, Y_b>, the FP64 Cholesky of -M with L^{-1}, and the
// small-matrix application out_o = sum_i C[o][i] X_i used by ACE (Sec. 3.1, Eqs. 11-13).
#include <algorithm>
#include <cstdint>

#include "dense.cuh"
#include "tcgen05_util.cuh"
#include "gemm_tcgen05.cuh"
#include "../../include/rsx.h"

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

// Register-tiled Gram partials (same result layout): each thread owns a 4 x 4 tile of
// outputs over a 1/S share of every chunk's points, S threads per tile (a power of two up
// to 32, so a tile's threads share a warp and are summed by shuffles at the end).  Points
// are staged transposed, [point][row], with a row stride of an odd number of 4-element
// groups, so that 4-element loads by consecutive points do not collide in shared memory.
// For up to 256 tiles.
__device__ inline void ld4(const float* p, float v[4]) {
  const float4 t = *reinterpret_cast<const float4*>(p);
  v[0] = t.x;
  v[1] = t.y;
  v[2] = t.z;
  v[3] = t.w;
}
__device__ inline void ld4(const double* p, double v[4]) {
  const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
  v[0] = a.x;
  v[1] = a.y;
  v[2] = b.x;
  v[3] = b.y;
}

__host__ __device__ inline int gram_stride(int n) { return ((((n + 3) >> 2)) | 1) * 4; }

// Stage rows [0, na) of X (times w when given) for points [r0, r0 + len) into xs[j][a]
// (rows na .. sx - 1 zero).  vec: R is float, X (and w) 16-byte aligned, N % 4 == 0 --
// every thread then issues its (at most kStageVec) 4-point loads before any store, rows
// along the lanes so that the transposed stores do not collide.
constexpr int kStageVec = 9;   // ceil(68 * 32 / 256): rows up to 64 (stride 68)
template <typename R>
__device__ inline void gram_stage(const R* __restrict__ X, int na, const R* __restrict__ w, size_t N, size_t r0,
                                  int len, R* __restrict__ xs, int sx, bool vec) {
  if constexpr (sizeof(R) == 4) {
    if (vec) {
      constexpr int Q = kGramChunk / 4;
      const int total = sx * Q;
      float4 v[kStageVec];
#pragma unroll
      for (int u = 0; u < kStageVec; ++u) {
        const int i = threadIdx.x + u * kGramThreads;
        const int q = i / sx, a = i - q * sx;
        v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (i < total && a < na && 4 * q < len) {
          v[u] = *reinterpret_cast<const float4*>(X + (size_t)a * N + r0 + 4 * q);
          if (w) {
            const float4 c = *reinterpret_cast<const float4*>(w + r0 + 4 * q);
            v[u] = make_float4(v[u].x * c.x, v[u].y * c.y, v[u].z * c.z, v[u].w * c.w);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < kStageVec; ++u) {
        const int i = threadIdx.x + u * kGramThreads;
        if (i < total) {
          const int q = i / sx, a = i - q * sx;
          float* d = reinterpret_cast<float*>(xs) + 4 * q * sx + a;
          d[0] = v[u].x;
          d[sx] = v[u].y;
          d[2 * sx] = v[u].z;
          d[3 * sx] = v[u].w;
        }
      }
      return;
    }
  }
  for (int i = threadIdx.x; i < sx * kGramChunk; i += kGramThreads) {
    const int a = i / kGramChunk, j = i - a * kGramChunk;
    R v = R(0);
    if (a < na && j < len) v = w ? X[(size_t)a * N + r0 + j] * w[r0 + j] : X[(size_t)a * N + r0 + j];
    xs[j * sx + a] = v;
  }
}

// sym: X == Y, na == nb, no weight -- one staged copy, tiles (i <= j) only, each written
// to both halves.
template <typename R>
__global__ void __launch_bounds__(kGramThreads) k_gram_tiled(const R* __restrict__ X, int na, const R* __restrict__ Y,
                                                             int nb, const R* __restrict__ w, size_t N, int S, int sym,
                                                             int vec, double* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ta = (na + 3) >> 2, tb = (nb + 3) >> 2;
  const int sx = gram_stride(na), sy = gram_stride(nb);
  R* xs = reinterpret_cast<R*>(smem_raw);            // [kGramChunk][sx]
  R* ys = sym ? xs : xs + kGramChunk * sx;           // [kGramChunk][sy]
  const int tile = threadIdx.x / S, split = threadIdx.x - tile * S;
  int ti = 0, tj = 0;
  bool active;
  if (sym) {
    // tile -> (ti, tj), ti <= tj, row-major over the upper triangle
    active = tile < ta * (ta + 1) / 2;
    int t = tile;
    while (active && t >= ta - ti) {
      t -= ta - ti;
      ++ti;
    }
    tj = ti + t;
  } else {
    active = tile < ta * tb;
    ti = tile / tb;
    tj = tile - ti * tb;
  }
  const int a0 = active ? ti * 4 : 0, b0 = active ? tj * 4 : 0;
  // The FP32 sums of each chunk are accumulated across chunks as double-float pairs
  // (hi + lo, the rounding error of every addition carried into lo by Knuth's TwoSum):
  // FP32 instructions only, where one FP64 addition per output and chunk cost as much as
  // the chunk's products on this part's few FP64 units.  FP64 inputs accumulate in FP64.
  double acc[16];
  float ah[16], al[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    acc[q] = 0.0;
    ah[q] = al[q] = 0.f;
  }
  const size_t nchunk = (N + kGramChunk - 1) / kGramChunk;
  for (size_t c = blockIdx.x; c < nchunk; c += gridDim.x) {
    const size_t r0 = c * kGramChunk;
    const int len = (int)min((size_t)kGramChunk, N - r0);
    __syncthreads();
    gram_stage<R>(X, na, nullptr, N, r0, len, xs, sx, vec != 0);
    if (!sym) gram_stage<R>(Y, nb, w, N, r0, len, ys, sy, vec != 0);
    __syncthreads();
    if (active) {
      R sacc[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) sacc[q] = R(0);
#pragma unroll 4
      for (int j = split; j < kGramChunk; j += S) {
        R xv[4], yv[4];
        ld4(xs + j * sx + a0, xv);
        ld4(ys + j * sy + b0, yv);
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
          for (int q = 0; q < 4; ++q) sacc[p * 4 + q] = fma(xv[p], yv[q], sacc[p * 4 + q]);
      }
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        if constexpr (sizeof(R) == 4) {
          const float a = ah[q], b = sacc[q];
          const float sm = a + b, bp = sm - a;
          al[q] += (a - (sm - bp)) + (b - bp);
          ah[q] = sm;
        } else {
          acc[q] += (double)sacc[q];
        }
      }
    }
  }
  if constexpr (sizeof(R) == 4) {
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q] = (double)ah[q] + (double)al[q];
  }
  for (int o = S >> 1; o > 0; o >>= 1)
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
  if (active && split == 0) {
    const int nout = na * nb;
    double* pb = part + (size_t)blockIdx.x * nout;
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (a0 + p < na && b0 + q < nb) {
          pb[(a0 + p) * nb + b0 + q] = acc[p * 4 + q];
          if (sym) pb[(b0 + q) * nb + a0 + p] = acc[p * 4 + q];
        }
  }
}

// out[a][b] (or out[b][a] when transpose) = scale * sum_blk part[blk][a][b]; optional
// R copy with the same layout.  32 outputs per block, 8 warps splitting the partials.
// (ldo: row stride of out / out_r; 0 means na or nb as implied by transpose)
constexpr int kRedGroups = 16;   // warps of k_gram_reduce, each over every 16th partial block

template <typename R>
__global__ void k_gram_reduce(const double* __restrict__ part, int nblk, int na, int nb, double scale,
                              int transpose, double* __restrict__ out, R* __restrict__ out_r, int ldo) {
  __shared__ double red[kRedGroups][33];
  const int nout = na * nb;
  const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
  const int o = blockIdx.x * 32 + lane;
  // four independent partial sums per thread, so that four loads are in flight at a time
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  if (o < nout) {
    int k = g;
    for (; k + 3 * kRedGroups < nblk; k += 4 * kRedGroups) {
      s0 += part[(size_t)k * nout + o];
      s1 += part[(size_t)(k + kRedGroups) * nout + o];
      s2 += part[(size_t)(k + 2 * kRedGroups) * nout + o];
      s3 += part[(size_t)(k + 3 * kRedGroups) * nout + o];
    }
    for (; k < nblk; k += kRedGroups) s0 += part[(size_t)k * nout + o];
  }
  red[g][lane] = (s0 + s1) + (s2 + s3);
  __syncthreads();
  if (g == 0 && o < nout) {
    double t = 0.0;
    for (int q = 0; q < kRedGroups; ++q) t += red[q][lane];
    t *= scale;
    const int a = o / nb, b = o - a * nb;
    const size_t d = transpose ? (size_t)b * (ldo ? ldo : na) + a : (size_t)a * (ldo ? ldo : nb) + b;
    if (out) out[d] = t;
    if (out_r) out_r[d] = (R)t;
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
  __shared__ double rinv[64];   // 1 / L_jj (FP64 division and square root are long sequences
                                // on this part: one rsqrt per column, multiplications after)
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
      const double rs = rsqrt(d);
      L[j * k + j] = d * rs;
      rinv[j] = rs;
    }
    __syncthreads();
    for (int i = j + 1 + threadIdx.x; i < k; i += blockDim.x) {
      double s = B[i * k + j];
      for (int p = 0; p < j; ++p) s -= L[i * k + p] * L[j * k + p];
      L[i * k + j] = s * rinv[j];
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
      B[i * k + c] = s * rinv[i];
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

// FP32 combination with the outputs in registers: each thread owns PTS consecutive points
// and NO outputs (output group blockIdx.y); X is read straight from global memory as
// PTS-wide vectors, the coefficients are staged transposed, ct[i][NO] (zero-padded), and
// read as 4-wide broadcasts -- 4 NO x PTS / (NO + 4 PTS) FMAs per shared-memory word
// instead of the 1/2 of k_combine.  Same summation order over i as k_combine.
// N % PTS == 0; X, out PTS*4-byte aligned; with one output group out may equal X.
template <int NO, int PTS>
__global__ void __launch_bounds__(256) k_combine_reg(const float* __restrict__ C, int no, int ni, const float* X,
                                                     size_t N, float* out) {
  extern __shared__ __align__(16) float ct[];   // [ni][NO]
  const int o0 = blockIdx.y * NO;
  for (int q = threadIdx.x; q < ni * NO; q += blockDim.x) {
    const int i = q / NO, o = q - i * NO;
    ct[q] = o0 + o < no ? C[(size_t)(o0 + o) * ni + i] : 0.f;
  }
  __syncthreads();
  const size_t ng = N / PTS;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < ng; g += (size_t)gridDim.x * blockDim.x) {
    float acc[NO][PTS];
#pragma unroll
    for (int o = 0; o < NO; ++o)
#pragma unroll
      for (int p = 0; p < PTS; ++p) acc[o][p] = 0.f;
    const float* xp = X + g * PTS;
#pragma unroll 2
    for (int i = 0; i < ni; ++i) {
      float xv[PTS];
      if constexpr (PTS == 4) {
        const float4 t = *reinterpret_cast<const float4*>(xp + (size_t)i * N);
        xv[0] = t.x;
        xv[1] = t.y;
        xv[2] = t.z;
        xv[3] = t.w;
      } else {
        const float2 t = *reinterpret_cast<const float2*>(xp + (size_t)i * N);
        xv[0] = t.x;
        xv[1] = t.y;
      }
#pragma unroll
      for (int o4 = 0; o4 < NO; o4 += 4) {
        const float4 c = *reinterpret_cast<const float4*>(ct + i * NO + o4);
#pragma unroll
        for (int p = 0; p < PTS; ++p) {
          acc[o4][p] = fmaf(c.x, xv[p], acc[o4][p]);
          acc[o4 + 1][p] = fmaf(c.y, xv[p], acc[o4 + 1][p]);
          acc[o4 + 2][p] = fmaf(c.z, xv[p], acc[o4 + 2][p]);
          acc[o4 + 3][p] = fmaf(c.w, xv[p], acc[o4 + 3][p]);
        }
      }
    }
#pragma unroll
    for (int o = 0; o < NO; ++o) {
      if (o0 + o < no) {
        float* op = out + (size_t)(o0 + o) * N + g * PTS;
        if constexpr (PTS == 4)
          *reinterpret_cast<float4*>(op) = make_float4(acc[o][0], acc[o][1], acc[o][2], acc[o][3]);
        else
          *reinterpret_cast<float2*>(op) = make_float2(acc[o][0], acc[o][1]);
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

// Pass 2's FP32 copy of the kernel table in the order its lanes read it: after the
// 16-point z transforms lane t (< Az) holds kz = t + Az k2, k2 < 16, and reads the
// factors of one column (kx, |ky|) as four float4 at [(k2 / 4) Az + t], so that a
// half-warp's request covers 16 contiguous bytes per lane.  out[kx][iy][k2/4][t][k2%4] =
// T[kx][iy][fold(t + Az k2)], fold(kz) = min(kz, Mz - kz).
__global__ void k_vhat_lanes(const float* __restrict__ T, int rows, int hz, int Az, float* __restrict__ out) {
  const int Mz = 16 * Az;
  const size_t n = (size_t)rows * Mz;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const size_t row = i / Mz;
    const int p = (int)(i - row * Mz);
    const int q = p / (4 * Az), rem = p - q * 4 * Az;
    const int t = rem >> 2, k2 = 4 * q + (rem & 3);
    const int kz = t + Az * k2;
    out[i] = T[row * hz + (kz <= Mz / 2 ? kz : Mz - kz)];
  }
}

// 8-lane order: entry p of a row is lane s = p / (2 Az), j = (p % (2 Az)) / 8, k2 = p % 8
__global__ void k_vhat_lanes8(const float* __restrict__ T, int rows, int hz, int Az, float* __restrict__ out) {
  const int Mz = 16 * Az, A2 = 2 * Az;
  const size_t n = (size_t)rows * Mz;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const size_t row = i / Mz;
    const int p = (int)(i - row * Mz);
    const int s = p / A2, rem = p - s * A2;
    const int j = rem >> 3, k2 = rem & 7;
    const int kz = (s + 8 * j) + A2 * k2;
    out[i] = T[row * hz + (kz <= Mz / 2 ? kz : Mz - kz)];
  }
}

// ---------------------------------------------------------------------------------
// host launchers

cudaError_t launch_vhat_lanes8(const Geom& g, const float* table, float* out, cudaStream_t s) {
  const int rows = (g.Mx / 2 + 1) * (g.My / 2 + 1);
  k_vhat_lanes8<<<1024, 256, 0, s>>>(table, rows, g.Mz / 2 + 1, g.Az, out);
  return cudaGetLastError();
}

cudaError_t launch_vhat_lanes(const Geom& g, const float* table, float* out, cudaStream_t s) {
  const int rows = (g.Mx / 2 + 1) * (g.My / 2 + 1);
  k_vhat_lanes<<<1024, 256, 0, s>>>(table, rows, g.Mz / 2 + 1, g.Az, out);
  return cudaGetLastError();
}

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

// ---------------------------------------------------------------------------------
// Streaming FP32 Gram partials (N % 4 == 0, 16-byte aligned rows; up to 16 output groups:
// the ACE shapes 16 x 16 and 16 x 32, the eigensolver's 48 x 48).  The output is cut into
// 16 x 16 groups (grid.x, fastest); a CTA of chunk stream grid.y streams chunks of 256 points
// of its 16 X rows, 16 Y rows
// (and the weight row) into a 3-stage ring, each chunk as one 2-D TMA box per operand
// (16 rows x 256 points; rows past na / nb and points past N arrive as zeros) completing
// on the stage's mbarrier.  Thread (ti = warp & 3, tj = lane >> 3, split = lane & 7 +
// 8 (warp >> 2)) owns the 4 x 4 outputs (4 ti + p, 4 tj + q) and the 4-point quads split,
// split + 16, ... of each chunk; the eight lanes of a quarter-warp read eight consecutive
// quads of the same rows (16-byte loads, no bank conflicts).  The products of a quad are
// packed FP32x2 fused multiply-adds (even and odd points in the two halves); every two
// chunks the FP32 sums are carried into double-float pairs (Knuth's TwoSum), and the 16
// split lanes are combined as pairs too -- FP64 arithmetic is slow on this part.
//
// There is no CTA-wide barrier per chunk: every warp waits only for its chunk's mbarrier,
// multiplies, and counts itself out of the stage on a shared counter; the warp that counts
// out last (all eight have read the stage) re-arms the mbarrier and issues the chunk three
// ahead into it, so warps drift apart by up to two chunks.  The stage of chunk j is
// refilled only after every warp has finished chunk j, so no warp waits on a phase that has
// been overtaken.  Every wait is bounded: on a timeout the CTA stops, waits (bounded) for
// the copies it issued, writes NaN partials and raises RSX_ETIMEOUT in `status`.
constexpr int kGsChunk = 256, kGsStages = 3, kGsFold = 2, kGsThreads = 256, kGsSlots = 33;
// output groups served by the streaming kernel (up to 64 x 64 outputs; wider: the staged kernel)
constexpr int kGsMaxGroups = 16;

template <int CHUNK, int STAGES, int FOLD>
__global__ void __launch_bounds__(kGsThreads, 2) k_gram_stream(const float* __restrict__ X, int na,
                                                              const float* __restrict__ Y, int nb,
                                                              const float* __restrict__ w, size_t N, int ngb,
                                                              double* __restrict__ part, int* status,
                                                              const __grid_constant__ CUtensorMap map_x,
                                                              const __grid_constant__ CUtensorMap map_y,
                                                              const __grid_constant__ CUtensorMap map_w) {
  extern __shared__ __align__(1024) float gstream[];   // [stage][slot][CHUNK], then STAGES mbarriers
  float* gs = gstream;
  uint64_t* full = reinterpret_cast<uint64_t*>(gs + (size_t)STAGES * kGsSlots * CHUNK);
  __shared__ int abort_flag;
  __shared__ unsigned out_count[STAGES];          // warps done with the stage, all uses so far
  __shared__ unsigned long long issued;           // chunks whose copies have been issued
  // blockIdx.x: output group (fastest, so that the groups sharing a chunk's rows run
  // together and re-read them from L2); blockIdx.y: chunk stream, gridDim.y streams
  const int gx = blockIdx.x / ngb, gy = blockIdx.x - gx * ngb;
  const unsigned cb = blockIdx.y, ncb = gridDim.y;
  const int a_lo = 16 * gx, b_lo = 16 * gy;
  const int nra = min(16, na - a_lo), nrb = min(16, nb - b_lo);
  const bool shared_rows = X == Y && a_lo == b_lo && w == nullptr;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ti = warp & 3, tj = lane >> 3, split = (lane & 7) + 8 * (warp >> 2);
  const int a0 = 4 * ti, b0 = 4 * tj;
  constexpr int kWarps = kGsThreads / 32;
  const size_t nchunk = (N + CHUNK - 1) / CHUNK;
  const long long mine = cb < nchunk ? (long long)((nchunk - 1 - cb) / ncb) + 1 : 0;
  if (threadIdx.x == 0) {
    abort_flag = 0;
    issued = 0;
    for (int st = 0; st < STAGES; ++st) {
      tc::mbar_init(&full[st], 1);
      out_count[st] = 0;
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  auto issue = [&](long long i) {   // one whole warp
    const size_t r0 = (cb + (size_t)i * ncb) * CHUNK;
    float* base = gs + (size_t)(i % STAGES) * kGsSlots * CHUNK;
    uint64_t* bar = &full[i % STAGES];
    // whole boxes of 16 rows x CHUNK points (rows past the end and points past N read as 0)
    if (lane == 0) {
      const uint32_t box = 16u * CHUNK * 4u;
      tc::mbar_arrive_expect_tx(bar, box * (shared_rows ? 1u : 2u) + (w ? CHUNK * 4u : 0u));
      tc::tma_load_2d(base, &map_x, bar, (int)r0, a_lo);
      if (!shared_rows) tc::tma_load_2d(base + 16 * CHUNK, &map_y, bar, (int)r0, b_lo);
      if (w) tc::tma_load_2d(base + 32 * CHUNK, &map_w, bar, (int)r0, 0);
      atomicMax(&issued, (unsigned long long)(i + 1));
    }
    __syncwarp();
  };
  if (warp == 0)
    for (int i = 0; i < STAGES && i < mine; ++i) issue(i);
  float ah[16], al[16];
  float2 s2[16];
#pragma unroll
  for (int o = 0; o < 16; ++o) ah[o] = al[o] = 0.f;
  bool ok = true;
  for (long long i = 0; i < mine; ++i) {
    ok = tc::mbar_wait(&full[i % STAGES], (uint32_t)((i / STAGES) & 1), &abort_flag);
    if (!ok) break;
    const size_t r0 = (cb + (size_t)i * ncb) * CHUNK;
    const int q4 = (int)min((size_t)CHUNK, N - r0) >> 2;
    const float* xs = gs + (size_t)(i % STAGES) * kGsSlots * CHUNK;
    const float* ys = shared_rows ? xs : xs + 16 * CHUNK;
    const float* ws = xs + 32 * CHUNK;
    if (i % FOLD == 0) {
#pragma unroll
      for (int o = 0; o < 16; ++o) s2[o] = make_float2(0.f, 0.f);
    }
    for (int q = split; q < q4; q += 16) {
      float4 xv[4], yv[4];
#pragma unroll
      for (int p = 0; p < 4; ++p) xv[p] = *reinterpret_cast<const float4*>(xs + (a0 + p) * CHUNK + 4 * q);
#pragma unroll
      for (int p = 0; p < 4; ++p) yv[p] = *reinterpret_cast<const float4*>(ys + (b0 + p) * CHUNK + 4 * q);
      if (w) {
        const float4 wv = *reinterpret_cast<const float4*>(ws + 4 * q);
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          const float2 lo = __fmul2_rn(make_float2(yv[p].x, yv[p].y), make_float2(wv.x, wv.y));
          const float2 hi = __fmul2_rn(make_float2(yv[p].z, yv[p].w), make_float2(wv.z, wv.w));
          yv[p] = make_float4(lo.x, lo.y, hi.x, hi.y);
        }
      }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          float2 acc = s2[p * 4 + r];
          acc = __ffma2_rn(make_float2(xv[p].x, xv[p].y), make_float2(yv[r].x, yv[r].y), acc);
          acc = __ffma2_rn(make_float2(xv[p].z, xv[p].w), make_float2(yv[r].z, yv[r].w), acc);
          s2[p * 4 + r] = acc;
        }
    }
    if (i % FOLD == FOLD - 1 || i == mine - 1) {
#pragma unroll
      for (int o = 0; o < 16; ++o) {   // TwoSum: (ah, al) += the FP32 sum of FOLD chunks
        const float a = ah[o], b = s2[o].x + s2[o].y;
        const float sm = a + b, bp = sm - a;
        al[o] += (a - (sm - bp)) + (b - bp);
        ah[o] = sm;
      }
    }
    // count this warp out of the stage; the last one refills it with chunk i + STAGES
    __syncwarp();
    unsigned before = 0;
    if (lane == 0) {
      __threadfence_block();
      before = atomicAdd(&out_count[i % STAGES], 1u);
    }
    before = __shfl_sync(0xffffffffu, before, 0);
    if (before % kWarps == kWarps - 1 && i + STAGES < mine) issue(i + STAGES);
  }
  const bool failed = __syncthreads_or(!ok);
  if (failed) {
    if (threadIdx.x == 0) {
      // the last chunk issued into each stage may still be landing
      const long long last = (long long)issued;
      for (long long j = max(0ll, last - STAGES); j < last; ++j)
        for (uint32_t it = 0; it < tc::kWaitLimit; ++it)
          if (tc::mbar_try_wait(&full[j % STAGES], (uint32_t)((j / STAGES) & 1))) break;
      if (status) atomicMax(status, RSX_ETIMEOUT);
    }
    __syncthreads();
    const int a = threadIdx.x >> 4, b = threadIdx.x & 15;
    if (a < nra && b < nrb)
      part[(size_t)cb * na * nb + (size_t)(a_lo + a) * nb + (b_lo + b)] = __longlong_as_double(0x7ff8000000000000ll);
    return;
  }
#pragma unroll
  for (int o = 0; o < 16; ++o)
#pragma unroll
    for (int m = 1; m < 8; m <<= 1) {
      const float bh = __shfl_xor_sync(0xffffffffu, ah[o], m), bl = __shfl_xor_sync(0xffffffffu, al[o], m);
      const float sm = ah[o] + bh, bp = sm - ah[o];
      al[o] += bl + ((ah[o] - (sm - bp)) + (bh - bp));
      ah[o] = sm;
    }
  float2* red = reinterpret_cast<float2*>(gs);   // [2][16][16] (h, l); every copy has landed
  if ((lane & 7) == 0) {
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int r = 0; r < 4; ++r)
        red[((warp >> 2) * 16 + a0 + p) * 16 + b0 + r] = make_float2(ah[p * 4 + r], al[p * 4 + r]);
  }
  __syncthreads();
  const int a = threadIdx.x >> 4, b = threadIdx.x & 15;
  if (a < nra && b < nrb) {
    const float2 u = red[a * 16 + b], v = red[256 + a * 16 + b];
    part[(size_t)cb * na * nb + (size_t)(a_lo + a) * nb + (b_lo + b)] =
        ((double)u.x + (double)v.x) + ((double)u.y + (double)v.y);
  }
}

// 2-D tensor map of `rows` rows of N floats, boxes of box_rows x chunk
static bool gram_map(CUtensorMap* m, const float* base, int rows, size_t N, int box_rows, int chunk) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)N, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)N * 4};
  cuuint32_t box[2] = {(cuuint32_t)chunk, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// cudaErrorNotSupported when the tensor maps cannot be encoded (the caller takes the staged kernel)
static cudaError_t launch_gram_stream(const float* X, int na, const float* Y, int nb, size_t N, double* part,
                                      int nblk, cudaStream_t s, const float* w, int* status) {
  const int ngb = (nb + 15) / 16, ngrp = ((na + 15) / 16) * ngb;
  CUtensorMap mx{}, my{}, mw{};
  if (!gram_map(&mx, X, na, N, 16, kGsChunk) || !gram_map(&my, Y, nb, N, 16, kGsChunk) ||
      (w && !gram_map(&mw, w, 1, N, 1, kGsChunk)))
    return cudaErrorNotSupported;
  const size_t smem = sizeof(float) * (size_t)kGsStages * kGsSlots * kGsChunk + 8 * kGsStages;
  auto kern = k_gram_stream<kGsChunk, kGsStages, kGsFold>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<dim3(ngrp, nblk), kGsThreads, smem, s>>>(X, na, Y, nb, w, N, ngb, part, status, mx, my, mw);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_gram(const R* X, int na, const R* Y, int nb, size_t N, double* part, int nblk,
                        cudaStream_t s, const R* w, int* status) {
  if (na * nb > 16 * kGramThreads) return cudaErrorInvalidValue;
  if constexpr (sizeof(R) == 4) {
    auto al16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
    const int nga = (na + 15) / 16, ngb = (nb + 15) / 16;
    // each 16 x 16 group streams its own rows; the groups are the fastest grid index, so the
    // groups that share a chunk's rows run together and the re-reads hit L2 (the eigensolver's
    // 48 x 48 Grams: step 1.56 -> 1.48 ms against the staged kernel)
    if (N % 4 == 0 && al16(X) && al16(Y) && (w == nullptr || al16(w)) && nga * ngb <= kGsMaxGroups) {
      const cudaError_t e = launch_gram_stream(X, na, Y, nb, N, part, nblk, s, w, status);
      if (e != cudaErrorNotSupported) return e;
    }
  }
  const bool sym = X == Y && na == nb && w == nullptr;
  const int ta = (na + 3) / 4, tb = (nb + 3) / 4;
  const int tiles = sym ? ta * (ta + 1) / 2 : ta * tb;
  if (tiles <= kGramThreads && gram_stride(na) <= 68 && gram_stride(nb) <= 68) {
    int S = 1;
    while (S < 32 && 2 * S * tiles <= kGramThreads) S *= 2;
    auto al16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
    const bool vec = sizeof(R) == 4 && N % 4 == 0 && al16(X) && al16(Y) && (w == nullptr || al16(w));
    const size_t smem = sizeof(R) * (size_t)(gram_stride(na) + (sym ? 0 : gram_stride(nb))) * kGramChunk;
    cudaError_t e = cudaFuncSetAttribute(k_gram_tiled<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_gram_tiled<R><<<nblk, kGramThreads, smem, s>>>(X, na, Y, nb, w, N, S, sym ? 1 : 0, vec ? 1 : 0, part);
    return cudaGetLastError();
  }
  const size_t smem = sizeof(R) * (size_t)(na + nb) * (kGramChunk + 1);
  cudaError_t e = cudaFuncSetAttribute(k_gram<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_gram<R><<<nblk, kGramThreads, smem, s>>>(X, na, Y, nb, w, N, part);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_gram_reduce(const double* part, int nblk, int na, int nb, double scale, bool transpose,
                               double* out, R* out_r, cudaStream_t s, int ldo) {
  k_gram_reduce<R><<<(na * nb + 31) / 32, 32 * kRedGroups, 0, s>>>(part, nblk, na, nb, scale, transpose ? 1 : 0, out,
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
  if constexpr (sizeof(R) == 4) {
    auto al = [](const void* p, int a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; };
    const bool inplace = reinterpret_cast<const void*>(X) == reinterpret_cast<const void*>(out);
    const int ngrp16 = (no + 15) / 16;
    if (N % 4 == 0 && al(X, 16) && al(out, 16) && (!inplace || no <= 16) && ni <= 768) {
      const size_t smem = sizeof(float) * (size_t)ni * 16;
      const int bx = (int)std::max<size_t>(1, std::min<size_t>((size_t)nblk, (N / 4 + 255) / 256));
      k_combine_reg<16, 4><<<dim3(bx, ngrp16), 256, smem, s>>>(C, no, ni, X, N, out);
      return cudaGetLastError();
    }
    if (N % 2 == 0 && al(X, 8) && al(out, 8) && inplace && no <= 32 && ni <= 384) {
      const size_t smem = sizeof(float) * (size_t)ni * 32;
      const int bx = (int)std::max<size_t>(1, std::min<size_t>((size_t)nblk, (N / 2 + 255) / 256));
      k_combine_reg<32, 2><<<dim3(bx, 1), 256, smem, s>>>(C, no, ni, X, N, out);
      return cudaGetLastError();
    }
  }
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
                                      const R*, int*);                                                          \
  template cudaError_t launch_gram_reduce<R>(const double*, int, int, int, double, bool, double*, R*,      \
                                             cudaStream_t, int);                                          \
  template cudaError_t launch_combine<R>(const R*, int, int, const R*, size_t, R*, int, cudaStream_t);     \
  template cudaError_t launch_pair_products<R>(const R*, int, const R*, int, size_t, R*, cudaStream_t);
RSX_INST(float)
RSX_INST(double)
#undef RSX_INST

}  // namespace rsx
