// Plain block eigensolver for H = -1/2 Lap + V (fourth-order finite differences, zero
// boundary values): LOBPCG with the kinetic-energy preconditioner, optionally widened by
// the learned preconditioner's directions.  The paper's own eigensolvers are conjugate
// gradients and preconditioned Lanczos (Sec. 3.1); this block solver is the project's
// plain method.
//
// One step, k bands, basis B = [Psi | W_plain | P (| W_learned)], m = 2k .. 4k (P, the
// previous step's update direction, from the second step on):
//   R = H Psi - Psi diag(theta)              (k_residual)
//   T_i = theta_i - <psi_i, V psi_i>          (orbital kinetic energy, weighted Gram)
//   W_plain = (K + T)^-1 R by damped Jacobi   (k_ke_jacobi, K = -1/2 Lap)
//   W_learned = s net(R / s, V c)             (convnet.cu, s = |R_i|)
//   normalise the non-Psi blocks, apply H to them (k_ham_apply)
//   S = <B, B>, Hs = <B, H B> (FP64 Gram), Rayleigh-Ritz in one CTA (FP64, eigen-
//   decomposition of S with nearly dependent directions dropped)   (k_rayleigh_ritz)
//   P <- non-Psi part of Q^T B, Psi <- Q^T B (k_combine), H Psi applied afresh
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <vector>

#include "../../include/rsx.h"
#include "api_internal.cuh"
#include "dense.cuh"
#include "eig.cuh"

using namespace rsx;

namespace {

constexpr int kMaxBasis = 64;

// out = -1/2 Lap_FD4 f + V f  (or only the kinetic part when V is null; plus shift T_i f
// when shift is not null; times the domain mask when one is given, f being zero outside
// it).  f, out: [nb][n^3].  Block (x threads, rows of y), grid
// (y blocks, z, orbital): no index division, and the y / z boundary test is uniform over
// each warp (a warp holds one y row), so only the x neighbours are predicated per lane.
__device__ __forceinline__ bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

__global__ void k_ham_apply(const float* __restrict__ f, int nb, int n, float inv12h2, const float* __restrict__ V,
                            const double* __restrict__ shift, const float* __restrict__ mask, float* __restrict__ out) {
  const int x = threadIdx.x, y = blockIdx.x * blockDim.y + threadIdx.y, z = blockIdx.y, b = blockIdx.z;
  if (x >= n || y >= n) return;
  const int nn = n * n;
  const size_t N = (size_t)nn * n;
  const int v = z * nn + y * n + x;
  const float* p = f + (size_t)b * N + v;
  const float c = *p;
  // per axis 16 (f-1 + f+1) - (f-2 + f+2) - 30 c, summed as differences from c so that
  // the FP32 rounding is relative to the second differences, not to c
  auto g = [&](bool ok, int off) { return (ok ? p[off] : 0.f) - c; };
  const float a1 = g(x > 0, -1) + g(x < n - 1, 1);
  const float a2 = g(x > 1, -2) + g(x < n - 2, 2);
  float b1, b2, c1, c2;
  if (y >= 2 && y < n - 2 && z >= 2 && z < n - 2) {
    b1 = (p[-n] - c) + (p[n] - c);
    b2 = (p[-2 * n] - c) + (p[2 * n] - c);
    c1 = (p[-nn] - c) + (p[nn] - c);
    c2 = (p[-2 * nn] - c) + (p[2 * nn] - c);
  } else {
    b1 = g(y > 0, -n) + g(y < n - 1, n);
    b2 = g(y > 1, -2 * n) + g(y < n - 2, 2 * n);
    c1 = g(z > 0, -nn) + g(z < n - 1, nn);
    c2 = g(z > 1, -2 * nn) + g(z < n - 2, 2 * nn);
  }
  float lap = 16.f * a1 - a2;
  lap += 16.f * b1 - b2;
  lap += 16.f * c1 - c2;
  float r = -0.5f * lap * inv12h2;
  if (V) r += V[v] * c;
  if (shift) r += (float)shift[b] * c;
  if (mask) r *= mask[v];   // spherical domain: H restricted to the kept points
  out[(size_t)b * N + v] = r;
}

// The same operator by z-marching tiles: a block owns kHamTy rows y of 4-point float4
// columns along x (one per thread) for kHamZc consecutive planes z.  Each thread keeps
// its column's planes z-2 .. z+2 in registers (and z+3, loaded a plane ahead of its use,
// like every other global load of the loop); the plane z rows y0-2 .. y0+kHamTy+1 are
// staged in shared memory (with one zero float4 on each side in x) for the x and y
// neighbours.  One global load per point instead of thirteen; the arithmetic per point
// is that of k_ham_apply, term by term.  n % 4 == 0, every array 16-byte aligned.
// With jr given, the output is one damped Jacobi sweep on (H) x = jr instead (H with
// V = 0 and the shift T_b): out = f + omega (jr - H f) / (d0 + T_b), the arithmetic of
// k_ke_jacobi.
constexpr int kHamTy = 8;
constexpr int kHamZc = 12;

__device__ __forceinline__ float ham_point(float c, float xm2, float xm1, float xp1, float xp2, float ym2,
                                           float ym1, float yp1, float yp2, float zm2, float zm1, float zp1,
                                           float zp2, float inv12h2) {
  const float a1 = (xm1 - c) + (xp1 - c);
  const float a2 = (xm2 - c) + (xp2 - c);
  const float b1 = (ym1 - c) + (yp1 - c);
  const float b2 = (ym2 - c) + (yp2 - c);
  const float c1 = (zm1 - c) + (zp1 - c);
  const float c2 = (zm2 - c) + (zp2 - c);
  float lap = 16.f * a1 - a2;
  lap += 16.f * b1 - b2;
  lap += 16.f * c1 - c2;
  return -0.5f * lap * inv12h2;
}

__global__ void __launch_bounds__(512) k_ham_apply_z(const float* __restrict__ f, int n, float inv12h2,
                                                     const float* __restrict__ V, const double* __restrict__ shift,
                                                     const float* __restrict__ mask, const float* __restrict__ jr,
                                                     float d0, float omega, float* __restrict__ out) {
  extern __shared__ float4 hs4[];   // [kHamTy + 4][n/4 + 2]
  const int n4 = n >> 2, W = n4 + 2;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int y0 = blockIdx.x * kHamTy, y = y0 + ty;
  const int z0 = blockIdx.y * kHamZc, z1 = min(z0 + kHamZc, n);
  const int b = blockIdx.z;
  const size_t nn4 = (size_t)n * n4, N4 = nn4 * n;
  const float4* f4 = reinterpret_cast<const float4*>(f) + (size_t)b * N4;
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  auto ld = [&](int yy, int zz) {
    return (yy >= 0 && yy < n && zz >= 0 && zz < n) ? __ldg(f4 + (size_t)zz * nn4 + (size_t)yy * n4 + tx) : zero;
  };
  for (int r = ty; r < kHamTy + 4; r += kHamTy) {   // x halo: zeros, never overwritten
    if (tx == 0) hs4[r * W] = zero;
    if (tx == n4 - 1) hs4[r * W + n4 + 1] = zero;
  }
  // planes z-2 .. z+3 of this column, the halo row value of plane z (threads ty < 2 and
  // ty >= kHamTy - 2): every global load is issued one plane ahead of its use
  const bool halo_lo = ty < 2, halo_hi = ty >= kHamTy - 2;
  const int yh = halo_lo ? y0 - 2 + ty : y0 + ty + 2;
  float4 q0 = ld(y, z0 - 2), q1 = ld(y, z0 - 1), q2 = ld(y, z0), q3 = ld(y, z0 + 1), q4 = ld(y, z0 + 2);
  float4 q5 = ld(y, z0 + 3);
  float4 hv = (halo_lo || halo_hi) ? ld(yh, z0) : zero;
  const double sh = shift ? shift[b] : 0.0;
  const bool act = y < n;
  for (int z = z0; z < z1; ++z) {
    const size_t v4 = (size_t)z * nn4 + (size_t)(act ? y : 0) * n4 + tx;
    float4 vv = zero, m = zero, rr = zero;
    if (act && V) vv = __ldg(reinterpret_cast<const float4*>(V) + v4);
    if (act && mask) m = __ldg(reinterpret_cast<const float4*>(mask) + v4);
    if (act && jr) rr = __ldg(reinterpret_cast<const float4*>(jr) + (size_t)b * N4 + v4);
    const float4 qn = ld(y, z + 4);
    const float4 hn = ((halo_lo || halo_hi) && z + 1 < z1) ? ld(yh, z + 1) : zero;
    __syncthreads();   // the previous plane's neighbour reads are done
    hs4[(ty + 2) * W + 1 + tx] = q2;
    if (halo_lo) hs4[ty * W + 1 + tx] = hv;
    if (halo_hi) hs4[(ty + 4) * W + 1 + tx] = hv;
    __syncthreads();
    if (act) {
      const float4 c = q2;
      const float4 L = hs4[(ty + 2) * W + tx], R = hs4[(ty + 2) * W + 2 + tx];
      const float4 ym1 = hs4[(ty + 1) * W + 1 + tx], yp1 = hs4[(ty + 3) * W + 1 + tx];
      const float4 ym2 = hs4[ty * W + 1 + tx], yp2 = hs4[(ty + 4) * W + 1 + tx];
      float4 r;
      r.x = ham_point(c.x, L.z, L.w, c.y, c.z, ym2.x, ym1.x, yp1.x, yp2.x, q0.x, q1.x, q3.x, q4.x, inv12h2);
      r.y = ham_point(c.y, L.w, c.x, c.z, c.w, ym2.y, ym1.y, yp1.y, yp2.y, q0.y, q1.y, q3.y, q4.y, inv12h2);
      r.z = ham_point(c.z, c.x, c.y, c.w, R.x, ym2.z, ym1.z, yp1.z, yp2.z, q0.z, q1.z, q3.z, q4.z, inv12h2);
      r.w = ham_point(c.w, c.y, c.z, R.x, R.y, ym2.w, ym1.w, yp1.w, yp2.w, q0.w, q1.w, q3.w, q4.w, inv12h2);
      if (V) {
        r.x += vv.x * c.x;
        r.y += vv.y * c.y;
        r.z += vv.z * c.z;
        r.w += vv.w * c.w;
      }
      if (shift) {
        const float s = (float)sh;
        r.x += s * c.x;
        r.y += s * c.y;
        r.z += s * c.z;
        r.w += s * c.w;
      }
      if (mask) {
        r.x *= m.x;
        r.y *= m.y;
        r.z *= m.z;
        r.w *= m.w;
      }
      if (jr) {
        const float d = d0 + (float)sh;
        r.x = c.x + omega * (rr.x - r.x) / d;
        r.y = c.y + omega * (rr.y - r.y) / d;
        r.z = c.z + omega * (rr.z - r.z) / d;
        r.w = c.w + omega * (rr.w - r.w) / d;
      }
      reinterpret_cast<float4*>(out)[(size_t)b * N4 + v4] = r;
    }
    q0 = q1;
    q1 = q2;
    q2 = q3;
    q3 = q4;
    q4 = q5;
    q5 = qn;
    hv = hn;
  }
}

// launch shape of k_ham_apply: x along whole warps, as many y rows as fit in 256 threads
dim3 ham_block(int n) {
  const int xt = (n + 31) / 32 * 32;
  return dim3(xt, std::max(1, 256 / xt));
}
dim3 ham_grid(int nb, int n) {
  const dim3 bl = ham_block(n);
  return dim3((n + bl.y - 1) / bl.y, n, nb);
}

bool ham_tiles_ok(const float* f, int n, const float* V, const float* mask, const float* out, const float* jr) {
  auto al16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
  return n % 4 == 0 && (n / 4) * kHamTy <= 512 && al16(f) && al16(out) && (!V || al16(V)) && (!mask || al16(mask)) &&
         (!jr || al16(jr));
}
void launch_ham_tiles(const float* f, int nb, int n, float inv12h2, const float* V, const double* shift,
                      const float* mask, const float* jr, float d0, float omega, float* out, cudaStream_t s) {
  const int n4 = n / 4;
  const dim3 grid((n + kHamTy - 1) / kHamTy, (n + kHamZc - 1) / kHamZc, nb), block(n4, kHamTy);
  const size_t smem = sizeof(float4) * (size_t)(kHamTy + 4) * (n4 + 2);
  k_ham_apply_z<<<grid, block, smem, s>>>(f, n, inv12h2, V, shift, mask, jr, d0, omega, out);
}

// out = H f over nb bands: the z-marching tiles where the layout allows, else one thread
// per point
void launch_ham(const float* f, int nb, int n, float inv12h2, const float* V, const double* shift, const float* mask,
                float* out, cudaStream_t s) {
  if (ham_tiles_ok(f, n, V, mask, out, nullptr)) {
    launch_ham_tiles(f, nb, n, inv12h2, V, shift, mask, nullptr, 0.f, 0.f, out, s);
  } else {
    k_ham_apply<<<ham_grid(nb, n), ham_block(n), 0, s>>>(f, nb, n, inv12h2, V, shift, mask, out);
  }
}

// rows of X (row = blockIdx.y) times the domain mask
__global__ void k_mask_rows(float* __restrict__ X, const float* __restrict__ mask, size_t N) {
  float* x = X + (size_t)blockIdx.y * N;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x)
    x[i] *= mask[i];
}

// part[b * gridDim.x + blk] = this block's share of sum_v X_b(v) Y_b(v) (w(v)) for row
// b = blockIdx.y (FP32 products of four points, FP64 sums).  N % 4 == 0, rows 16-byte aligned.
__global__ void k_row_dots(const float* __restrict__ X, const float* __restrict__ Y, const float* __restrict__ w,
                           size_t N, double* __restrict__ part) {
  __shared__ double red[32];
  const int b = blockIdx.y;
  const float4* x4 = reinterpret_cast<const float4*>(X + (size_t)b * N);
  const float4* y4 = reinterpret_cast<const float4*>(Y + (size_t)b * N);
  const float4* w4 = reinterpret_cast<const float4*>(w);
  double acc = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N / 4; i += (size_t)gridDim.x * blockDim.x) {
    const float4 a = x4[i], c = y4[i];
    float4 p = make_float4(a.x * c.x, a.y * c.y, a.z * c.z, a.w * c.w);
    if (w) {
      const float4 q = w4[i];
      p = make_float4(p.x * q.x, p.y * q.y, p.z * q.z, p.w * q.w);
    }
    acc += (double)((p.x + p.y) + (p.z + p.w));
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) part[(size_t)b * gridDim.x + blockIdx.x] = t;
  }
}

// out[b] = scale * sum_p part[b * P + p], a warp per row
__global__ void k_row_reduce(const double* __restrict__ part, int P, int rows, double scale, double* __restrict__ out) {
  const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (b >= rows) return;
  double t = 0.0;
  for (int p = lane; p < P; p += 32) t += part[(size_t)b * P + p];
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if (lane == 0) out[b] = scale * t;
}

// R_i = HPsi_i - theta_i Psi_i
__global__ void k_residual(const float* __restrict__ psi, const float* __restrict__ hpsi, const double* __restrict__ th,
                           int k, size_t N, float* __restrict__ R) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  if ((N & 3) == 0 && aligned16(psi) && aligned16(hpsi) && aligned16(R)) {   // 4 points of one row per access
    const float4* p4 = reinterpret_cast<const float4*>(psi);
    const float4* h4 = reinterpret_cast<const float4*>(hpsi);
    float4* r4 = reinterpret_cast<float4*>(R);
    const size_t N4 = N / 4;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < (size_t)k * N4; i += stride) {
      const float t = (float)th[i / N4];
      const float4 p = p4[i], h = h4[i];
      r4[i] = make_float4(h.x - t * p.x, h.y - t * p.y, h.z - t * p.z, h.w - t * p.w);
    }
    return;
  }
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < (size_t)k * N; i += stride) {
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

// rows of X scaled by 1/sqrt(g[b]) (g: squared norms); zero rows stay zero.  Row b is
// blockIdx.y; the FP64 scale is formed once per thread.
__global__ void k_normalise_rows(float* __restrict__ X, const double* __restrict__ g, size_t N) {
  const double gs = g[blockIdx.y];
  const float sc = gs > 0.0 ? (float)(1.0 / sqrt(gs)) : 0.f;
  float* x = X + (size_t)blockIdx.y * N;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  if ((N & 3) == 0 && aligned16(x)) {
    float4* x4 = reinterpret_cast<float4*>(x);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N / 4; i += stride) {
      const float4 v = x4[i];
      x4[i] = make_float4(v.x * sc, v.y * sc, v.z * sc, v.w * sc);
    }
    return;
  }
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += stride) x[i] *= sc;
}

// net input [k][2][N]: channel 0 = R_i / |R_i|, channel 1 = V * vscale (row i = blockIdx.y)
__global__ void k_net_input(const float* __restrict__ R, const double* __restrict__ g, const float* __restrict__ V,
                            float vscale, size_t N, float* __restrict__ x) {
  const int b = blockIdx.y;
  const double gs = g[b];
  const float sc = gs > 0.0 ? (float)(1.0 / sqrt(gs)) : 0.f;
  for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < N; v += (size_t)gridDim.x * blockDim.x) {
    x[(2 * (size_t)b) * N + v] = R[(size_t)b * N + v] * sc;
    x[(2 * (size_t)b + 1) * N + v] = V[v] * vscale;
  }
}

// ---------------------------------------------------------------------------------
// Rayleigh-Ritz in one CTA (FP64) for m <= kMaxBasis, robust to a nearly dependent basis
// (the LOBPCG blocks W and P become nearly parallel near convergence):
//  1. S = L L^T by a right-looking Cholesky that drops direction j when its pivot falls
//     below kRrDrop S_jj (B_j within ~1e-3 rad of the span of the directions before it:
//     the FP32-summed Gram matrices leave smaller pivots, and the directions they would
//     add, dominated by rounding);
//  2. C = L^-1 Hs L^-T over the m' kept directions;
//  3. an approximate eigenbasis of C in FP32 (Householder reduction, every root of the
//     tridiagonal matrix, inverse iteration, back-transformation), then FP64 Newton
//     corrections of the k lowest vectors against C and their Rayleigh quotients;
//  4. the new orbitals' coefficients over the basis, Q = L^-T Z.
// Outputs theta[k] and qt[k][m] (float).  Fewer than k kept directions raise RSX_ENOTPD.
constexpr double kRrDrop = 1e-6;
constexpr int kRrThreads = 512;
constexpr int kRrWarps = kRrThreads / 32;
constexpr int kRrNewton = 2;   // FP64 correction steps of the Rayleigh-Ritz eigenvectors

__global__ void __launch_bounds__(kRrThreads) k_rayleigh_ritz(const double* __restrict__ Sg, const double* __restrict__ Hg,
                                                              int m, int k, double* __restrict__ theta,
                                                              float* __restrict__ qt, int* status) {
  extern __shared__ double rr_smem[];   // 4 m x m: L, Li, C, T (then Z); solve scratch 4 m per warp
  double* L = rr_smem;
  double* Li = L + m * m;
  double* C = Li + m * m;
  double* T = C + m * m;
  double* SCR = T + m * m;
  __shared__ double dg0[kMaxBasis], lam[kMaxBasis], lamh[kMaxBasis], rdg[kMaxBasis];
  __shared__ float d32[kMaxBasis], e32[kMaxBasis], e2f[kMaxBasis], lam32[kMaxBasis];
  __shared__ float tau32[kMaxBasis], vv32[kMaxBasis], pp32[kMaxBasis];
  __shared__ int kept[kMaxBasis], dropped[kMaxBasis];
  __shared__ int piv[kRrWarps][kMaxBasis];
  __shared__ int nkeep;
  __shared__ float sh_beta32, sh_tau32, sh_scale32;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  for (int q = tid; q < m * m; q += kRrThreads) {
    const int r = q / m, c = q - r * m;
    L[q] = 0.5 * (Sg[r * m + c] + Sg[c * m + r]);
    C[q] = 0.5 * (Hg[r * m + c] + Hg[c * m + r]);
  }
  if (tid < m) dg0[tid] = Sg[tid * m + tid];
  __syncthreads();
  // 1. dropping Cholesky, lower triangle of L
  for (int j = 0; j < m; ++j) {
    if (tid == 0) {
      const double pv = L[j * m + j];
      const int dr = !(pv > kRrDrop * dg0[j]);
      dropped[j] = dr;
      const double rs = dr ? 1.0 : rsqrt(pv);
      L[j * m + j] = dr ? 1.0 : pv * rs;
      rdg[j] = rs;   // 1 / L_jj
    }
    __syncthreads();
    const double rl = rdg[j];
    const int dr = dropped[j];
    for (int i = j + 1 + tid; i < m; i += kRrThreads) L[i * m + j] = dr ? 0.0 : L[i * m + j] * rl;
    __syncthreads();
    const int t = m - j - 1;
    for (int q = tid; q < t * t; q += kRrThreads) {
      const int i = j + 1 + q / t, l = j + 1 + q % t;
      if (l <= i) L[i * m + l] -= L[i * m + j] * L[l * m + j];
    }
    __syncthreads();
  }
  // L^-1, one column per thread
  if (tid < m) {
    const int c = tid;
    for (int i = 0; i < c; ++i) Li[i * m + c] = 0.0;
    Li[c * m + c] = rdg[c];
    for (int i = c + 1; i < m; ++i) {
      // four partial sums: shorter dependent chains
      double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
      int p = c;
      for (; p + 3 < i; p += 4) {
        s0 += L[i * m + p] * Li[p * m + c];
        s1 += L[i * m + p + 1] * Li[(p + 1) * m + c];
        s2 += L[i * m + p + 2] * Li[(p + 2) * m + c];
        s3 += L[i * m + p + 3] * Li[(p + 3) * m + c];
      }
      for (; p < i; ++p) s0 += L[i * m + p] * Li[p * m + c];
      Li[i * m + c] = -((s0 + s1) + (s2 + s3)) * rdg[i];
    }
  }
  if (tid == 0) {
    int nk = 0;
    for (int j = 0; j < m; ++j)
      if (!dropped[j]) kept[nk++] = j;
    nkeep = nk;
  }
  __syncthreads();
  const int n = nkeep;
  if (n < k) {
    if (tid < k) theta[tid] = 0.0;
    for (int q = tid; q < k * m; q += kRrThreads) qt[q] = 0.f;
    if (tid == 0 && status) atomicMax(status, RSX_ENOTPD);
    return;
  }
  // 2. T = Li Hs (rows of kept directions), C' = T Li^T over kept pairs (n x n, in C)
  for (int q = tid; q < n * m; q += kRrThreads) {
    const int a = q / m, c = q - a * m, i = kept[a];
    double s = 0.0;
    for (int p = 0; p <= i; ++p) s += Li[i * m + p] * C[p * m + c];
    T[a * m + c] = s;
  }
  __syncthreads();
  for (int q = tid; q < n * n; q += kRrThreads) {
    const int a = q / n, b = q - a * n;
    if (b > a) continue;
    const int l = kept[b];
    double s = 0.0;
    for (int p = 0; p <= l; ++p) s += T[a * m + p] * Li[l * m + p];
    C[a * n + b] = s;
    C[b * n + a] = s;
  }
  __syncthreads();
  // 3. Eigenpairs of C' (n x n).  FP64 latency is long on this part, so an approximate
  //    eigenbasis comes from FP32 (Householder reduction of C' rounded, every root of T
  //    by Sturm multisection, inverse iteration, back-transformation), and the k wanted
  //    vectors are then corrected against C' itself in FP64 (Newton steps of the
  //    correction equation in that basis, as in the dense eigensolver), which converges
  //    quadratically from FP32 accuracy; their Rayleigh quotients are the Ritz values.
  float* C32 = reinterpret_cast<float*>(L);     // n x n (L is dead after L^-1)
  float* X32 = C32 + n * n;                     // n x n: vectors of T, then of C'32
  float* SC32 = reinterpret_cast<float*>(SCR);  // 4 n floats per warp
  for (int q = tid; q < n * n; q += kRrThreads) C32[q] = (float)C[q];
  __syncthreads();
  // 3a. FP32 Householder reduction (reflectors below the subdiagonal, tau32)
  for (int kk = 0; kk + 2 < n; ++kk) {
    const int m0 = kk + 1;
    if (warp == 0) {
      float sq = 0.f;
      for (int i = m0 + 1 + lane; i < n; i += 32) sq += C32[i * n + kk] * C32[i * n + kk];
      const float xn2 = warp_sum(sq);
      if (lane == 0) {
        const float alpha = C32[m0 * n + kk];
        if (xn2 == 0.f) {
          sh_tau32 = 0.f;
          sh_beta32 = alpha;
          sh_scale32 = 0.f;
        } else {
          const float s2 = alpha * alpha + xn2, rs = rsqrtf(s2);
          const float beta = -copysignf(s2 * rs, alpha);
          sh_tau32 = 1.f + fabsf(alpha) * rs;
          sh_scale32 = 1.f / (alpha - beta);
          sh_beta32 = beta;
        }
        e32[kk] = sh_beta32;
        tau32[kk] = sh_tau32;
        d32[kk] = C32[kk * n + kk];
      }
    }
    __syncthreads();
    const float tk = sh_tau32;
    for (int i = m0 + tid; i < n; i += kRrThreads) {
      const float vi = (i == m0) ? 1.f : C32[i * n + kk] * sh_scale32;
      vv32[i] = vi;
      if (i > m0) C32[i * n + kk] = vi;
    }
    __syncthreads();
    if (tk != 0.f) {
      {  // p = tk C v over the trailing block: 8 threads per row (n <= 64 rows)
        const int g = tid & 7, i = m0 + (tid >> 3);
        float acc = 0.f;
        if (i < n)
          for (int jj = m0 + g; jj < n; jj += 8) acc += C32[i * n + jj] * vv32[jj];
        acc += __shfl_xor_sync(0xffffffffu, acc, 1);
        acc += __shfl_xor_sync(0xffffffffu, acc, 2);
        acc += __shfl_xor_sync(0xffffffffu, acc, 4);
        if (g == 0 && i < n) pp32[i] = tk * acc;
      }
      __syncthreads();
      if (warp == 0) {   // w = p - (tau/2)(p^T v) v
        float pv = 0.f;
        for (int i = m0 + lane; i < n; i += 32) pv += pp32[i] * vv32[i];
        const float cc = 0.5f * tk * warp_sum(pv);
        for (int i = m0 + lane; i < n; i += 32) pp32[i] -= cc * vv32[i];
      }
      __syncthreads();
      const int t = n - m0;
      for (int q = tid; q < t * t; q += kRrThreads) {
        const int i = m0 + q / t, jj = m0 + q % t;
        C32[i * n + jj] -= vv32[i] * pp32[jj] + pp32[i] * vv32[jj];
      }
      __syncthreads();
    }
  }
  if (tid == 0) {
    if (n >= 2) {
      d32[n - 2] = C32[(n - 2) * n + (n - 2)];
      e32[n - 2] = C32[(n - 1) * n + (n - 2)];
    }
    if (n >= 3) tau32[n - 2] = 0.f;
    d32[n - 1] = C32[(n - 1) * n + (n - 1)];
  }
  __syncthreads();
  if (tid < n - 1) e2f[tid] = e32[tid] * e32[tid];
  __syncthreads();
  // 3b. every root of T: Sturm multisection, a warp per root (32 points per round)
  float lo0 = d32[0], hi0 = d32[0], emax = 0.f;
  for (int i = 0; i < n; ++i) {
    const float r = (i > 0 ? fabsf(e32[i - 1]) : 0.f) + (i < n - 1 ? fabsf(e32[i]) : 0.f);
    lo0 = fminf(lo0, d32[i] - r);
    hi0 = fmaxf(hi0, d32[i] + r);
    if (i < n - 1) emax = fmaxf(emax, fabsf(e32[i]));
  }
  const float scale = fmaxf(fabsf(lo0), fabsf(hi0));
  lo0 -= 1e-6f * scale + 1e-30f;
  hi0 += 1e-6f * scale + 1e-30f;
  const float pivmin = 1.2e-38f * fmaxf(1.f, emax * emax);
  for (int r = warp; r < n; r += kRrWarps) {
    float lo = lo0, hi = hi0;
    for (int round = 0; round < 8; ++round) {
      if (!(hi - lo > 2.4e-7f * fmaxf(fabsf(lo), fabsf(hi)))) break;
      const float x = lo + (hi - lo) * (float)(lane + 1) / 33.f;
      const unsigned above = __ballot_sync(0xffffffffu, sturm_count_f32(d32, e2f, n, x, pivmin) > r);
      const int f = above ? __ffs(above) - 1 : 32;
      const float nlo = (f == 0) ? lo : lo + (hi - lo) * (float)f / 33.f;
      const float nhi = (f == 32) ? hi : lo + (hi - lo) * (float)(f + 1) / 33.f;
      lo = nlo;
      hi = nhi;
    }
    if (lane == 0) lam32[r] = 0.5f * (lo + hi);
  }
  __syncthreads();
  // 3c. vectors of T by inverse iteration; among the wanted roots and a margin above
  //     them, roots closer than gap32 to the previous one are redone in order, orthogonal
  //     to the earlier members of their run (higher vectors only carry the small
  //     corrections along far directions, where a duplicate costs nothing measurable)
  const float gap32 = 1e-5f * fmaxf(1.f, scale);
  for (int r = warp; r < n; r += kRrWarps) {
    float* z = X32 + r * n;
    for (int i = lane; i < n; i += 32) z[i] = 1.f + 0.001f * (float)((i * 7919 + r * 104729) % 997);
    __syncwarp();
    warp_inverse_iteration<float>(d32, e32, n, lam32[r], z, SC32 + warp * 4 * n, piv[warp], 3, X32, n, 0u);
  }
  __syncthreads();
  if (warp == 0) {
    for (int r = 1; r < min(n, k + 8); ++r) {
      int j0 = r;
      while (j0 > 0 && lam32[r] - lam32[j0 - 1] < gap32) --j0;
      if (j0 == r) continue;
      float* z = X32 + r * n;
      for (int i = lane; i < n; i += 32) z[i] = 1.f + 0.001f * (float)((i * 7919 + r * 104729) % 997);
      __syncwarp();
      if (lane == 0) tri_factor_shifted<float>(d32, e32, n, lam32[r], SC32, piv[0]);
      __syncwarp();
      for (int it = 0; it < 3; ++it) {
        if (lane == 0) tri_solve_factored<float>(n, z, SC32, piv[0]);
        __syncwarp();
        for (int j = j0; j < r; ++j) {
          const float* zj = X32 + j * n;
          float dot = 0.f;
          for (int i = lane; i < n; i += 32) dot += zj[i] * z[i];
          dot = warp_sum(dot);
          for (int i = lane; i < n; i += 32) z[i] -= dot * zj[i];
          __syncwarp();
        }
        float nn = 0.f;
        for (int i = lane; i < n; i += 32) nn += z[i] * z[i];
        nn = warp_sum(nn);
        const float inv = nn > 0.f ? 1.f / sqrtf(nn) : 0.f;
        for (int i = lane; i < n; i += 32) z[i] *= inv;
        __syncwarp();
      }
    }
  }
  __syncthreads();
  // 3d. back-transformation of every vector, z <- H_0 ... H_{n-3} z (two entries per lane)
  for (int r = warp; r < n; r += kRrWarps) {
    float* z = X32 + r * n;
    const int i0 = lane, i1 = lane + 32;
    float z0 = i0 < n ? z[i0] : 0.f, z1 = i1 < n ? z[i1] : 0.f;
    for (int kk = n - 3; kk >= 0; --kk) {
      const float tk = tau32[kk];
      if (tk == 0.f) continue;
      const float v0 = i0 > kk + 1 && i0 < n ? C32[i0 * n + kk] : (i0 == kk + 1 ? 1.f : 0.f);
      const float v1 = i1 > kk + 1 && i1 < n ? C32[i1 * n + kk] : (i1 == kk + 1 ? 1.f : 0.f);
      const float sd = tk * warp_sum(v0 * z0 + v1 * z1);
      z0 -= sd * v0;
      z1 -= sd * v1;
    }
    if (i0 < n) z[i0] = z0;
    if (i1 < n) z[i1] = z1;
  }
  __syncthreads();
  // 3e. FP64 Newton corrections of the k lowest vectors against C' (FP64, in C):
  //     r_j = C' x_j - theta_j x_j, x_j <- x_j - sum_i xh_i <xh_i, r_j> / (lambda_i - theta_j)
  //     over the roots i farther than gthr from theta_j; then the final Rayleigh quotients.
  double* Z = T;                   // k x n: the corrected vectors (read by step 4)
  double* Yk = SCR;                // k x n: C' x
  double* Rk = Yk + k * n;         // k x n: residuals, then correction coefficients
  double* Cm = Rk + k * n;         // n x k: <xh_i, r_j>
  if (tid < n) lamh[tid] = (double)lam32[tid];
  for (int q = tid; q < k * n; q += kRrThreads) Z[q] = (double)X32[q];
  const double gthr = 1e-5 * fmax(1.0, (double)scale);
  __syncthreads();
  for (int it = 0; it <= kRrNewton; ++it) {
    for (int q = tid; q < k * n; q += kRrThreads) {   // Yk = Z C' (C' symmetric)
      const int j = q / n, i = q - j * n;
      const double* zr = Z + j * n;
      double a0 = 0.0, a1 = 0.0;
      int l = 0;
      for (; l + 1 < n; l += 2) {
        a0 += zr[l] * C[l * n + i];
        a1 += zr[l + 1] * C[(l + 1) * n + i];
      }
      if (l < n) a0 += zr[l] * C[l * n + i];
      Yk[q] = a0 + a1;
    }
    __syncthreads();
    for (int j = warp; j < k; j += kRrWarps) {   // Rayleigh quotients
      double a = 0.0, b = 0.0;
      for (int i = lane; i < n; i += 32) {
        a += Z[j * n + i] * Yk[j * n + i];
        b += Z[j * n + i] * Z[j * n + i];
      }
      a = warp_sum(a);
      b = warp_sum(b);
      if (lane == 0) lam[j] = a / b;
    }
    __syncthreads();
    if (it == kRrNewton) break;
    for (int q = tid; q < k * n; q += kRrThreads) Rk[q] = Yk[q] - lam[q / n] * Z[q];
    __syncthreads();
    // the correction's own error is second order, so its two products run in FP32
    // (the residual above needs FP64: it is a difference of nearly equal terms)
    for (int q = tid; q < n * k; q += kRrThreads) {   // Cm[i][j] = <xh_i, r_j>
      const int i = q / k, j = q - i * k;
      const float* xr = X32 + i * n;
      const double* rr = Rk + j * n;
      float a0 = 0.f, a1 = 0.f;
      int l = 0;
      for (; l + 1 < n; l += 2) {
        a0 = fmaf(xr[l], (float)rr[l], a0);
        a1 = fmaf(xr[l + 1], (float)rr[l + 1], a1);
      }
      if (l < n) a0 = fmaf(xr[l], (float)rr[l], a0);
      Cm[q] = (double)(a0 + a1);
    }
    __syncthreads();
    for (int q = tid; q < k * n; q += kRrThreads) {   // coefficients, into Rk
      const int j = q / n, i = q - j * n;
      const double dl = lamh[i] - lam[j];
      Rk[q] = fabs(dl) > gthr ? -Cm[i * k + j] / dl : 0.0;
    }
    __syncthreads();
    for (int q = tid; q < k * n; q += kRrThreads) {   // Z += coefficients x Xh
      const int j = q / n, i = q - j * n;
      const double* cr = Rk + j * n;
      float a0 = 0.f, a1 = 0.f;
      int l = 0;
      for (; l + 1 < n; l += 2) {
        a0 = fmaf((float)cr[l], X32[l * n + i], a0);
        a1 = fmaf((float)cr[l + 1], X32[(l + 1) * n + i], a1);
      }
      if (l < n) a0 = fmaf((float)cr[l], X32[l * n + i], a0);
      Z[q] += (double)(a0 + a1);
    }
    __syncthreads();
  }
  // 4. qt[o][r] = sum_a Li[kept[a]][r] Z[o][a]
  for (int q = tid; q < k * m; q += kRrThreads) {
    const int o = q / m, r = q - o * m;
    double s = 0.0;
    for (int a = 0; a < n; ++a) s += Li[kept[a] * m + r] * Z[o * n + a];
    qt[q] = (float)s;
  }
  if (tid < k) theta[tid] = lam[tid];
}

// out[b][v] -= sum_a C[a][b] xi[a][v]  (the ACE term -xi <xi, f> of Eq. 13, C = <xi, f>).
// The projectors are taken 16 at a time into registers; C is staged in shared memory,
// zero-padded to a multiple of 16 rows (16 * ceil(nxi / 16) * nb <= 64 * kMaxBasis).
__global__ void k_ace_accumulate(float* __restrict__ out, const float* __restrict__ xi, const double* __restrict__ C,
                                 int nxi, int nb, size_t N) {
  __shared__ float cs[64 * kMaxBasis];
  const int na = (nxi + 15) & ~15;
  for (int i = threadIdx.x; i < na * nb; i += blockDim.x) cs[i] = i < nxi * nb ? (float)C[i] : 0.f;
  __syncthreads();
  for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < N; v += (size_t)gridDim.x * blockDim.x) {
    for (int a0 = 0; a0 < na; a0 += 16) {
      float x[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) x[j] = a0 + j < nxi ? xi[(size_t)(a0 + j) * N + v] : 0.f;
      for (int b = 0; b < nb; ++b) {
        float acc = 0.f;
#pragma unroll
        for (int j = 0; j < 16; ++j) acc = fmaf(cs[(a0 + j) * nb + b], x[j], acc);
        out[(size_t)b * N + v] -= acc;
      }
    }
  }
}

// out += x (n elements)
__global__ void k_accumulate(float* __restrict__ out, const float* __restrict__ x, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] += x[i];
}

// closed-shell density rho = 2 sum_i phi_i^2
__global__ void k_density(const float* __restrict__ phi, int nocc, size_t N, float* __restrict__ rho) {
  for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < N; v += (size_t)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int i = 0; i < nocc; ++i) {
      const float f = phi[(size_t)i * N + v];
      s = fmaf(f, f, s);
    }
    rho[v] = 2.f * s;
  }
}

// part[blk] = partial sums of |a - b| (FP64); a_next = alpha a + (1 - alpha) b (the linear
// mixing of the input density a with the output density b) when mix != 0
__global__ void k_absdiff_mix(float* __restrict__ a, const float* __restrict__ b, size_t N, float alpha, int mix,
                              double* __restrict__ part) {
  __shared__ double red[8];
  double s = 0.0;
  for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < N; v += (size_t)gridDim.x * blockDim.x) {
    const float av = a[v], bv = b[v];
    s += fabs((double)av - (double)bv);
    if (mix) a[v] = alpha * av + (1.f - alpha) * bv;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    part[blockIdx.x] = t;
  }
}

// out = a + b (n elements)
__global__ void k_add(const float* __restrict__ a, const float* __restrict__ b, size_t n, float* __restrict__ out) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = a[i] + b[i];
}

// qp[i][j] = qt[i][k + j]: the coefficients of the new orbitals over the non-Psi blocks
__global__ void k_tail_cols(const float* __restrict__ qt, int k, int m, float* __restrict__ qp) {
  for (int i = threadIdx.x; i < k * (m - k); i += blockDim.x) {
    const int r = i / (m - k), c = i - r * (m - k);
    qp[i] = qt[r * m + k + c];
  }
}

// coef[j][i] (k x 2k) over [phi_in; phi_out]: alpha on input orbital j and (1 - alpha)
// O[i][j] = (1 - alpha) <out_i, in_j> on output orbital i, so that row j is
// alpha phi_in_j + (1 - alpha) (projection of phi_in_j on the span of the outputs)
__global__ void k_state_mix_coeffs(const double* __restrict__ O, int k, float alpha, float* __restrict__ coef) {
  for (int q = threadIdx.x; q < 2 * k * k; q += blockDim.x) {
    const int j = q / (2 * k), i = q - j * 2 * k;
    coef[q] = i < k ? (i == j ? alpha : 0.f) : (float)((1.0 - (double)alpha) * O[(i - k) * k + j]);
  }
}

// S = L L^T (k <= 32, FP64, one warp); linv[j][i] = (L^-1)[j][i] as float, so that
// rows linv X are orthonormal when S is the Gram matrix of the rows of X.  A pivot
// that is not positive raises RSX_ENOTPD in *status (the rows are then left unscaled).
__global__ void k_chol_inv_small(const double* __restrict__ S, int k, float* __restrict__ linv, int* status) {
  __shared__ double L[32 * 32], Li[32 * 32];
  const int lane = threadIdx.x;
  for (int q = lane; q < k * k; q += 32) {
    L[q] = S[q];
    Li[q] = 0.0;
  }
  __syncwarp();
  for (int j = 0; j < k; ++j) {
    if (lane == 0) {
      double d = L[j * k + j];
      if (!(d > 0.0)) {
        atomicMax(status, RSX_ENOTPD);
        d = 1.0;
      }
      L[j * k + j] = sqrt(d);
    }
    __syncwarp();
    const double rl = 1.0 / L[j * k + j];
    if (lane > j && lane < k) L[lane * k + j] *= rl;
    __syncwarp();
    for (int i = j + 1 + lane; i < k; i += 32)
      for (int l = j + 1; l <= i; ++l) L[i * k + l] -= L[i * k + j] * L[l * k + j];
    __syncwarp();
  }
  if (lane < k) {
    const int c = lane;
    Li[c * k + c] = 1.0 / L[c * k + c];
    for (int i = c + 1; i < k; ++i) {
      double sum = 0.0;
      for (int p = c; p < i; ++p) sum += L[i * k + p] * Li[p * k + c];
      Li[i * k + c] = -sum / L[i * k + i];
    }
  }
  __syncwarp();
  for (int q = lane; q < k * k; q += 32) linv[q] = (float)Li[q];
}

size_t blocks_for(size_t n) { return std::min<size_t>((n + 255) / 256, 4096); }
// x-blocks of a (blocks, rows) grid over `rows` rows of N elements (256 threads)
size_t row_blocks(size_t N, int rows) { return std::max<size_t>(1, std::min<size_t>((N + 255) / 256, 4096 / rows)); }

}  // namespace

namespace {

// ---- FP64 energy of the current block (rsx_eig_energy64)
__global__ void k_cast64(const float* __restrict__ x, size_t n, double* __restrict__ y) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = (double)x[i];
}

// out = (-1/2 Lap_FD4 + V) f in FP64 (times the domain mask), f: [nb][n^3], zero values
// outside the box; the stencil of k_ham_apply in double precision
__global__ void k_ham_apply64(const double* __restrict__ f, int nb, int n, double inv12h2, const float* __restrict__ V,
                              const float* __restrict__ mask, double* __restrict__ out) {
  const int nn = n * n;
  const size_t N = (size_t)nn * n, tot = N * nb;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < tot; i += (size_t)gridDim.x * blockDim.x) {
    const size_t b = i / N;
    const int v = (int)(i - b * N);
    const int z = v / nn, y = (v - z * nn) / n, x = v - z * nn - y * n;
    const double* p = f + i;
    const double c = *p;
    auto g = [&](bool ok, int off) { return (ok ? p[off] : 0.0) - c; };
    const double a1 = g(x > 0, -1) + g(x < n - 1, 1), a2 = g(x > 1, -2) + g(x < n - 2, 2);
    const double b1 = g(y > 0, -n) + g(y < n - 1, n), b2 = g(y > 1, -2 * n) + g(y < n - 2, 2 * n);
    const double c1 = g(z > 0, -nn) + g(z < n - 1, nn), c2 = g(z > 1, -2 * nn) + g(z < n - 2, 2 * nn);
    const double lap = (16.0 * a1 - a2) + (16.0 * b1 - b2) + (16.0 * c1 - c2);
    double r = -0.5 * lap * inv12h2 + (double)V[v] * c;
    if (mask) r *= (double)mask[v];
    out[i] = r;
  }
}

// energy = trace(S^-1 Hs) = trace(L^-1 Hs L^-T), S = L L^T (k x k, FP64, one warp)
__global__ void k_rr_trace(const double* __restrict__ S, const double* __restrict__ Hs, int k,
                           double* __restrict__ out) {
  __shared__ double L[32 * 32], W[32 * 32], T[32 * 32];
  const int lane = threadIdx.x;
  for (int i = lane; i < k * k; i += 32) {
    L[i] = 0.0;
    const int r = i / k, c = i - r * k;
    W[i] = 0.5 * (Hs[r * k + c] + Hs[c * k + r]);
  }
  __syncwarp();
  for (int j = 0; j < k; ++j) {
    if (lane == 0) {
      double d = S[j * k + j];
      for (int p = 0; p < j; ++p) d -= L[j * k + p] * L[j * k + p];
      L[j * k + j] = sqrt(d > 0.0 ? d : 1e-300);
    }
    __syncwarp();
    for (int i = j + 1 + lane; i < k; i += 32) {
      double a = 0.5 * (S[i * k + j] + S[j * k + i]);
      for (int p = 0; p < j; ++p) a -= L[i * k + p] * L[j * k + p];
      L[i * k + j] = a / L[j * k + j];
    }
    __syncwarp();
  }
  // T = L^-1 W (columns over lanes), then W = L^-1 T^T, trace of the result
  for (int pass = 0; pass < 2; ++pass) {
    for (int c = lane; c < k; c += 32)
      for (int i = 0; i < k; ++i) {
        double a = pass == 0 ? W[i * k + c] : T[c * k + i];
        for (int p = 0; p < i; ++p) a -= L[i * k + p] * (pass == 0 ? T[p * k + c] : W[p * k + c]);
        (pass == 0 ? T : W)[i * k + c] = a / L[i * k + i];
      }
    __syncwarp();
  }
  if (lane == 0) {
    double tr = 0.0;
    for (int i = 0; i < k; ++i) tr += W[i * k + i];
    *out = tr;
  }
}

}  // namespace

struct rsx_eig {
  rsx_ctx* ctx = nullptr;        // owns the Gram / combine workspace
  int n = 0, k = 0;
  double h = 0.0;
  const float* V = nullptr;      // caller's potential (device)
  float vscale = 1.f;
  float* B = nullptr;            // [4k][N] basis: Psi | W_plain | P (| W_learned)
  float* HB = nullptr;           // [4k][N]
  float* R = nullptr;            // [k][N] residual of the last step
  float* tmp = nullptr;          // [2k][N] Jacobi scratch / net input
  float* xnet = nullptr;         // [k][2][N]
  double* sm = nullptr;          // small FP64: theta, T, gram outputs, S, Hs
  float* qt = nullptr;           // [k][4k]
  float* qp = nullptr;           // [k][3k] coefficients over the non-Psi blocks
  bool started = false;
  bool has_p = false;            // P (the previous update direction) is in the basis
  // non-local exchange term of H (rsx_eig_set_exchange): 0 none, 1 ACE -xi xi^T with
  // projectors xsrc [xcount][N], 2 exact exchange Vx[xsrc] of orbitals xsrc through xctx
  int xmode = 0;
  const float* xsrc = nullptr;
  int xcount = 0;
  rsx_ctx* xctx = nullptr;
  float* xbuf = nullptr;         // [4k][N] exact-exchange output
  const float* mask = nullptr;   // spherical domain (rsx_eig_set_mask), caller's [N] 0/1
  double* e64 = nullptr;         // rsx_eig_energy64: Psi and H Psi in FP64 [2k][N] + small matrices
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
  rc = check_cuda(c, launch_gram<float>(X, na, Y, nb, N, c->dsm, nblk, s, w, c->status), "gram");
  if (rc) return rc;
  return check_cuda(c, launch_gram_reduce<float>(c->dsm, nblk, na, nb, e->h * e->h * e->h, false, out, (float*)nullptr, s),
                    "gram reduce");
}

// out[b] = h^3 <X_b, Y_b w> for b < rows (w may be null)
int row_dots(rsx_eig* e, const float* X, const float* Y, const float* w, int rows, double* out, cudaStream_t s) {
  rsx_ctx* c = e->ctx;
  const size_t N = (size_t)e->n * e->n * e->n;
  const int P = std::max(1, std::min(256, 4 * c->nsm / rows));
  int rc = grow(c, (void**)&c->dsm, &c->dsm_bytes, sizeof(double) * ((size_t)2 * c->nsm * 4096 + 3 * 4096), "small FP64");
  if (rc) return rc;
  k_row_dots<<<dim3(P, rows), 256, 0, s>>>(X, Y, w, N, c->dsm);
  k_row_reduce<<<(rows + 7) / 8, 256, 0, s>>>(c->dsm, P, rows, e->h * e->h * e->h, out);
  return ecuda(e, cudaGetLastError(), "row dots");
}

// out = H f (the full operator, with the exchange term, when V is given; the kinetic part
// plus shift when V is null)
int ham(rsx_eig* e, const float* f, int nb, float* out, const double* shift, const float* V, cudaStream_t s) {
  const size_t N = (size_t)e->n * e->n * e->n;
  launch_ham(f, nb, e->n, (float)(1.0 / (12.0 * e->h * e->h)), V, shift, e->mask, out, s);
  int rc = ecuda(e, cudaGetLastError(), "hamiltonian");
  if (rc || !V || e->xmode == 0) return rc;
  if (e->xmode == 1) {
    double* C = e->sm + 256 + 2 * kMaxBasis * kMaxBasis;   // [xcount][nb], past the Rayleigh-Ritz matrices
    rc = gram(e, e->xsrc, e->xcount, f, nb, nullptr, C, s);
    if (rc) return rc;
    k_ace_accumulate<<<(unsigned)std::min<size_t>((N + 255) / 256, 2048), 256, 0, s>>>(out, e->xsrc, C, e->xcount, nb, N);
    return ecuda(e, cudaGetLastError(), "ACE term");
  }
  rc = rsx_exchange_apply(e->xctx, e->xsrc, e->xcount, f, nb, e->xbuf, s);
  if (rc) return efail(e, rc, "exact exchange in H failed");
  k_accumulate<<<(unsigned)blocks_for(nb * N), 256, 0, s>>>(out, e->xbuf, nb * N);
  return ecuda(e, cudaGetLastError(), "exchange term");
}

// Rayleigh-Ritz over the first m rows of B / HB, update Psi (in place), P (when keep_p)
// and H Psi
int rr_update(rsx_eig* e, int m, bool keep_p, cudaStream_t s) {
  const int k = e->k;
  const size_t N = (size_t)e->n * e->n * e->n;
  double* S = e->sm + 256;
  double* Hs = S + kMaxBasis * kMaxBasis;
  double* theta = e->sm;
  int rc = gram(e, e->B, m, e->B, m, nullptr, S, s);
  if (!rc) rc = gram(e, e->B, m, e->HB, m, nullptr, Hs, s);
  if (rc) return rc;
  const size_t smem = (4 * (size_t)m * m + 4 * (size_t)kRrWarps * m) * sizeof(double);
  cudaFuncSetAttribute(k_rayleigh_ritz, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_rayleigh_ritz<<<1, kRrThreads, smem, s>>>(S, Hs, m, k, theta, e->qt, e->ctx->status);
  rc = ecuda(e, cudaGetLastError(), "rayleigh-ritz");
  if (rc) return rc;
  // LOBPCG direction P = (new Psi minus its Psi-block part), from the old non-Psi blocks,
  // into scratch before Psi is updated in place; then moved into the P slot (rows 2k..3k)
  const bool with_p = m > k && keep_p;
  if (with_p) {
    k_tail_cols<<<1, 256, 0, s>>>(e->qt, k, m, e->qp);
    rc = check_cuda(e->ctx, launch_combine<float>(e->qp, k, m - k, e->B + (size_t)k * N, N, e->tmp, 4 * e->ctx->nsm, s),
                    "p update");
    if (rc) return rc;
  }
  rc = check_cuda(e->ctx, launch_combine<float>(e->qt, k, m, e->B, N, e->B, 4 * e->ctx->nsm, s), "psi update");
  if (!rc && with_p)
    rc = ecuda(e, cudaMemcpyAsync(e->B + 2 * (size_t)k * N, e->tmp, (size_t)k * N * sizeof(float),
                                  cudaMemcpyDeviceToDevice, s), "p move");
  e->has_p = with_p && rc == RSX_OK;
  // H Psi is applied afresh (not combined from H B) so that rounding does not accumulate
  // over the iterations
  if (!rc) rc = ham(e, e->B, k, e->HB, nullptr, e->V, s);
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
  if (cudaMalloc(&e->B, 4 * nband * N * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&e->HB, 4 * nband * N * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&e->R, nband * N * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&e->tmp, 2 * nband * N * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&e->xnet, 2 * nband * N * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&e->sm, (256 + 3 * kMaxBasis * kMaxBasis) * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&e->qt, kMaxBasis * kMaxBasis * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&e->qp, kMaxBasis * kMaxBasis * sizeof(float)) != cudaSuccess) {
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
  if (!rc && e->mask) {
    k_mask_rows<<<dim3((unsigned)row_blocks(N, e->k), e->k), 256, 0, s>>>(e->B, e->mask, N);
    rc = ecuda(e, cudaGetLastError(), "init mask");
  }
  if (!rc) rc = ham(e, e->B, e->k, e->HB, nullptr, e->V, s);
  e->has_p = false;
  if (!rc) rc = rr_update(e, e->k, false, s);
  e->started = rc == RSX_OK;
  return rc;
}

// One step; net may be NULL (plain).  theta_host[k] receives the new Ritz values; the
// residual used in this step is kept (rsx_eig_residual).  Synchronises the stream.
int rsx_eig_step(rsx_eig* e, rsx_net* net, int jacobi_sweeps, double* theta_host, void* stream) {
  rsx::NvtxRange nvtx_range("rsx_eig_step");
  if (!e || !e->started || jacobi_sweeps < 0) return RSX_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const int k = e->k;
  const size_t N = (size_t)e->n * e->n * e->n;
  double* theta = e->sm;
  double* T = e->sm + 64;
  double* diag = e->sm + 128;
  float* psi = e->B;
  float* hpsi = e->HB;
  float* wp = e->B + k * N;
  // residual
  k_residual<<<(unsigned)blocks_for(k * N), 256, 0, s>>>(psi, hpsi, theta, k, N, e->R);
  // kinetic energies T_i = theta_i - <psi_i, V psi_i>
  int rc = row_dots(e, psi, psi, e->V, k, diag, s);
  if (rc) return rc;
  k_kinetic<<<1, 64, 0, s>>>(theta, diag, k, T);
  rc = ecuda(e, cudaGetLastError(), "kinetic");
  if (rc) return rc;
  // plain preconditioner: damped Jacobi sweeps on (K + T) x = R
  const float d0 = (float)(3.75 / (e->h * e->h));
  const float omega = 2.f / 3.f;
  float* x = wp;
  float* ax = e->tmp;
  if (ham_tiles_ok(wp, e->n, nullptr, e->mask, e->tmp + k * N, e->R) &&
      ham_tiles_ok(e->tmp + k * N, e->n, nullptr, e->mask, wp, e->R)) {
    // each sweep one fused stencil launch, alternating between W and a scratch block so
    // that the last sweep writes W
    float* buf[2] = {wp, e->tmp + k * N};
    int cur = jacobi_sweeps % 2;
    k_ke_jacobi<<<(unsigned)blocks_for(k * N), 256, 0, s>>>(e->R, nullptr, nullptr, T, k, N, d0, omega, buf[cur]);
    for (int sw = 0; sw < jacobi_sweeps; ++sw, cur ^= 1)
      launch_ham_tiles(buf[cur], k, e->n, (float)(1.0 / (12.0 * e->h * e->h)), nullptr, T, e->mask, e->R, d0, omega,
                       buf[cur ^ 1], s);
    rc = ecuda(e, cudaGetLastError(), "jacobi sweeps");
    if (rc) return rc;
  } else {
    k_ke_jacobi<<<(unsigned)blocks_for(k * N), 256, 0, s>>>(e->R, nullptr, nullptr, T, k, N, d0, omega, x);
    for (int sw = 0; sw < jacobi_sweeps; ++sw) {
      rc = ham(e, x, k, ax, T, nullptr, s);
      if (rc) return rc;
      k_ke_jacobi<<<(unsigned)blocks_for(k * N), 256, 0, s>>>(e->R, x, ax, T, k, N, d0, omega, e->tmp + k * N);
      rc = ecuda(e, cudaMemcpyAsync(x, e->tmp + k * N, k * N * sizeof(float), cudaMemcpyDeviceToDevice, s), "jacobi copy");
      if (rc) return rc;
    }
  }
  // basis: Psi | W | P (LOBPCG, from the second step on) | W_learned (with a network)
  int m = e->has_p ? 3 * k : 2 * k;
  // learned directions
  if (net) {
    rc = row_dots(e, e->R, e->R, nullptr, k, diag, s);
    if (rc) return rc;
    k_net_input<<<dim3((unsigned)row_blocks(N, k), k), 256, 0, s>>>(e->R, diag, e->V, e->vscale, N, e->xnet);
    float* wl = e->B + (size_t)m * N;
    rc = rsx_net_forward(net, e->xnet, k, e->n, e->n, e->n, wl, s);
    if (rc) return efail(e, rc, "learned preconditioner forward failed");
    if (e->mask) k_mask_rows<<<dim3((unsigned)row_blocks(N, k), k), 256, 0, s>>>(wl, e->mask, N);
    m += k;
  }
  // normalise the W blocks, apply H to them
  rc = row_dots(e, wp, wp, nullptr, m - k, diag, s);
  if (rc) return rc;
  k_normalise_rows<<<dim3((unsigned)row_blocks(N, m - k), m - k), 256, 0, s>>>(wp, diag, N);
  rc = ham(e, wp, m - k, e->HB + k * N, nullptr, e->V, s);
  if (rc) return rc;
  // keep a P block for the next step when Psi | W | P (| W_learned) still fits
  rc = rr_update(e, m, (3 + (net ? 1 : 0)) * k <= kMaxBasis, s);
  if (rc) return rc;
  if (theta_host) rc = ecuda(e, cudaMemcpyAsync(theta_host, theta, k * sizeof(double), cudaMemcpyDeviceToHost, s), "theta");
  if (!rc) rc = ecuda(e, cudaStreamSynchronize(s), "step sync");
  if (!rc && net && rsx_net_sync_status(net, stream) != RSX_OK)
    rc = efail(e, RSX_ETIMEOUT, "learned preconditioner: a tensor-core convolution timed out");
  return rc;
}

// Non-local exchange term of H: mode 0 none; 1 the ACE operator -xi <xi, .> of the
// projectors src [count][N] (Eq. 13); 2 the exact exchange Vx[src] of the orbitals src
// [count][N] (Eq. 2) through the context ctx (same grid, FP32).  src stays the caller's.
// The next step (or rsx_eig_refresh) uses it.
int rsx_eig_set_exchange(rsx_eig* e, rsx_ctx* ctx, const float* src, int count, int mode) {
  if (!e || mode < 0 || mode > 2 || (mode && (!src || count < 1 || count > 64))) return RSX_EINVAL;
  if (mode == 1 && ((count + 15) & ~15) * 4 * e->k > kMaxBasis * kMaxBasis)
    return efail(e, RSX_EINVAL, "too many ACE projectors for the block size");
  if (mode == 2) {
    if (!ctx || ctx->precision != RSX_FP32 || ctx->g.nx != e->n || ctx->g.ny != e->n || ctx->g.nz != e->n)
      return efail(e, RSX_EINVAL, "exact exchange needs an FP32 context on the eigensolver's grid");
    if (!e->xbuf) {
      const size_t N = (size_t)e->n * e->n * e->n;
      if (cudaMalloc(&e->xbuf, 4 * (size_t)e->k * N * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        return efail(e, RSX_ENOMEM, "exchange scratch");
      }
    }
  }
  e->xmode = mode;
  e->xsrc = mode ? src : nullptr;
  e->xcount = mode ? count : 0;
  e->xctx = ctx;
  return RSX_OK;
}

// Spherical domain: H restricted to the points where mask (caller's [N], 0 or 1) is 1;
// the next rsx_eig_init masks the starting orbitals.  NULL restores the whole box.
int rsx_eig_set_mask(rsx_eig* e, const float* mask) {
  if (!e) return RSX_EINVAL;
  e->mask = mask;
  return RSX_OK;
}

// H has changed (the potential's contents or the exchange term): H Psi and Rayleigh-Ritz
// on the current orbitals, the LOBPCG direction dropped.
int rsx_eig_refresh(rsx_eig* e, double* theta_host, void* stream) {
  rsx::NvtxRange nvtx_range("rsx_eig_refresh");
  if (!e || !e->started) return RSX_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = ham(e, e->B, e->k, e->HB, nullptr, e->V, s);
  e->has_p = false;
  if (!rc) rc = rr_update(e, e->k, false, s);
  if (!rc && theta_host)
    rc = ecuda(e, cudaMemcpyAsync(theta_host, e->sm, e->k * sizeof(double), cudaMemcpyDeviceToHost, s), "theta");
  if (!rc) rc = ecuda(e, cudaStreamSynchronize(s), "refresh sync");
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

// FP64 energy of the current orbitals (see rsx.h)
int rsx_eig_energy64(rsx_eig* e, double* energy_host, void* stream) {
  rsx::NvtxRange nvtx_range("rsx_eig_energy64");
  if (!e || !energy_host) return RSX_EINVAL;
  if (!e->started) return efail(e, RSX_EINVAL, "energy64: call rsx_eig_init first");
  if (e->xmode != 0) return efail(e, RSX_EUNSUPPORTED, "energy64: H with an exchange term is not covered");
  cudaStream_t s = (cudaStream_t)stream;
  rsx_ctx* c = e->ctx;
  const int k = e->k;
  const size_t N = (size_t)e->n * e->n * e->n;
  if (!e->e64 && cudaMalloc(&e->e64, (2 * (size_t)k * N + 2 * 4096 + 8) * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    e->e64 = nullptr;
    return efail(e, RSX_ENOMEM, "energy64: cannot allocate the FP64 workspace");
  }
  double* P = e->e64;
  double* HP = P + (size_t)k * N;
  double* Sm = HP + (size_t)k * N;
  double* Hm = Sm + 4096;
  double* res = Hm + 4096;
  const int nblk = 2 * c->nsm;
  int rc = grow(c, (void**)&c->dsm, &c->dsm_bytes, sizeof(double) * ((size_t)nblk * 4096 + 3 * 4096), "small FP64");
  if (rc) return efail(e, rc, rsx_last_error(c));
  k_cast64<<<4 * c->nsm, 256, 0, s>>>(e->B, (size_t)k * N, P);
  k_ham_apply64<<<8 * c->nsm, 256, 0, s>>>(P, k, e->n, 1.0 / (12.0 * e->h * e->h), e->V, e->mask, HP);
  rc = ecuda(e, cudaGetLastError(), "energy64 H");
  const double h3 = e->h * e->h * e->h;
  if (!rc) rc = ecuda(e, launch_gram<double>(P, k, P, k, N, c->dsm, nblk, s), "energy64 S");
  if (!rc) rc = ecuda(e, launch_gram_reduce<double>(c->dsm, nblk, k, k, h3, false, Sm, (double*)nullptr, s), "energy64 S");
  if (!rc) rc = ecuda(e, launch_gram<double>(P, k, HP, k, N, c->dsm, nblk, s), "energy64 H");
  if (!rc) rc = ecuda(e, launch_gram_reduce<double>(c->dsm, nblk, k, k, h3, false, Hm, (double*)nullptr, s), "energy64 H");
  if (rc) return rc;
  k_rr_trace<<<1, 32, 0, s>>>(Sm, Hm, k, res);
  rc = ecuda(e, cudaMemcpyAsync(energy_host, res, sizeof(double), cudaMemcpyDeviceToHost, s), "energy64 copy");
  if (!rc) rc = ecuda(e, cudaStreamSynchronize(s), "energy64 sync");
  return rc;
}

const char* rsx_eig_last_error(const rsx_eig* e) { return e ? e->err : "null eigensolver"; }

int rsx_eig_destroy(rsx_eig* e) {
  if (!e) return RSX_OK;
  void* bufs[] = {e->B, e->HB, e->R, e->tmp, e->xnet, e->sm, e->qt, e->qp, e->xbuf, e->e64};
  for (void* p : bufs)
    if (p) cudaFree(p);
  rsx_destroy(e->ctx);
  delete e;
  return RSX_OK;
}

// ---------------------------------------------------------------------------------
// Closed-shell Hartree-Fock SCF (Sec. 3.1-3.2): per iteration the exchange operator is
// rebuilt from the current orbitals (ACE: Eqs. 11-13 once per iteration; exact: Eq. 2
// applied inside every H application), the Hartree potential of the mixed input density
// is added to V_ext, the block eigensolver takes a few steps, and the output density is
// mixed linearly into the next input (Eq. 14); the relative density error (Eq. 15) and the
// HF energy of the orbitals entering the iteration are reported.

}  // extern "C"

struct rsx_scf {
  rsx_ctx* ctx = nullptr;        // caller's FP32 context on the grid (exchange, Poisson)
  rsx_eig* eig = nullptr;
  int n = 0, nocc = 0, mode = 1, iter = 0;
  double h = 0.0;
  float alpha = 0.3f;
  const float* vext = nullptr;   // caller's
  float* V = nullptr;            // V_ext + V_H, the eigensolver's potential
  float* rho_in = nullptr;       // mixed input density
  float* rho = nullptr;          // density of the current orbitals
  float* vh = nullptr;           // scratch potential
  float* phi = nullptr;          // [nocc][N] orbitals entering the iteration
  float* xi = nullptr;           // [nocc][N] ACE projectors
  float* hphi = nullptr;         // [nocc][N] (T + V_ext) phi
  double* dsm = nullptr;         // M (nocc^2), Gram results, reduction partials
  // mixing of states (rsx_scf_set_mixing): [phi_in; phi_out] [2 nocc][N], coefficients
  int mix_states = 0;
  float* mix2 = nullptr;
  float* fsm = nullptr;          // [nocc][2 nocc] mixing coefficients, [nocc][nocc] L^-1
  char err[256] = {0};
};

namespace {

int sfail(rsx_scf* c, int code, const char* msg) {
  snprintf(c->err, sizeof(c->err), "%s", msg);
  return code;
}
int scuda(rsx_scf* c, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return RSX_OK;
  snprintf(c->err, sizeof(c->err), "%s: %s", what, cudaGetErrorString(e));
  return RSX_ECUDA;
}
constexpr int kScfRedBlocks = 256;

// out[a][b] = h^3 <X_a, Y_b> (device FP64, na * nb <= 1024)
int scf_gram(rsx_scf* c, const float* X, int na, const float* Y, int nb, double* out, cudaStream_t s) {
  rsx_ctx* x = c->ctx;
  const int nblk = 2 * x->nsm;
  int rc = grow(x, (void**)&x->dsm, &x->dsm_bytes, sizeof(double) * ((size_t)nblk * 4096 + 3 * 4096), "small FP64");
  if (!rc) rc = check_cuda(x, launch_gram<float>(X, na, Y, nb, x->g.N(), x->dsm, nblk, s), "gram");
  if (!rc)
    rc = check_cuda(x, launch_gram_reduce<float>(x->dsm, nblk, na, nb, c->h * c->h * c->h, false, out, (float*)nullptr, s),
                    "gram reduce");
  return rc ? sfail(c, rc, x->err) : RSX_OK;
}

}  // namespace

extern "C" {

int rsx_scf_create(rsx_scf** out, rsx_ctx* ctx, const float* V_ext, int nocc, int use_ace, float alpha) {
  if (!out || !ctx || !V_ext || nocc < 1 || nocc > 16 || !(alpha >= 0.f && alpha < 1.f)) return RSX_EINVAL;
  *out = nullptr;
  if (ctx->precision != RSX_FP32 || ctx->g.nx != ctx->g.ny || ctx->g.ny != ctx->g.nz) return RSX_EINVAL;
  rsx_scf* c = new rsx_scf();
  c->ctx = ctx;
  c->n = ctx->g.nx;
  c->nocc = nocc;
  c->mode = use_ace ? 1 : 2;
  c->alpha = alpha;
  c->h = ctx->h;
  c->vext = V_ext;
  cudaSetDevice(ctx->device);
  const size_t N = ctx->g.N();
  if (cudaMalloc(&c->V, N * sizeof(float)) != cudaSuccess || cudaMalloc(&c->rho_in, N * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&c->rho, N * sizeof(float)) != cudaSuccess || cudaMalloc(&c->vh, N * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&c->phi, nocc * N * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&c->xi, nocc * N * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&c->hphi, nocc * N * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&c->dsm, (4096 + kScfRedBlocks) * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&c->fsm, 1024 * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    rsx_scf_destroy(c);
    return RSX_ENOMEM;
  }
  cudaMemcpy(c->V, V_ext, N * sizeof(float), cudaMemcpyDeviceToDevice);
  const int rc = rsx_eig_create(&c->eig, c->n, c->h, c->V, 1.f, nocc, ctx->device);
  if (rc) {
    rsx_scf_destroy(c);
    return rc;
  }
  *out = c;
  return RSX_OK;
}

// Starting orbitals psi0 [nocc][N]: Rayleigh-Ritz with H = T + V_ext, input density of
// the first iteration = their density.
int rsx_scf_init(rsx_scf* c, const float* psi0, void* stream) {
  if (!c || !psi0) return RSX_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t N = c->ctx->g.N();
  int rc = rsx_eig_set_exchange(c->eig, nullptr, nullptr, 0, 0);
  if (!rc) rc = scuda(c, cudaMemcpyAsync(c->V, c->vext, N * sizeof(float), cudaMemcpyDeviceToDevice, s), "V");
  if (!rc) rc = rsx_eig_init(c->eig, psi0, stream);
  if (rc) return sfail(c, rc, "eigensolver start failed");
  rc = rsx_eig_orbitals(c->eig, c->phi, stream);
  if (rc) return sfail(c, rc, "orbitals");
  k_density<<<(unsigned)blocks_for(N), 256, 0, s>>>(c->phi, c->nocc, N, c->rho_in);
  c->iter = 0;
  return scuda(c, cudaStreamSynchronize(s), "init sync");
}

// One SCF iteration with `inner` eigensolver steps (3 Jacobi sweeps each).  out_host[6]:
// HF energy of the orbitals entering the iteration and its parts (one-body, Hartree,
// exchange), the relative density error of the previous iteration (Eq. 15; 0 on the
// first), and the sum of the new Ritz values.  Synchronises the stream.
int rsx_scf_step(rsx_scf* c, int inner, double* out_host, void* stream) {
  rsx::NvtxRange nvtx_range("rsx_scf_step");
  if (!c || inner < 1 || !out_host) return RSX_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const int k = c->nocc;
  const size_t N = c->ctx->g.N();
  const double h3 = c->h * c->h * c->h;
  double* M = c->dsm;                 // [k][k]
  double* part = c->dsm + 4096;
  // Output orbitals of the previous iteration (the eigensolver's current ones), their
  // density, the reldens of the previous iteration (Eq. 15), and the input of this one:
  // density mixing (Eq. 14 on rho; the entering orbitals are the outputs) or state
  // mixing (Eq. 14 on the orbitals, aligned through the projector on the output span).
  const bool states = c->mix_states != 0;
  float* phi_e = states ? c->mix2 : c->phi;               // orbitals entering this iteration
  float* phi_out = states ? c->mix2 + (size_t)k * N : c->phi;
  int rc = rsx_eig_orbitals(c->eig, phi_out, stream);
  if (rc) return sfail(c, rc, "orbitals");
  k_density<<<(unsigned)blocks_for(N), 256, 0, s>>>(phi_out, k, N, c->rho);
  double reldens = 0.0;
  if (c->iter > 0) {
    k_absdiff_mix<<<kScfRedBlocks, 256, 0, s>>>(c->rho_in, c->rho, N, c->alpha, states ? 0 : 1, part);
    double hp[kScfRedBlocks];
    rc = scuda(c, cudaMemcpyAsync(hp, part, sizeof(hp), cudaMemcpyDeviceToHost, s), "reldens");
    if (!rc) rc = scuda(c, cudaStreamSynchronize(s), "reldens sync");
    if (rc) return rc;
    for (int b = 0; b < kScfRedBlocks; ++b) reldens += hp[b];
    reldens *= h3 / (2.0 * k);
  }
  if (states) {
    if (c->iter == 0) {
      rc = scuda(c, cudaMemcpyAsync(phi_e, phi_out, (size_t)k * N * sizeof(float), cudaMemcpyDeviceToDevice, s), "states");
    } else {
      double* O = c->dsm + 3072;
      float* coef = c->fsm;
      float* linv = c->fsm + 2 * k * k;
      float* tmp = c->hphi;
      rc = scf_gram(c, phi_out, k, phi_e, k, O, s);
      if (rc) return rc;
      k_state_mix_coeffs<<<1, 256, 0, s>>>(O, k, c->alpha, coef);
      rc = check_cuda(c->ctx, launch_combine<float>(coef, k, 2 * k, c->mix2, N, tmp, 4 * c->ctx->nsm, s), "state mix");
      if (!rc) rc = scf_gram(c, tmp, k, tmp, k, O, s);
      if (rc) return rc;
      k_chol_inv_small<<<1, 32, 0, s>>>(O, k, linv, c->ctx->status);
      rc = check_cuda(c->ctx, launch_combine<float>(linv, k, k, tmp, N, phi_e, 4 * c->ctx->nsm, s), "orthonormalise");
    }
    if (rc) return rc;
    k_density<<<(unsigned)blocks_for(N), 256, 0, s>>>(phi_e, k, N, c->rho_in);
  } else if (c->iter == 0) {
    rc = scuda(c, cudaMemcpyAsync(c->rho_in, c->rho, N * sizeof(float), cudaMemcpyDeviceToDevice, s), "rho_in");
    if (rc) return rc;
  }
  const float* rho_e = states ? c->rho_in : c->rho;       // density of the entering orbitals
  // exchange from the entering orbitals: W, M (E_x = tr M) and the ACE projectors
  rc = rsx_ace_build(c->ctx, phi_e, k, c->xi, M, stream);
  if (rc) return sfail(c, rc, "ACE build failed");
  // energy parts of the entering orbitals: one-body, Hartree
  rc = rsx_poisson(c->ctx, rho_e, c->vh, stream);
  if (rc) return sfail(c, rc, "Poisson (energy) failed");
  launch_ham(phi_e, k, c->n, (float)(1.0 / (12.0 * c->h * c->h)), c->vext, nullptr, c->eig->mask, c->hphi, s);
  rc = scf_gram(c, phi_e, k, c->hphi, k, c->dsm + 1024, s);
  if (!rc) rc = scf_gram(c, rho_e, 1, c->vh, 1, c->dsm + 2048, s);
  if (rc) return rc;
  double hm[3 * 1024];
  rc = scuda(c, cudaMemcpyAsync(hm, c->dsm, sizeof(hm), cudaMemcpyDeviceToHost, s), "energies");
  if (!rc) rc = scuda(c, cudaStreamSynchronize(s), "energy sync");
  if (!rc) rc = rsx_sync_status(c->ctx, stream);
  if (rc) return sfail(c, rc, "energy evaluation failed (ACE or overlap matrix not definite)");
  double one = 0.0, ex = 0.0;
  for (int i = 0; i < k; ++i) {
    one += 2.0 * hm[1024 + i * k + i];
    ex += hm[i * k + i];
  }
  const double eh = 0.5 * hm[2048];
  // Fock operator of this iteration: V = V_ext + V_H[rho_in], exchange of the entering
  // orbitals (with state mixing rho_in is their density, and V_H was just computed)
  if (!states) {
    rc = rsx_poisson(c->ctx, c->rho_in, c->vh, stream);
    if (rc) return sfail(c, rc, "Poisson failed");
  }
  k_add<<<(unsigned)blocks_for(N), 256, 0, s>>>(c->vext, c->vh, N, c->V);
  rc = rsx_eig_set_exchange(c->eig, c->ctx, c->mode == 1 ? c->xi : phi_e, k, c->mode);
  if (!rc) rc = rsx_eig_refresh(c->eig, nullptr, stream);
  double theta[64] = {0};
  for (int it = 0; it < inner && !rc; ++it) rc = rsx_eig_step(c->eig, nullptr, 3, theta, stream);
  if (rc) return sfail(c, rc, rsx_eig_last_error(c->eig));
  double ts = 0.0;
  for (int i = 0; i < k; ++i) ts += theta[i];
  out_host[0] = one + eh + ex;
  out_host[1] = one;
  out_host[2] = eh;
  out_host[3] = ex;
  out_host[4] = reldens;
  out_host[5] = ts;
  ++c->iter;
  return RSX_OK;
}

// Spherical domain for the SCF orbitals (see rsx_eig_set_mask); before rsx_scf_init.
int rsx_scf_set_mask(rsx_scf* c, const float* mask) {
  if (!c) return RSX_EINVAL;
  return rsx_eig_set_mask(c->eig, mask);
}

// What Eq. 14 mixes: 0 the density (default), 1 the states.  Before the first step only.
int rsx_scf_set_mixing(rsx_scf* c, int mix_states) {
  if (!c || c->iter > 0 || (mix_states != 0 && mix_states != 1)) return RSX_EINVAL;
  if (mix_states && !c->mix2) {
    if (cudaMalloc(&c->mix2, 2 * (size_t)c->nocc * c->ctx->g.N() * sizeof(float)) != cudaSuccess) {
      cudaGetLastError();
      return sfail(c, RSX_ENOMEM, "state mixing buffer");
    }
  }
  c->mix_states = mix_states;
  return RSX_OK;
}

int rsx_scf_orbitals(rsx_scf* c, float* psi_out, void* stream) {
  if (!c || !psi_out) return RSX_EINVAL;
  return rsx_eig_orbitals(c->eig, psi_out, stream);
}

const char* rsx_scf_last_error(const rsx_scf* c) { return c ? c->err : "null SCF"; }

int rsx_scf_destroy(rsx_scf* c) {
  if (!c) return RSX_OK;
  cudaDeviceSynchronize();
  if (c->eig) rsx_eig_destroy(c->eig);
  void* bufs[] = {c->V, c->rho_in, c->rho, c->vh, c->phi, c->xi, c->hphi, c->dsm, c->mix2, c->fsm};
  for (void* p : bufs)
    if (p) cudaFree(p);
  delete c;
  return RSX_OK;
}

}  // extern "C"
