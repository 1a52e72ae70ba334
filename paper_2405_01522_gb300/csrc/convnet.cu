// Learned preconditioner network: conv3d(2->16) ReLU conv3d(16->16) ReLU conv3d(16->1),
// 3^3 kernels, stride 1, zero padding 1; weights rounded to bf16 for every use (FP32
// masters updated by Adam), FP32 activations and accumulation.  The paper has no
// learned component; this is the eigensolver preconditioner the project adds.
//
// Kernels: k_conv_tc (the convolution as an implicit GEMM on the tcgen05 tensor cores,
// see below), the data gradient as the same convolution with flipped, transposed weights
// (k_flip_weights), k_wgrad_tc (the weight gradient as an implicit GEMM on the tensor
// cores, per-block partial sums reduced in fixed order by k_wgrad_reduce), masked MSE
// loss, ReLU backward and Adam.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>

#include <cuda_bf16.h>

#include "../../include/rsx.h"
#include "api_internal.cuh"
#include "tcgen05_util.cuh"

namespace {

constexpr int kC1 = 2, kC2 = 16, kC3 = 16, kC4 = 1;   // channels in -> hidden -> hidden -> out
constexpr int kT = 8;                                   // output block edge
constexpr int kHalo = kT + 2;
constexpr int kConvThreads = 256;
// parameter layout (floats): w1 [16][2][27], b1 [16], w2 [16][16][27], b2 [16], w3 [1][16][27], b3 [1]
constexpr int kW1 = kC2 * kC1 * 27, kW2 = kC3 * kC2 * 27, kW3 = kC4 * kC3 * 27;
constexpr int kOffW1 = 0, kOffB1 = kW1, kOffW2 = kOffB1 + kC2, kOffB2 = kOffW2 + kW2, kOffW3 = kOffB2 + kC3,
              kOffB3 = kOffW3 + kW3, kNParams = kOffB3 + kC4;

__device__ __forceinline__ float bf16_round(float f) {
  const uint32_t u = __float_as_uint(f);
  return __uint_as_float(((u + 0x7FFFu + ((u >> 16) & 1u)) >> 16) << 16);
}

// ---------------------------------------------------------------------------------
// 3^3 convolution as an implicit GEMM on the tensor cores:
//   out[b][co][v] = bias[co] + sum_{t, ci} w[co][ci][t] act(in[b][ci][v + t - 1])
// (act = ReLU of the previous layer's pre-activation when relu_in, else identity).
// A CTA owns an 8 (x) by 16 (y) block of output voxels over kTcZ consecutive z slices.
// Per slice the GEMM has rows m = 8 yl + xl (128 voxels), columns n = output channel
// (16, zero-padded when CO < 16) and K = 27 taps x 16 input channels (zero-padded when
// CI < 16): one tcgen05.mma (M = 128, N = 16, K = 16) per tap and activation part.  The
// activations are split into bf16 hi + lo (x - hi - lo ~ 2^-17 |x|) and both parts are
// multiplied by the bf16-rounded weights, so the products keep FP32-level accuracy; the
// accumulation is FP32 in TMEM (two 16-column buffers: slice i accumulates while slice
// i - 1 is read back and stored).
//
// The input planes z - 1, z, z + 1 of the halo (18 y x 10 x voxels, 16 channels) sit in
// a 3-slot ring in the no-swizzle K-major operand layout plane[yh][khalf][xh][8 ch]
// (16 B per (yh, khalf, xh)), so that the A operand of tap (dz, dy, dx) is the plane of
// slot (slice + dz) % 3 started dy rows and dx voxels in: row m = 8 yl + xl sits at
// (yl + dy) 320 + (xl + dx) 16 bytes, the two K halves 160 bytes apart (leading byte
// offset) and 8-row groups 320 bytes apart (stride byte offset).  No im2col copy exists.
// Weights: tap t at 512 t bytes, element (co, ci) at (co/8) 256 + (ci/8) 128 + (co%8) 16
// + (ci%8) 2.  Every wait is bounded; a timeout sets RSX_ETIMEOUT in the status word and
// the CTA drains, frees its TMEM and returns.
constexpr int kTcThreads = 128;
constexpr int kTcX = 8, kTcY = 16, kTcZ = 16;         // output block of one CTA
constexpr int kHY = kTcY + 2, kHX = kTcX + 2;          // halo plane 18 x 10
constexpr int kHalfBytes = kHX * 16;                   // 160: one K half of a halo row
constexpr int kRowBytes = 2 * kHalfBytes;              // 320: one halo row (both K halves)
constexpr int kPlaneBytes = kHY * kRowBytes;           // 5760
constexpr int kTapBytes = 512;                         // 16 x 16 bf16 weights of one tap
constexpr int kTcSmem = 6 * kPlaneBytes + 27 * kTapBytes;   // 3 slots x (hi, lo) + weights
constexpr int kHaloVox = kHY * kHX;                    // 180
constexpr int kStageRounds = (kHaloVox + kTcThreads - 1) / kTcThreads;
// instruction descriptor, kind::f16: D f32, A and B bf16, both K-major, M = 128, N = 16
constexpr uint32_t kConvIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((16u >> 3) << 17) | ((128u >> 4) << 24);

// shared-memory matrix descriptor, K-major without swizzle: 8 x 16 B core matrices,
// `lbo` bytes between K-adjacent and `sbo` bytes between M/N-adjacent core matrices
__device__ __forceinline__ uint64_t kmajor_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;   // descriptor version for tcgen05; swizzle bits 61-63 stay 0
  return d;
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo_half, float hi_half) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo_half, hi_half);
  return *reinterpret_cast<const uint32_t*>(&v);
}

template <int CI, int CO>
__global__ void __launch_bounds__(kTcThreads) k_conv_tc(const float* __restrict__ in, const float* __restrict__ w,
                                                        const float* __restrict__ bias, float* __restrict__ out, int D,
                                                        int H, int W, int relu_in, int* status) {
  static_assert(CI <= 16 && CO <= 16, "channels per layer <= 16");
  using namespace rsx::tc;
  extern __shared__ __align__(128) unsigned char sm[];
  unsigned char* ring = sm;                             // slot s, part p (0 hi, 1 lo): (2 s + p) * kPlaneBytes
  unsigned char* wsm = sm + 6 * kPlaneBytes;
  __shared__ __align__(8) uint64_t mma_bar;
  __shared__ uint32_t tmem_sh;
  __shared__ int abort_sh;

  const int nbx = (W + kTcX - 1) / kTcX, nby = (H + kTcY - 1) / kTcY;
  int blk = blockIdx.x;
  const int bx = blk % nbx;
  blk /= nbx;
  const int by = blk % nby;
  const int bz = blk / nby;
  const int b = blockIdx.y;
  const int x0 = bx * kTcX, y0 = by * kTcY, z0 = bz * kTcZ;
  const int nzl = min(kTcZ, D - z0);
  const size_t vol = (size_t)D * H * W;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // zero the ring (channels >= CI stay zero), weights into the B operand layout
  for (int i = tid; i < 6 * kPlaneBytes / 16; i += kTcThreads) reinterpret_cast<uint4*>(ring)[i] = make_uint4(0, 0, 0, 0);
  for (int i = tid; i < 27 * 256; i += kTcThreads) {
    const int t = i >> 8, co = (i >> 4) & 15, ci = i & 15;
    const float v = (co < CO && ci < CI) ? w[((size_t)co * CI + ci) * 27 + t] : 0.f;
    *reinterpret_cast<__nv_bfloat16*>(wsm + t * kTapBytes + (co >> 3) * 256 + (ci >> 3) * 128 + (co & 7) * 16 +
                                      (ci & 7) * 2) = __float2bfloat16_rn(v);
  }
  if (tid == 0) {
    abort_sh = 0;
    mbar_init(&mma_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_sh)), "r"(32)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }

  // halo voxel e = tid + 128 r of a plane: (yh, xh) = (e / 10, e % 10)
  float v[kStageRounds][CI];
  auto load_plane = [&](int z) {
#pragma unroll
    for (int r = 0; r < kStageRounds; ++r) {
      const int e = tid + r * kTcThreads;
      const int yh = e / kHX, xh = e - yh * kHX;
      const int y = y0 - 1 + yh, x = x0 - 1 + xh;
      const bool inside = e < kHaloVox && z >= 0 && z < D && y >= 0 && y < H && x >= 0 && x < W;
      const float* src = in + (size_t)b * CI * vol + ((size_t)(inside ? z : 0) * H + (inside ? y : 0)) * W + (inside ? x : 0);
#pragma unroll
      for (int ci = 0; ci < CI; ++ci) {
        float a = inside ? __ldg(src + (size_t)ci * vol) : 0.f;
        v[r][ci] = relu_in ? fmaxf(a, 0.f) : a;
      }
    }
  };
  auto store_plane = [&](int slot) {
#pragma unroll
    for (int r = 0; r < kStageRounds; ++r) {
      const int e = tid + r * kTcThreads;
      if (e >= kHaloVox) continue;
      const int yh = e / kHX, xh = e - yh * kHX;
#pragma unroll
      for (int half = 0; half < (CI + 7) / 8; ++half) {
        uint32_t hv[4], lv[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int c0 = half * 8 + 2 * j, c1 = c0 + 1;
          const float a0 = c0 < CI ? v[r][c0 < CI ? c0 : 0] : 0.f;
          const float a1 = c1 < CI ? v[r][c1 < CI ? c1 : 0] : 0.f;
          const __nv_bfloat162 h2 = __floats2bfloat162_rn(a0, a1);
          const float2 hf = __bfloat1622float2(h2);
          hv[j] = *reinterpret_cast<const uint32_t*>(&h2);
          lv[j] = pack_bf16x2(a0 - hf.x, a1 - hf.y);
        }
        const size_t off = (size_t)yh * kRowBytes + half * kHalfBytes + xh * 16;
        *reinterpret_cast<uint4*>(ring + (size_t)(2 * slot) * kPlaneBytes + off) = make_uint4(hv[0], hv[1], hv[2], hv[3]);
        *reinterpret_cast<uint4*>(ring + (size_t)(2 * slot + 1) * kPlaneBytes + off) =
            make_uint4(lv[0], lv[1], lv[2], lv[3]);
      }
    }
  };

  __syncthreads();   // ring zeroed before the first plane is written
  // planes z0 - 1 + j live in slot j % 3
  load_plane(z0 - 1);
  store_plane(0);
  load_plane(z0);
  store_plane(1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_sh;
  const uint32_t ring_s = smem_u32(ring), w_s = smem_u32(wsm);
  volatile int* abort_flag = &abort_sh;
  int issued = 0, waited = 0;

  auto epilogue = [&](int i) {
    const int m = warp * 32 + lane;                     // TMEM lane = GEMM row
    const int yl = m >> 3, xl = m & 7;
    const int z = z0 + i, y = y0 + yl, x = x0 + xl;
    float acc[16];
    tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)((i & 1) * 16), acc);
    if (y < H && x < W) {
#pragma unroll
      for (int co = 0; co < CO; ++co)
        out[((size_t)b * CO + co) * vol + ((size_t)z * H + y) * W + x] = acc[co] + (bias ? __ldg(bias + co) : 0.f);
    }
  };

  for (int i = 0; i < nzl; ++i) {
    load_plane(z0 + i + 1);                             // loads in flight while slice i - 1 finishes
    if (i > 0) {
      if (tid == 0) {
        if (!mbar_wait(&mma_bar, (uint32_t)((i - 1) & 1), abort_flag)) *abort_flag = 1;
        else waited = i;
      }
      __syncthreads();
      if (*abort_flag) break;
    }
    store_plane((i + 2) % 3);                           // its slot held plane i - 1, last read by slice i - 1
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == 0) {
      const uint32_t acc = tmem + (uint32_t)((i & 1) * 16);
#pragma unroll 1
      for (int t = 0; t < 27; ++t) {
        const int dz = t / 9, dy = (t / 3) % 3, dx = t % 3;
        const uint32_t pl = ring_s + (uint32_t)(2 * ((i + dz) % 3)) * kPlaneBytes + dy * kRowBytes + dx * 16;
        const uint64_t bd = kmajor_desc(w_s + t * kTapBytes, 128, 256);
        mma_f16(acc, kmajor_desc(pl, kHalfBytes, kRowBytes), bd, kConvIdesc, t > 0 ? 1u : 0u);
        mma_f16(acc, kmajor_desc(pl + kPlaneBytes, kHalfBytes, kRowBytes), bd, kConvIdesc, 1u);
      }
      mma_commit(&mma_bar);
      issued = i + 1;
    }
    if (i > 0) epilogue(i - 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }
  // last slice (or, after a timeout, drain what was issued)
  if (tid == 0) {
    if (!*abort_flag && issued == nzl) {
      if (!mbar_wait(&mma_bar, (uint32_t)((nzl - 1) & 1), abort_flag)) *abort_flag = 1;
    } else if (issued > waited) {
      for (uint32_t k = 0; k < kWaitLimit && !mbar_try_wait(&mma_bar, (uint32_t)((issued - 1) & 1)); ++k) {
      }
    }
    if (*abort_flag && status) atomicMax(status, RSX_ETIMEOUT);
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!*abort_flag) epilogue(nzl - 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(32) : "memory");
}

// wt[ci][co][26 - t] = w[co][ci][t]: the data gradient is the forward convolution of
// dout with these weights (no bias)
__global__ void k_flip_weights(const float* __restrict__ w, float* __restrict__ wt, int CI, int CO) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < CI * CO * 27; i += gridDim.x * blockDim.x) {
    const int co = i / (CI * 27), r = i - co * CI * 27, ci = r / 27, t = r - ci * 27;
    wt[((size_t)ci * CO + co) * 27 + (26 - t)] = w[i];
  }
}

// dz = da * (z > 0)  (ReLU backward), in place on da
__global__ void k_relu_back(float* __restrict__ da, const float* __restrict__ z, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    if (!(z[i] > 0.f)) da[i] = 0.f;
}

// Weight and bias gradients of one layer on the tensor cores, per CTA partial sums:
//   part[blk][co][ci][t] = sum_v dout[co][v] act(in[ci][v + t - 1]),  part[blk][CO*CI*27 + co] = sum_v dout[co][v]
// over the CTA's 16 (x) x 8 (y) x 8 (z) block of output voxels of one sample.  The
// contraction is an implicit GEMM with rows (t, ci) -- four groups of 8 taps x 16 input
// channels, M = 128 rows per MMA (the last group holds taps 24..26 and zero rows) -- columns
// co (N = 16, zero rows for co >= CO) and K = the voxels, 16 consecutive x positions of one
// (z, y) row per K step.  Per output plane z the input rows the plane's 8 K steps need (3
// planes x 10 rows x 16 channels x 18 x, ReLU applied) and its dout rows are staged once in
// shared memory.  For each K step thread (ci, 8-voxel chunk, dz) writes the 9 taps
// (dy, dx) of its channel from those rows into the A operand (the shifted input windows:
// one copy per tap, the operand layout having no room for a shifted view), 32 threads
// write the B operand (dout), both in the no-swizzle K-major core-matrix layout (element
// (row, k) at (row / 8) 256 + (k / 8) 128 + (row % 8) 16 + (k % 8) 2 bytes) and split into
// bf16 hi + lo; one thread issues hi.hi + hi.lo + lo.hi per group into four 16-column FP32
// accumulators in TMEM.  The tiles are double-buffered: building step s overlaps the MMAs
// of step s - 1 (an mbarrier per buffer).  Every wait is bounded; a
// timeout sets RSX_ETIMEOUT, the CTA waits (bounded) for its issued MMAs, frees its TMEM and
// returns without writing.
constexpr int kWgX = 16, kWgY = 8, kWgZ = 8;
constexpr int kWgThreads = 128;
constexpr int kWgATile = 4096;                          // 128 rows x 16 K bf16
constexpr int kWgBTile = 512;                           // 16 rows x 16 K bf16
constexpr int kWgBuf = 4 * 2 * kWgATile + 2 * kWgBTile; // (4 groups x hi, lo) + (hi, lo) of B
constexpr int kWgRow = kWgX + 2;                        // 18 x values per staged input row
constexpr int kWgSlabRows = 3 * (kWgY + 2) * 16;        // (dz, y, ci) rows of one plane's K steps
constexpr int kWgSlab = kWgSlabRows * kWgRow * 4;       // 34560 bytes
constexpr int kWgDslab = kWgY * 16 * kWgX * 4;          // dout rows of one plane: [y][co][x], 8192 bytes
constexpr int kWgSmem = 2 * kWgBuf + kWgSlab + kWgDslab;

template <int CI, int CO>
__global__ void __launch_bounds__(kWgThreads, 1) k_wgrad_tc(const float* __restrict__ in, const float* __restrict__ dout,
                                                         float* __restrict__ part, int D, int H, int W, int relu_in,
                                                         int* status) {
  static_assert(CI <= 16 && CO <= 16, "channels per layer <= 16");
  static_assert(kWgThreads == 128, "96 A-builder threads (ci, chunk, dz) + 32 B-builder threads (co, chunk)");
  using namespace rsx::tc;
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ uint32_t tmem_sh;
  __shared__ int abort_sh;
  __shared__ float bsum[16];
  const int nbx = (W + kWgX - 1) / kWgX, nby = (H + kWgY - 1) / kWgY;
  int blk = blockIdx.x;
  const int bx = blk % nbx;
  blk /= nbx;
  const int by = blk % nby;
  const int bz = blk / nby;
  const int b = blockIdx.y;
  const int x0 = bx * kWgX, y0 = by * kWgY, z0 = bz * kWgZ;
  const size_t vol = (size_t)D * H * W;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  constexpr int NOUT = CO * CI * 27 + CO;
  float* dst = part + ((size_t)b * gridDim.x + blockIdx.x) * NOUT;

  for (int i = tid; i < 2 * kWgBuf / 16; i += kWgThreads) reinterpret_cast<uint4*>(sm)[i] = make_uint4(0, 0, 0, 0);
  float* slab = reinterpret_cast<float*>(sm + 2 * kWgBuf);   // [dz][y - y0 + 1][ci][x - x0 + 1]
  float* dslab = slab + kWgSlab / 4;                          // [y - y0][co][x - x0]
  if (tid < 16) bsum[tid] = 0.f;
  if (tid == 0) {
    abort_sh = 0;
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_sh)), "r"(64)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_sh;
  const uint32_t sm_s = smem_u32(sm);
  volatile int* abort_flag = &abort_sh;
  float bacc = 0.f;
  int issued = 0;
  constexpr int nsteps = kWgY * kWgZ;
  // operand descriptors of both buffers, made once (the issuing thread only)
  uint64_t dah[2][4], dal[2][4], dbh[2], dbl[2];
  if (tid == 0) {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const uint32_t a_s = sm_s + (uint32_t)q * kWgBuf, b_s = a_s + 8 * kWgATile;
      dbh[q] = kmajor_desc(b_s, 128, 256);
      dbl[q] = kmajor_desc(b_s + kWgBTile, 128, 256);
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        dah[q][g] = kmajor_desc(a_s + (uint32_t)g * 2 * kWgATile, 128, 256);
        dal[q][g] = kmajor_desc(a_s + (uint32_t)g * 2 * kWgATile + kWgATile, 128, 256);
      }
    }
  }
  for (int s = 0; s < nsteps; ++s) {
    const int buf = s & 1;
    if (s >= 2) {   // buffer buf was read by the MMAs of step s - 2
      if (tid == 0 && !mbar_wait(&bar[buf], (uint32_t)(((s - 2) >> 1) & 1), abort_flag)) *abort_flag = 1;
      __syncthreads();
      if (*abort_flag) break;
    }
    const int zl = s / kWgY, yl = s % kWgY;
    const int z = z0 + zl, y = y0 + yl;
    if (yl == 0) {   // stage the input rows of plane z's K steps (every reader of the last slab is done)
      __syncthreads();
      for (int e = tid; e < kWgSlabRows * kWgRow; e += kWgThreads) {
        const int row = e / kWgRow, xo = e - row * kWgRow;
        const int ci = row & 15, yy = (row >> 4) % (kWgY + 2), dz = (row >> 4) / (kWgY + 2);
        const int zz = z + dz - 1, yg = y0 - 1 + yy, xg = x0 - 1 + xo;
        float a = 0.f;
        if (ci < CI && zz >= 0 && zz < D && yg >= 0 && yg < H && xg >= 0 && xg < W)
          a = __ldg(in + ((size_t)b * CI + ci) * vol + ((size_t)zz * H + yg) * W + xg);
        slab[e] = relu_in ? fmaxf(a, 0.f) : a;
      }
      for (int e = tid; e < kWgY * 16 * kWgX; e += kWgThreads) {
        const int yy = e / (16 * kWgX), co = (e / kWgX) & 15, xo = e % kWgX;
        const int yg = y0 + yy, xg = x0 + xo;
        dslab[e] = (co < CO && z < D && yg < H && xg < W)
                       ? __ldg(dout + ((size_t)b * CO + co) * vol + ((size_t)z * H + yg) * W + xg) : 0.f;
      }
      __syncthreads();
    }
    unsigned char* At = sm + (size_t)buf * kWgBuf;
    unsigned char* Bt = At + 8 * kWgATile;
    auto put = [&](unsigned char* dstp, int lo_off, const float* v) {
      uint32_t hv[4], lv[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const __nv_bfloat162 h2 = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
        const float2 hf = __bfloat1622float2(h2);
        hv[q] = *reinterpret_cast<const uint32_t*>(&h2);
        lv[q] = pack_bf16x2(v[2 * q] - hf.x, v[2 * q + 1] - hf.y);
      }
      *reinterpret_cast<uint4*>(dstp) = make_uint4(hv[0], hv[1], hv[2], hv[3]);
      *reinterpret_cast<uint4*>(dstp + lo_off) = make_uint4(lv[0], lv[1], lv[2], lv[3]);
    };
    if (tid < 96) {   // A: channel ci, chunk c, plane offset dz -> taps (dz, dy, dx)
      const int ci = tid & 15, c = (tid >> 4) & 1, dz = tid >> 5;
      if (ci < CI) {
#pragma unroll
        for (int dy = 0; dy < 3; ++dy) {
          const float2* rp = reinterpret_cast<const float2*>(
              slab + ((dz * (kWgY + 2) + yl + dy) * 16 + ci) * kWgRow + 8 * c);
          float r[10];
#pragma unroll
          for (int q = 0; q < 5; ++q) {
            const float2 u = rp[q];
            r[2 * q] = u.x;
            r[2 * q + 1] = u.y;
          }
#pragma unroll
          for (int dx = 0; dx < 3; ++dx) {
            const int t = 9 * dz + 3 * dy + dx;
            const int g = t >> 3, m = ((t & 7) << 4) | ci;
            put(At + (size_t)g * 2 * kWgATile + (m >> 3) * 256 + c * 128 + (m & 7) * 16, kWgATile, r + dx);
          }
        }
      }
    } else {          // B: dout of channel co, chunk c (and the bias gradient)
      const int j = tid - 96, co = j >> 1, c = j & 1;
      const float4* dp = reinterpret_cast<const float4*>(dslab + (yl * 16 + co) * kWgX + 8 * c);
      const float4 d0 = dp[0], d1 = dp[1];
      const float v[8] = {d0.x, d0.y, d0.z, d0.w, d1.x, d1.y, d1.z, d1.w};
#pragma unroll
      for (int k = 0; k < 8; ++k) bacc += v[k];
      put(Bt + (co >> 3) * 256 + c * 128 + (co & 7) * 16, kWgBTile, v);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == 0) {
      const uint32_t first = s > 0 ? 1u : 0u;
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        const uint32_t d = tmem + (uint32_t)(16 * g);
        const uint64_t ah = buf ? dah[1][g] : dah[0][g], al = buf ? dal[1][g] : dal[0][g];
        const uint64_t bh = buf ? dbh[1] : dbh[0], bl = buf ? dbl[1] : dbl[0];
        mma_f16(d, ah, bh, kConvIdesc, first);
        mma_f16(d, ah, bl, kConvIdesc, 1u);
        mma_f16(d, al, bh, kConvIdesc, 1u);
      }
      mma_commit(&bar[buf]);
      issued = s + 1;
    }
  }
  // wait for the last commit of each barrier (no arrival may land after the CTA exits; the
  // last commit also covers every MMA issued before it); bounded in every case
  if (tid == 0 && issued > 0) {
    for (int st = issued - 1; st >= 0 && st >= issued - 2; --st) {
      const uint32_t par = (uint32_t)((st >> 1) & 1);
      if (!*abort_flag) {
        if (!mbar_wait(&bar[st & 1], par, abort_flag)) *abort_flag = 1;
      } else {
        for (uint32_t k = 0; k < kWaitLimit && !mbar_try_wait(&bar[st & 1], par); ++k) {
        }
      }
    }
    if (*abort_flag && status) atomicMax(status, RSX_ETIMEOUT);
  }
  if (tid >= 96) atomicAdd(&bsum[(tid - 96) >> 1], bacc);
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!*abort_flag) {
    const int m = warp * 32 + lane;
#pragma unroll 1
    for (int g = 0; g < 4; ++g) {
      float acc[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(16 * g), acc);
      const int t = 8 * g + (m >> 4), ci = m & 15;
      if (t < 27 && ci < CI) {
#pragma unroll
        for (int co = 0; co < CO; ++co) dst[((size_t)co * CI + ci) * 27 + t] = acc[co];
      }
    }
    if (tid < CO) dst[CO * CI * 27 + tid] = bsum[tid];
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(64) : "memory");
}

// grad[o] = sum over nparts of part[p][o], FP64 accumulation in a fixed order: a block owns
// 32 consecutive outputs (lane = output, coalesced reads), warp w sums the partials
// p = w, w + 8, ..., and the 8 warp sums are added in warp order
__global__ void __launch_bounds__(256) k_wgrad_reduce(const float* __restrict__ part, int nparts, int nout,
                                                      float* __restrict__ gw, float* __restrict__ gb, int nw) {
  __shared__ double red[8][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int o = blockIdx.x * 32 + lane;
  double sum = 0.0;
  if (o < nout)
    for (int p = warp; p < nparts; p += 8) sum += (double)part[(size_t)p * nout + o];
  red[warp][lane] = sum;
  __syncthreads();
  if (warp == 0 && o < nout) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w][lane];
    if (o < nw)
      gw[o] = (float)t;
    else
      gb[o - nw] = (float)t;
  }
}

// masked mean squared error: loss = sum m (y - t)^2 / sum m over the batch; dy = 2 m (y - t) / sum m.
// The mask excludes `border` voxels at every face of each sample.
__global__ void k_mse(const float* __restrict__ y, const float* __restrict__ t, float* __restrict__ dy, int B, int D,
                      int H, int W, int border, double* __restrict__ loss_acc) {
  const size_t vol = (size_t)D * H * W;
  const double cnt = (double)B * (D - 2 * border) * (H - 2 * border) * (W - 2 * border);
  double s = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < (size_t)B * vol;
       i += (size_t)gridDim.x * blockDim.x) {
    const size_t v = i % vol;
    const int x = (int)(v % W), yy = (int)((v / W) % H), z = (int)(v / ((size_t)W * H));
    const bool in = x >= border && x < W - border && yy >= border && yy < H - border && z >= border && z < D - border;
    const float d = in ? y[i] - t[i] : 0.f;
    dy[i] = (float)(2.0 * d / cnt);
    s += (double)d * d;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss_acc, s / cnt);
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       int n, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

}  // namespace

struct rsx_net {
  int device = 0;
  float* params = nullptr;   // FP32 masters
  float* grads = nullptr;
  float* adam_m = nullptr;
  float* adam_v = nullptr;
  float* wflip = nullptr;    // flipped weights of one layer (scratch)
  float* act = nullptr;      // z1, z2 [B][16][vol] each
  size_t act_elems = 0;
  float* gout = nullptr;     // gradients of activations [B][16][vol] x 2 + output
  size_t gout_elems = 0;
  float* part = nullptr;
  size_t part_elems = 0;
  double* loss = nullptr;
  int* status = nullptr;     // device status word (RSX_ETIMEOUT from a bounded wait)
  long long step = 0;
  char err[256] = {0};
};

namespace {

int nfail(rsx_net* n, int code, const char* msg) {
  snprintf(n->err, sizeof(n->err), "%s", msg);
  return code;
}

int ncuda(rsx_net* n, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return RSX_OK;
  snprintf(n->err, sizeof(n->err), "%s: %s", what, cudaGetErrorString(e));
  return RSX_ECUDA;
}

int ngrow(rsx_net* n, float** p, size_t* have, size_t need) {
  if (need <= *have) return RSX_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *have = 0;
  if (cudaMalloc(p, need * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    return nfail(n, RSX_ENOMEM, "network workspace allocation failed");
  }
  *have = need;
  return RSX_OK;
}

dim3 conv_grid(int B, int D, int H, int W) {
  return dim3((unsigned)(((W + kT - 1) / kT) * ((H + kT - 1) / kT) * ((D + kT - 1) / kT)), (unsigned)B);
}

// one 3^3 convolution layer on the tensor cores (k_conv_tc)
template <int CI, int CO>
void conv(rsx_net* n, const float* in, const float* w, const float* bias, float* out, int B, int D, int H, int W,
          int relu_in, cudaStream_t s) {
  const dim3 g((unsigned)(((W + kTcX - 1) / kTcX) * ((H + kTcY - 1) / kTcY) * ((D + kTcZ - 1) / kTcZ)), (unsigned)B);
  k_conv_tc<CI, CO><<<g, kTcThreads, kTcSmem, s>>>(in, w, bias, out, D, H, W, relu_in, n->status);
}

int forward(rsx_net* n, const float* x, int B, int D, int H, int W, float* out, cudaStream_t s) {
  const size_t vol = (size_t)D * H * W;
  int rc = ngrow(n, &n->act, &n->act_elems, 2 * (size_t)B * kC2 * vol);
  if (rc) return rc;
  float* z1 = n->act;
  float* z2 = n->act + (size_t)B * kC2 * vol;
  const dim3 g = conv_grid(B, D, H, W);
  const float* P = n->params;
  conv<kC1, kC2>(n, x, P + kOffW1, P + kOffB1, z1, B, D, H, W, 0, s);
  conv<kC2, kC3>(n, z1, P + kOffW2, P + kOffB2, z2, B, D, H, W, 1, s);
  conv<kC3, kC4>(n, z2, P + kOffW3, P + kOffB3, out, B, D, H, W, 1, s);
  return ncuda(n, cudaGetLastError(), "network forward");
}

// gradients of the masked MSE loss w.r.t. all parameters into n->grads; loss (device double) += value
int backward(rsx_net* n, const float* x, const float* target, int B, int D, int H, int W, int border, cudaStream_t s) {
  const size_t vol = (size_t)D * H * W;
  int rc = ngrow(n, &n->gout, &n->gout_elems, 2 * (size_t)B * kC2 * vol + (size_t)B * vol * 2);
  if (rc) return rc;
  const int nblk = ((W + kWgX - 1) / kWgX) * ((H + kWgY - 1) / kWgY) * ((D + kWgZ - 1) / kWgZ);
  rc = ngrow(n, &n->part, &n->part_elems, (size_t)B * nblk * (kW2 + kC3));
  if (rc) return rc;
  float* g2 = n->gout;                                  // d z2  [B][16][vol]
  float* g1 = n->gout + (size_t)B * kC2 * vol;          // d z1  [B][16][vol]
  float* y = g1 + (size_t)B * kC2 * vol;                // output [B][vol]
  float* gy = y + (size_t)B * vol;                      // d output
  rc = forward(n, x, B, D, H, W, y, s);                 // (re)sizes n->act
  if (rc) return rc;
  float* z1 = n->act;                                   // pre-activations of layers 1 and 2
  float* z2 = n->act + (size_t)B * kC2 * vol;
  k_mse<<<512, 256, 0, s>>>(y, target, gy, B, D, H, W, border, n->loss);
  const dim3 g((unsigned)nblk, (unsigned)B);
  const float* P = n->params;
  for (auto k : {k_wgrad_tc<kC3, kC4>, k_wgrad_tc<kC2, kC3>, k_wgrad_tc<kC1, kC2>})
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kWgSmem) != cudaSuccess)
      return ncuda(n, cudaGetLastError(), "wgrad attributes");
  // layer 3: w3 grads from relu(z2) and gy; d relu(z2) = conv(gy, flip(w3)); dz2 = * (z2 > 0)
  k_wgrad_tc<kC3, kC4><<<g, kWgThreads, kWgSmem, s>>>(z2, gy, n->part, D, H, W, 1, n->status);
  k_wgrad_reduce<<<(kW3 + kC4 + 31) / 32, 256, 0, s>>>(n->part, B * nblk, kW3 + kC4, n->grads + kOffW3, n->grads + kOffB3, kW3);
  k_flip_weights<<<16, 256, 0, s>>>(P + kOffW3, n->wflip, kC3, kC4);
  conv<kC4, kC3>(n, gy, n->wflip, nullptr, g2, B, D, H, W, 0, s);
  k_relu_back<<<512, 256, 0, s>>>(g2, z2, (size_t)B * kC2 * vol);
  // layer 2
  k_wgrad_tc<kC2, kC3><<<g, kWgThreads, kWgSmem, s>>>(z1, g2, n->part, D, H, W, 1, n->status);
  k_wgrad_reduce<<<(kW2 + kC3 + 31) / 32, 256, 0, s>>>(n->part, B * nblk, kW2 + kC3, n->grads + kOffW2, n->grads + kOffB2, kW2);
  k_flip_weights<<<32, 256, 0, s>>>(P + kOffW2, n->wflip, kC2, kC3);
  conv<kC3, kC2>(n, g2, n->wflip, nullptr, g1, B, D, H, W, 0, s);
  k_relu_back<<<512, 256, 0, s>>>(g1, z1, (size_t)B * kC2 * vol);
  // layer 1
  k_wgrad_tc<kC1, kC2><<<g, kWgThreads, kWgSmem, s>>>(x, g1, n->part, D, H, W, 0, n->status);
  k_wgrad_reduce<<<(kW1 + kC2 + 31) / 32, 256, 0, s>>>(n->part, B * nblk, kW1 + kC2, n->grads + kOffW1, n->grads + kOffB1, kW1);
  return ncuda(n, cudaGetLastError(), "network backward");
}

}  // namespace

extern "C" {

int rsx_net_create(rsx_net** out, int device) {
  if (!out) return RSX_EINVAL;
  *out = nullptr;
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return RSX_ECUDA;
  }
  rsx_net* n = new rsx_net();
  n->device = device;
  if (cudaMalloc(&n->params, kNParams * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&n->grads, kNParams * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&n->adam_m, kNParams * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&n->adam_v, kNParams * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&n->wflip, kW2 * sizeof(float)) != cudaSuccess || cudaMalloc(&n->loss, sizeof(double)) != cudaSuccess ||
      cudaMalloc(&n->status, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    rsx_net_destroy(n);
    return RSX_ENOMEM;
  }
  cudaMemset(n->params, 0, kNParams * sizeof(float));
  cudaMemset(n->adam_m, 0, kNParams * sizeof(float));
  cudaMemset(n->adam_v, 0, kNParams * sizeof(float));
  cudaMemset(n->status, 0, sizeof(int));
  *out = n;
  return RSX_OK;
}

int rsx_net_param_count(void) { return kNParams; }

int rsx_net_set_params(rsx_net* n, const float* host, int count) {
  if (!n || !host || count != kNParams) return RSX_EINVAL;
  cudaSetDevice(n->device);
  n->step = 0;
  cudaMemset(n->adam_m, 0, kNParams * sizeof(float));
  cudaMemset(n->adam_v, 0, kNParams * sizeof(float));
  return ncuda(n, cudaMemcpy(n->params, host, kNParams * sizeof(float), cudaMemcpyHostToDevice), "set params");
}

int rsx_net_get_params(rsx_net* n, float* host, int count) {
  if (!n || !host || count != kNParams) return RSX_EINVAL;
  cudaSetDevice(n->device);
  return ncuda(n, cudaMemcpy(host, n->params, kNParams * sizeof(float), cudaMemcpyDeviceToHost), "get params");
}

int rsx_net_forward(rsx_net* n, const float* x, int B, int D, int H, int W, float* out, void* stream) {
  rsx::NvtxRange nvtx_range("rsx_net_forward");
  if (!n || !x || !out || B < 1 || D < 1 || H < 1 || W < 1) return RSX_EINVAL;
  cudaSetDevice(n->device);
  return forward(n, x, B, D, H, W, out, (cudaStream_t)stream);
}

int rsx_net_loss_grad(rsx_net* n, const float* x, const float* target, int B, int D, int H, int W, int border,
                      double* loss_host, float* grad_host, void* stream) {
  rsx::NvtxRange nvtx_range("rsx_net_loss_grad");
  if (!n || !x || !target || B < 1 || D <= 2 * border || H <= 2 * border || W <= 2 * border) return RSX_EINVAL;
  cudaSetDevice(n->device);
  cudaStream_t s = (cudaStream_t)stream;
  cudaMemsetAsync(n->loss, 0, sizeof(double), s);
  int rc = backward(n, x, target, B, D, H, W, border, s);
  if (rc) return rc;
  if (loss_host) rc = ncuda(n, cudaMemcpyAsync(loss_host, n->loss, sizeof(double), cudaMemcpyDeviceToHost, s), "loss");
  if (!rc && grad_host)
    rc = ncuda(n, cudaMemcpyAsync(grad_host, n->grads, kNParams * sizeof(float), cudaMemcpyDeviceToHost, s), "grads");
  if (!rc) rc = ncuda(n, cudaStreamSynchronize(s), "sync");
  return rc;
}

int rsx_net_train_step(rsx_net* n, const float* x, const float* target, int B, int D, int H, int W, int border,
                       float lr, double* loss_host, void* stream) {
  rsx::NvtxRange nvtx_range("rsx_net_train_step");
  if (!n || !x || !target || B < 1 || D <= 2 * border || H <= 2 * border || W <= 2 * border || !(lr > 0.f))
    return RSX_EINVAL;
  cudaSetDevice(n->device);
  cudaStream_t s = (cudaStream_t)stream;
  cudaMemsetAsync(n->loss, 0, sizeof(double), s);
  int rc = backward(n, x, target, B, D, H, W, border, s);
  if (rc) return rc;
  ++n->step;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)n->step), c2 = 1.f - powf(b2, (float)n->step);
  k_adam<<<(kNParams + 255) / 256, 256, 0, s>>>(n->params, n->grads, n->adam_m, n->adam_v, kNParams, lr, b1, b2, 1e-8f,
                                                 c1, c2);
  rc = ncuda(n, cudaGetLastError(), "adam");
  if (!rc && loss_host)
    rc = ncuda(n, cudaMemcpyAsync(loss_host, n->loss, sizeof(double), cudaMemcpyDeviceToHost, s), "loss");
  return rc;
}

// Synchronises the stream, then reports (and clears) a deferred device error of the
// network kernels: RSX_ETIMEOUT when a tensor-core convolution gave up a bounded wait.
int rsx_net_sync_status(rsx_net* n, void* stream) {
  if (!n) return RSX_EINVAL;
  cudaSetDevice(n->device);
  int rc = ncuda(n, cudaStreamSynchronize((cudaStream_t)stream), "sync");
  if (rc) return rc;
  int st = 0;
  rc = ncuda(n, cudaMemcpy(&st, n->status, sizeof(int), cudaMemcpyDeviceToHost), "status");
  if (rc) return rc;
  if (st != RSX_OK) {
    cudaMemset(n->status, 0, sizeof(int));
    return nfail(n, st, "network kernel gave up a bounded wait (timeout)");
  }
  return RSX_OK;
}

const char* rsx_net_last_error(const rsx_net* n) { return n ? n->err : "null network"; }

int rsx_net_destroy(rsx_net* n) {
  if (!n) return RSX_OK;
  cudaSetDevice(n->device);
  cudaDeviceSynchronize();
  void* bufs[] = {n->params, n->grads, n->adam_m, n->adam_v, n->wflip, n->act, n->gout, n->part, n->loss, n->status};
  for (void* p : bufs)
    if (p) cudaFree(p);
  delete n;
  return RSX_OK;
}

}  // extern "C"
