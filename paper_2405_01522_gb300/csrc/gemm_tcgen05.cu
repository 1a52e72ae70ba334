// Split-BF16 symmetric contraction on the 5th-generation tensor cores (sm_103a):
//
//     C = H H^T + H L^T + L H^T        H, L: [n][ld] bf16 (hi and lo parts of one FP32
//                                      panel S = H + L, row-major, K contiguous)
//
// which is S S^T to ~16 mantissa bits; for the Casida coupling S_t(G) holds the
// weighted pair spectra and C = K (Eqs. 6-7, K = sum_G w_G ghat(G) Re conj R_t R_s).
//
// Tiling: 128 x 128 output tiles of the upper triangle (I <= J), split-K over the
// K dimension so that tiles x splits ~ one CTA per SM.  Per CTA, a 3-stage ring of
// 64-wide K blocks (H_I, L_I, H_J, L_J: 4 x 16 KB, 128B-swizzled) is filled by TMA
// (cp.async.bulk.tensor) from one producer thread; one thread issues tcgen05.mma
// (kind::f16, bf16 x bf16 -> f32, M = N = 128, K = 16) into a 128-column TMEM
// accumulator; tcgen05.commit frees each stage.  The tensor-core FP32 accumulation
// is not round-to-nearest over long sums (its error grows with the number of
// accumulations), so the accumulator is double-buffered in TMEM (2 x 128 columns) and
// restarted every kChunk K blocks: 16 epilogue warps read each finished chunk with
// tcgen05.ld and add it into double-float (TwoSum) registers while the next chunk
// accumulates.  Each CTA writes an FP64 partial tile; a second kernel sums the split
// partials in FP64 and mirrors the upper triangle.
//
// Every mbarrier wait is bounded: on timeout the kernel raises RSX_ETIMEOUT in the
// status word, stops issuing, drains what it issued (bounded), frees TMEM and returns.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/rsx.h"
#include "api_internal.cuh"
#include "gemm_tcgen05.cuh"
#include "tcgen05_util.cuh"

namespace rsx {
namespace {

using namespace tc;

constexpr int kBM = 128, kBN = 128, kBK = 64;
constexpr int kStages = 3;
constexpr int kTileBytes = kBM * kBK * 2;           // 16 KB per operand tile
constexpr int kStageBytes = 4 * kTileBytes;         // H_I, L_I, H_J, L_J
constexpr int kEpiWarps = 16;                       // four per TMEM lane quarter, 32 columns each
constexpr int kGemmThreads = 32 * (2 + kEpiWarps);  // producer, MMA, epilogue warps
constexpr int kTmemCols = 2 * kBN;                  // double-buffered 128-column accumulator
constexpr int kChunk = 4;                           // K blocks per TMEM accumulation chunk

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row core groups 1024 B apart
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);   // start address (16-byte units)
  d |= (uint64_t)1 << 16;                      // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;           // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                      // descriptor version for tcgen05
  d |= (uint64_t)2 << 61;                      // 128-byte swizzle
  return d;
}

// instruction descriptor, kind::f16: D f32, A/B bf16, both K-major, M = 128, N = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kBN >> 3) << 17) |
                            ((uint32_t)(kBM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accum) {
  asm volatile(
      "{\n"
      " .reg .pred p;\n"
      " setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
      "}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accum)
      : "memory");
}

// upper-triangle tile index -> (I, J), I <= J, row-major over nb blocks
__device__ __forceinline__ void tile_ij(int tile, int nb, int& I, int& J) {
  int i = 0, rem = tile;
  while (rem >= nb - i) {
    rem -= nb - i;
    ++i;
  }
  I = i;
  J = i + rem;
}

__global__ void __launch_bounds__(kGemmThreads, 1)
    k_syrk_bf16x3(const __grid_constant__ CUtensorMap tm_hi, const __grid_constant__ CUtensorMap tm_lo, int nb,
                  int nkb, int nsplit, int blocked, double* __restrict__ part, int* status) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte aligned operand ring
  unsigned char* ring = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  __shared__ __align__(8) uint64_t full_bar[kStages];
  __shared__ __align__(8) uint64_t empty_bar[kStages];
  __shared__ __align__(8) uint64_t tfull_bar[2];
  __shared__ __align__(8) uint64_t tempty_bar[2];
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_sh;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tile = blockIdx.x / nsplit;
  const int split = blockIdx.x - tile * nsplit;
  int I, J;
  tile_ij(tile, nb, I, J);
  const int kb0 = (int)((long long)nkb * split / nsplit);
  const int kb1 = (int)((long long)nkb * (split + 1) / nsplit);
  const int nchunk = (kb1 - kb0 + kChunk - 1) / kChunk;

  if (threadIdx.x == 0) {
    abort_sh = 0;
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull_bar[b], 1);
      mbar_init(&tempty_bar[b], kEpiWarps);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base_sh;
  volatile int* abort_flag = &abort_sh;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer
      int issued = 0;
      for (int kb = kb0; kb < kb1; ++kb) {
        const int it = kb - kb0;
        const int s = it % kStages;
        const uint32_t ph = (uint32_t)((it / kStages) & 1);
        if (it >= kStages && !mbar_wait(&empty_bar[s], ph ^ 1u, abort_flag)) break;
        unsigned char* st = ring + (size_t)s * kStageBytes;
        // diagonal tiles (I == J) read one operand pair and use it on both sides
        mbar_arrive_expect_tx(&full_bar[s], I == J ? 2 * kTileBytes : kStageBytes);
        // row-major panel: box at (k, row); tile-major panel: box (kb, row block) is the
        // contiguous 128 x 64 block number kb * nb + row block
        const int kx = blocked ? 0 : kb * kBK;
        const int ri = blocked ? (kb * nb + I) * kBM : I * kBM;
        const int rj = blocked ? (kb * nb + J) * kBN : J * kBN;
        tma_load_2d(st + 0 * kTileBytes, &tm_hi, &full_bar[s], kx, ri);
        tma_load_2d(st + 1 * kTileBytes, &tm_lo, &full_bar[s], kx, ri);
        if (I != J) {
          tma_load_2d(st + 2 * kTileBytes, &tm_hi, &full_bar[s], kx, rj);
          tma_load_2d(st + 3 * kTileBytes, &tm_lo, &full_bar[s], kx, rj);
        }
        issued = it + 1;
      }
      // drain: every issued stage's copies must have landed before the CTA exits
      const int first = issued > kStages ? issued - kStages : 0;
      for (int it = first; it < issued; ++it) {
        const int s = it % kStages;
        const uint32_t ph = (uint32_t)((it / kStages) & 1);
        for (uint32_t i = 0; i < kWaitLimit && !mbar_try_wait(&full_bar[s], ph); ++i) {
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer: chunks of kChunk K blocks into alternating TMEM buffers
      bool live = true;
      for (int ch = 0; ch < nchunk && live; ++ch) {
        const int b = ch & 1, use = ch >> 1;
        if (use > 0 && !mbar_wait(&tempty_bar[b], (uint32_t)((use - 1) & 1), abort_flag)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t acc = tmem + (uint32_t)(b * kBN);
        const int c0 = kb0 + ch * kChunk;
        const int c1 = min(c0 + kChunk, kb1);
        for (int kb = c0; kb < c1; ++kb) {
          const int it = kb - kb0;
          const int s = it % kStages;
          const uint32_t ph = (uint32_t)((it / kStages) & 1);
          if (!mbar_wait(&full_bar[s], ph, abort_flag)) {
            live = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t base = smem_u32(ring + (size_t)s * kStageBytes);
          const uint64_t dh_i = sw128_desc(base + 0 * kTileBytes);
          const uint64_t dl_i = sw128_desc(base + 1 * kTileBytes);
          const uint64_t dh_j = I == J ? dh_i : sw128_desc(base + 2 * kTileBytes);
          const uint64_t dl_j = I == J ? dl_i : sw128_desc(base + 3 * kTileBytes);
#pragma unroll
          for (int j = 0; j < kBK / 16; ++j) {
            const uint64_t adv = (uint64_t)((j * 32) >> 4);   // 16 bf16 = 32 bytes along K
            mma_bf16(acc, dh_i + adv, dh_j + adv, (kb > c0 || j > 0) ? 1u : 0u);
            mma_bf16(acc, dh_i + adv, dl_j + adv, 1u);
            mma_bf16(acc, dl_i + adv, dh_j + adv, 1u);
          }
          mma_commit(&empty_bar[s]);
        }
        mma_commit(&tfull_bar[b]);   // fires when this chunk's MMAs have completed
      }
    }
  } else {
    // ---------------- epilogue warps: drain each chunk into double-float registers
    const int e = warp - 2;                  // 0..15
    const int quarter = warp & 3;            // TMEM lanes this warp may access
    const int cg = e >> 2;                   // columns [32 cg, 32 cg + 32)
    const int row = quarter * 32 + lane;
    float sh[32], sl[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) sh[i] = sl[i] = 0.f;
    bool ok = true;
    for (int ch = 0; ch < nchunk; ++ch) {
      const int b = ch & 1, use = ch >> 1;
      ok = mbar_wait(&tfull_bar[b], (uint32_t)(use & 1), abort_flag);
      if (!ok) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * kBN + cg * 32);
      float v[32];
      tmem_ld32(taddr, v);
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0)
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&tempty_bar[b])) : "memory");
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        // TwoSum: (sh, sl) += v exactly up to the final rounding of sl
        const float t = sh[i] + v[i];
        const float bp = t - sh[i];
        const float err = (sh[i] - (t - bp)) + (v[i] - bp);
        sh[i] = t;
        sl[i] += err;
      }
    }
    double* dst = part + ((size_t)tile * nsplit + split) * (kBM * kBN) + (size_t)row * kBN + cg * 32;
    const bool good = ok && !*abort_flag;
#pragma unroll
    for (int i = 0; i < 32; ++i) dst[i] = good ? (double)sh[i] + (double)sl[i] : 0.0;
  }
  if (threadIdx.x == 0 && *abort_flag && status) atomicMax(status, RSX_ETIMEOUT);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

// C[t][s] = sum over splits of the partial tiles (FP64), mirrored; diagonal tiles are
// symmetrised by averaging (t, s) and (s, t).
__global__ void k_syrk_reduce(const double* __restrict__ part, int n, int nb, int nsplit, double* __restrict__ C) {
  const long long total = (long long)n * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int t = (int)(e / n), s = (int)(e - (long long)t * n);
    const int a = t < s ? t : s, b = t < s ? s : t;
    const int I = a / kBM, J = b / kBN;
    const int tile = I * nb - I * (I - 1) / 2 + (J - I);
    const int ra = a - I * kBM, cb = b - J * kBN;
    double v = 0.0;
    const double* p = part + (size_t)tile * nsplit * (kBM * kBN);
    for (int sp = 0; sp < nsplit; ++sp) {
      const double* q = p + (size_t)sp * (kBM * kBN);
      v += q[ra * kBN + cb];
      if (I == J) v += q[cb * kBN + ra];
    }
    if (I == J) v *= 0.5;
    C[e] = v;
  }
}

}  // namespace

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

namespace {

// 2-D view of a panel: row-major [rows][ld], or tile-major as [rows * ld / 64][64]
bool make_map(CUtensorMap* m, const void* base, int rows, long long ld, bool blocked) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const long long inner = blocked ? kBK : ld;
  const long long outer = blocked ? (long long)rows * (ld / kBK) : rows;
  cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
  cuuint64_t strides[1] = {(cuuint64_t)inner * 2};
  cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)kBM};
  cuuint32_t es[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

int syrk_splits(int nsm, int n) {
  const int nb = (n + kBM - 1) / kBM;
  const int tiles = nb * (nb + 1) / 2;
  int s = nsm / tiles;
  return s < 1 ? 1 : s;
}

size_t syrk_partial_bytes(int n, int nsplit) {
  const int nb = (n + kBM - 1) / kBM;
  const int tiles = nb * (nb + 1) / 2;
  return (size_t)tiles * nsplit * kBM * kBN * sizeof(double);
}

// hi, lo: bf16 panels of n_pad = 128 * ceil(n / 128) rows (rows >= n zero) and ld % 64 == 0
// columns, row-major [n_pad][ld] or (blocked) tile-major [ld / 64][n_pad / 128][128][64]
int syrk_bf16x3(rsx_ctx* c, const uint16_t* hi, const uint16_t* lo, int n, long long ld, int nsplit, double* part,
                double* C, cudaStream_t s, bool blocked) {
  if (n < 1 || ld < kBK || ld % kBK) return set_error(c, RSX_EINVAL, "syrk: need n >= 1 and ld a multiple of 64");
  if ((reinterpret_cast<uintptr_t>(hi) | reinterpret_cast<uintptr_t>(lo)) & 15)
    return set_error(c, RSX_EINVAL, "syrk: panels must be 16-byte aligned");
  const int nb = (n + kBM - 1) / kBM;
  const int tiles = nb * (nb + 1) / 2;
  CUtensorMap mh, ml;
  if (!make_map(&mh, hi, nb * kBM, ld, blocked) || !make_map(&ml, lo, nb * kBM, ld, blocked))
    return set_error(c, RSX_ECUDA, "syrk: cuTensorMapEncodeTiled failed");
  const int nkb = (int)(ld / kBK);
  const size_t smem = (size_t)kStages * kStageBytes + 1024;
  cudaError_t e = cudaFuncSetAttribute(k_syrk_bf16x3, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return check_cuda(c, e, "syrk smem attribute");
  {
    ProfScope ps(c, kKGemm, s);
    k_syrk_bf16x3<<<tiles * nsplit, kGemmThreads, smem, s>>>(mh, ml, nb, nkb, nsplit, blocked ? 1 : 0, part,
                                                              c->status);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return check_cuda(c, e, "syrk launch");
  {
    ProfScope ps(c, kKGemmReduce, s);
    k_syrk_reduce<<<512, 256, 0, s>>>(part, n, nb, nsplit, C);
    e = cudaGetLastError();
  }
  return check_cuda(c, e, "syrk reduce");
}

}  // namespace rsx
