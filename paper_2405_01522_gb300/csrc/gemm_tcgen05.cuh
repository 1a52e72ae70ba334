// Split-BF16 symmetric contraction on tcgen05 tensor cores (gemm_tcgen05.cu).
#pragma once
#include <cuda.h>
#include <cstdint>

#include "rsx_internal.cuh"

struct rsx_ctx;

namespace rsx {
// cuTensorMapEncodeTiled from the driver (null if the driver does not provide it)
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_fn();
// number of K splits for an n x n output on nsm SMs (about one CTA per SM)
int syrk_splits(int nsm, int n);
// bytes of the FP32 split partials
size_t syrk_partial_bytes(int n, int nsplit);
// C = H H^T + H L^T + L H^T (FP64 out, n x n row-major, symmetric).  hi, lo: 128*ceil(n/128) rows
// (rows >= n zero) x ld columns (ld % 64 == 0), 16-byte aligned; row-major, or with `blocked`
// tile-major [ld/64][rows/128][128][64] so that every 128 x 64 TMA box is contiguous.
int syrk_bf16x3(rsx_ctx* c, const uint16_t* hi, const uint16_t* lo, int n, long long ld, int nsplit, double* part,
                double* C, cudaStream_t s, bool blocked = false);
}  // namespace rsx
