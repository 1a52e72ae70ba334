// Casida pair-spectrum launcher (fp32 spectra, bf16 hi/lo panel)
#include "poisson_launch.cuh"

namespace rsx {

constexpr int spectrum_threads(int A) { return A <= 12 ? 512 : 448; }

// wsq[kx][iy][iz] = sqrt(w_kx * vhat[kx][iy][iz] * h^3), w = 1 at kx = 0, Mx/2 and 2
// otherwise (vhat = ghat h^3 / N_pad): the Casida panel weights
static __global__ void k_spectrum_weights(const float* __restrict__ vhat, int Hx, int Hy, int Hz, int Mx, float h3,
                                   float* __restrict__ wsq) {
  const size_t n = (size_t)Hx * Hy * Hz;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int kx = (int)(i / ((size_t)Hy * Hz));
    const float w = (kx == 0 || 2 * kx == Mx) ? 1.0f : 2.0f;
    wsq[i] = sqrtf(w * vhat[i] * h3);
  }
}

cudaError_t launch_spectrum_weights(const Geom& g, const float* vhat, float h3, float* wsq, cudaStream_t s) {
  k_spectrum_weights<<<512, 256, 0, s>>>(vhat, g.Hx, g.My / 2 + 1, g.Mz / 2 + 1, g.Mx, h3, wsq);
  return cudaGetLastError();
}

cudaError_t launch_spectrum_f32(const Geom& g, int nq, const Cx<float>* inter, const Cx<float>* twy,
                                const Cx<float>* twz, const float* wsq, uint16_t* hi,
                                uint16_t* lo, size_t ld, int nrb, cudaStream_t s) {
  if (nq <= 0) return cudaSuccess;
  if (g.Ay != g.Az) return cudaErrorInvalidValue;
  // 512 threads (32 lines in flight) where the kernel fits 128 registers (A <= 12); 448
  // (28 lines, a divisor of n = 112) for A = 14; 256 when that does not fit in shared
  // memory.  (Dividing n evenly with fewer lines, e.g. 320 threads at n = 80, measured
  // slower than 512 with one partial round.)
  int nt = spectrum_threads(g.Ay);
  size_t smem = pass2_scratch_smem<float>(g.Ay, g.Az, nt) + pass2_plane_bytes<float>(g);
  if (smem > (size_t)max_dyn_smem()) {
    nt = 256;
    smem = pass2_scratch_smem<float>(g.Ay, g.Az, nt) + pass2_plane_bytes<float>(g);
  }
  if (smem > (size_t)max_dyn_smem()) return cudaErrorInvalidValue;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const long long nwork = (long long)nq * g.Hx;
  switch (g.Ay) {
#define RSX_CASE(a)                                                                              \
  case a: {                                                                                      \
    auto k = nt == 256 ? k_spectrum<a, a, 256> : k_spectrum<a, a, spectrum_threads(a)>;          \
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
    if (e != cudaSuccess) return e;                                                              \
    int per_sm = 1;                                                                              \
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, nt, smem) != cudaSuccess) {    \
      cudaGetLastError();                                                                        \
      per_sm = 1;                                                                                \
    }                                                                                            \
    const long long cap = (long long)(per_sm > 0 ? per_sm : 1) * nsm;                            \
    const int grid = (int)(nwork < cap ? nwork : cap);                                           \
    k<<<grid, nt, smem, s>>>(g, nq, inter, twy, twz, wsq, hi, lo, ld, nrb);                \
    return cudaGetLastError();                                                                   \
  }
    RSX_FOR_EACH_A(RSX_CASE)
#undef RSX_CASE
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace rsx
