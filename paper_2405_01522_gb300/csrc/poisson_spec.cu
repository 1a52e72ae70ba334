// Casida pair-spectrum launcher (fp32 spectra, bf16 hi/lo panel)
#include "poisson_launch.cuh"

namespace rsx {

cudaError_t launch_spectrum_f32(const Geom& g, int nq, const Cx<float>* inter, const Cx<float>* twy,
                                const Cx<float>* twz, const float* vhat, float h3, uint16_t* hi,
                                uint16_t* lo, size_t ld, int nrb, cudaStream_t s) {
  if (nq <= 0) return cudaSuccess;
  if (g.Ay != g.Az) return cudaErrorInvalidValue;
  // 512 threads (32 lines in flight) where the kernel fits 128 registers without spills
  // (A <= 12) and the shared memory allows it, else 256
  int nt = 512;
  size_t smem = pass2_scratch_smem<float>(g.Ay, g.Az, nt) + pass2_plane_bytes<float>(g);
  if (g.Ay > 12 || smem > (size_t)max_dyn_smem()) {
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
    auto k = (nt == 512 && a <= 12) ? k_spectrum<a, a, 512> : k_spectrum<a, a, 256>;             \
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
    if (e != cudaSuccess) return e;                                                              \
    int per_sm = 1;                                                                              \
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, nt, smem) != cudaSuccess) {    \
      cudaGetLastError();                                                                        \
      per_sm = 1;                                                                                \
    }                                                                                            \
    const long long cap = (long long)(per_sm > 0 ? per_sm : 1) * nsm;                            \
    const int grid = (int)(nwork < cap ? nwork : cap);                                           \
    k<<<grid, nt, smem, s>>>(g, nq, inter, twy, twz, vhat, h3, hi, lo, ld, nrb);                \
    return cudaGetLastError();                                                                   \
  }
    RSX_FOR_EACH_A(RSX_CASE)
#undef RSX_CASE
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace rsx
