// pass 3 (x inverse + exchange accumulation) launchers, both precisions
#include "poisson_launch.cuh"

namespace rsx {

template <typename R>
cudaError_t launch_pass3(const Geom& g, const PairMap<R>& pm, int q0, int p0, int np, int pot, const Cx<R>* inter,
                         const Cx<R>* twx, R* out, cudaStream_t s) {
  if (np <= 0) return cudaSuccess;
  const size_t smem = pass3_smem<R>(g.Ax, g.nx);
  const int nyb = (g.ny + kRowsPerCta - 1) / kRowsPerCta;
  const long long nblk = (long long)nyb * g.nz * np;
  if (nblk > 0x7fffffffLL) return cudaErrorInvalidValue;
  switch (g.Ax) {
#define RSX_CASE(a)                                                                              \
  case a: {                                                                                      \
    auto k = k_pass3<R, a>;                                                                      \
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
    if (e != cudaSuccess) return e;                                                              \
    k<<<(unsigned)nblk, kThreads, smem, s>>>(g, pm, q0, p0, pot, inter, twx, out);                    \
    return cudaGetLastError();                                                                   \
  }
    RSX_FOR_EACH_A(RSX_CASE)
#undef RSX_CASE
    default: return cudaErrorInvalidValue;
  }
}

template cudaError_t launch_pass3<float>(const Geom&, const PairMap<float>&, int, int, int, int, const Cx<float>*,
                                         const Cx<float>*, float*, cudaStream_t);
template cudaError_t launch_pass3<double>(const Geom&, const PairMap<double>&, int, int, int, int, const Cx<double>*,
                                          const Cx<double>*, double*, cudaStream_t);

}  // namespace rsx
