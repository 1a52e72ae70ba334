// pass 1 (x forward) launchers, both precisions
#include "poisson_launch.cuh"

namespace rsx {

template <typename R>
cudaError_t launch_pass1(const Geom& g, const PairMap<R>& pm, int q0, int nq, Cx<R>* inter,
                         const Cx<R>* twx, cudaStream_t s) {
  if (nq <= 0) return cudaSuccess;
  const size_t smem = pass1_smem<R>(g.Ax);
  const int nyb = (g.ny + kRowsPerCta - 1) / kRowsPerCta;
  const int G = g.p1_group > 0 ? (g.p1_group < nq ? g.p1_group : nq) : 0;
  Geom gg = g;
  gg.p1_group = G;
  const long long nblk = G > 0 ? (long long)((nq + G - 1) / G) * G * nyb * g.nz : (long long)nyb * g.nz * nq;
  if (nblk > 0x7fffffffLL) return cudaErrorInvalidValue;
  switch (g.Ax) {
#define RSX_CASE(a)                                                                              \
  case a: {                                                                                      \
    auto k = k_pass1<R, a>;                                                                      \
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
    if (e != cudaSuccess) return e;                                                              \
    k<<<(unsigned)nblk, kThreads, smem, s>>>(gg, pm, q0, nq, inter, twx);                        \
    return cudaGetLastError();                                                                   \
  }
    RSX_FOR_EACH_A(RSX_CASE)
#undef RSX_CASE
    default: return cudaErrorInvalidValue;
  }
}

template cudaError_t launch_pass1<float>(const Geom&, const PairMap<float>&, int, int, Cx<float>*,
                                         const Cx<float>*, cudaStream_t);
template cudaError_t launch_pass1<double>(const Geom&, const PairMap<double>&, int, int, Cx<double>*,
                                          const Cx<double>*, cudaStream_t);

bool axis_supported(int A) { return axis_supported_impl(A); }

}  // namespace rsx
