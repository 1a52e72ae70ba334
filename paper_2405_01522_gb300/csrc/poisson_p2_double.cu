// pass 2 (y/z transforms with the kernel multiply), double
#include "poisson_launch.cuh"

namespace rsx {
template size_t pass2_smem_bytes<double>(const Geom&, bool*);
template int pass2_occupancy<double>(const Geom&);
template cudaError_t launch_pass2<double>(const Geom&, int, Cx<double>*, const Cx<double>*, const Cx<double>*, const double*,
                                        const float*, double*, int, cudaStream_t, const Cx<float>*, const float*);
}  // namespace rsx
