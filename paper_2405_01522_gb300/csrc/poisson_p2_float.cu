// pass 2 (y/z transforms with the kernel multiply), float
#include "poisson_launch.cuh"

namespace rsx {
template size_t pass2_smem_bytes<float>(const Geom&, bool*);
template int pass2_occupancy<float>(const Geom&);
template cudaError_t launch_pass2<float>(const Geom&, int, Cx<float>*, const Cx<float>*, const Cx<float>*, const float*,
                                       const float*, float*, int, cudaStream_t);
}  // namespace rsx
