// pass 2 (y/z transforms with the kernel multiply), float
#include "poisson_launch.cuh"

namespace rsx {
template size_t pass2_smem_bytes<float>(const Geom&, bool*);
template int pass2_occupancy<float>(const Geom&);
template cudaError_t launch_pass2<float>(const Geom&, int, Cx<float>*, const Cx<float>*, const Cx<float>*, const float*,
                                        const float*, float*, int, cudaStream_t, const Cx<float>*, const float*);
bool pass2_l8_active(const Geom& g, const void* tw8, const void* vl8) { return pass2_l8_ok(g, tw8, vl8); }
}  // namespace rsx
