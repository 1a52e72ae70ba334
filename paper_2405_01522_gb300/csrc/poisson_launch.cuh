// Launchers of the pair Poisson passes for one precision R (included once per TU).
#pragma once
#include "poisson_kernels.cuh"
#include "poisson_pass2_l8.cuh"

namespace rsx {

#define RSX_FOR_EACH_A(X) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(10) X(12) X(14)

inline bool axis_supported_impl(int A) {
  switch (A) {
#define RSX_CASE(a) case a: return true;
    RSX_FOR_EACH_A(RSX_CASE)
#undef RSX_CASE
    default: return false;
  }
}

// line scratch and the row-block staging buffer share the same bytes (pass1_item)
template <typename R>
inline size_t pass1_smem(int AX) {
  const int L = 16 * AX, H = L / 2 + 1;
  const size_t scr = (size_t)kLinesPerCta * AX * kScrPitch, xs = (size_t)H * kRowsPerCta;
  return sizeof(Cx<R>) * (scr > xs ? scr : xs);
}
template <typename R>
inline size_t pass3_smem(int AX, int nx) {
  return sizeof(Cx<R>) * (size_t)kLinesPerCta * AX * kScrPitch + 2 * pass3_buffer_elems<R>(AX, nx);
}
inline int max_dyn_smem() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return v;
}

// threads per CTA of pass 2 (g.p2_threads): 256 (default), 384 (FP32 only: 12 warps at
// <= 168 registers) or 512 (<= 128 registers), each used only when its line scratch and
// the plane fit in shared memory
template <typename R>
inline int pass2_threads(const Geom& g) {
  int nt = g.p2_threads;
  if (nt != 384 && nt != 512) return 256;
  if (nt == 384 && sizeof(R) != 4) return 256;
  const int A = g.Ay > g.Az ? g.Ay : g.Az;
  const size_t sc = sizeof(Cx<R>) * (size_t)(nt / 16) * A * p2_pitch<R>(A);
  const size_t pl = sizeof(Cx<R>) * (size_t)g.nz * (g.My + 1);
  return (sc + pl <= (size_t)max_dyn_smem()) ? nt : 256;
}

// the shared-memory pass-2 kernel for transform size A and nt threads
template <typename R, int A>
inline auto pass2_kernel(int nt) {
  if constexpr (sizeof(R) == 4) {
    if (nt == 384) return k_pass2<R, A, A, true, 384>;
  }
  return nt == 512 ? k_pass2<R, A, A, true, 512> : k_pass2<R, A, A, true, 256>;
}
template <typename R>
inline size_t pass2_scratch_smem(int AY, int AZ, int nt = kThreads) {
  const int A = AY > AZ ? AY : AZ;
  return sizeof(Cx<R>) * (size_t)(nt / 16) * A * p2_pitch<R>(A);
}
template <typename R>
inline size_t pass2_plane_bytes(const Geom& g) {
  return sizeof(Cx<R>) * (size_t)g.nz * (g.My + 1);
}



template <typename R>
size_t pass2_smem_bytes(const Geom& g, bool* fits) {
  const bool global = g.p2_global != 0;
  const size_t sc = pass2_scratch_smem<R>(g.Ay, g.Az, global ? kThreads : pass2_threads<R>(g));
  const size_t pl = pass2_plane_bytes<R>(g);
  const bool f = !global && sc + pl <= (size_t)max_dyn_smem();
  if (fits) *fits = f;
  return f ? sc + pl : sc;
}

template <typename R>
int pass2_occupancy(const Geom& g) {
  bool fits = false;
  const size_t smem = pass2_smem_bytes<R>(g, &fits);
  int nb = 1;
  switch (g.Ay) {
#define RSX_CASE(a)                                                                                  \
  case a: {                                                                                          \
    const int nt = pass2_threads<R>(g);                                                              \
    auto k = pass2_kernel<R, a>(nt);                                                                 \
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess || \
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, nt, smem) != cudaSuccess) {            \
      cudaGetLastError();                                                                            \
      nb = 1;                                                                                        \
    }                                                                                                \
    break;                                                                                           \
  }
    RSX_FOR_EACH_A(RSX_CASE)
#undef RSX_CASE
    default: break;
  }
  return nb;
}

// threads per CTA of the 8-lane kernel (384 where its scratch and the plane fit, else
// 256), 0 when it does not serve this geometry
template <int A>
inline int pass2_l8_threads(const Geom& g) {
  const int want = g.p2_threads == 256 ? 256 : 384;
  for (int nt : {want, 256})
    if (pass2_l8_smem<A>(nt) <= (size_t)max_dyn_smem()) return nt;
  return 0;
}

inline bool pass2_l8_ok(const Geom& g, const void* tw8, const void* vl8) {
  if (g.p2_lanes != 8 || g.p2_global || !tw8 || !vl8 || g.Ay != g.Az) return false;
  switch (g.Ay) {
    case 4: return pass2_l8_threads<4>(g) > 0;
    case 8: return pass2_l8_threads<8>(g) > 0;
    case 12: return pass2_l8_threads<12>(g) > 0;
    default: return false;
  }
}

template <int A>
cudaError_t launch_pass2_l8(const Geom& g, int nq, Cx<float>* inter, const Cx<float>* tw8, const float* vl8, int grid,
                            cudaStream_t s) {
  const int nt = pass2_l8_threads<A>(g);
  const size_t smem = pass2_l8_smem<A>(nt);
  // twiddles held in registers (153 registers at A = 12: 384 threads fit without spills)
  auto k = nt == 384 ? k_pass2_l8<A, 384, false> : k_pass2_l8<A, 256, false>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k<<<grid, nt, smem, s>>>(g, nq, inter, tw8, vl8);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_pass2(const Geom& g, int nq, Cx<R>* inter, const Cx<R>* twy, const Cx<R>* twz,
                         const R* vhat, const float* vhat_lanes, R* gscratch, int grid, cudaStream_t s,
                         const Cx<float>* tw8, const float* vl8) {
  if (nq <= 0) return cudaSuccess;
  if (g.Ay != g.Az) return cudaErrorInvalidValue;
  if (sizeof(R) == 4 && vhat_lanes == nullptr) return cudaErrorInvalidValue;   // FP32 reads the lane-order table
  if constexpr (sizeof(R) == 4) {
    if (pass2_l8_ok(g, tw8, vl8)) {
      Cx<float>* in = reinterpret_cast<Cx<float>*>(inter);
      switch (g.Ay) {
        case 4: return launch_pass2_l8<4>(g, nq, in, tw8, vl8, grid, s);
        case 8: return launch_pass2_l8<8>(g, nq, in, tw8, vl8, grid, s);
        case 12: return launch_pass2_l8<12>(g, nq, in, tw8, vl8, grid, s);
        default: break;
      }
    }
  }
  bool fits = false;
  const size_t smem = pass2_smem_bytes<R>(g, &fits);
  if (!fits && gscratch == nullptr) return cudaErrorInvalidValue;
  switch (g.Ay) {
#define RSX_CASE(a)                                                                                  \
  case a: {                                                                                          \
    if (fits) {                                                                                      \
      const int nt = pass2_threads<R>(g);                                                            \
      auto k = pass2_kernel<R, a>(nt);                                                               \
      cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
      if (e != cudaSuccess) return e;                                                                \
      k<<<grid, nt, smem, s>>>(g, nq, inter, twy, twz, vhat, vhat_lanes, gscratch);                  \
    } else {                                                                                         \
      auto k = k_pass2<R, a, a, false, 256>;                                                         \
      cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
      if (e != cudaSuccess) return e;                                                                \
      k<<<grid, kThreads, smem, s>>>(g, nq, inter, twy, twz, vhat, vhat_lanes, gscratch);            \
    }                                                                                                \
    return cudaGetLastError();                                                                       \
  }
    RSX_FOR_EACH_A(RSX_CASE)
#undef RSX_CASE
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace rsx
