// Context object behind the C ABI and helpers shared by the host-side TUs.
#pragma once
#include <algorithm>
#include <cstddef>

#include <nvtx3/nvToolsExt.h>

#include <vector>

#include "rsx_internal.cuh"

namespace rsx {
// Kernel identifiers for the per-context launch profiler (CUDA events around launches).
enum KernelId {
  kKPass1 = 0, kKPass2, kKPass3, kKSpectrum, kKGram, kKGramReduce, kKChol, kKCombine, kKPairProd,
  kKGemm, kKGemmReduce, kKEig, kKKdSolve, kKCount
};
const char* kernel_name(int id);
}  // namespace rsx

struct rsx_ctx {
  int device = 0;
  int precision = 1;
  double h = 0.0;
  rsx::Geom g{};
  int nsm = 0;
  size_t work_limit = 0;
  // device buffers owned by the context
  void* vhat = nullptr;                 // kernel table T[kx][ky][kz] (R)
  void* vhatz = nullptr;                // FP32: the same in pass 2's lane order (launch_vhat_lanes)
  void* vhatz8 = nullptr;               // FP32, Ay % 4 == 0: the order of the 8-lane y/z kernel
  void* tw8 = nullptr;                  // FP32, Ay % 4 == 0: twiddles w_M^{-t k1}, t < 8, k1 < 2 Ay
  void* tw[3] = {nullptr, nullptr, nullptr};
  void* work = nullptr;   size_t work_bytes = 0;     // FFT intermediates
  void* gscr = nullptr;   size_t gscr_bytes = 0;     // pass-2 planes when shared memory is too small
  double* dsm = nullptr;  size_t dsm_bytes = 0;      // FP64 partials and small matrices
  void* smallr = nullptr; size_t smallr_bytes = 0;   // small R-typed coefficient matrices
  int* status = nullptr;                             // deferred device status word
  void* panel_hi = nullptr; size_t panel_hi_bytes = 0;  // Casida spectrum panel, bf16 hi
  void* panel_lo = nullptr; size_t panel_lo_bytes = 0;  // bf16 lo
  void* gemm_part = nullptr; size_t gemm_part_bytes = 0;
  void* eig_work = nullptr; size_t eig_work_bytes = 0;
  void* gscr_kd = nullptr; size_t gscr_kd_bytes = 0;     // occupied pair potentials (K_d)
  void* pos = nullptr; size_t pos_bytes = 0;             // grid coordinates [3][N] (R), dipoles
  void* specw = nullptr; size_t specw_bytes = 0;         // Casida panel weights (float)
  void* ones = nullptr; size_t ones_bytes = 0;           // unit field (R), Poisson solves of a density
  void* tdhf_work = nullptr; size_t tdhf_work_bytes = 0; // full TDHF: L, A + B, products
  int p2_occ[2] = {0, 0};
  int chunk_outputs = 0;   // tuning: output orbitals per exchange chunk (0 = as many as fit)
  long long wait_limit = -1;   // spin rounds of the bounded grid waits (-1: the kernels' default)
  // host-side fault injection (testing aid): fail the workspace allocation after
  // fault_alloc_after more successful ones (-1: off); flip the sign of the next ACE matrix
  int fault_alloc_after = -1;
  bool fault_pivot = false;
  // launch profiler: events recorded around every kernel while enabled
  bool prof_on = false;
  struct ProfRec { int id; cudaEvent_t a, b; };
  std::vector<ProfRec> prof_pending;
  std::vector<cudaEvent_t> prof_pool;
  double prof_ms[rsx::kKCount] = {0};
  long long prof_n[rsx::kKCount] = {0};
  char err[512] = {0};

  size_t elem_size() const { return precision == 1 ? 4 : 8; }
  template <typename R>
  int pass2_ctas_per_sm() {
    int& o = p2_occ[sizeof(R) == 8 ? 1 : 0];
    if (o == 0) o = std::max(1, rsx::pass2_occupancy<R>(g));
    return o;
  }
};

namespace rsx {
// NVTX range around a C-ABI call (tracing with Nsight Systems; a few nanoseconds when no
// tool is attached)
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
int check_cuda(rsx_ctx* c, cudaError_t e, const char* what);
int grow(rsx_ctx* c, void** p, size_t* have, size_t need, const char* what);
int set_error(rsx_ctx* c, int code, const char* msg);
// RAII timer: records a start event at construction and a stop event at destruction
// on stream s when the context profiler is on.
struct ProfScope {
  rsx_ctx* c;
  int id;
  cudaStream_t s;
  cudaEvent_t a = nullptr, b = nullptr;
  ProfScope(rsx_ctx* c_, int id_, cudaStream_t s_);
  ~ProfScope();
};
// pot = 0: out_p accumulates -partner * V over p's pairs (exchange);
// pot = 1: out_p is the potential of pair q0 + (p - p0) itself.
template <typename R>
int solve_pairs(rsx_ctx* c, const PairMap<R>& pm, int q0, int nq, int p0, int np, R* out, cudaStream_t s,
                int pot = 0);
}  // namespace rsx
