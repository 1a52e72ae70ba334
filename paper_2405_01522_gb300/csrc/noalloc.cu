// rsx_exchange_apply_noalloc: the exchange action of rsx_exchange_apply with its FFT
// intermediates in a fixed, file-scope device array instead of context workspace.
//
// Who needs it: callers that may not allocate device memory once they are running,
// for example a host program whose device memory is handed out by its own pool
// allocator sized at start-up (a cudaMalloc behind the pool's back can fail or
// fragment that budget), or a latency-sensitive loop that must not hit the implicit
// device-wide synchronisation of cudaFree when a workspace is regrown.  They create the
// context (kernel table and twiddles) once at start-up; this call then allocates
// nothing: no cudaMalloc, no cudaFree, no allocating library routine.
//
// The array is kNoAllocScratchBytes (64 MiB) of device memory held by every GPU that
// loads the library, from module load until process exit.  One output orbital is
// processed at a time, so the limit is nocc pair intermediates:
//     nocc * (nx + 1) * nz * ny * 2 * sizeof(element) <= 64 MiB
// (e.g. FP32 32^3: nocc <= 248; FP32 64^3: nocc <= 31; FP32 96^3: nocc <= 9).
// Larger requests are rejected with RSX_EINVAL before anything is launched.  Only boxes
// whose y/z pass fits in shared memory are served (FP32 edges up to 112, FP64 up to 64);
// others return RSX_EUNSUPPORTED.
//
// Every call on a device shares the one array and it keeps the last call's contents.
// Nothing in it has to start at zero: pass 1 writes every intermediate element that
// passes 2 and 3 read.  Calls whose work overlaps on the GPU (different streams, or
// different host threads) race on the array and give wrong results; serialise them.
//
// Set-up: the first call on each device looks up the array's device address with
// cudaGetSymbolAddress while that device is current, checks the result and caches it
// (the array's name is only a host-side stand-in in host code).  With lazy module
// loading (the CUDA default) that lookup is also the moment the driver loads the module
// holding the array and maps its 64 MiB, and the first launch of each FFT pass kernel
// loads that kernel's module, so the FIRST call on a device can allocate driver memory;
// every later call allocates nothing.  Make one call on each device at start-up, before
// any stream capture begins and before the caller's allocation budget is fixed.  The
// cached address stays valid until process exit; a cudaDeviceReset invalidates it (the
// library is then not usable on that device until the process restarts).  The caller's
// current device is restored before each call returns.
#include <mutex>

#include "../../include/rsx.h"
#include "api_internal.cuh"

using namespace rsx;

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_setup_mu;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of g_noalloc_scratch on `device` (which must be current).
int scratch_address(rsx_ctx* c, int device, void** out) {
  if (device < 0 || device >= kMaxDevices) return set_error(c, RSX_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (g_scratch_ptr[device] == nullptr) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return check_cuda(c, e == cudaSuccess ? cudaErrorInvalidSymbol : e, "cudaGetSymbolAddress(noalloc scratch)");
    }
    g_scratch_ptr[device] = p;
  }
  *out = g_scratch_ptr[device];
  return RSX_OK;
}

template <typename R>
int exchange_noalloc(rsx_ctx* c, const void* phi, int nocc, const void* psi, int npsi, void* out, void* scratch,
                     cudaStream_t s) {
  Geom g = c->g;
  g.p2_global = 0;   // the y/z pass always in shared memory here (no plane scratch to allocate)
  const size_t N = g.N();
  PairMap<R> pm;
  pm.mode = kProd;
  pm.A = (const R*)phi;
  pm.B = (const R*)psi;
  pm.na = nocc;
  pm.nb = npsi;
  pm.N = N;
  Cx<R>* inter = (Cx<R>*)scratch;
  const Cx<R>* twz = (const Cx<R>*)c->tw[0];
  const Cx<R>* twy = (const Cx<R>*)c->tw[1];
  const Cx<R>* twx = (const Cx<R>*)c->tw[2];
  const int per_sm = std::max(1, pass2_occupancy<R>(g));
  const int grid = (int)std::min<long long>((long long)nocc * g.Hx, (long long)per_sm * c->nsm);
  for (int p = 0; p < npsi; ++p) {
    int rc = check_cuda(c, launch_pass1<R>(g, pm, p * nocc, nocc, inter, twx, s), "noalloc pass 1");
    if (rc) return rc;
    rc = check_cuda(c, launch_pass2<R>(g, nocc, inter, twy, twz, (const R*)c->vhat, (const float*)c->vhatz, nullptr, grid, s),
                    "noalloc pass 2");
    if (rc) return rc;
    rc = check_cuda(c, launch_pass3<R>(g, pm, p * nocc, p, 1, 0, inter, twx, (R*)out + (size_t)p * N, s),
                    "noalloc pass 3");
    if (rc) return rc;
  }
  return RSX_OK;
}

bool overlap(const void* a, size_t na, const void* b, size_t nb) {
  const char* pa = (const char*)a;
  const char* pb = (const char*)b;
  return pa < pb + nb && pb < pa + na;
}

int noalloc_on_device(rsx_ctx* c, const void* phi, int nocc, const void* psi, int npsi, void* out, void* stream);

}  // namespace

extern "C" int rsx_exchange_apply_noalloc(rsx_ctx* c, const void* phi, int nocc, const void* psi, int npsi,
                                          void* out, void* stream) {
  rsx::NvtxRange nvtx_range("rsx_exchange_apply_noalloc");
  if (!c) return RSX_EINVAL;
  c->err[0] = 0;
  if (!phi || !psi || !out || nocc < 1 || npsi < 1) return set_error(c, RSX_EINVAL, "bad exchange arguments");
  const size_t N = c->g.N(), es = c->elem_size();
  if (overlap(out, npsi * N * es, phi, nocc * N * es) || overlap(out, npsi * N * es, psi, npsi * N * es))
    return set_error(c, RSX_EINVAL, "out aliases an input");
  const size_t need = (size_t)nocc * c->g.inter_elems() * 2 * es;
  if (need > kNoAllocScratchBytes)
    return set_error(c, RSX_EINVAL,
                     "noalloc exchange: nocc * (nx+1) * nz * ny * 2 * element size exceeds the 64 MiB static scratch");
  // the work runs on the context's device; the caller's current device is put back on return
  int prev_device = -1;
  if (cudaGetDevice(&prev_device) != cudaSuccess) {
    cudaGetLastError();
    prev_device = -1;
  }
  if (cudaSetDevice(c->device) != cudaSuccess) {
    cudaGetLastError();
    return set_error(c, RSX_ECUDA, "cudaSetDevice failed");
  }
  const int rc = noalloc_on_device(c, phi, nocc, psi, npsi, out, stream);
  if (prev_device >= 0 && prev_device != c->device) cudaSetDevice(prev_device);
  return rc;
}

namespace {

int noalloc_on_device(rsx_ctx* c, const void* phi, int nocc, const void* psi, int npsi, void* out, void* stream) {
  bool fits = false;
  Geom g = c->g;
  g.p2_global = 0;
  if (c->precision == RSX_FP32)
    pass2_smem_bytes<float>(g, &fits);
  else
    pass2_smem_bytes<double>(g, &fits);
  if (!fits) return set_error(c, RSX_EUNSUPPORTED, "noalloc exchange: box too large for the shared-memory y/z pass");
  void* scratch = nullptr;
  const int rc = scratch_address(c, c->device, &scratch);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  return c->precision == RSX_FP32 ? exchange_noalloc<float>(c, phi, nocc, psi, npsi, out, scratch, s)
                                  : exchange_noalloc<double>(c, phi, nocc, psi, npsi, out, scratch, s);
}

}  // namespace
