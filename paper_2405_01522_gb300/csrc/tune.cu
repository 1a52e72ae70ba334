// Autotuner for the pair-solve path.
//
// Candidates (per box size, precision and device):
//   - threads per CTA of the y/z pass: 256, 384 or 512 (FP32; each only where its
//     scratch fits);
//   - output orbitals per exchange chunk: 1, 2, 4 or all.  Small chunks keep each
//     chunk's pair intermediates (nocc x 7.15 MB at 96^3) near L2 size between passes,
//     large chunks launch fewer, fuller grids.
// Each candidate runs the exchange apply on synthetic orbitals on the device (one
// warm-up, best of two timed runs with CUDA events); the fastest is applied to the
// context and appended to a text cache keyed by (edges, precision, nocc, npsi, SMs,
// device name) so later contexts skip the timing.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/rsx.h"
#include "api_internal.cuh"

using namespace rsx;

namespace {

template <typename R>
__global__ void k_fill_synthetic(R* x, size_t n, uint32_t seed) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    uint32_t h = (uint32_t)i * 2654435761u ^ seed;
    h ^= h >> 16;
    h *= 0x7feb352du;
    h ^= h >> 15;
    x[i] = (R)((double)(h & 0xffffff) / 16777216.0 - 0.5);
  }
}

std::string cache_key(const rsx_ctx* c, int nocc, int npsi) {
  cudaDeviceProp prop;
  cudaGetDeviceProperties(&prop, c->device);
  char buf[512];
  snprintf(buf, sizeof(buf), "rsx1 %d %d %d %s %d %d %d %s", c->g.nz, c->g.ny, c->g.nx,
           c->precision == RSX_FP32 ? "fp32" : "fp64", nocc, npsi, c->nsm, prop.name);
  for (char* p = buf; *p; ++p)
    if (*p == '\n') *p = ' ';
  return buf;
}

bool cache_lookup(const char* path, const std::string& key, int* p2, int* chunk) {
  if (!path || !*path) return false;
  FILE* f = fopen(path, "r");
  if (!f) return false;
  char line[1024];
  bool found = false;
  while (fgets(line, sizeof(line), f)) {
    const size_t kl = key.size();
    if (strncmp(line, key.c_str(), kl) == 0 && line[kl] == '|') {
      if (sscanf(line + kl + 1, "%d %d", p2, chunk) == 2) found = true;  // last entry wins
    }
  }
  fclose(f);
  return found;
}

void cache_store(const char* path, const std::string& key, int p2, int chunk, double ms) {
  if (!path || !*path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s|%d %d %.4f\n", key.c_str(), p2, chunk, ms);
  fclose(f);
}

}  // namespace

extern "C" int rsx_autotune(rsx_ctx* c, int nocc, int npsi, const char* cache_path, int* p2_threads,
                            int* chunk_outputs, double* best_ms) {
  if (!c || nocc < 1 || npsi < 1) return RSX_EINVAL;
  c->err[0] = 0;
  if (cudaSetDevice(c->device) != cudaSuccess) {
    cudaGetLastError();
    return set_error(c, RSX_ECUDA, "cudaSetDevice failed");
  }
  const std::string key = cache_key(c, nocc, npsi);
  int bp2 = 256, bch = 0;
  double bms = -1.0;
  if (cache_lookup(cache_path, key, &bp2, &bch)) {
    c->g.p2_threads = bp2;
    c->p2_occ[0] = c->p2_occ[1] = 0;
    c->chunk_outputs = bch;
  } else {
    const size_t N = c->g.N(), es = c->elem_size();
    void *phi = nullptr, *psi = nullptr, *out = nullptr;
    if (cudaMalloc(&phi, nocc * N * es) != cudaSuccess || cudaMalloc(&psi, npsi * N * es) != cudaSuccess ||
        cudaMalloc(&out, npsi * N * es) != cudaSuccess) {
      cudaGetLastError();
      if (phi) cudaFree(phi);
      if (psi) cudaFree(psi);
      return set_error(c, RSX_ENOMEM, "autotune: cannot allocate synthetic orbitals");
    }
    if (c->precision == RSX_FP32) {
      k_fill_synthetic<float><<<1024, 256>>>((float*)phi, nocc * N, 1u);
      k_fill_synthetic<float><<<1024, 256>>>((float*)psi, npsi * N, 2u);
    } else {
      k_fill_synthetic<double><<<1024, 256>>>((double*)phi, nocc * N, 1u);
      k_fill_synthetic<double><<<1024, 256>>>((double*)psi, npsi * N, 2u);
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int saved_p2 = c->g.p2_threads, saved_ch = c->chunk_outputs;
    const int p2s[3] = {256, 384, 512};
    const int chs[4] = {1, 2, 4, 0};
    int rc = RSX_OK;
    for (int a = 0; a < 3 && !rc; ++a) {
      if (a > 0 && c->precision != RSX_FP32) break;
      for (int b = 0; b < 4 && !rc; ++b) {
        if (chs[b] >= npsi) continue;
        c->g.p2_threads = p2s[a];
        c->p2_occ[0] = c->p2_occ[1] = 0;
        c->chunk_outputs = chs[b];
        rc = rsx_exchange_apply(c, phi, nocc, psi, npsi, out, nullptr);
        if (rc) break;
        double best = 1e30;
        for (int r = 0; r < 2 && !rc; ++r) {
          cudaEventRecord(e0, 0);
          rc = rsx_exchange_apply(c, phi, nocc, psi, npsi, out, nullptr);
          cudaEventRecord(e1, 0);
          cudaEventSynchronize(e1);
          float ms = 0.f;
          cudaEventElapsedTime(&ms, e0, e1);
          if (ms < best) best = ms;
        }
        if (!rc && (bms < 0 || best < bms)) {
          bms = best;
          bp2 = p2s[a];
          bch = chs[b];
        }
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(phi);
    cudaFree(psi);
    cudaFree(out);
    if (rc) {
      c->g.p2_threads = saved_p2;
      c->chunk_outputs = saved_ch;
      return rc;
    }
    c->g.p2_threads = bp2;
    c->p2_occ[0] = c->p2_occ[1] = 0;
    c->chunk_outputs = bch;
    cache_store(cache_path, key, bp2, bch, bms);
  }
  if (p2_threads) *p2_threads = c->g.p2_threads;
  if (chunk_outputs) *chunk_outputs = c->chunk_outputs;
  if (best_ms) *best_ms = bms;
  return RSX_OK;
}

extern "C" int rsx_set_tuning(rsx_ctx* c, int p2_threads, int chunk_outputs) {
  if (!c || (p2_threads != 256 && p2_threads != 384 && p2_threads != 512) || chunk_outputs < 0) return RSX_EINVAL;
  c->g.p2_threads = p2_threads;
  c->p2_occ[0] = c->p2_occ[1] = 0;
  c->chunk_outputs = chunk_outputs;
  return RSX_OK;
}
