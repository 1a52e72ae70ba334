// Autotuner for the pair-solve path.
//
// Knobs (rsx_tuning, per box size, precision and device):
//   - p2_threads: threads per CTA of the y/z pass, 256, 384 (FP32) or 512, each used only
//     where its line scratch and the work plane fit in shared memory;
//   - p2_global: the y/z pass keeps its (nz x My) work plane in shared memory (one CTA per
//     SM, next plane prefetched behind the current one) or in a global scratch slice per
//     CTA that stays in L2 (only the line scratch in shared memory);
//   - p2_lanes: the radix split of the y/z line transforms (M = 16 A points), 16 lanes x A
//     or 8 lanes x 2A (FP32, A in {4, 8, 12});
//   - p1_group: the x pass's block order, pair-major (0) or pairs fastest in groups of G
//     (CTAs in flight share their orbital rows in L2);
//   - chunk_outputs: output orbitals per exchange chunk, 1, 2, 4 or all (small chunks keep
//     a chunk's pair intermediates near L2 size between the passes, large chunks launch
//     fewer, fuller grids).
// The search is coordinate descent from the current knobs: the pass-2 configuration
// (threads x plane staging x line split) first, then the pass-1 order, then the chunking, each
// candidate timed on the exchange apply of synthetic orbitals on the device (one warm-up,
// best of two runs, CUDA events).  The winner is applied to the context and appended to
// a text cache keyed by (edges, precision, nocc, npsi, SMs, device name), so later
// contexts skip the timing.  Only p2_lanes changes the arithmetic (the rounding order of
// the line transforms); under the other knobs the results are bitwise the same.
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
  snprintf(buf, sizeof(buf), "rsx3 %d %d %d %s %d %d %d %s", c->g.nz, c->g.ny, c->g.nx,
           c->precision == RSX_FP32 ? "fp32" : "fp64", nocc, npsi, c->nsm, prop.name);
  for (char* p = buf; *p; ++p)
    if (*p == '\n' || *p == '|') *p = ' ';
  return buf;
}

bool cache_lookup(const char* path, const std::string& key, rsx_tuning* t) {
  if (!path || !*path) return false;
  FILE* f = fopen(path, "r");
  if (!f) return false;
  char line[1024];
  bool found = false;
  while (fgets(line, sizeof(line), f)) {
    const size_t kl = key.size();
    rsx_tuning v;
    if (strncmp(line, key.c_str(), kl) == 0 && line[kl] == '|' &&
        sscanf(line + kl + 1, "%d %d %d %d %d", &v.p2_threads, &v.chunk_outputs, &v.p1_group, &v.p2_global,
               &v.p2_lanes) == 5) {
      *t = v;   // last entry wins
      found = true;
    }
  }
  fclose(f);
  return found;
}

void cache_store(const char* path, const std::string& key, const rsx_tuning& t, double ms) {
  if (!path || !*path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s|%d %d %d %d %d %.4f\n", key.c_str(), t.p2_threads, t.chunk_outputs, t.p1_group, t.p2_global,
          t.p2_lanes, ms);
  fclose(f);
}

bool valid(const rsx_tuning& t) {
  return (t.p2_threads == 256 || t.p2_threads == 384 || t.p2_threads == 512) && t.chunk_outputs >= 0 &&
         t.p1_group >= 0 && (t.p2_global == 0 || t.p2_global == 1) && (t.p2_lanes == 16 || t.p2_lanes == 8);
}

void apply(rsx_ctx* c, const rsx_tuning& t) {
  c->g.p2_threads = t.p2_threads;
  c->g.p1_group = t.p1_group;
  c->g.p2_global = t.p2_global;
  c->g.p2_lanes = t.p2_lanes;
  c->p2_occ[0] = c->p2_occ[1] = 0;
  c->chunk_outputs = t.chunk_outputs;
}

rsx_tuning current(const rsx_ctx* c) {
  rsx_tuning t;
  t.p2_threads = c->g.p2_threads;
  t.chunk_outputs = c->chunk_outputs;
  t.p1_group = c->g.p1_group;
  t.p2_global = c->g.p2_global;
  t.p2_lanes = c->g.p2_lanes;
  return t;
}

// best of two timed exchange applies (after one warm-up) under knobs t
int time_candidate(rsx_ctx* c, const rsx_tuning& t, const void* phi, int nocc, const void* psi, int npsi, void* out,
                   cudaEvent_t e0, cudaEvent_t e1, double* ms_out) {
  apply(c, t);
  int rc = rsx_exchange_apply(c, phi, nocc, psi, npsi, out, nullptr);
  if (rc) return rc;
  double best = 1e30;
  for (int r = 0; r < 2; ++r) {
    cudaEventRecord(e0, 0);
    rc = rsx_exchange_apply(c, phi, nocc, psi, npsi, out, nullptr);
    cudaEventRecord(e1, 0);
    if (rc) return rc;
    if (cudaEventSynchronize(e1) != cudaSuccess) return check_cuda(c, cudaGetLastError(), "autotune timing");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  *ms_out = best;
  return RSX_OK;
}

}  // namespace

extern "C" int rsx_get_tuning(rsx_ctx* c, rsx_tuning* out) {
  if (!c || !out) return RSX_EINVAL;
  *out = current(c);
  return RSX_OK;
}

extern "C" int rsx_set_tuning_ex(rsx_ctx* c, const rsx_tuning* t) {
  if (!c || !t || !valid(*t)) return RSX_EINVAL;
  apply(c, *t);
  return RSX_OK;
}

extern "C" int rsx_set_tuning(rsx_ctx* c, int p2_threads, int chunk_outputs) {
  if (!c) return RSX_EINVAL;
  rsx_tuning t = current(c);
  t.p2_threads = p2_threads;
  t.chunk_outputs = chunk_outputs;
  return rsx_set_tuning_ex(c, &t);
}

extern "C" int rsx_autotune_ex(rsx_ctx* c, int nocc, int npsi, const char* cache_path, rsx_tuning* chosen,
                               double* best_ms) {
  rsx::NvtxRange nvtx_range("rsx_autotune_ex");
  if (!c || nocc < 1 || npsi < 1) return RSX_EINVAL;
  c->err[0] = 0;
  if (cudaSetDevice(c->device) != cudaSuccess) {
    cudaGetLastError();
    return set_error(c, RSX_ECUDA, "cudaSetDevice failed");
  }
  const std::string key = cache_key(c, nocc, npsi);
  rsx_tuning best = current(c);
  double bms = -1.0;
  if (cache_lookup(cache_path, key, &best) && valid(best)) {
    apply(c, best);
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
    const rsx_tuning saved = current(c);
    int rc = time_candidate(c, best, phi, nocc, psi, npsi, out, e0, e1, &bms);
    auto consider = [&](const rsx_tuning& t) {
      if (rc) return;
      double ms = 0.0;
      rc = time_candidate(c, t, phi, nocc, psi, npsi, out, e0, e1, &ms);
      if (!rc && ms < bms) {
        bms = ms;
        best = t;
      }
    };
    // 1. pass-2 configuration: CTA size x plane staging x line split
    const int p2s[3] = {256, 384, 512};
    const bool l8 = c->precision == RSX_FP32 && pass2_l8_active(
        [&] { Geom g8 = c->g; g8.p2_lanes = 8; g8.p2_global = 0; return g8; }(), c->tw8, c->vhatz8);
    for (int a = 0; a < 3; ++a) {
      if (a > 0 && c->precision != RSX_FP32) break;
      for (int gl = 0; gl < 2; ++gl) {
        if (gl == 1 && a > 0) continue;   // the global-plane kernel runs at 256 threads
        for (int ln = 0; ln < 2; ++ln) {
          if (ln == 1 && (!l8 || gl == 1 || a == 2)) continue;   // 8 lanes: shared plane, 256 or 384 threads
          rsx_tuning t = best;
          t.p2_threads = p2s[a];
          t.p2_global = gl;
          t.p2_lanes = ln ? 8 : 16;
          consider(t);
        }
      }
    }
    // 2. pass-1 block order
    const int groups[5] = {0, 4, 16, 64, 1 << 30};
    for (int gi = 0; gi < 5; ++gi) {
      rsx_tuning t = best;
      t.p1_group = groups[gi];
      consider(t);
    }
    // 3. output orbitals per chunk
    const int chs[4] = {1, 2, 4, 0};
    for (int b = 0; b < 4; ++b) {
      if (chs[b] >= npsi) continue;
      rsx_tuning t = best;
      t.chunk_outputs = chs[b];
      consider(t);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(phi);
    cudaFree(psi);
    cudaFree(out);
    if (rc) {
      apply(c, saved);
      return rc;
    }
    apply(c, best);
    cache_store(cache_path, key, best, bms);
  }
  if (chosen) *chosen = current(c);
  if (best_ms) *best_ms = bms;
  return RSX_OK;
}

extern "C" int rsx_autotune(rsx_ctx* c, int nocc, int npsi, const char* cache_path, int* p2_threads,
                            int* chunk_outputs, double* best_ms) {
  rsx_tuning t;
  const int rc = rsx_autotune_ex(c, nocc, npsi, cache_path, &t, best_ms);
  if (rc) return rc;
  if (p2_threads) *p2_threads = t.p2_threads;
  if (chunk_outputs) *chunk_outputs = t.chunk_outputs;
  return RSX_OK;
}
