// Uneven batch of independent molecules in persistent launches under one CUDA graph.
//
// For every molecule m (cubic box of edge n_m, N_occ,m orbitals phi_m) the batch computes
//   W_m  = Vx[phi_m] phi_m                 (Eq. 2 with psi = phi: the exchange apply)
//   xi_m = L_m^{-1} W_m, -M_m = L_m L_m^T  (ACE projectors, Eqs. 11-12)
// The x passes of all molecules run as two persistent kernels whose CTAs pull work items
// (molecule, pair or output, plane, row block) from a device queue (an atomic counter)
// in descending molecule work and dispatch on the molecule's transform length.  The
// pair intermediates are laid out grouped by edge, so the y/z pass runs as one
// prefetching launch of the single-problem kernel per distinct edge (all pairs of all
// molecules of that edge share the kernel table and twiddles).  The ACE steps are three
// batched kernels.  The first run records
// the whole sequence in a CUDA graph; later runs replay it.  Descriptors live on the
// device, so rebinding arrays does not invalidate the graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <cmath>
#include <numeric>
#include <vector>

#include "../../include/rsx.h"
#include "api_internal.cuh"
#include "dense.cuh"
#include "poisson_kernels.cuh"

using namespace rsx;

namespace {

constexpr int kBatchBlocksPerMol = 8;    // CTAs per molecule in the batched ACE kernels
constexpr int kGramChunkB = 128;
constexpr int kMaxOccBatch = 32;

struct MolDesc {
  Geom g;
  int nocc, npairs;
  const float* phi;
  float* W;
  float* xi;
  Cx<float>* inter;        // pair intermediates of this molecule
  const Cx<float>* tw;     // twiddles (all three axes have the same length)
  const float* vhat;       // kernel table for this edge and spacing
  long long off[3];        // first item of this molecule in the pass-1/2/3 queues
  long long cnt[3];        // items of this molecule per pass
};

__device__ __forceinline__ int find_mol(const MolDesc* md, int nmol, int pass, long long item) {
  int lo = 0, hi = nmol - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (md[mid].off[pass] <= item)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ long long next_item(unsigned long long* ctr, long long* sh) {
  __syncthreads();
  if (threadIdx.x == 0) *sh = (long long)atomicAdd(ctr, 1ull);
  __syncthreads();
  return *sh;
}

template <int A>
__device__ __noinline__ void batch_p1(const MolDesc& m, long long local, unsigned char* smem) {
  const int nyb = (m.g.ny + kRowsPerCta - 1) / kRowsPerCta;
  const int yblk = (int)(local % nyb);
  long long r = local / nyb;
  const int z = (int)(r % m.g.nz);
  const int q = (int)(r / m.g.nz);
  PairMap<float> pm;
  pm.mode = kSym;
  pm.A = m.phi;
  pm.B = nullptr;
  pm.na = m.nocc;
  pm.nb = 0;
  pm.N = m.g.N();
  const float* f1;
  const float* f2;
  pm.pair(q, f1, f2);
  pass1_item<float, A>(m.g, f1, f2, z, yblk, m.inter + (size_t)q * m.g.inter_elems(), m.tw, smem);
}

__global__ void __launch_bounds__(kThreads, 2) k_batch_pass1(const MolDesc* __restrict__ md, int nmol, long long total,
                                                          unsigned long long* ctr) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ long long item_sh;
  for (long long it = next_item(ctr, &item_sh); it < total; it = next_item(ctr, &item_sh)) {
    const int mi = find_mol(md, nmol, 0, it);
    const MolDesc& m = md[mi];
    const long long local = it - m.off[0];
    switch (m.g.Ax) {
      case 6: batch_p1<6>(m, local, smem_raw); break;
      case 8: batch_p1<8>(m, local, smem_raw); break;
      case 10: batch_p1<10>(m, local, smem_raw); break;
      case 12: batch_p1<12>(m, local, smem_raw); break;
      case 14: batch_p1<14>(m, local, smem_raw); break;
      default: break;
    }
  }
}

template <int A>
__device__ __noinline__ void batch_p3(const MolDesc& m, long long local, unsigned char* smem) {
  const int nyb = (m.g.ny + kRowsPerCta - 1) / kRowsPerCta;
  const int yblk = (int)(local % nyb);
  long long r = local / nyb;
  const int z = (int)(r % m.g.nz);
  const int p = (int)(r / m.g.nz);
  PairMap<float> pm;
  pm.mode = kSym;
  pm.A = m.phi;
  pm.B = nullptr;
  pm.na = m.nocc;
  pm.nb = 0;
  pm.N = m.g.N();
  pass3_item<float, A>(m.g, pm, 0, p, z, yblk, 0, m.inter, m.tw, m.W + (size_t)p * m.g.N(), smem);
}

__global__ void __launch_bounds__(kThreads, 2) k_batch_pass3(const MolDesc* __restrict__ md, int nmol, long long total,
                                                          unsigned long long* ctr) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ long long item_sh;
  for (long long it = next_item(ctr, &item_sh); it < total; it = next_item(ctr, &item_sh)) {
    const int mi = find_mol(md, nmol, 2, it);
    const MolDesc& m = md[mi];
    const long long local = it - m.off[2];
    switch (m.g.Ax) {
      case 6: batch_p3<6>(m, local, smem_raw); break;
      case 8: batch_p3<8>(m, local, smem_raw); break;
      case 10: batch_p3<10>(m, local, smem_raw); break;
      case 12: batch_p3<12>(m, local, smem_raw); break;
      case 14: batch_p3<14>(m, local, smem_raw); break;
      default: break;
    }
  }
}

// part[m][b][k][l] = partial sums of phi_k W_l over this block's chunks of molecule m
__global__ void __launch_bounds__(256) k_batch_gram(const MolDesc* __restrict__ md, double* __restrict__ part) {
  __shared__ float xs[kMaxOccBatch][kGramChunkB + 1];
  __shared__ float ys[kMaxOccBatch][kGramChunkB + 1];
  const int mi = blockIdx.x / kBatchBlocksPerMol, sub = blockIdx.x % kBatchBlocksPerMol;
  const MolDesc& m = md[mi];
  const int k = m.nocc;
  const size_t N = m.g.N();
  const int nout = k * k;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  const size_t nchunk = (N + kGramChunkB - 1) / kGramChunkB;
  for (size_t c = sub; c < nchunk; c += kBatchBlocksPerMol) {
    const size_t r0 = c * kGramChunkB;
    const int len = (int)min((size_t)kGramChunkB, N - r0);
    __syncthreads();
    for (int i = threadIdx.x; i < k * kGramChunkB; i += 256) {
      const int a = i / kGramChunkB, j = i - a * kGramChunkB;
      xs[a][j] = j < len ? m.phi[(size_t)a * N + r0 + j] : 0.f;
      ys[a][j] = j < len ? m.W[(size_t)a * N + r0 + j] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int o = threadIdx.x + q * 256;
      if (o < nout) {
        const int a = o / k, b = o - a * k;
        float s = 0.f;
        for (int j = 0; j < kGramChunkB; ++j) s += xs[a][j] * ys[b][j];
        acc[q] += (double)s;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int o = threadIdx.x + q * 256;
    if (o < nout) part[((size_t)mi * kBatchBlocksPerMol + sub) * 1024 + o] = acc[q];
  }
}

// one CTA per molecule: M = h^3 sum of partials, symmetrise, -M = L L^T, L^{-1} (float)
__global__ void __launch_bounds__(256) k_batch_chol(const MolDesc* __restrict__ md, const double* __restrict__ part,
                                                    double h3, float* __restrict__ linv, int* status) {
  __shared__ double B[kMaxOccBatch * kMaxOccBatch];
  __shared__ double L[kMaxOccBatch * kMaxOccBatch];
  const int mi = blockIdx.x;
  const int k = md[mi].nocc;
  for (int o = threadIdx.x; o < k * k; o += blockDim.x) {
    const int a = o / k, b = o - a * k;
    double s = 0.0, st = 0.0;
    for (int j = 0; j < kBatchBlocksPerMol; ++j) {
      s += part[((size_t)mi * kBatchBlocksPerMol + j) * 1024 + o];
      st += part[((size_t)mi * kBatchBlocksPerMol + j) * 1024 + b * k + a];
    }
    B[o] = -0.5 * h3 * (s + st);
  }
  __syncthreads();
  const bool ok = chol_linv_block(B, L, k);
  const float nan = __int_as_float(0x7fc00000);
  for (int o = threadIdx.x; o < k * k; o += blockDim.x) linv[(size_t)mi * 1024 + o] = ok ? (float)B[o] : nan;
  if (threadIdx.x == 0 && !ok && status) atomicMax(status, RSX_ENOTPD);
}

// xi_m = L_m^{-1} W_m, one point per thread
__global__ void __launch_bounds__(256) k_batch_combine(const MolDesc* __restrict__ md,
                                                       const float* __restrict__ linv) {
  __shared__ float cs[kMaxOccBatch * kMaxOccBatch];
  const int mi = blockIdx.x / kBatchBlocksPerMol, sub = blockIdx.x % kBatchBlocksPerMol;
  const MolDesc& m = md[mi];
  const int k = m.nocc;
  const size_t N = m.g.N();
  for (int o = threadIdx.x; o < k * k; o += blockDim.x) cs[o] = linv[(size_t)mi * 1024 + o];
  __syncthreads();
  for (size_t r = (size_t)sub * 256 + threadIdx.x; r < N; r += (size_t)kBatchBlocksPerMol * 256) {
    float w[kMaxOccBatch];
    for (int i = 0; i < k; ++i) w[i] = m.W[(size_t)i * N + r];
    for (int o = 0; o < k; ++o) {
      float s = 0.f;
      for (int i = 0; i <= o; ++i) s += cs[o * k + i] * w[i];
      m.xi[(size_t)o * N + r] = s;
    }
  }
}

}  // namespace

struct PairGroup {
  int size;          // index into size_ctx
  size_t off;        // byte offset of the group's intermediates
  int npairs;
};

struct rsx_batch {
  int device = 0;
  int nmol = 0;
  double h = 0.0;
  std::vector<int> edge, nocc, order;      // order: molecules sorted by decreasing work
  std::vector<rsx_ctx*> size_ctx;          // one FP32 context per distinct edge (tables)
  std::vector<int> size_of_mol;            // index into size_ctx
  std::vector<MolDesc> desc;               // host copy, in queue order
  std::vector<PairGroup> groups;           // contiguous pair intermediates per size
  MolDesc* d_desc = nullptr;
  void* inter = nullptr;
  size_t inter_bytes = 0;
  double* part = nullptr;
  float* linv = nullptr;
  unsigned long long* ctr = nullptr;
  int* status = nullptr;
  long long total[3] = {0, 0, 0};
  size_t smem[3] = {0, 0, 0};
  int grid[3] = {0, 0, 0};
  bool bound = false;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  char err[512] = {0};
};

namespace {

int bfail(rsx_batch* b, int code, const char* msg) {
  snprintf(b->err, sizeof(b->err), "%s", msg);
  return code;
}

int bcuda(rsx_batch* b, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return RSX_OK;
  snprintf(b->err, sizeof(b->err), "%s: %s", what, cudaGetErrorString(e));
  return RSX_ECUDA;
}

int record(rsx_batch* b, cudaStream_t s) {
  int rc = bcuda(b, cudaMemsetAsync(b->ctr, 0, 3 * sizeof(unsigned long long), s), "queue reset");
  if (rc) return rc;
  k_batch_pass1<<<b->grid[0], kThreads, b->smem[0], s>>>(b->d_desc, b->nmol, b->total[0], b->ctr + 0);
  for (const PairGroup& grp : b->groups) {
    rsx_ctx* c = b->size_ctx[grp.size];
    Cx<float>* inter = reinterpret_cast<Cx<float>*>((char*)b->inter + grp.off);
    const long long nwork = (long long)grp.npairs * c->g.Hx;
    const int grid = (int)std::min<long long>(nwork, (long long)c->pass2_ctas_per_sm<float>() * c->nsm);
    rc = bcuda(b, launch_pass2<float>(c->g, grp.npairs, inter, (const Cx<float>*)c->tw[1], (const Cx<float>*)c->tw[0],
                                      (const float*)c->vhat, (const float*)c->vhatz, nullptr, grid, s),
               "batch pass 2");
    if (rc) return rc;
  }
  k_batch_pass3<<<b->grid[2], kThreads, b->smem[2], s>>>(b->d_desc, b->nmol, b->total[2], b->ctr + 2);
  k_batch_gram<<<b->nmol * kBatchBlocksPerMol, 256, 0, s>>>(b->d_desc, b->part);
  k_batch_chol<<<b->nmol, 256, 0, s>>>(b->d_desc, b->part, b->h * b->h * b->h, b->linv, b->status);
  k_batch_combine<<<b->nmol * kBatchBlocksPerMol, 256, 0, s>>>(b->d_desc, b->linv);
  return bcuda(b, cudaGetLastError(), "batch launches");
}

}  // namespace

extern "C" {

int rsx_batch_create(rsx_batch** out, int nmol, const int* edges, const int* nocc, double h, int device) {
  if (!out) return RSX_EINVAL;
  *out = nullptr;
  if (nmol < 1 || !edges || !nocc || !(h > 0.0)) return RSX_EINVAL;
  for (int m = 0; m < nmol; ++m) {
    const int e = edges[m];
    if (e % 8 || (e / 8 != 6 && e / 8 != 8 && e / 8 != 10 && e / 8 != 12 && e / 8 != 14)) return RSX_EUNSUPPORTED;
    if (nocc[m] < 1 || nocc[m] > kMaxOccBatch) return RSX_EINVAL;
  }
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return RSX_ECUDA;
  }
  rsx_batch* b = new rsx_batch();
  b->device = device;
  b->nmol = nmol;
  b->h = h;
  b->edge.assign(edges, edges + nmol);
  b->nocc.assign(nocc, nocc + nmol);
  // distinct sizes -> one context each (kernel table and twiddles)
  std::vector<int> sizes(b->edge);
  std::sort(sizes.begin(), sizes.end());
  sizes.erase(std::unique(sizes.begin(), sizes.end()), sizes.end());
  for (int e : sizes) {
    rsx_ctx* c = nullptr;
    const int rc = rsx_create(&c, e, e, e, h, RSX_FP32, device);
    if (rc) {
      rsx_batch_destroy(b);
      return rc;
    }
    c->g.p2_threads = 384;   // 12 warps where the plane fits (else 256)
    b->size_ctx.push_back(c);
  }
  b->size_of_mol.resize(nmol);
  for (int m = 0; m < nmol; ++m)
    b->size_of_mol[m] = (int)(std::lower_bound(sizes.begin(), sizes.end(), b->edge[m]) - sizes.begin());
  // queue order: decreasing pair-solve work (largest first balances the tail)
  b->order.resize(nmol);
  std::iota(b->order.begin(), b->order.end(), 0);
  auto work = [&](int m) { return (double)b->nocc[m] * (b->nocc[m] + 1) / 2 * std::pow((double)b->edge[m], 3.0); };
  std::stable_sort(b->order.begin(), b->order.end(), [&](int x, int y) { return work(x) > work(y); });
  // descriptors (pointers bound later), item counts, intermediates
  size_t off_inter = 0;
  b->desc.resize(nmol);
  for (int qi = 0; qi < nmol; ++qi) {
    const int m = b->order[qi];
    MolDesc& d = b->desc[qi];
    const rsx_ctx* c = b->size_ctx[b->size_of_mol[m]];
    d.g = c->g;
    d.nocc = b->nocc[m];
    d.npairs = d.nocc * (d.nocc + 1) / 2;
    d.tw = (const Cx<float>*)c->tw[2];
    d.vhat = (const float*)c->vhat;
    const int nyb = (d.g.ny + kRowsPerCta - 1) / kRowsPerCta;
    d.cnt[0] = (long long)d.npairs * d.g.nz * nyb;
    d.cnt[1] = (long long)d.npairs * d.g.Hx;
    d.cnt[2] = (long long)d.nocc * d.g.nz * nyb;
    for (int p = 0; p < 3; ++p) {
      d.off[p] = b->total[p];
      b->total[p] += d.cnt[p];
    }
    d.phi = nullptr;
    d.W = nullptr;
    d.xi = nullptr;
  }
  // intermediates grouped by size: the pairs of all molecules of one edge are contiguous,
  // so that the y/z pass runs as one tuned, prefetching launch per size
  for (int si = (int)b->size_ctx.size() - 1; si >= 0; --si) {
    PairGroup grp;
    grp.size = si;
    grp.off = off_inter;
    grp.npairs = 0;
    for (int qi = 0; qi < nmol; ++qi) {
      if (b->size_of_mol[b->order[qi]] != si) continue;
      MolDesc& d = b->desc[qi];
      d.inter = reinterpret_cast<Cx<float>*>(off_inter);  // offset, rebased below
      off_inter += (size_t)d.npairs * d.g.inter_elems() * sizeof(Cx<float>);
      grp.npairs += d.npairs;
    }
    if (grp.npairs > 0) b->groups.push_back(grp);
    off_inter = (off_inter + 255) / 256 * 256;
  }
  b->inter_bytes = off_inter;
  if (cudaMalloc(&b->inter, off_inter) != cudaSuccess || cudaMalloc(&b->d_desc, nmol * sizeof(MolDesc)) != cudaSuccess ||
      cudaMalloc(&b->part, (size_t)nmol * kBatchBlocksPerMol * 1024 * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&b->linv, (size_t)nmol * 1024 * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&b->ctr, 3 * sizeof(unsigned long long)) != cudaSuccess ||
      cudaMalloc(&b->status, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    rsx_batch_destroy(b);
    return RSX_ENOMEM;
  }
  cudaMemset(b->status, 0, sizeof(int));
  for (auto& d : b->desc) d.inter = reinterpret_cast<Cx<float>*>((char*)b->inter + reinterpret_cast<size_t>(d.inter));
  // launch shapes: dynamic shared memory of the largest size class, persistent grids
  int maxA = 0, nmaxx = 0;
  for (auto& d : b->desc) {
    maxA = std::max(maxA, d.g.Ax);
    nmaxx = std::max(nmaxx, d.g.nx);
  }
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
  const int L = 16 * maxA, H = L / 2 + 1;
  b->smem[0] = sizeof(Cx<float>) * std::max((size_t)kLinesPerCta * maxA * kScrPitch, (size_t)H * kRowsPerCta);
  b->smem[2] = sizeof(Cx<float>) * (size_t)kLinesPerCta * maxA * kScrPitch + 2 * pass3_buffer_elems<float>(maxA, nmaxx);
  const void* kern[3] = {(const void*)k_batch_pass1, nullptr, (const void*)k_batch_pass3};
  for (int p = 0; p < 3; p += 2) {
    if (cudaFuncSetAttribute(kern[p], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem[p]) != cudaSuccess) {
      cudaGetLastError();
      rsx_batch_destroy(b);
      return RSX_EUNSUPPORTED;
    }
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern[p], kThreads, b->smem[p]);
    b->grid[p] = std::max(1, per_sm) * nsm;
  }
  *out = b;
  return RSX_OK;
}

int rsx_batch_bind(rsx_batch* b, const void* const* phi, void* const* W, void* const* xi) {
  if (!b || !phi || !W || !xi) return RSX_EINVAL;
  for (int qi = 0; qi < b->nmol; ++qi) {
    const int m = b->order[qi];
    if (!phi[m] || !W[m] || !xi[m]) return bfail(b, RSX_EINVAL, "batch bind: null pointer");
    b->desc[qi].phi = (const float*)phi[m];
    b->desc[qi].W = (float*)W[m];
    b->desc[qi].xi = (float*)xi[m];
  }
  if (cudaSetDevice(b->device) != cudaSuccess) return bcuda(b, cudaGetLastError(), "cudaSetDevice");
  const int rc = bcuda(b, cudaMemcpy(b->d_desc, b->desc.data(), b->nmol * sizeof(MolDesc), cudaMemcpyHostToDevice),
                       "descriptor upload");
  if (rc) return rc;
  b->bound = true;
  return RSX_OK;
}

int rsx_batch_run(rsx_batch* b, void* stream) {
  if (!b) return RSX_EINVAL;
  if (!b->bound) return bfail(b, RSX_EINVAL, "batch run: bind the molecule arrays first");
  if (cudaSetDevice(b->device) != cudaSuccess) return bcuda(b, cudaGetLastError(), "cudaSetDevice");
  cudaStream_t s = (cudaStream_t)stream;
  if (!b->exec) {
    cudaStream_t cap = nullptr;
    int rc = bcuda(b, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "capture stream");
    if (rc) return rc;
    rc = bcuda(b, cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal), "begin capture");
    if (!rc) {
      const int rrc = record(b, cap);
      cudaGraph_t g = nullptr;
      const cudaError_t ec = cudaStreamEndCapture(cap, &g);
      rc = rrc ? rrc : bcuda(b, ec, "end capture");
      if (!rc) {
        b->graph = g;
        rc = bcuda(b, cudaGraphInstantiate(&b->exec, g, 0), "graph instantiate");
      }
    }
    cudaStreamDestroy(cap);
    if (rc) return rc;
  }
  return bcuda(b, cudaGraphLaunch(b->exec, s), "graph launch");
}

int rsx_batch_sync_status(rsx_batch* b, void* stream) {
  if (!b) return RSX_EINVAL;
  cudaSetDevice(b->device);
  int rc = bcuda(b, cudaStreamSynchronize((cudaStream_t)stream), "stream synchronise");
  if (rc) return rc;
  int st = 0;
  rc = bcuda(b, cudaMemcpy(&st, b->status, sizeof(int), cudaMemcpyDeviceToHost), "status read");
  if (rc) return rc;
  cudaMemset(b->status, 0, sizeof(int));
  if (st) return bfail(b, st, st == RSX_ENOTPD ? "ACE: -M not positive definite" : "deferred device error");
  return RSX_OK;
}

const char* rsx_batch_last_error(const rsx_batch* b) { return b ? b->err : "null batch"; }

int rsx_batch_destroy(rsx_batch* b) {
  if (!b) return RSX_OK;
  cudaSetDevice(b->device);
  cudaDeviceSynchronize();
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  void* bufs[] = {b->inter, b->d_desc, b->part, b->linv, b->ctr, b->status};
  for (void* p : bufs)
    if (p) cudaFree(p);
  for (rsx_ctx* c : b->size_ctx) rsx_destroy(c);
  delete b;
  return RSX_OK;
}

}  // extern "C"
