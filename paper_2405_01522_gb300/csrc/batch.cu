// Uneven batch of independent molecules under one CUDA graph.
//
// For every molecule m (cubic box of edge n_m, N_occ,m orbitals phi_m) the batch computes
//   W_m  = Vx[phi_m] phi_m                 (Eq. 2 with psi = phi: the exchange apply)
//   xi_m = L_m^{-1} W_m, -M_m = L_m L_m^T  (ACE projectors, Eqs. 11-12)
// The molecules are grouped by box edge.  The pair intermediates of a group are
// contiguous, so each of the three FFT passes runs as one launch of the single-problem
// kernel per group over all pairs of all its molecules: a device list gives each pair
// its two orbitals and each output its orbital set, index and first pair (the LIST mode
// of PairMap), so the tuned kernels (pass 1 at 5 CTAs per SM, the prefetching pass 2,
// the double-buffered pass 3) serve the batch unchanged, and a group's launch is as large
// as its pair count.  Then per molecule the ACE Gram M_m = h^3 <phi_m, W_m> and, after one
// FP64 Cholesky kernel over all molecules, xi_m = L_m^{-1} W_m by the dense kernels of the
// single-problem path.  The first run records the whole sequence in a CUDA graph and later
// runs replay it; binding new arrays makes the next run record it again.
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

constexpr int kMaxOccBatch = 32;

struct MolDesc {
  Geom g;
  int nocc, npairs;
  const float* phi;
  float* W;
  float* xi;
  Cx<float>* inter;        // pair intermediates of this molecule
  int q0;                  // its first pair within its size group
};

// one CTA per molecule: M_m (the Gram sums, scaled here by h^3), symmetrised, -M = L L^T,
// L^{-1} (float, [k][k] row-major at linv + 1024 m)
__global__ void __launch_bounds__(256) k_batch_chol(const MolDesc* __restrict__ md, const double* __restrict__ Mm,
                                                    double h3, float* __restrict__ linv, int* status) {
  __shared__ double B[kMaxOccBatch * kMaxOccBatch];
  __shared__ double L[kMaxOccBatch * kMaxOccBatch];
  const int mi = blockIdx.x;
  const int k = md[mi].nocc;
  const double* M = Mm + (size_t)mi * 1024;
  for (int o = threadIdx.x; o < k * k; o += blockDim.x) {
    const int a = o / k, b = o - a * k;
    B[o] = -0.5 * h3 * (M[o] + M[b * k + a]);
  }
  __syncthreads();
  const bool ok = chol_linv_block(B, L, k);
  const float nan = __int_as_float(0x7fc00000);
  for (int o = threadIdx.x; o < k * k; o += blockDim.x) linv[(size_t)mi * 1024 + o] = ok ? (float)B[o] : nan;
  if (threadIdx.x == 0 && !ok && status) atomicMax(status, RSX_ENOTPD);
}

}  // namespace

struct PairGroup {
  int size;          // index into size_ctx
  size_t off;        // byte offset of the group's intermediates
  int npairs, nout;
  std::vector<int> mols;                 // queue positions of the group's molecules
  const float** plist = nullptr;         // device: two orbital pointers per pair
  OutRef<float>* olist = nullptr;        // device: one entry per output orbital
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
  double* part = nullptr;                  // Gram partials (reused molecule by molecule)
  double* Mm = nullptr;                    // per molecule M (Gram sums), [nmol][1024]
  float* linv = nullptr;                   // per molecule L^{-1}, [nmol][1024]
  int* status = nullptr;
  int nsm = 0;
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
  int rc = RSX_OK;
  for (const PairGroup& grp : b->groups) {
    rsx_ctx* c = b->size_ctx[grp.size];
    Cx<float>* inter = reinterpret_cast<Cx<float>*>((char*)b->inter + grp.off);
    PairMap<float> pm;
    pm.mode = kList;
    pm.A = pm.B = nullptr;
    pm.na = pm.nb = 0;
    pm.N = c->g.N();
    pm.plist = grp.plist;
    pm.olist = grp.olist;
    const Cx<float>* twx = (const Cx<float>*)c->tw[2];
    rc = bcuda(b, launch_pass1<float>(c->g, pm, 0, grp.npairs, inter, twx, s), "batch pass 1");
    if (rc) return rc;
    const long long nwork = (long long)grp.npairs * c->g.Hx;
    const int grid = (int)std::min<long long>(nwork, (long long)c->pass2_ctas_per_sm<float>() * c->nsm);
    rc = bcuda(b, launch_pass2<float>(c->g, grp.npairs, inter, (const Cx<float>*)c->tw[1], (const Cx<float>*)c->tw[0],
                                      (const float*)c->vhat, (const float*)c->vhatz, nullptr, grid, s,
                                      (const Cx<float>*)c->tw8, (const float*)c->vhatz8),
               "batch pass 2");
    if (rc) return rc;
    rc = bcuda(b, launch_pass3<float>(c->g, pm, 0, 0, grp.nout, 0, inter, twx, nullptr, s), "batch pass 3");
    if (rc) return rc;
  }
  // ACE: M_m = <phi_m, W_m> per molecule (the partials buffer is reused in stream order)
  const int nblk = 2 * b->nsm;
  for (int qi = 0; qi < b->nmol; ++qi) {
    const MolDesc& d = b->desc[qi];
    rc = bcuda(b, launch_gram<float>(d.phi, d.nocc, d.W, d.nocc, d.g.N(), b->part, nblk, s, nullptr, b->status), "batch gram");
    if (!rc)
      rc = bcuda(b, launch_gram_reduce<float>(b->part, nblk, d.nocc, d.nocc, 1.0, false, b->Mm + (size_t)qi * 1024,
                                              (float*)nullptr, s),
                 "batch gram reduce");
    if (rc) return rc;
  }
  k_batch_chol<<<b->nmol, 256, 0, s>>>(b->d_desc, b->Mm, b->h * b->h * b->h, b->linv, b->status);
  rc = bcuda(b, cudaGetLastError(), "batch cholesky");
  for (int qi = 0; qi < b->nmol && !rc; ++qi) {
    const MolDesc& d = b->desc[qi];
    rc = bcuda(b, launch_combine<float>(b->linv + (size_t)qi * 1024, d.nocc, d.nocc, d.W, d.g.N(), d.xi, 4 * b->nsm, s),
               "batch combine");
  }
  return rc;
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
    // y/z transforms: the 8-lane x 2A split where its tables exist (edges a multiple of 32:
    // every lane busy in both DFT stages, the autotuner's choice at 96^3), else 16 lanes x A
    // at 12 warps where the plane fits (else 256 threads)
    if (c->tw8 != nullptr && c->vhatz8 != nullptr) {
      c->g.p2_lanes = 8;
      c->g.p2_threads = 256;
    } else {
      c->g.p2_threads = 384;
    }
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
  // descriptors (pointers bound later), intermediates
  size_t off_inter = 0;
  b->desc.resize(nmol);
  for (int qi = 0; qi < nmol; ++qi) {
    const int m = b->order[qi];
    MolDesc& d = b->desc[qi];
    const rsx_ctx* c = b->size_ctx[b->size_of_mol[m]];
    d.g = c->g;
    d.nocc = b->nocc[m];
    d.npairs = d.nocc * (d.nocc + 1) / 2;
    d.phi = nullptr;
    d.W = nullptr;
    d.xi = nullptr;
  }
  // intermediates grouped by size: the pairs of all molecules of one edge are contiguous,
  // so that each FFT pass runs as one launch per size over all of them
  for (int si = (int)b->size_ctx.size() - 1; si >= 0; --si) {
    PairGroup grp;
    grp.size = si;
    grp.off = off_inter;
    grp.npairs = grp.nout = 0;
    for (int qi = 0; qi < nmol; ++qi) {
      if (b->size_of_mol[b->order[qi]] != si) continue;
      MolDesc& d = b->desc[qi];
      d.inter = reinterpret_cast<Cx<float>*>(off_inter);  // offset, rebased below
      d.q0 = grp.npairs;
      off_inter += (size_t)d.npairs * d.g.inter_elems() * sizeof(Cx<float>);
      grp.npairs += d.npairs;
      grp.nout += d.nocc;
      grp.mols.push_back(qi);
    }
    if (grp.npairs > 0) b->groups.push_back(grp);
    off_inter = (off_inter + 255) / 256 * 256;
  }
  b->inter_bytes = off_inter;
  cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, device);
  bool ok = cudaMalloc(&b->inter, off_inter) == cudaSuccess &&
            cudaMalloc(&b->d_desc, nmol * sizeof(MolDesc)) == cudaSuccess &&
            cudaMalloc(&b->part, (size_t)2 * b->nsm * 4096 * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&b->Mm, (size_t)nmol * 1024 * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&b->linv, (size_t)nmol * 1024 * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&b->status, sizeof(int)) == cudaSuccess;
  for (PairGroup& grp : b->groups)
    ok = ok && cudaMalloc((void**)&grp.plist, (size_t)2 * grp.npairs * sizeof(float*)) == cudaSuccess &&
         cudaMalloc((void**)&grp.olist, (size_t)grp.nout * sizeof(OutRef<float>)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    rsx_batch_destroy(b);
    return RSX_ENOMEM;
  }
  cudaMemset(b->status, 0, sizeof(int));
  for (auto& d : b->desc) d.inter = reinterpret_cast<Cx<float>*>((char*)b->inter + reinterpret_cast<size_t>(d.inter));
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
  int rc = bcuda(b, cudaMemcpy(b->d_desc, b->desc.data(), b->nmol * sizeof(MolDesc), cudaMemcpyHostToDevice),
                 "descriptor upload");
  // pair and output lists of every size group (SYM pair order within a molecule)
  for (PairGroup& grp : b->groups) {
    if (rc) break;
    std::vector<const float*> pl;
    std::vector<OutRef<float>> ol;
    pl.reserve(2 * (size_t)grp.npairs);
    for (int qi : grp.mols) {
      const MolDesc& d = b->desc[qi];
      const size_t N = d.g.N();
      for (int i = 0; i < d.nocc; ++i) {
        for (int j = i; j < d.nocc; ++j) {
          pl.push_back(d.phi + (size_t)i * N);
          pl.push_back(d.phi + (size_t)j * N);
        }
        OutRef<float> o;
        o.phi = d.phi;
        o.out = d.W + (size_t)i * N;
        o.nocc = d.nocc;
        o.i = i;
        o.q0 = d.q0;
        o.pad = 0;
        ol.push_back(o);
      }
    }
    rc = bcuda(b, cudaMemcpy(grp.plist, pl.data(), pl.size() * sizeof(float*), cudaMemcpyHostToDevice), "pair list");
    if (!rc)
      rc = bcuda(b, cudaMemcpy(grp.olist, ol.data(), ol.size() * sizeof(OutRef<float>), cudaMemcpyHostToDevice),
                 "output list");
  }
  if (rc) return rc;
  // the recorded graph holds the previous arrays' pointers: record again at the next run
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  b->bound = true;
  return RSX_OK;
}

int rsx_batch_run(rsx_batch* b, void* stream) {
  rsx::NvtxRange nvtx_range("rsx_batch_run");
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
  void* bufs[] = {b->inter, b->d_desc, b->part, b->Mm, b->linv, b->status};
  for (void* p : bufs)
    if (p) cudaFree(p);
  for (PairGroup& grp : b->groups) {
    if (grp.plist) cudaFree((void*)grp.plist);
    if (grp.olist) cudaFree(grp.olist);
  }
  for (rsx_ctx* c : b->size_ctx) rsx_destroy(c);
  delete b;
  return RSX_OK;
}

}  // extern "C"
