// C ABI of librsx (include/rsx.h): context, workspace and the host side of each call.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "../../include/rsx.h"
#include "api_internal.cuh"
#include "dense.cuh"

using namespace rsx;

namespace {

int fail(rsx_ctx* c, int code, const char* fmt, ...) {
  if (c) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(c->err, sizeof(c->err), fmt, ap);
    va_end(ap);
  }
  return code;
}

}  // namespace

namespace rsx {

int check_cuda(rsx_ctx* c, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return RSX_OK;
  return fail(c, RSX_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

int grow(rsx_ctx* c, void** p, size_t* have, size_t need, const char* what) {
  if (need <= *have) return RSX_OK;
  if (c && c->fault_alloc_after >= 0) {   // injected failure: nothing is allocated or freed
    if (c->fault_alloc_after == 0) {
      c->fault_alloc_after = -1;
      return fail(c, RSX_ENOMEM, "injected allocation failure (%zu bytes for %s)", need, what);
    }
    --c->fault_alloc_after;
  }
  if (*p) cudaFree(*p);
  *p = nullptr;
  *have = 0;
  if (cudaMalloc(p, need) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(c, RSX_ENOMEM, "cannot allocate %zu bytes for %s", need, what);
  }
  *have = need;
  return RSX_OK;
}

int set_error(rsx_ctx* c, int code, const char* msg) { return fail(c, code, "%s", msg); }

const char* kernel_name(int id) {
  static const char* names[kKCount] = {"pass1_x_forward", "pass2_yz_kernel", "pass3_x_inverse_accumulate",
                                       "spectrum_panel", "gram", "gram_reduce", "cholesky_linv", "combine",
                                       "pair_products", "k_gemm_tcgen05", "gemm_reduce", "tda_eigensolve",
                                       "kd_contract"};
  return (id >= 0 && id < kKCount) ? names[id] : "";
}

static cudaEvent_t prof_event(rsx_ctx* c) {
  if (!c->prof_pool.empty()) {
    cudaEvent_t e = c->prof_pool.back();
    c->prof_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

ProfScope::ProfScope(rsx_ctx* c_, int id_, cudaStream_t s_) : c(c_), id(id_), s(s_) {
  if (c && c->prof_on) {
    a = prof_event(c);
    b = prof_event(c);
    cudaEventRecord(a, s);
  }
}

ProfScope::~ProfScope() {
  if (a) {
    cudaEventRecord(b, s);
    c->prof_pending.push_back({id, a, b});
  }
}

static void prof_collect(rsx_ctx* c) {
  for (auto& r : c->prof_pending) {
    cudaEventSynchronize(r.b);
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      c->prof_ms[r.id] += ms;
      c->prof_n[r.id] += 1;
    }
    cudaGetLastError();
    c->prof_pool.push_back(r.a);
    c->prof_pool.push_back(r.b);
  }
  c->prof_pending.clear();
}

}  // namespace rsx

namespace {

bool edge_ok(int n) { return n >= 16 && n % 8 == 0 && axis_supported(n / 8); }

template <typename R>
int make_tables(rsx_ctx* c) {
  const Geom& g = c->g;
  // twiddles tw[t][k1] = exp(-2 pi i t k1 / M), t < 16, k1 < A, per axis (z, y, x)
  const int Ms[3] = {g.Mz, g.My, g.Mx};
  const int As[3] = {g.Az, g.Ay, g.Ax};
  for (int ax = 0; ax < 3; ++ax) {
    std::vector<Cx<R>> tw(16 * As[ax]);
    for (int t = 0; t < 16; ++t)
      for (int k1 = 0; k1 < As[ax]; ++k1) {
        const long long e = (long long)t * k1 % Ms[ax];
        const double ang = 2.0 * M_PI * (double)e / (double)Ms[ax];
        tw[t * As[ax] + k1].x = (R)cos(ang);
        tw[t * As[ax] + k1].y = (R)(-sin(ang));
      }
    size_t have = 0;
    int rc = grow(c, &c->tw[ax], &have, tw.size() * sizeof(Cx<R>), "twiddles");
    if (rc) return rc;
    rc = check_cuda(c, cudaMemcpy(c->tw[ax], tw.data(), tw.size() * sizeof(Cx<R>), cudaMemcpyHostToDevice),
                    "twiddle upload");
    if (rc) return rc;
  }
  // kernel spectrum table
  const int hz = g.Mz / 2 + 1, hy = g.My / 2 + 1, hx = g.Mx / 2 + 1;
  const size_t nt = (size_t)hz * hy * hx;
  std::vector<double> cosv;
  double* dcos[3] = {nullptr, nullptr, nullptr};
  for (int ax = 0; ax < 3; ++ax) {
    cosv.resize(Ms[ax]);
    for (int j = 0; j < Ms[ax]; ++j) cosv[j] = cos(2.0 * M_PI * (double)j / (double)Ms[ax]);
    if (cudaMalloc(&dcos[ax], Ms[ax] * sizeof(double)) != cudaSuccess) return fail(c, RSX_ENOMEM, "cos table");
    cudaMemcpy(dcos[ax], cosv.data(), Ms[ax] * sizeof(double), cudaMemcpyHostToDevice);
  }
  double *b0 = nullptr, *b1 = nullptr;
  if (cudaMalloc(&b0, nt * sizeof(double)) != cudaSuccess || cudaMalloc(&b1, nt * sizeof(double)) != cudaSuccess)
    return fail(c, RSX_ENOMEM, "kernel table scratch");
  size_t have = 0;
  int rc = grow(c, &c->vhat, &have, nt * sizeof(R), "kernel table");
  if (rc) return rc;
  const double npad = (double)g.Mz * g.My * g.Mx;
  const double scale = c->h * c->h * c->h / npad;
  cudaError_t e = launch_ghat(g, c->h, scale, dcos[0], dcos[1], dcos[2], b0, b1, c->vhat, sizeof(R) == 8, 0);
  if (e == cudaSuccess && sizeof(R) == 4) {
    size_t hz_have = 0;
    if (grow(c, &c->vhatz, &hz_have, (size_t)hx * hy * g.Mz * sizeof(float), "kernel table (lane order)") != RSX_OK)
      e = cudaErrorMemoryAllocation;
    else
      e = launch_vhat_lanes(g, (const float*)c->vhat, (float*)c->vhatz, 0);
  }
  if (e == cudaSuccess && sizeof(R) == 4 && g.Ay == g.Az && g.Ay % 4 == 0) {
    // the 8-lane y/z kernel: its lane-order table and twiddles w_M^{-t k1}, t < 8, k1 < 2 A
    size_t have8 = 0, have_tw = 0;
    const int A2 = 2 * g.Az;
    std::vector<Cx<float>> tw8(8 * A2);
    for (int t = 0; t < 8; ++t)
      for (int k1 = 0; k1 < A2; ++k1) {
        const long long ex = (long long)t * k1 % g.Mz;
        const double ang = 2.0 * M_PI * (double)ex / (double)g.Mz;
        tw8[t * A2 + k1].x = (float)cos(ang);
        tw8[t * A2 + k1].y = (float)(-sin(ang));
      }
    if (grow(c, &c->vhatz8, &have8, (size_t)hx * hy * g.Mz * sizeof(float), "kernel table (8-lane order)") != RSX_OK ||
        grow(c, &c->tw8, &have_tw, tw8.size() * sizeof(Cx<float>), "8-lane twiddles") != RSX_OK)
      e = cudaErrorMemoryAllocation;
    else
      e = cudaMemcpy(c->tw8, tw8.data(), tw8.size() * sizeof(Cx<float>), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_vhat_lanes8(g, (const float*)c->vhat, (float*)c->vhatz8, 0);
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  cudaFree(b0);
  cudaFree(b1);
  for (int ax = 0; ax < 3; ++ax) cudaFree(dcos[ax]);
  return check_cuda(c, e, "kernel table");
}

template <typename R>
PairMap<R> pair_map(int mode, const void* A, const void* B, int na, int nb, size_t N) {
  PairMap<R> pm;
  pm.mode = mode;
  pm.A = (const R*)A;
  pm.B = (const R*)B;
  pm.na = na;
  pm.nb = nb;
  pm.N = N;
  return pm;
}

bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
  const char* pa = (const char*)a;
  const char* pb = (const char*)b;
  return pa < pb + nb && pb < pa + na;
}

}  // namespace

namespace rsx {

// Pair solves for pairs [q0, q0 + nq) of pm, accumulated into outputs [p0, p0 + np).
// Requires the intermediate workspace to hold nq pairs (grown here).
template <typename R>
int solve_pairs(rsx_ctx* c, const PairMap<R>& pm, int q0, int nq, int p0, int np, R* out, cudaStream_t s,
                int pot) {
  Geom g = c->g;
  g.dbg_nq = nq;   // pairs of this launch's intermediate (read by bounds-checked builds)
  const size_t need = (size_t)nq * g.inter_elems() * sizeof(Cx<R>);
  int rc = grow(c, &c->work, &c->work_bytes, need, "FFT intermediates");
  if (rc) return rc;
  Cx<R>* inter = (Cx<R>*)c->work;
  const Cx<R>* twz = (const Cx<R>*)c->tw[0];
  const Cx<R>* twy = (const Cx<R>*)c->tw[1];
  const Cx<R>* twx = (const Cx<R>*)c->tw[2];
  {
    ProfScope ps(c, kKPass1, s);
    rc = check_cuda(c, launch_pass1<R>(g, pm, q0, nq, inter, twx, s), "pass 1");
  }
  if (rc) return rc;
  bool fits = false;
  pass2_smem_bytes<R>(g, &fits);
  const long long nwork = (long long)nq * g.Hx;
  int grid;
  R* gscr = nullptr;
  if (fits) {
    const int per_sm = c->pass2_ctas_per_sm<R>();
    grid = (int)std::min<long long>(nwork, (long long)per_sm * c->nsm);
  } else {
    grid = (int)std::min<long long>(nwork, 2LL * c->nsm);
    const size_t gneed = (size_t)grid * g.nz * (g.My + 1) * sizeof(Cx<R>);
    rc = grow(c, &c->gscr, &c->gscr_bytes, gneed, "pass-2 plane scratch");
    if (rc) return rc;
    gscr = (R*)c->gscr;
  }
  {
    ProfScope ps(c, kKPass2, s);
    rc = check_cuda(c, launch_pass2<R>(g, nq, inter, twy, twz, (const R*)c->vhat, (const float*)c->vhatz, gscr, grid, s,
                                       (const Cx<float>*)c->tw8, (const float*)c->vhatz8),
                    "pass 2");
  }
  if (rc) return rc;
  if (out != nullptr) {
    ProfScope ps(c, kKPass3, s);
    rc = check_cuda(c, launch_pass3<R>(g, pm, q0, p0, np, pot, inter, twx, out, s), "pass 3");
  }
  return rc;
}

template <typename R>
int exchange_apply(rsx_ctx* c, const void* phi, int nocc, const void* psi, int npsi, void* out, cudaStream_t s) {
  const Geom& g = c->g;
  const size_t N = g.N();
  const PairMap<R> pm = pair_map<R>(kProd, phi, psi, nocc, npsi, N);
  const size_t per_pair = g.inter_elems() * sizeof(Cx<R>);
  // outputs per chunk: all of p's nocc pairs must be resident for pass 3
  long long pmax = (long long)(c->work_limit / ((size_t)nocc * per_pair));
  if (pmax < 1) return set_error(c, RSX_ENOMEM, "workspace limit below one output orbital's pairs");
  if (c->chunk_outputs > 0 && c->chunk_outputs < pmax) pmax = c->chunk_outputs;
  for (int p0 = 0; p0 < npsi; p0 += (int)pmax) {
    const int np = (int)std::min<long long>(pmax, npsi - p0);
    int rc = solve_pairs<R>(c, pm, p0 * nocc, np * nocc, p0, np, (R*)out + (size_t)p0 * N, s);
    if (rc) return rc;
  }
  return RSX_OK;
}

template <typename R>
int ace_build(rsx_ctx* c, const void* phi, int nocc, void* xi, double* M_out, cudaStream_t s) {
  const Geom& g = c->g;
  const size_t N = g.N();
  const PairMap<R> pm = pair_map<R>(kSym, phi, nullptr, nocc, 0, N);
  const int npairs = nocc * (nocc + 1) / 2;
  if ((size_t)npairs * g.inter_elems() * sizeof(Cx<R>) > c->work_limit)
    return set_error(c, RSX_ENOMEM, "ACE build needs all nocc(nocc+1)/2 pairs resident; raise the workspace limit");
  // W = Vx[phi] phi, written into xi
  int rc = solve_pairs<R>(c, pm, 0, npairs, 0, nocc, (R*)xi, s);
  if (rc) return rc;
  // M = h^3 <phi, W>
  const int nblk = 2 * c->nsm;
  rc = grow(c, (void**)&c->dsm, &c->dsm_bytes, sizeof(double) * ((size_t)nblk * 4096 + 3 * 4096), "small FP64");
  if (rc) return rc;
  double* part = c->dsm;
  double* M = c->dsm + (size_t)nblk * 4096;
  double* Linv = M + 4096;
  rc = grow(c, &c->smallr, &c->smallr_bytes, sizeof(R) * 4096 * 2, "small coefficients");
  if (rc) return rc;
  R* linv_r = (R*)c->smallr;
  const double h3 = c->h * c->h * c->h;
  {
    ProfScope ps(c, kKGram, s);
    rc = check_cuda(c, launch_gram<R>((const R*)phi, nocc, (const R*)xi, nocc, N, part, nblk, s, nullptr, c->status), "gram");
  }
  if (rc) return rc;
  {
    // an injected bad pivot flips M's sign, so that -M is negative definite
    const double msc = c->fault_pivot ? -h3 : h3;
    c->fault_pivot = false;
    ProfScope ps(c, kKGramReduce, s);
    rc = check_cuda(c, launch_gram_reduce<R>(part, nblk, nocc, nocc, msc, false, M, (R*)nullptr, s), "gram reduce");
  }
  if (rc) return rc;
  {
    ProfScope ps(c, kKChol, s);
    rc = check_cuda(c,
                    launch_chol_linv(M, nocc, Linv, sizeof(R) == 4 ? (float*)linv_r : nullptr,
                                     sizeof(R) == 8 ? (double*)linv_r : nullptr, c->status, s),
                    "cholesky");
  }
  if (rc) return rc;
  {
    ProfScope ps(c, kKCombine, s);
    rc = check_cuda(c, launch_combine<R>(linv_r, nocc, nocc, (const R*)xi, N, (R*)xi, 4 * c->nsm, s),
                    "xi = L^-1 W");
  }
  if (rc) return rc;
  if (M_out)
    rc = check_cuda(c, cudaMemcpyAsync(M_out, M, sizeof(double) * nocc * nocc, cudaMemcpyDeviceToDevice, s),
                    "M copy");
  return rc;
}

template <typename R>
int ace_apply(rsx_ctx* c, const void* xi, int nxi, const void* psi, int npsi, void* out, cudaStream_t s) {
  const size_t N = c->g.N();
  const int nblk = 2 * c->nsm;
  int rc = grow(c, (void**)&c->dsm, &c->dsm_bytes, sizeof(double) * ((size_t)nblk * 4096 + 3 * 4096), "small FP64");
  if (rc) return rc;
  rc = grow(c, &c->smallr, &c->smallr_bytes, sizeof(R) * 4096 * 2, "small coefficients");
  if (rc) return rc;
  double* part = c->dsm;
  R* cm = (R*)c->smallr + 4096;
  const double h3 = c->h * c->h * c->h;
  // C_kp = h^3 <xi_k, psi_p>; Cm[p][k] = -C_kp
  {
    ProfScope ps(c, kKGram, s);
    rc = check_cuda(c, launch_gram<R>((const R*)xi, nxi, (const R*)psi, npsi, N, part, nblk, s, nullptr, c->status), "gram");
  }
  if (rc) return rc;
  {
    ProfScope ps(c, kKGramReduce, s);
    rc = check_cuda(c, launch_gram_reduce<R>(part, nblk, nxi, npsi, -h3, true, (double*)nullptr, cm, s),
                    "gram reduce");
  }
  if (rc) return rc;
  ProfScope ps(c, kKCombine, s);
  return check_cuda(c, launch_combine<R>(cm, npsi, nxi, (const R*)xi, N, (R*)out, 4 * c->nsm, s), "ace apply");
}

template int solve_pairs<float>(rsx_ctx*, const PairMap<float>&, int, int, int, int, float*, cudaStream_t, int);
template int solve_pairs<double>(rsx_ctx*, const PairMap<double>&, int, int, int, int, double*, cudaStream_t, int);

}  // namespace rsx

// ==================================================================================
// exported C ABI

namespace rsx {
namespace {

template <typename R>
__global__ void k_fill(R* x, size_t n, R v) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) x[i] = v;
}

// V = potential of the density rho: the pair (rho, 1) through the three passes, pass 3
// writing the potential itself
template <typename R>
int poisson(rsx_ctx* c, const void* rho, void* V, cudaStream_t s) {
  const size_t N = c->g.N();
  if (!c->ones) {
    int rc = grow(c, &c->ones, &c->ones_bytes, N * sizeof(R), "unit field");
    if (rc) return rc;
    k_fill<R><<<512, 256, 0, s>>>((R*)c->ones, N, R(1));
    rc = check_cuda(c, cudaGetLastError(), "unit field");
    if (rc) return rc;
  }
  const PairMap<R> pm = pair_map<R>(kProd, rho, c->ones, 1, 1, N);
  return solve_pairs<R>(c, pm, 0, 1, 0, 1, (R*)V, s, 1);
}

}  // namespace
}  // namespace rsx

namespace rsx {
namespace {
template <typename R>
int ace_factor(rsx_ctx* c, double* M, const void* W, int nocc, void* xi, cudaStream_t s) {
  const size_t N = c->g.N();
  int rc = grow(c, (void**)&c->dsm, &c->dsm_bytes, sizeof(double) * ((size_t)2 * c->nsm * 4096 + 3 * 4096), "small FP64");
  if (rc) return rc;
  rc = grow(c, &c->smallr, &c->smallr_bytes, sizeof(R) * 4096 * 2, "small coefficients");
  if (rc) return rc;
  double* Linv = c->dsm + (size_t)2 * c->nsm * 4096 + 4096;
  R* linv_r = (R*)c->smallr;
  {
    ProfScope ps(c, kKChol, s);
    rc = check_cuda(c,
                    launch_chol_linv(M, nocc, Linv, sizeof(R) == 4 ? (float*)linv_r : nullptr,
                                     sizeof(R) == 8 ? (double*)linv_r : nullptr, c->status, s),
                    "cholesky");
  }
  if (rc) return rc;
  ProfScope ps(c, kKCombine, s);
  return check_cuda(c, launch_combine<R>(linv_r, nocc, nocc, (const R*)W, N, (R*)xi, 4 * c->nsm, s), "xi = L^-1 W");
}
}  // namespace
}  // namespace rsx

extern "C" {

int rsx_create(rsx_ctx** out, int nz, int ny, int nx, double h, int precision, int device) {
  if (!out) return RSX_EINVAL;
  *out = nullptr;
  if (!(h > 0.0) || (precision != RSX_FP32 && precision != RSX_FP64)) return RSX_EINVAL;
  if (!edge_ok(nz) || !edge_ok(ny) || !edge_ok(nx) || nz != ny) return RSX_EUNSUPPORTED;
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return RSX_ECUDA;
  }
  rsx_ctx* c = new rsx_ctx();
  c->device = device;
  c->precision = precision;
  c->h = h;
  Geom& g = c->g;
  g.nz = nz; g.ny = ny; g.nx = nx;
  g.Mz = 2 * nz; g.My = 2 * ny; g.Mx = 2 * nx;
  g.Az = g.Mz / 16; g.Ay = g.My / 16; g.Ax = g.Mx / 16;
  g.Hx = g.Mx / 2 + 1;
  g.p2_threads = 256;
  if (const char* e = getenv("RSX_PASS2_THREADS")) g.p2_threads = (atoi(e) == 512 || atoi(e) == 384) ? atoi(e) : 256;
  g.p1_group = 1 << 30;   // pass-1 blocks pair-fastest over the whole launch (orbital rows shared in L2)
  if (const char* e = getenv("RSX_PASS1_GROUP")) g.p1_group = atoi(e) > 0 ? atoi(e) : 0;
  g.p2_global = 0;
  g.p2_lanes = 16;
  if (const char* e = getenv("RSX_PASS2_LANES")) g.p2_lanes = atoi(e) == 8 ? 8 : 16;
  cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, device);
  size_t freeb = 0, totalb = 0;
  cudaMemGetInfo(&freeb, &totalb);
  c->work_limit = std::min<size_t>((size_t)(0.4 * (double)freeb), (size_t)64 << 30);
  if (cudaMalloc(&c->status, sizeof(int)) != cudaSuccess) {
    delete c;
    return RSX_ENOMEM;
  }
  cudaMemset(c->status, 0, sizeof(int));
#ifdef RSX_CHECKED
  g.dbg = c->status;   // out-of-range indices of the FFT passes are reported here
#endif
  const int rc = precision == RSX_FP32 ? make_tables<float>(c) : make_tables<double>(c);
  if (rc) {
    rsx_destroy(c);
    return rc;
  }
  // host-side fault injection from the environment, armed once the context exists (the
  // same faults as rsx_inject_fault): RSX_INJECT_FAULT=alloc:N (the workspace allocation
  // after N successful ones fails) or pivot
  if (const char* e = getenv("RSX_INJECT_FAULT")) {
    if (strncmp(e, "alloc:", 6) == 0 && atoi(e + 6) >= 0) c->fault_alloc_after = atoi(e + 6);
    if (strcmp(e, "pivot") == 0) c->fault_pivot = true;
  }
  *out = c;
  return RSX_OK;
}

int rsx_destroy(rsx_ctx* c) {
  if (!c) return RSX_OK;
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  prof_collect(c);
  for (cudaEvent_t e : c->prof_pool) cudaEventDestroy(e);
  void* bufs[] = {c->vhat, c->vhatz, c->vhatz8, c->tw8, c->tw[0], c->tw[1], c->tw[2], c->work, c->gscr, c->dsm, c->smallr, c->status,
                  c->panel_hi, c->panel_lo, c->gemm_part, c->eig_work, c->gscr_kd, c->pos, c->tdhf_work, c->specw, c->ones};
  for (void* b : bufs)
    if (b) cudaFree(b);
  delete c;
  return RSX_OK;
}

const char* rsx_last_error(const rsx_ctx* c) { return c ? c->err : "null context"; }

int rsx_set_workspace_limit(rsx_ctx* c, size_t bytes) {
  if (!c || bytes == 0) return RSX_EINVAL;
  c->work_limit = bytes;
  return RSX_OK;
}

#define RSX_PREP(c)                                         \
  if (!(c)) return RSX_EINVAL;                              \
  (c)->err[0] = 0;                                          \
  if (cudaSetDevice((c)->device) != cudaSuccess) {          \
    cudaGetLastError();                                     \
    return set_error((c), RSX_ECUDA, "cudaSetDevice failed"); \
  }

int rsx_build_pair_densities(rsx_ctx* c, const void* a, int na, const void* b, int nb, void* rho, void* stream) {
  rsx::NvtxRange nvtx_range("rsx_build_pair_densities");
  RSX_PREP(c);
  if (!a || !b || !rho || na < 1 || nb < 1) return set_error(c, RSX_EINVAL, "bad pair-density arguments");
  const size_t N = c->g.N(), es = c->elem_size();
  if (overlaps(rho, (size_t)na * nb * N * es, a, na * N * es) || overlaps(rho, (size_t)na * nb * N * es, b, nb * N * es))
    return set_error(c, RSX_EINVAL, "rho aliases an input");
  cudaStream_t s = (cudaStream_t)stream;
  ProfScope ps(c, kKPairProd, s);
  cudaError_t e = c->precision == RSX_FP32
                      ? launch_pair_products<float>((const float*)a, na, (const float*)b, nb, N, (float*)rho, s)
                      : launch_pair_products<double>((const double*)a, na, (const double*)b, nb, N, (double*)rho, s);
  return check_cuda(c, e, "pair densities");
}

int rsx_exchange_apply(rsx_ctx* c, const void* phi, int nocc, const void* psi, int npsi, void* out, void* stream) {
  rsx::NvtxRange nvtx_range("rsx_exchange_apply");
  RSX_PREP(c);
  if (!phi || !psi || !out || nocc < 1 || npsi < 1) return set_error(c, RSX_EINVAL, "bad exchange arguments");
  const size_t N = c->g.N(), es = c->elem_size();
  if (overlaps(out, npsi * N * es, phi, nocc * N * es) || overlaps(out, npsi * N * es, psi, npsi * N * es))
    return set_error(c, RSX_EINVAL, "out aliases an input");
  cudaStream_t s = (cudaStream_t)stream;
  return c->precision == RSX_FP32 ? exchange_apply<float>(c, phi, nocc, psi, npsi, out, s)
                                  : exchange_apply<double>(c, phi, nocc, psi, npsi, out, s);
}

int rsx_poisson(rsx_ctx* c, const void* rho, void* V, void* stream) {
  rsx::NvtxRange nvtx_range("rsx_poisson");
  RSX_PREP(c);
  if (!rho || !V) return set_error(c, RSX_EINVAL, "bad Poisson arguments");
  const size_t bytes = c->g.N() * c->elem_size();
  if (overlaps(V, bytes, rho, bytes)) return set_error(c, RSX_EINVAL, "V aliases rho");
  cudaStream_t s = (cudaStream_t)stream;
  return c->precision == RSX_FP32 ? poisson<float>(c, rho, V, s) : poisson<double>(c, rho, V, s);
}

int rsx_ace_build(rsx_ctx* c, const void* phi, int nocc, void* xi, double* M_out, void* stream) {
  rsx::NvtxRange nvtx_range("rsx_ace_build");
  RSX_PREP(c);
  if (!phi || !xi || nocc < 1 || nocc > 64) return set_error(c, RSX_EINVAL, "bad ACE build arguments");
  const size_t N = c->g.N(), es = c->elem_size();
  if (overlaps(xi, nocc * N * es, phi, nocc * N * es)) return set_error(c, RSX_EINVAL, "xi aliases phi");
  cudaStream_t s = (cudaStream_t)stream;
  return c->precision == RSX_FP32 ? ace_build<float>(c, phi, nocc, xi, M_out, s)
                                  : ace_build<double>(c, phi, nocc, xi, M_out, s);
}

int rsx_ace_apply(rsx_ctx* c, const void* xi, int nxi, const void* psi, int npsi, void* out, void* stream) {
  rsx::NvtxRange nvtx_range("rsx_ace_apply");
  RSX_PREP(c);
  if (!xi || !psi || !out || nxi < 1 || npsi < 1 || nxi * npsi > 4096 || nxi > 64)
    return set_error(c, RSX_EINVAL, "bad ACE apply arguments");
  const size_t N = c->g.N(), es = c->elem_size();
  if (overlaps(out, npsi * N * es, xi, nxi * N * es)) return set_error(c, RSX_EINVAL, "out aliases xi");
  if (out != psi && overlaps(out, npsi * N * es, psi, npsi * N * es))
    return set_error(c, RSX_EINVAL, "out partially aliases psi");
  cudaStream_t s = (cudaStream_t)stream;
  return c->precision == RSX_FP32 ? ace_apply<float>(c, xi, nxi, psi, npsi, out, s)
                                  : ace_apply<double>(c, xi, nxi, psi, npsi, out, s);
}

int rsx_gram(rsx_ctx* c, const void* a, int na, const void* b, int nb, double* C, void* stream) {
  rsx::NvtxRange nvtx_range("rsx_gram");
  RSX_PREP(c);
  if (!a || !b || !C || na < 1 || nb < 1 || na * nb > 4096) return set_error(c, RSX_EINVAL, "bad Gram arguments");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t N = c->g.N();
  const int nblk = 2 * c->nsm;
  int rc = grow(c, (void**)&c->dsm, &c->dsm_bytes, sizeof(double) * ((size_t)nblk * 4096 + 3 * 4096), "small FP64");
  if (rc) return rc;
  const double h3 = c->h * c->h * c->h;
  {
    ProfScope ps(c, kKGram, s);
    rc = check_cuda(c, c->precision == RSX_FP32
                           ? launch_gram<float>((const float*)a, na, (const float*)b, nb, N, c->dsm, nblk, s, nullptr, c->status)
                           : launch_gram<double>((const double*)a, na, (const double*)b, nb, N, c->dsm, nblk, s),
                    "gram");
  }
  if (rc) return rc;
  ProfScope ps(c, kKGramReduce, s);
  return check_cuda(c, c->precision == RSX_FP32
                           ? launch_gram_reduce<float>(c->dsm, nblk, na, nb, h3, false, C, (float*)nullptr, s)
                           : launch_gram_reduce<double>(c->dsm, nblk, na, nb, h3, false, C, (double*)nullptr, s),
                    "gram reduce");
}


int rsx_ace_factor(rsx_ctx* c, double* M, const void* W, int nocc, void* xi, void* stream) {
  rsx::NvtxRange nvtx_range("rsx_ace_factor");
  RSX_PREP(c);
  if (!M || !W || !xi || nocc < 1 || nocc > 64) return set_error(c, RSX_EINVAL, "bad ACE factor arguments");
  const size_t bytes = (size_t)nocc * c->g.N() * c->elem_size();
  if (xi != W && overlaps(xi, bytes, W, bytes)) return set_error(c, RSX_EINVAL, "xi partially aliases W");
  cudaStream_t s = (cudaStream_t)stream;
  return c->precision == RSX_FP32 ? ace_factor<float>(c, M, W, nocc, xi, s) : ace_factor<double>(c, M, W, nocc, xi, s);
}

int rsx_set_wait_limit(rsx_ctx* c, long long spins) {
  if (!c) return RSX_EINVAL;
  c->wait_limit = spins < 0 ? -1 : spins;
  return RSX_OK;
}

int rsx_inject_fault(rsx_ctx* c, int kind, int after) {
  if (!c) return RSX_EINVAL;
  switch (kind) {
    case RSX_FAULT_NONE:
      c->fault_alloc_after = -1;
      c->fault_pivot = false;
      return RSX_OK;
    case RSX_FAULT_ALLOC:
      if (after < 0) return RSX_EINVAL;
      c->fault_alloc_after = after;
      return RSX_OK;
    case RSX_FAULT_PIVOT:
      c->fault_pivot = true;
      return RSX_OK;
    default:
      return RSX_EINVAL;
  }
}

int rsx_profile_enable(rsx_ctx* c, int on) {
  if (!c) return RSX_EINVAL;
  c->prof_on = on != 0;
  return RSX_OK;
}

int rsx_profile_reset(rsx_ctx* c) {
  if (!c) return RSX_EINVAL;
  prof_collect(c);
  for (int i = 0; i < kKCount; ++i) {
    c->prof_ms[i] = 0.0;
    c->prof_n[i] = 0;
  }
  return RSX_OK;
}

int rsx_profile_read(rsx_ctx* c, int kernel, double* total_ms, long long* launches) {
  if (!c || kernel < 0 || kernel >= kKCount) return RSX_EINVAL;
  prof_collect(c);
  if (total_ms) *total_ms = c->prof_ms[kernel];
  if (launches) *launches = c->prof_n[kernel];
  return RSX_OK;
}

int rsx_kernel_count(void) { return kKCount; }

const char* rsx_kernel_name(int kernel) { return kernel_name(kernel); }

int rsx_sync_status(rsx_ctx* c, void* stream) {
  RSX_PREP(c);
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return check_cuda(c, e, "stream synchronise");
  int st = 0;
  e = cudaMemcpy(&st, c->status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return check_cuda(c, e, "status read");
  cudaMemset(c->status, 0, sizeof(int));
  if (st == RSX_ENOTPD) return set_error(c, RSX_ENOTPD, "ACE: -M is not positive definite");
  if (st == RSX_ETIMEOUT) return set_error(c, RSX_ETIMEOUT, "a bounded device wait timed out");
  if (st == RSX_EBOUNDS) return set_error(c, RSX_EBOUNDS, "bounds-checked build: an FFT-pass index left its array");
  if (st) return set_error(c, st, "deferred device error");
  return RSX_OK;
}

}  // extern "C"
