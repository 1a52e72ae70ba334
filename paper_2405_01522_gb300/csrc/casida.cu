// Tamm-Dancoff Casida calls of the C ABI (Sec. 2, Eqs. 6-7).
//
// rsx_casida_K   K_{ia,jb} = (ia|jb) for transitions t = i * nvirt + a.
//   FP32 context: pair densities rho_t -> x forward (pass 1) -> y, z forward with the
//   weights sqrt(w_G ghat h^6 / N_pad) -> bf16 hi/lo panel S [t][G] -> tcgen05
//   K = S S^T in three split products (gemm_tcgen05.cu).
//   FP64 context (plain form): V_t for every transition (full pair solves), then
//   K = h^3 rho^T V in FP64 (Gram blocks of 64 x 64).
// rsx_casida_Kd  K_d[ia,jb] = (ab|ji) = h^3 sum_r phi_a phi_b V_ij, V_ij for the
//   unordered occupied pairs (i, j); symmetric in (i, j), so each block fills two places.
// rsx_casida_solve  FP64 eigen-solve of A = diag(de) + delta_M K - K_d (eig.cu).
// rsx_casida_K_uhf / rsx_casida_solve_uhf  the spin-polarised form: K over the alpha
//   then the beta transitions in one panel (every spin block of the Coulomb-type term),
//   A = diag(de) + K - blockdiag(K_d alpha, K_d beta).
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/rsx.h"
#include "api_internal.cuh"
#include "dense.cuh"
#include "eig.cuh"
#include "gemm_tcgen05.cuh"

using namespace rsx;

namespace {

__global__ void k_symmetrise(double* K, int n) {
  const long long total = (long long)n * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int t = (int)(e / n), s = (int)(e - (long long)t * n);
    if (t < s) {
      const long long et = (long long)s * n + t;
      const double v = 0.5 * (K[e] + K[et]);
      K[e] = v;
      K[et] = v;
    }
  }
}

template <typename R>
PairMap<R> prod_map(const void* A, int na, const void* B, int nb, size_t N) {
  PairMap<R> pm;
  pm.mode = kProd;
  pm.A = (const R*)A;
  pm.B = (const R*)B;
  pm.na = na;
  pm.nb = nb;
  pm.N = N;
  return pm;
}

template <typename R>
PairMap<R> sym_map(const void* A, int na, size_t N) {
  PairMap<R> pm;
  pm.mode = kSym;
  pm.A = (const R*)A;
  pm.B = nullptr;
  pm.na = na;
  pm.nb = 0;
  pm.N = N;
  return pm;
}

// K as the Gram matrix h^3 X Y^T of two [n][N] sets, 64 x 64 blocks, row stride n
template <typename R>
int gram_blocks(rsx_ctx* c, const R* X, const R* Y, int n, size_t N, double scale, double* K, const R* w,
                int ldo, cudaStream_t s) {
  const int nblk = 2 * c->nsm;
  int rc = grow(c, (void**)&c->dsm, &c->dsm_bytes, sizeof(double) * ((size_t)nblk * 4096 + 3 * 4096), "small FP64");
  if (rc) return rc;
  for (int b0 = 0; b0 < n; b0 += 64) {
    const int na = std::min(64, n - b0);
    for (int b1 = 0; b1 < n; b1 += 64) {
      const int nb = std::min(64, n - b1);
      {
        ProfScope ps(c, kKGram, s);
        rc = check_cuda(c, launch_gram<R>(X + (size_t)b0 * N, na, Y + (size_t)b1 * N, nb, N, c->dsm, nblk, s, w, c->status),
                        "gram block");
      }
      if (rc) return rc;
      ProfScope ps(c, kKGramReduce, s);
      rc = check_cuda(c,
                      launch_gram_reduce<R>(c->dsm, nblk, na, nb, scale, false, K + (size_t)b0 * ldo + b1,
                                            (R*)nullptr, s, ldo),
                      "gram block reduce");
      if (rc) return rc;
    }
  }
  return RSX_OK;
}

// A set of transitions (occupied x virtual of one spin), t = i * nv + a within the set;
// sets follow one another in K.
struct TSet {
  const void* po;
  int no;
  const void* pv;
  int nv;
  int nt() const { return no * nv; }
};

int casida_K_f32(rsx_ctx* c, const TSet* sets, int nsets, double* K, cudaStream_t s) {
  const Geom& g = c->g;
  const size_t N = g.N();
  int nt = 0;
  for (int k = 0; k < nsets; ++k) nt += sets[k].nt();
  const size_t inter_bytes = (size_t)nt * g.inter_elems() * sizeof(Cx<float>);
  const long long ng = 2LL * g.Hx * g.My * g.Mz;
  const long long ld = (ng + 63) / 64 * 64;
  const int nt_pad = (nt + 127) / 128 * 128;
  const size_t panel_bytes = (size_t)nt_pad * ld * sizeof(uint16_t);
  if (inter_bytes + 2 * panel_bytes > c->work_limit)
    return set_error(c, RSX_ENOMEM, "casida_K: intermediates and panels exceed the workspace limit");
  int rc = grow(c, &c->work, &c->work_bytes, inter_bytes, "FFT intermediates");
  if (rc) return rc;
  rc = grow(c, &c->panel_hi, &c->panel_hi_bytes, panel_bytes, "K panel (hi)");
  if (rc) return rc;
  rc = grow(c, &c->panel_lo, &c->panel_lo_bytes, panel_bytes, "K panel (lo)");
  if (rc) return rc;
  uint16_t* hi = (uint16_t*)c->panel_hi;
  uint16_t* lo = (uint16_t*)c->panel_lo;
  // tile-major panel [ld/64][nrb][128][64]; zero what the spectrum kernel does not write:
  // whole column blocks past ng, and rows nt .. nt_pad - 1 of the last row block
  const int nrb = nt_pad / 128;
  const long long nkb = ld / 64, nkb_used = ng / 64;   // ng is a multiple of 64 for supported edges
  const size_t kb_bytes = (size_t)nrb * 8192 * 2;
  for (uint16_t* P : {hi, lo}) {
    if (nkb > nkb_used) {
      rc = check_cuda(c, cudaMemsetAsync(P + (size_t)nkb_used * nrb * 8192, 0, (size_t)(nkb - nkb_used) * kb_bytes, s),
                      "panel tail");
      if (rc) return rc;
    }
    if (nt_pad > nt) {
      const int r0 = nt % 128;
      rc = check_cuda(c,
                      cudaMemset2DAsync(P + (size_t)(nrb - 1) * 8192 + (size_t)r0 * 64, kb_bytes, 0,
                                        (size_t)(128 - r0) * 64 * 2, nkb, s),
                      "panel pad");
      if (rc) return rc;
    }
  }
  if (ng % 64) return set_error(c, RSX_EUNSUPPORTED, "casida_K: spectrum length not a multiple of 64");
  Cx<float>* inter = (Cx<float>*)c->work;
  {
    ProfScope ps(c, kKPass1, s);
    size_t off = 0;
    for (int k = 0; k < nsets && !rc; ++k) {
      if (!sets[k].nt()) continue;
      const PairMap<float> pm = prod_map<float>(sets[k].pv, sets[k].nv, sets[k].po, sets[k].no, N);  // q = i * nv + a
      rc = check_cuda(c, launch_pass1<float>(g, pm, 0, sets[k].nt(), inter + off * g.inter_elems(),
                                             (const Cx<float>*)c->tw[2], s),
                      "pass 1");
      off += sets[k].nt();
    }
  }
  if (rc) return rc;
  if (!c->specw) {   // panel weights, once per context
    const size_t nw = (size_t)g.Hx * (g.My / 2 + 1) * (g.Mz / 2 + 1);
    rc = grow(c, &c->specw, &c->specw_bytes, nw * sizeof(float), "panel weights");
    if (!rc)
      rc = check_cuda(c, launch_spectrum_weights(g, (const float*)c->vhat, (float)(c->h * c->h * c->h), (float*)c->specw, s),
                      "panel weights");
    if (rc) return rc;
  }
  {
    ProfScope ps(c, kKSpectrum, s);
    rc = check_cuda(c,
                    launch_spectrum_f32(g, nt, inter, (const Cx<float>*)c->tw[1], (const Cx<float>*)c->tw[0],
                                        (const float*)c->specw, hi, lo, (size_t)ld, nrb, s),
                    "spectrum panel");
  }
  if (rc) return rc;
  const int nsplit = syrk_splits(c->nsm, nt);
  rc = grow(c, &c->gemm_part, &c->gemm_part_bytes, syrk_partial_bytes(nt, nsplit), "K split partials");
  if (rc) return rc;
  return syrk_bf16x3(c, hi, lo, nt, ld, nsplit, (double*)c->gemm_part, K, s, true);
}

template <typename R>
int casida_K_plain(rsx_ctx* c, const TSet* sets, int nsets, double* K, cudaStream_t s) {
  const Geom& g = c->g;
  const size_t N = g.N();
  int nt = 0, ntmax = 0;
  for (int k = 0; k < nsets; ++k) {
    nt += sets[k].nt();
    ntmax = std::max(ntmax, sets[k].nt());
  }
  const size_t need = (size_t)ntmax * g.inter_elems() * sizeof(Cx<R>) + 2 * (size_t)nt * N * sizeof(R);
  if (need > c->work_limit) return set_error(c, RSX_ENOMEM, "casida_K: workspace limit exceeded");
  int rc = grow(c, &c->panel_hi, &c->panel_hi_bytes, 2 * (size_t)nt * N * sizeof(R), "potentials and densities");
  if (rc) return rc;
  R* V = (R*)c->panel_hi;
  R* rho = V + (size_t)nt * N;
  size_t off = 0;
  for (int k = 0; k < nsets && !rc; ++k) {
    const TSet& t = sets[k];
    if (!t.nt()) continue;
    const PairMap<R> pm = prod_map<R>(t.pv, t.nv, t.po, t.no, N);
    rc = solve_pairs<R>(c, pm, 0, t.nt(), 0, t.nt(), V + off * N, s, 1);
    if (rc) return rc;
    ProfScope ps(c, kKPairProd, s);
    rc = check_cuda(c, launch_pair_products<R>((const R*)t.po, t.no, (const R*)t.pv, t.nv, N, rho + off * N, s),
                    "densities");
    off += t.nt();
  }
  if (rc) return rc;
  rc = gram_blocks<R>(c, rho, V, nt, N, c->h * c->h * c->h, K, (const R*)nullptr, nt, s);
  if (rc) return rc;
  k_symmetrise<<<256, 256, 0, s>>>(K, nt);
  return check_cuda(c, cudaGetLastError(), "symmetrise");
}

template <typename R>
int casida_Kd(rsx_ctx* c, const void* po, int no, const void* pv, int nv, double* Kd, cudaStream_t s) {
  const Geom& g = c->g;
  const size_t N = g.N();
  const int nt = no * nv;
  const int npairs = no * (no + 1) / 2;
  const PairMap<R> pm = sym_map<R>(po, no, N);
  const size_t need = (size_t)npairs * g.inter_elems() * sizeof(Cx<R>) + (size_t)npairs * N * sizeof(R);
  if (need > c->work_limit) return set_error(c, RSX_ENOMEM, "casida_Kd: workspace limit exceeded");
  int rc = grow(c, &c->gscr_kd, &c->gscr_kd_bytes, (size_t)npairs * N * sizeof(R), "occupied pair potentials");
  if (rc) return rc;
  R* V = (R*)c->gscr_kd;
  rc = solve_pairs<R>(c, pm, 0, npairs, 0, npairs, V, s, 1);
  if (rc) return rc;
  const double h3 = c->h * c->h * c->h;
  int q = 0;
  for (int i = 0; i < no; ++i)
    for (int j = i; j < no; ++j, ++q) {
      const R* w = V + (size_t)q * N;
      rc = gram_blocks<R>(c, (const R*)pv, (const R*)pv, nv, N, h3, Kd + (size_t)i * nv * nt + (size_t)j * nv, w, nt,
                          s);
      if (rc) return rc;
      if (j != i) {
        rc = check_cuda(c,
                        cudaMemcpy2DAsync(Kd + (size_t)j * nv * nt + (size_t)i * nv, nt * sizeof(double),
                                          Kd + (size_t)i * nv * nt + (size_t)j * nv, nt * sizeof(double),
                                          nv * sizeof(double), nv, cudaMemcpyDeviceToDevice, s),
                        "Kd mirror");
        if (rc) return rc;
      }
    }
  return RSX_OK;
}

bool overlap(const void* a, size_t na, const void* b, size_t nb) {
  const char* pa = (const char*)a;
  const char* pb = (const char*)b;
  return pa < pb + nb && pb < pa + na;
}

int check_casida_args(rsx_ctx* c, const void* po, int no, const void* pv, int nv, const double* K) {
  if (!po || !pv || !K || no < 1 || nv < 1 || no * nv > 4096)
    return set_error(c, RSX_EINVAL, "casida: bad arguments (need nocc, nvirt >= 1, nocc * nvirt <= 4096)");
  const size_t N = c->g.N(), es = c->elem_size(), nt = (size_t)no * nv;
  if (overlap(K, nt * nt * 8, po, no * N * es) || overlap(K, nt * nt * 8, pv, nv * N * es))
    return set_error(c, RSX_EINVAL, "casida: output aliases an input");
  return RSX_OK;
}

}  // namespace

extern "C" {

#define RSX_PREP_C(c)                                            \
  if (!(c)) return RSX_EINVAL;                                   \
  (c)->err[0] = 0;                                               \
  if (cudaSetDevice((c)->device) != cudaSuccess) {               \
    cudaGetLastError();                                          \
    return set_error((c), RSX_ECUDA, "cudaSetDevice failed");    \
  }

int rsx_casida_K(rsx_ctx* c, const void* phi_occ, int nocc, const void* phi_virt, int nvirt, double* K,
                 void* stream) {
  rsx::NvtxRange nvtx_range("rsx_casida_K");
  RSX_PREP_C(c);
  int rc = check_casida_args(c, phi_occ, nocc, phi_virt, nvirt, K);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const TSet set{phi_occ, nocc, phi_virt, nvirt};
  if (c->precision == RSX_FP32) {
    if (c->g.Ay != c->g.Az) return set_error(c, RSX_EUNSUPPORTED, "casida_K: ny must equal nz");
    return casida_K_f32(c, &set, 1, K, s);
  }
  return casida_K_plain<double>(c, &set, 1, K, s);
}

int rsx_casida_K_uhf(rsx_ctx* c, const void* occ_a, int nocc_a, const void* virt_a, int nvirt_a, const void* occ_b,
                     int nocc_b, const void* virt_b, int nvirt_b, double* K, void* stream) {
  rsx::NvtxRange nvtx_range("rsx_casida_K_uhf");
  RSX_PREP_C(c);
  int rc = check_casida_args(c, occ_a, nocc_a, virt_a, nvirt_a, K);
  if (rc) return rc;
  const bool has_b = nocc_b > 0 && nvirt_b > 0;
  if (nocc_b < 0 || nvirt_b < 0 || (has_b && (!occ_b || !virt_b)))
    return set_error(c, RSX_EINVAL, "casida_K_uhf: bad beta arguments");
  const size_t N = c->g.N(), es = c->elem_size();
  const size_t nt = (size_t)nocc_a * nvirt_a + (has_b ? (size_t)nocc_b * nvirt_b : 0);
  if (nt > 4096) return set_error(c, RSX_EINVAL, "casida_K_uhf: more than 4096 transitions");
  if (has_b && (overlap(K, nt * nt * 8, occ_b, nocc_b * N * es) || overlap(K, nt * nt * 8, virt_b, nvirt_b * N * es) ||
                overlap(K, nt * nt * 8, occ_a, nocc_a * N * es) || overlap(K, nt * nt * 8, virt_a, nvirt_a * N * es)))
    return set_error(c, RSX_EINVAL, "casida_K_uhf: output aliases an input");
  cudaStream_t s = (cudaStream_t)stream;
  const TSet sets[2] = {{occ_a, nocc_a, virt_a, nvirt_a}, {occ_b, has_b ? nocc_b : 0, virt_b, has_b ? nvirt_b : 0}};
  if (c->precision == RSX_FP32) {
    if (c->g.Ay != c->g.Az) return set_error(c, RSX_EUNSUPPORTED, "casida_K: ny must equal nz");
    return casida_K_f32(c, sets, 2, K, s);
  }
  return casida_K_plain<double>(c, sets, 2, K, s);
}

int rsx_casida_solve_uhf(rsx_ctx* c, const double* eo_a, int nocc_a, const double* ev_a, int nvirt_a,
                         const double* eo_b, int nocc_b, const double* ev_b, int nvirt_b, const double* K,
                         const double* Kd_a, const double* Kd_b, int nroots, double* omega, double* X, void* stream) {
  rsx::NvtxRange nvtx_range("rsx_casida_solve_uhf");
  RSX_PREP_C(c);
  const bool has_b = nocc_b > 0 && nvirt_b > 0;
  const int nt = nocc_a * nvirt_a + (has_b ? nocc_b * nvirt_b : 0);
  if (!eo_a || !ev_a || !K || !omega || nocc_a < 1 || nvirt_a < 1 || nocc_b < 0 || nvirt_b < 0 ||
      (has_b && (!eo_b || !ev_b)) || nt > 4096 || nroots < 1 || nroots > nt)
    return set_error(c, RSX_EINVAL, "casida_solve_uhf: bad arguments");
  int rc = grow(c, &c->eig_work, &c->eig_work_bytes, tda_work_doubles(nt, nroots) * sizeof(double), "eigensolver");
  if (rc) return rc;
  return uhf_tda_solve(c, eo_a, nocc_a, ev_a, nvirt_a, eo_b, has_b ? nocc_b : 0, ev_b, has_b ? nvirt_b : 0, K, Kd_a,
                       has_b ? Kd_b : nullptr, nroots, omega, X, (double*)c->eig_work, (cudaStream_t)stream);
}

int rsx_casida_Kd(rsx_ctx* c, const void* phi_occ, int nocc, const void* phi_virt, int nvirt, double* Kd,
                  void* stream) {
  rsx::NvtxRange nvtx_range("rsx_casida_Kd");
  RSX_PREP_C(c);
  int rc = check_casida_args(c, phi_occ, nocc, phi_virt, nvirt, Kd);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  return c->precision == RSX_FP32 ? casida_Kd<float>(c, phi_occ, nocc, phi_virt, nvirt, Kd, s)
                                  : casida_Kd<double>(c, phi_occ, nocc, phi_virt, nvirt, Kd, s);
}

int rsx_casida_solve(rsx_ctx* c, const double* eps_occ, int nocc, const double* eps_virt, int nvirt, const double* K,
                     const double* Kd, double delta_M, int nroots, double* omega, double* X, void* stream) {
  rsx::NvtxRange nvtx_range("rsx_casida_solve");
  RSX_PREP_C(c);
  const int nt = nocc * nvirt;
  if (!eps_occ || !eps_virt || !K || !omega || nocc < 1 || nvirt < 1 || nt > 4096 || nroots < 1 || nroots > nt)
    return set_error(c, RSX_EINVAL, "casida_solve: bad arguments");
  int rc = grow(c, &c->eig_work, &c->eig_work_bytes, tda_work_doubles(nt, nroots) * sizeof(double), "eigensolver");
  if (rc) return rc;
  return tda_solve(c, eps_occ, nocc, eps_virt, nvirt, K, Kd, delta_M, nroots, omega, X, (double*)c->eig_work,
                   (cudaStream_t)stream);
}

// C = H H^T + H L^T + L H^T for bf16 panels H, L: [n][ld] (n % 128 == 0, ld % 64 == 0)
int rsx_syrk_bf16x3(rsx_ctx* c, const void* hi, const void* lo, int n, long long ld, double* C, void* stream) {
  rsx::NvtxRange nvtx_range("rsx_syrk_bf16x3");
  RSX_PREP_C(c);
  if (!hi || !lo || !C || n < 128 || n % 128 || ld < 64 || ld % 64)
    return set_error(c, RSX_EINVAL, "syrk: need n % 128 == 0 and ld % 64 == 0");
  const int nsplit = syrk_splits(c->nsm, n);
  int rc = grow(c, &c->gemm_part, &c->gemm_part_bytes, syrk_partial_bytes(n, nsplit), "split partials");
  if (rc) return rc;
  return syrk_bf16x3(c, (const uint16_t*)hi, (const uint16_t*)lo, n, ld, nsplit, (double*)c->gemm_part, C,
                     (cudaStream_t)stream);
}

}  // extern "C"
