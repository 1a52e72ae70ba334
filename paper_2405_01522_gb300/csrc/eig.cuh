// FP64 Tamm-Dancoff eigen-solve on the device (eig.cu).
#pragma once
#include <cuda_runtime.h>

struct rsx_ctx;

namespace rsx {
// number of eigenvalues of the symmetric tridiagonal matrix (diagonal d, off-diagonal e)
// below x, by the signs of the LDL^T pivots (Sturm sequence); pivots smaller than pivmin in
// magnitude are replaced by -pivmin
__device__ inline int sturm_count(const double* d, const double* e, int n, double x, double pivmin) {
  int cnt = 0;
  double q = d[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  if (q < 0) ++cnt;
  for (int i = 1; i < n; ++i) {
    q = d[i] - x - e[i - 1] * e[i - 1] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    if (q < 0) ++cnt;
  }
  return cnt;
}

__device__ inline double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ inline float warp_sum(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// FP32 count of eigenvalues of T below x (the ratio form above in single precision, with
// the single-precision pivmin, and the fast approximate division: a Sturm count only needs
// the pivots' signs, and the count it returns is that of a slightly perturbed T); for an
// approximate eigenbasis that FP64 steps then refine
__device__ inline int sturm_count_f32(const float* d, const float* e2, int n, float x, float pivmin) {
  int cnt = 0;
  float q = d[0] - x;
  if (fabsf(q) < pivmin) q = -pivmin;
  if (q < 0.f) ++cnt;
  for (int i = 1; i < n; ++i) {
    q = (d[i] - x) - __fdividef(e2[i - 1], q);
    if (fabsf(q) < pivmin) q = -pivmin;
    if (q < 0.f) ++cnt;
  }
  return cnt;
}

// LU with partial pivoting of T - lam I (serial, one thread): sc holds 4 n values
// (reciprocal pivots, first and second superdiagonal of U, multipliers), piv n ints.
// R = double, or float for a first approximation.  The recurrence carries the current
// pivot row's diagonal and superdiagonal in registers; the factors are only stored, so
// the dependent chain is one reciprocal and one fused multiply-add per row.
template <typename R>
__device__ inline void tri_factor_shifted(const R* __restrict__ d, const R* __restrict__ e, int n, R lam,
                                          R* __restrict__ sc, int* __restrict__ piv) {
  R* dg = sc;
  R* u1 = sc + n;
  R* u2 = sc + 2 * n;
  R* lw = sc + 3 * n;
  const R eps_shift = R(sizeof(R) == 8 ? 1e-14 : 1e-6) * fmax(R(1), fabs(lam));
  R cur = d[0] - lam;                    // row i's diagonal, as updated by the previous step
  R cu1 = n > 1 ? e[0] : R(0);           // row i's first superdiagonal, likewise
#pragma unroll 4
  for (int i = 0; i < n - 1; ++i) {
    const R sub = e[i];
    const R dn = d[i + 1] - lam;                   // row i + 1 before this step
    const R en = (i + 1 < n - 1) ? e[i + 1] : R(0);
    if (fabs(cur) >= fabs(sub)) {
      piv[i] = 0;
      if (cur == R(0)) cur = eps_shift;
      const R r = R(1) / cur;
      const R l = sub * r;
      lw[i] = l;
      dg[i] = r;
      u1[i] = cu1;
      u2[i] = R(0);
      cur = dn - l * cu1;
      cu1 = en;
    } else {
      // rows i and i + 1 swapped: U's row i is the old row i + 1
      piv[i] = 1;
      const R r = R(1) / sub;
      const R l = cur * r;
      lw[i] = l;
      dg[i] = r;
      u1[i] = dn;
      u2[i] = en;
      cur = cu1 - l * dn;
      cu1 = -l * en;
    }
  }
  if (cur == R(0)) cur = eps_shift;
  dg[n - 1] = R(1) / cur;   // dg now holds the reciprocal pivots the solves multiply by
}

// z <- (T - lam I)^{-1} z with the factors of tri_factor_shifted (serial, one thread; the
// running entries of z in registers, the factors read ahead)
template <typename R>
__device__ inline void tri_solve_factored(int n, R* __restrict__ z, const R* __restrict__ sc,
                                          const int* __restrict__ piv) {
  const R* rdg = sc;
  const R* u1 = sc + n;
  const R* u2 = sc + 2 * n;
  const R* lw = sc + 3 * n;
  R c = z[0];   // entry i of the forward sweep, as updated by the previous step
#pragma unroll 4
  for (int i = 0; i < n - 1; ++i) {
    const R zn = z[i + 1];
    const R l = lw[i];
    if (piv[i]) {
      z[i] = zn;
      c = c - l * zn;
    } else {
      z[i] = c;
      c = zn - l * c;
    }
  }
  z[n - 1] = c;
  R z1 = R(0), z2 = R(0);   // the solution's entries i + 1 and i + 2
#pragma unroll 4
  for (int i = n - 1; i >= 0; --i) {
    R s = z[i];
    if (i + 1 < n) s -= u1[i] * z1;
    if (i + 2 < n) s -= u2[i] * z2;
    const R zi = s * rdg[i];
    z[i] = zi;
    z2 = z1;
    z1 = zi;
  }
}

// one warp: `iters` inverse iterations for root r (vector z, length n), each followed by
// orthogonalisation against the roots j in `ortho` (bit j set) and normalisation; the
// shifted matrix is factored once
template <typename R>
__device__ inline void warp_inverse_iteration(const R* d, const R* e, int n, R lam, R* z, R* sc, int* piv, int iters,
                                              const R* Z, int ldz, unsigned ortho) {
  const int lane = threadIdx.x & 31;
  if (lane == 0) tri_factor_shifted<R>(d, e, n, lam, sc, piv);
  __syncwarp();
  for (int it = 0; it < iters; ++it) {
    if (lane == 0) tri_solve_factored<R>(n, z, sc, piv);
    __syncwarp();
    for (unsigned bits = ortho; bits; bits &= bits - 1) {
      const int j = __ffs(bits) - 1;
      R sdot = R(0);
      for (int i = lane; i < n; i += 32) sdot += Z[j * ldz + i] * z[i];
      sdot = warp_sum(sdot);
      for (int i = lane; i < n; i += 32) z[i] -= sdot * Z[j * ldz + i];
      __syncwarp();
    }
    R nn = R(0);
    for (int i = lane; i < n; i += 32) nn += z[i] * z[i];
    nn = warp_sum(nn);
    const R inv = nn > R(0) ? R(1) / sqrt(nn) : R(0);
    for (int i = lane; i < n; i += 32) z[i] *= inv;
    __syncwarp();
  }
}

// The same count without divisions (FP64 division is a long sequence on this part's few
// FP64 units): the leading principal minors p_i of T - x I follow
// p_0 = 1, p_1 = d_0 - x, p_{i+1} = (d_i - x) p_i - e_{i-1}^2 p_{i-1}, and the LDL^T pivot
// q_i = p_i / p_{i-1} is negative exactly when p_i and p_{i-1} differ in sign.  e2 holds
// e_i^2.  After every step the binary exponent of the larger of |p_{i-1}|, |p_i| is checked
// with integer operations and the pair is rescaled by a power of two when it has left
// [2^-400, 2^400] (one step cannot overflow from there unless the Gershgorin radius exceeds
// 2^300); an exact zero minor is replaced by -2^-60 times its predecessor (a tiny negative
// pivot, the role pivmin plays above; relative, so that it cannot underflow).
__device__ inline int sturm_count_prod(const double* d, const double* e2, int n, double x) {
  double pm = 1.0, p = d[0] - x;
  if (p == 0.0) p = -0x1p-60;
  int cnt = p < 0.0;
  for (int i = 1; i < n; ++i) {
    double pn = fma(d[i] - x, p, -e2[i - 1] * pm);
    if (pn == 0.0) pn = -0x1p-60 * p;
    cnt += (pn < 0.0) != (p < 0.0);
    pm = p;
    p = pn;
    // rescale both by a power of two when the larger leaves [2^-400, 2^400]
    const int ex = ((__double2hiint(fmax(fabs(p), fabs(pm))) >> 20) & 0x7FF) - 1023;
    if (ex > 400 || ex < -400) {
      p = ldexp(p, -ex);
      pm = ldexp(pm, -ex);
    }
  }
  return cnt;
}

// doubles of workspace for an n x n problem with nroots roots
size_t tda_work_doubles(int n, int nroots);
// lowest nroots eigenvalues (ascending) of the symmetric n x n matrix held in the first
// n^2 doubles of `work` (overwritten; tda_work_doubles(n, nroots) in all) and, if X is not
// null, the eigenvectors [nroots][n].  All pointers are device memory.
int sym_eig_lowest(rsx_ctx* c, double* work, int n, int nroots, double* omega, double* X, cudaStream_t s);
// A = diag(ev_a - eo_i) + dm K - Kd (Kd may be null), lowest nroots eigenvalues (ascending) and,
// if X is not null, eigenvectors [nroots][n].  All pointers are device memory.
// spin-polarised form: A = diag(de per spin) + K - blockdiag(Kda, Kdb) over the alpha then
// beta transitions (nob * nvb may be 0; Kda / Kdb may be null)
int uhf_tda_solve(rsx_ctx* c, const double* eoa, int noa, const double* eva, int nva, const double* eob, int nob,
                  const double* evb, int nvb, const double* K, const double* Kda, const double* Kdb, int nroots,
                  double* omega, double* X, double* work, cudaStream_t s);
int tda_solve(rsx_ctx* c, const double* eo, int no, const double* ev, int nv, const double* K, const double* Kd,
              double dm, int nroots, double* omega, double* X, double* work, cudaStream_t s);
}  // namespace rsx
