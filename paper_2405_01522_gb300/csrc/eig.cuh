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

// doubles of workspace for an n x n problem with nroots roots
size_t tda_work_doubles(int n, int nroots);
// lowest nroots eigenvalues (ascending) of the symmetric n x n matrix held in the first
// n^2 doubles of `work` (overwritten; tda_work_doubles(n, nroots) in all) and, if X is not
// null, the eigenvectors [nroots][n].  All pointers are device memory.
int sym_eig_lowest(rsx_ctx* c, double* work, int n, int nroots, double* omega, double* X, cudaStream_t s);
// A = diag(ev_a - eo_i) + dm K - Kd (Kd may be null), lowest nroots eigenvalues (ascending) and,
// if X is not null, eigenvectors [nroots][n].  All pointers are device memory.
int tda_solve(rsx_ctx* c, const double* eo, int no, const double* ev, int nv, const double* K, const double* Kd,
              double dm, int nroots, double* omega, double* X, double* work, cudaStream_t s);
}  // namespace rsx
