// FP64 Tamm-Dancoff eigen-solve on the device (eig.cu).
#pragma once
#include <cuda_runtime.h>

struct rsx_ctx;

namespace rsx {
// doubles of workspace for an n x n problem with nroots roots
size_t tda_work_doubles(int n, int nroots);
// A = diag(ev_a - eo_i) + dm K - Kd (Kd may be null), lowest nroots eigenvalues (ascending) and,
// if X is not null, eigenvectors [nroots][n].  All pointers are device memory.
int tda_solve(rsx_ctx* c, const double* eo, int no, const double* ev, int nv, const double* K, const double* Kd,
              double dm, int nroots, double* omega, double* X, double* work, cudaStream_t s);
}  // namespace rsx
