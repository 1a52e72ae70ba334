"""The register DFT codelets of the line transforms, built for the host and checked
against numpy's FFT: every length and sign the kernels instantiate, the complete
transforms and the pruned ones (zero upper half of the inputs, lower half of the outputs
kept), in double and in float.  The pair Poisson solve of Eq. 2 (Sec. 3.1) is built from
these transforms, so a wrong constant or index map in one of them shows up here first."""
import os
import subprocess

import numpy as np
import pytest

from paper_2405_01522_gb300 import build as pkg_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2405_01522_gb300", "csrc")

FULL = [2, 3, 4, 5, 6, 7, 8, 10, 12, 14, 16, 24]
HALF = [4, 6, 8, 10, 12, 14, 16, 24]

PROGRAM = r"""
#include <cstdio>
#include <cmath>
#include "fft_small.cuh"
using namespace rsx;

template <typename R> Cx<R> inp(int n, int j) {
  return cx<R>(R(std::sin(1.3 * j + 0.7 * n) + 0.25 * j), R(std::cos(0.9 * j - 0.2 * n)));
}
template <typename R> void put(const char* tag, int n, int s, const Cx<R>* o, int m) {
  std::printf("%s %d %d %d", tag, n, s, (int)sizeof(R));
  for (int k = 0; k < m; ++k) std::printf(" %.17g %.17g", (double)o[k].x, (double)o[k].y);
  std::printf("\n");
}
template <int N, int S, typename R> void full() {
  Cx<R> v[N];
  for (int j = 0; j < N; ++j) v[j] = inp<R>(N, j);
  Dft<N, S>::run(v);
  put<R>("full", N, S, v, N);
}
template <int A, int S, typename R> void half() {
  Cx<R> v[A], o[A];
  for (int j = 0; j < A; ++j) v[j] = inp<R>(A, j);
  DftHalfIn<A, S>::run(v, o);     // reads v[0 .. A/2) only
  put<R>("halfin", A, S, o, A);
  DftHalfOut<A, S>::run(v, o);    // forms out[0 .. A/2)
  put<R>("halfout", A, S, o, A / 2);
}
template <typename R> void all() {
#define F(N) full<N, -1, R>(); full<N, 1, R>();
  F(2) F(3) F(4) F(5) F(6) F(7) F(8) F(10) F(12) F(14) F(16) F(24)
#undef F
#define H(A) half<A, -1, R>(); half<A, 1, R>();
  H(4) H(6) H(8) H(10) H(12) H(14) H(16) H(24)
#undef H
}
int main() {
  all<double>();
  all<float>();
  return 0;
}
"""


def _inputs(n):
    j = np.arange(n)
    return (np.sin(1.3 * j + 0.7 * n) + 0.25 * j) + 1j * np.cos(0.9 * j - 0.2 * n)


def _dft(x, s):
    n = len(x)
    return np.fft.fft(x) if s < 0 else np.fft.ifft(x) * n


@pytest.fixture(scope="module")
def codelet_output(tmp_path_factory):
    d = tmp_path_factory.mktemp("codelets")
    src = os.path.join(d, "codelets.cu")
    exe = os.path.join(d, "codelets")
    with open(src, "w") as f:
        f.write(PROGRAM)
    r = subprocess.run([pkg_build.NVCC, "-O2", "-std=c++17", "-I", CSRC, src, "-o", exe],
                       capture_output=True, text=True)
    if r.returncode != 0:
        pytest.fail("host build of the codelets failed:\n" + r.stderr[-4000:])
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    rows = {}
    for line in out.strip().splitlines():
        tag, n, s, size, *vals = line.split()
        z = np.array(vals, dtype=float).reshape(-1, 2)
        rows[(tag, int(n), int(s), int(size))] = z[:, 0] + 1j * z[:, 1]
    return rows


@pytest.mark.parametrize("size,tol", [(8, 1e-13), (4, 3e-6)])
def test_complete_transforms(codelet_output, size, tol):
    for n in FULL:
        for s in (-1, 1):
            ref = _dft(_inputs(n), s)
            got = codelet_output[("full", n, s, size)]
            assert np.max(np.abs(got - ref)) <= tol * np.max(np.abs(ref)), (n, s, size)


@pytest.mark.parametrize("size,tol", [(8, 1e-13), (4, 3e-6)])
def test_pruned_transforms(codelet_output, size, tol):
    for a in HALF:
        x = _inputs(a)
        for s in (-1, 1):
            lower = x.copy()
            lower[a // 2:] = 0          # the padded half of a line: inputs that are zero
            ref_in = _dft(lower, s)
            got_in = codelet_output[("halfin", a, s, size)]
            assert np.max(np.abs(got_in - ref_in)) <= tol * np.max(np.abs(ref_in)), ("in", a, s, size)
            ref_out = _dft(x, s)[: a // 2]   # the outputs a transform back onto the box keeps
            got_out = codelet_output[("halfout", a, s, size)]
            assert np.max(np.abs(got_out - ref_out)) <= tol * np.max(np.abs(ref_out)), ("out", a, s, size)
