"""bench.py's flop counts of the register DFT codelets (the numerator of the pass-2 ALU
roofline) against the codelets themselves: the header is built for the host with a
scalar type that counts its additions and multiplications (a fused multiply-add counts
as both, as in the 2-flops-per-FMA peak), every codelet the kernels use is run once, and
the counts must equal the model's, so that the reported flops are the ones the code does."""
import os
import subprocess

import pytest

import bench
from paper_2405_01522_gb300 import build as pkg_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2405_01522_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include <cmath>
#include "fft_small.cuh"
using namespace rsx;

static long g_flops = 0;
struct F {
  double v;
  __host__ __device__ F() : v(0.0) {}
  __host__ __device__ F(double x) : v(x) {}
};
__host__ __device__ inline void count(int n) {
#ifndef __CUDA_ARCH__
  g_flops += n;
#endif
}
__host__ __device__ inline F operator+(F a, F b) { count(1); return F(a.v + b.v); }
__host__ __device__ inline F operator-(F a, F b) { count(1); return F(a.v - b.v); }
__host__ __device__ inline F operator-(F a) { return F(-a.v); }
__host__ __device__ inline F operator*(F a, F b) { count(1); return F(a.v * b.v); }
__host__ __device__ inline F fma(F a, F b, F c) { count(2); return F(a.v * b.v + c.v); }

template <int N> void full() {
  Cx<F> v[N];
  for (int j = 0; j < N; ++j) v[j] = cx<F>(F(j + 1.0), F(0.5 * j));
  g_flops = 0;
  Dft<N, -1>::run(v);
  std::printf("full %d %ld\n", N, g_flops);
}
template <int A> void half() {
  Cx<F> v[A], o[A];
  for (int j = 0; j < A; ++j) v[j] = cx<F>(F(j + 1.0), F(0.5 * j));
  g_flops = 0;
  DftHalfIn<A, -1>::run(v, o);
  std::printf("halfin %d %ld\n", A, g_flops);
  g_flops = 0;
  DftHalfOut<A, 1>::run(v, o);
  std::printf("halfout %d %ld\n", A, g_flops);
}
int main() {
  full<2>(); full<3>(); full<4>(); full<5>(); full<6>(); full<7>(); full<8>(); full<10>();
  full<12>(); full<14>(); full<16>(); full<24>();
  half<4>(); half<6>(); half<8>(); half<10>(); half<12>(); half<14>(); half<16>(); half<24>();
  return 0;
}
"""


@pytest.fixture(scope="module")
def counts(tmp_path_factory):
    d = tmp_path_factory.mktemp("flops")
    src, exe = os.path.join(d, "flops.cu"), os.path.join(d, "flops")
    with open(src, "w") as f:
        f.write(PROGRAM)
    r = subprocess.run([pkg_build.NVCC, "-O1", "-std=c++17", "-I", CSRC, src, "-o", exe],
                       capture_output=True, text=True)
    if r.returncode != 0:
        pytest.fail("host build of the counting codelets failed:\n" + r.stderr[-4000:])
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    res = {}
    for line in out.strip().splitlines():
        kind, n, c = line.split()
        res[(kind, int(n))] = int(c)
    return res


def test_complete_dft_flops(counts):
    got = {n: counts[("full", n)] for n in (2, 3, 4, 5, 6, 7, 8, 10, 12, 14, 16, 24)}
    want = {n: bench.DFT_FLOPS[n] for n in got}
    assert got == want


def test_pruned_dft_flops(counts):
    for a in (4, 6, 8, 10, 12, 14, 16, 24):
        assert counts[("halfin", a)] == bench._half_in(a), ("half in", a)
        assert counts[("halfout", a)] == bench._half_out(a), ("half out", a)
