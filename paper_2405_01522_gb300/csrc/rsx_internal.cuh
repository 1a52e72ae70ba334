// Internal declarations shared by the CUDA translation units of librsx.
#pragma once
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

#include "fft_small.cuh"

namespace rsx {

// Line transforms: an FFT of length M = 16 * A along one axis is done by a half-warp
// (16 lanes) in two register stages: A-point DFTs over stride-16 inputs, a twiddle,
// a transpose through shared memory, then 16-point DFTs (see poisson_kernels.cuh).
constexpr int kLinesPerCta = 16;      // 8 warps x 2 half-warps
constexpr int kThreads = 256;
constexpr int kScrPitch = 17;         // scratch row pitch (complex), avoids bank conflicts
constexpr int kRowsPerCta = 32;       // rows (y) per CTA in the x passes

// Which pair densities a batch holds and which pairs each output accumulates.
//   PROD: pair q = b * na + a  has density A[a] * B[b]  (exchange: A = phi, B = psi;
//         Casida: A = virtual, B = occupied, so q = i * n_virt + a);
//         output p (an element of B) accumulates pairs q = p * na + a, partner A[a].
//   SYM:  unique pairs a <= b of one set A (upper triangle, row-major);
//         output p accumulates every pair containing p, partner the other orbital.
//   LIST: pairs and outputs of several independent orbital sets (the uneven batch):
//         pair q has density plist[2q] * plist[2q + 1]; output p is orbital i of a set of
//         nocc orbitals phi whose symmetric pairs start at q0 (SYM order within the set),
//         accumulates -sum_e phi_e V[phi_i phi_e] and is written to olist[p].out.
enum PairMode { kProd = 0, kSym = 1, kList = 2 };

template <typename R>
struct OutRef {
  const R* phi;   // the output's orbital set [nocc][N]
  R* out;         // the output array [N]
  int nocc, i, q0, pad;
};

template <typename R>
struct PairMap {
  int mode;
  const R* A;
  const R* B;
  int na, nb;
  size_t N;  // points per orbital
  const R* const* plist = nullptr;   // LIST: two orbital pointers per pair
  const OutRef<R>* olist = nullptr;  // LIST: one entry per output

  __device__ __forceinline__ void pair(int q, const R*& f1, const R*& f2) const {
    if (mode == kProd) {
      const int b = q / na, a = q - b * na;
      f1 = A + (size_t)a * N;
      f2 = B + (size_t)b * N;
    } else if (mode == kSym) {
      int i = 0, rem = q;
      while (rem >= na - i) { rem -= na - i; ++i; }
      f1 = A + (size_t)i * N;
      f2 = A + (size_t)(i + rem) * N;
    } else {
      f1 = plist[2 * q];
      f2 = plist[2 * q + 1];
    }
  }
  __device__ __forceinline__ int nentries(int p) const { return mode == kList ? olist[p].nocc : na; }
  // entry e of output p: pair index and the orbital multiplied into the accumulator
  __device__ __forceinline__ void entry(int p, int e, int& q, const R*& partner) const {
    if (mode == kProd) {
      q = p * na + e;
      partner = A + (size_t)e * N;
    } else if (mode == kSym) {
      const int i = p < e ? p : e, j = p < e ? e : p;
      q = i * na - i * (i - 1) / 2 + (j - i);
      partner = A + (size_t)e * N;
    } else {
      const OutRef<R> o = olist[p];
      const int i = o.i < e ? o.i : e, j = o.i < e ? e : o.i;
      q = o.q0 + i * o.nocc - i * (i - 1) / 2 + (j - i);
      partner = o.phi + (size_t)e * N;
    }
  }
  // the array output p (local index pl of a launch starting at out) is written to
  __device__ __forceinline__ R* out_row(int p, R* out, int pl) const {
    return mode == kList ? olist[p].out : out + (size_t)pl * N;
  }
};

struct Geom {
  int nz, ny, nx;     // box
  int Mz, My, Mx;     // padded (2n)
  int Az, Ay, Ax;     // M / 16
  int Hx;             // Mx / 2 + 1 (half spectrum along x)
  int p2_threads;     // tuning: threads per CTA of the y/z pass (256 or 512)
  int p1_group;       // tuning: pass-1 block order (0: pair-major; G > 0: pairs fastest in groups of G)
  int p2_global;      // tuning: 1 = the y/z pass keeps its work plane in global scratch even where
                      // shared memory would hold it (0 = shared memory whenever it fits)
  int p2_lanes;       // tuning: lanes per line of the y/z transforms, 16 (16 x A) or 8 (8 x 2A;
                      // FP32, A a multiple of 4, shared-memory plane)
  int* dbg = nullptr; // bounds-checked builds: the status word an out-of-range index is reported in
  int dbg_nq = 0;     // bounds-checked builds: pairs the launch's intermediate holds (0: unknown)
  __host__ __device__ size_t N() const { return (size_t)nz * ny * nx; }
  __host__ __device__ size_t inter_elems() const { return (size_t)Hx * nz * ny; }  // complex per pair
};

// Bounds-checked builds (-DRSX_CHECKED, `librsx_checked.so`): the FFT passes test the
// indices they compute against the arrays they address, report the first violation as
// RSX_EBOUNDS in the context's status word and skip the access.  In the normal build the
// test is the constant true and compiles away.
#ifdef RSX_CHECKED
__device__ inline bool in_range_checked(int* dbg, long long i, long long n) {
  if (i >= 0 && i < n) return true;
  if (dbg) atomicMax(dbg, 7);   // RSX_EBOUNDS
  return false;
}
#define RSX_IN_RANGE(g, i, n) ::rsx::in_range_checked((g).dbg, (long long)(i), (long long)(n))
#else
#define RSX_IN_RANGE(g, i, n) true
#endif

// ---- launchers (defined per precision in poisson_f32.cu / poisson_f64.cu)
template <typename R>
cudaError_t launch_pass1(const Geom& g, const PairMap<R>& pm, int q0, int nq, Cx<R>* inter,
                         const Cx<R>* twx, cudaStream_t s);
// tw8 / vl8: twiddles and lane-order kernel table of the 8-lane split (FP32; NULL: the
// 16-lane kernel runs whatever g.p2_lanes says)
template <typename R>
cudaError_t launch_pass2(const Geom& g, int nq, Cx<R>* inter, const Cx<R>* twy, const Cx<R>* twz,
                         const R* vhat, const float* vhat_lanes, R* gscratch, int grid, cudaStream_t s,
                         const Cx<float>* tw8 = nullptr, const float* vl8 = nullptr);
// true when the 8-lane y/z kernel serves geometry g (FP32) with these tables
bool pass2_l8_active(const Geom& g, const void* tw8, const void* vl8);
template <typename R>
cudaError_t launch_pass3(const Geom& g, const PairMap<R>& pm, int q0, int p0, int np, int pot, const Cx<R>* inter,
                         const Cx<R>* twx, R* out, cudaStream_t s);
// forward y/z transform of each pair plane, weighted by sqrt(w_G vhat(G) h^3) and split
// into bf16 hi/lo of the K panel, tile-major [ld/64][nrb][128][64] (nrb row blocks of 128)
cudaError_t launch_spectrum_f32(const Geom& g, int nq, const Cx<float>* inter, const Cx<float>* twy,
                                const Cx<float>* twz, const float* wsq, uint16_t* hi,
                                uint16_t* lo, size_t ld, int nrb, cudaStream_t s);
// panel weights wsq = sqrt(w_kx vhat h^3) on the folded half spectrum (Hx, My/2+1, Mz/2+1)
cudaError_t launch_spectrum_weights(const Geom& g, const float* vhat, float h3, float* wsq, cudaStream_t s);
template <typename R>
size_t pass2_smem_bytes(const Geom& g, bool* fits);
template <typename R>
int pass2_occupancy(const Geom& g);  // resident pass-2 CTAs per SM (shared-memory variant)

bool axis_supported(int A);

}  // namespace rsx
