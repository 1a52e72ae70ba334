// Pass 2 of the pair Poisson solve with the line transforms split 8 lanes x 2A.
//
// Same work as k_pass2 (per (pair, kx) plane: y forward on the nz rows, z forward x
// kernel x z inverse on the My columns, y inverse keeping y < ny), but a line of length
// M = 16 A = 8 x 2A is transformed by 8 lanes instead of 16:
//   stage 1  lane t (< 8) holds x[t + 8 a], a < A (the non-zero half), does the 2A-point
//            DFT over a in registers, multiplies by w_M^{-t k1} and stores row k1 of the
//            line's scratch;
//   stage 2  lane s does the 8-point DFTs over t of rows k1 = s + 8 j (j < 2A / 8), giving
//            X[k1 + 2A k2].
// With 16 lanes x A the 16-point stage keeps only A of 16 lanes busy (12 of 16 at
// M = 192); here both stages keep all lanes busy (2A / 8 rows per lane).  The inverse
// runs the same steps backwards and keeps the outputs z < nz (y < ny) only.
// FP32, A in {4, 8, 12} (M = 64, 128, 192: 2A a multiple of 8).
#pragma once
#include "poisson_kernels.cuh"

namespace rsx {

// Line scratch: 2A rows of 8 complex (64 bytes).  Row k1 of line l is stored at physical
// row k1 ^ (l & 1), and the four 16-byte chunks of physical row r are XOR-swizzled by
// (r >> 1) & 3.  Then (i) the two lines of a half-warp (l even, l + 1) put the same row in
// opposite halves of the banks, so the 8-byte accesses of stage 1 are conflict-free, and
// (ii) the eight lanes of a line reading rows s + 8 j as 16-byte chunks in stage 2 hit
// eight distinct bank groups.
__device__ __forceinline__ int l8_off(int r, int t) { return r * 8 + 2 * ((t >> 1) ^ ((r >> 1) & 3)) + (t & 1); }

__device__ __forceinline__ void l8_load_row(Cx<float> (&u)[8], const Cx<float>* sc, int r) {
  const int sw = (r >> 1) & 3;
  const float4* rp = reinterpret_cast<const float4*>(sc + r * 8);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float4 v = rp[q ^ sw];
    u[2 * q] = cx<float>(v.x, v.y);
    u[2 * q + 1] = cx<float>(v.z, v.w);
  }
}

__device__ __forceinline__ void l8_store_row(Cx<float>* sc, int r, const Cx<float> (&u)[8]) {
  const int sw = (r >> 1) & 3;
  float4* rp = reinterpret_cast<float4*>(sc + r * 8);
#pragma unroll
  for (int q = 0; q < 4; ++q) rp[q ^ sw] = make_float4(u[2 * q].x, u[2 * q].y, u[2 * q + 1].x, u[2 * q + 1].y);
}

// Row pitch of the work plane, M + 2 complex: every row starts on a 16-byte boundary (the
// next plane is prefetched with 16-byte copies).  Bank pairs (8-byte units) of an access
// are then 2 row + column mod 16: the two lines of a half-warp take rows 4 apart (the
// 8 consecutive columns of a row access land 8 bank pairs apart) and z columns 1 apart
// (the 8 rows t + 8 a of a column access fall on even bank pairs for one line, odd ones
// for the other).
template <int A>
__host__ __device__ constexpr int l8_pitch() { return 16 * A + 2; }

// the next plane P (NB x NB complex, contiguous) into the upper halves of D's rows,
// columns [NB, 2 NB), as 16-byte cp.async copies
template <int A, int NT>
__device__ __forceinline__ void l8_prefetch_plane(Cx<float>* D, const Cx<float>* P) {
  constexpr int NB = 8 * A, DP = l8_pitch<A>(), G = NB / 2;   // granules (2 complex) per row
  for (int i = threadIdx.x; i < NB * G; i += NT) {
    const int z = i / G, y = 2 * (i - z * G);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(D + z * DP + NB + y)),
                 "l"(P + z * NB + y)
                 : "memory");
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

// This lane's stage-1 twiddles w_M^{-t k1}, k1 < 2A: held in registers (TWS = false) or
// read from a shared table [k1][t] (TWS = true: 46 fewer live registers at A = 12; the
// eight lanes of a line read 64 contiguous bytes, the lines of a warp the same ones).
template <int A, bool TWS>
struct L8Tw {
  Cx<float> reg[TWS ? 1 : 2 * A];
  const Cx<float>* sh;
  int t;
  __device__ __forceinline__ void init(const Cx<float>* __restrict__ tw8, const Cx<float>* shared_tab, int t_) {
    t = t_;
    sh = shared_tab;
    if constexpr (!TWS) {
#pragma unroll
      for (int k1 = 1; k1 < 2 * A; ++k1) reg[k1] = tw8[t * 2 * A + k1];
    }
  }
  __device__ __forceinline__ Cx<float> operator[](int k1) const {
    if constexpr (TWS) return sh[k1 * 8 + t];
    else return reg[k1];
  }
};

// stage 1 forward: inputs src[(t + 8 a) * es], a < A (the rest of the line is zero)
template <int A, class TW>
__device__ __forceinline__ void l8_stage1_fwd(const Cx<float>* src, int es, int t, int par, const TW& tw,
                                              Cx<float>* sc) {
  constexpr int A2 = 2 * A;
  Cx<float> v[A], x[A2];
#pragma unroll
  for (int a = 0; a < A; ++a) v[a] = src[(t + 8 * a) * es];
  DftHalfIn<A2, -1>::run(v, x);
#pragma unroll
  for (int k1 = 1; k1 < A2; ++k1) x[k1] = cmul(x[k1], tw[k1]);
#pragma unroll
  for (int k1 = 0; k1 < A2; ++k1) sc[l8_off(k1 ^ par, t)] = x[k1];
}

// stage 1 inverse: rows k1 of the scratch (lane t's column), conjugate twiddles, 2A-point
// inverse DFT keeping outputs a < A, written to dst[(t + 8 a) * es]
template <int A, class TW>
__device__ __forceinline__ void l8_stage1_inv(Cx<float>* dst, int es, int t, int par, const TW& tw,
                                              const Cx<float>* sc) {
  constexpr int A2 = 2 * A;
  Cx<float> r[A2], o[A];
#pragma unroll
  for (int k1 = 0; k1 < A2; ++k1) r[k1] = sc[l8_off(k1 ^ par, t)];
#pragma unroll
  for (int k1 = 1; k1 < A2; ++k1) r[k1] = cmul(r[k1], conj(tw[k1]));
  DftHalfOut<A2, 1>::run(r, o);
#pragma unroll
  for (int a = 0; a < A; ++a) dst[(t + 8 * a) * es] = o[a];
}

// this lane's kernel factors of one folded column |ky| (lane order: kz = (t + 8 j) + 2A k2,
// j < 2A / 8, k2 < 8), 2 x 2A / 8 16-byte loads
template <int J>
__device__ __forceinline__ void l8_load_factors(float4 (&fac)[2 * J], const float* __restrict__ src) {
  const float4* vq = reinterpret_cast<const float4*>(src);
#pragma unroll
  for (int i = 0; i < 2 * J; ++i) fac[i] = __ldg(vq + i);
}

// z forward, kernel multiply, z inverse of one column (col = D + ky, row pitch l8_pitch)
template <int A, class TW>
__device__ __forceinline__ void l8_z_column(Cx<float>* col, int t, int par, unsigned lmask, const TW& tw,
                                            Cx<float>* sc, const float4 (&fac)[2 * (2 * A / 8)]) {
  constexpr int A2 = 2 * A, J = A2 / 8, DP = l8_pitch<A>();
  l8_stage1_fwd<A>(col, DP, t, par, tw, sc);
  __syncwarp(lmask);
#pragma unroll
  for (int j = 0; j < J; ++j) {
    const int r = (t + 8 * j) ^ par;
    Cx<float> u[8];
    l8_load_row(u, sc, r);
    Dft<8, -1>::run(u);
    const float4 m0 = fac[2 * j], m1 = fac[2 * j + 1];
    u[0] = cscale(u[0], m0.x);
    u[1] = cscale(u[1], m0.y);
    u[2] = cscale(u[2], m0.z);
    u[3] = cscale(u[3], m0.w);
    u[4] = cscale(u[4], m1.x);
    u[5] = cscale(u[5], m1.y);
    u[6] = cscale(u[6], m1.z);
    u[7] = cscale(u[7], m1.w);
    Dft<8, 1>::run(u);
    l8_store_row(sc, r, u);   // row r is read and written by this lane only
  }
  __syncwarp(lmask);
  l8_stage1_inv<A>(col, DP, t, par, tw, sc);
  __syncwarp(lmask);
}

// one (pair, kx) plane; D: (nz x My) work plane, row pitch l8_pitch, input rows staged in
// columns [ny, 2 ny) (prefetched); the y inverse writes the result to the plane P in
// global memory
template <int A, int NT, class TW>
__device__ __forceinline__ void l8_plane(Cx<float>* P, int kx, int Hy, const float* __restrict__ vl8, Cx<float>* D,
                                         Cx<float>* sc, int lrow, int litem, int t, int par, unsigned lmask, const TW& tw,
                                         const Cx<float>* Pnext) {
  constexpr int A2 = 2 * A, J = A2 / 8, M = 16 * A, NB = 8 * A, DP = l8_pitch<A>(), NL = NT / 8;
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  __syncthreads();
  // ---- y forward of the nz rows (input columns [NB, 2 NB), outputs all M columns)
  for (int z = lrow; z < NB; z += NL) {
    Cx<float>* row = D + z * DP;
    l8_stage1_fwd<A>(row + NB, 1, t, par, tw, sc);
    __syncwarp(lmask);
#pragma unroll
    for (int j = 0; j < J; ++j) {
      const int k1 = t + 8 * j;
      Cx<float> u[8];
      l8_load_row(u, sc, k1 ^ par);
      Dft<8, -1>::run(u);
#pragma unroll
      for (int k2 = 0; k2 < 8; ++k2) row[k1 + A2 * k2] = u[k2];
    }
    __syncwarp(lmask);
  }
  __syncthreads();
  // ---- z forward, kernel multiply, z inverse on the M columns ky.  Columns ky and M - ky
  // use the same kernel factors (the table is folded in |ky|): a line takes them as one
  // item (item 0: the two unpaired columns 0 and M / 2), 2 columns per item.  The factors
  // of a column's row |ky| are loaded one column ahead (the DFTs of the column before cover
  // the loads' latency): fa holds the current row, fb the next one.
  const float* vrow = vl8 + (size_t)kx * Hy * M + t * A2;
  const int ncol = 2 * ((M / 2 - litem + NL - 1) / NL);
  float4 fa[2 * J], fb[2 * J];
  if (ncol > 0) l8_load_factors<J>(fa, vrow + (size_t)litem * M);   // lines without an item load nothing
  for (int c = 0; c < ncol; ++c) {
    const int it = litem + NL * (c >> 1);
    const int col = (c & 1) ? (it == 0 ? M / 2 : M - it) : it;
    // the next column's row differs at the start of every item and inside item 0
    const int itn = litem + NL * ((c + 1) >> 1);
    const int rown = ((c + 1) & 1) ? (itn == 0 ? M / 2 : itn) : itn;
    const bool next = c + 1 < ncol && (((c + 1) & 1) == 0 || itn == 0);
    if (next) l8_load_factors<J>(fb, vrow + (size_t)rown * M);
    l8_z_column<A>(D + col, t, par, lmask, tw, sc, fa);
    if (next) {
#pragma unroll
      for (int i = 0; i < 2 * J; ++i) fa[i] = fb[i];
    }
  }
  __syncthreads();
  // ---- y inverse of the nz rows, keeping y < ny: the rows go from registers straight to
  // the plane in global memory
  for (int z = lrow; z < NB; z += NL) {
    Cx<float>* row = D + z * DP;
#pragma unroll
    for (int j = 0; j < J; ++j) {
      const int k1 = t + 8 * j;
      Cx<float> u[8];
#pragma unroll
      for (int k2 = 0; k2 < 8; ++k2) u[k2] = row[k1 + A2 * k2];
      Dft<8, 1>::run(u);
      l8_store_row(sc, k1 ^ par, u);
    }
    __syncwarp(lmask);
    l8_stage1_inv<A>(P + z * NB, 1, t, par, tw, sc);
    __syncwarp(lmask);
  }
  __syncthreads();   // every read of D's upper halves is done
  if (Pnext) l8_prefetch_plane<A, NT>(D, Pnext);
}

// Persistent grid over the work items (pair, kx); the plane lives in shared memory and the
// next plane is prefetched into the upper halves of its rows behind the current one.
// tw8[t][k1] = w_M^{-t k1} (t < 8, k1 < 2A); vl8: the kernel table in this kernel's lane
// order, [kx][|ky|][s][j][k2] with kz = (s + 8 j) + 2A k2.
// Shared memory: [twiddle table A2 x 8] [line scratch NL x A2 x 8] [plane NB x l8_pitch].
template <int A, int NT, bool TWS>
__global__ void __launch_bounds__(NT, 1) k_pass2_l8(Geom g, int nq, Cx<float>* __restrict__ inter,
                                                    const Cx<float>* __restrict__ tw8, const float* __restrict__ vl8) {
  constexpr int A2 = 2 * A, M = 16 * A, NB = 8 * A, NL = NT / 8;
  static_assert(NL % 16 == 0, "lines per CTA: a multiple of 16 (line pairing)");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Cx<float>* twtab = reinterpret_cast<Cx<float>*>(smem_raw);
  Cx<float>* scr = twtab + A2 * 8;
  Cx<float>* D = scr + NL * A2 * 8;
  const int lane = threadIdx.x & 31, t = lane & 7, line = threadIdx.x >> 3, par = line & 1;
  const unsigned lmask = 0xFFu << (lane & 24);
  // the two lines of a half-warp (line 2k, 2k + 1) take rows 4 apart and z items (columns)
  // 1 apart, see l8_pitch
  const int k = (line >> 1) & 7;
  const int lrow = (line & ~15) | (k & 3) | ((k & 4) << 1) | ((line & 1) << 2);
  const int litem = line;
  Cx<float>* sc = scr + line * A2 * 8;
  if constexpr (TWS) {
    for (int i = threadIdx.x; i < A2 * 8; i += NT) {   // [k1][t] from the table's [t][k1]
      const int k1 = i >> 3, tt = i & 7;
      twtab[i] = tw8[tt * A2 + k1];
    }
    __syncthreads();
  }
  L8Tw<A, TWS> tw;
  tw.init(tw8, twtab, t);
  const int Hy = M / 2 + 1;
  const int nplane = NB * NB;
  const int nwork = nq * g.Hx;
  auto plane_ptr = [&](int w) {
    const int ql = w / g.Hx, kx = w - ql * g.Hx;
    return inter + (size_t)ql * g.inter_elems() + (size_t)kx * nplane;
  };
  if ((int)blockIdx.x < nwork) l8_prefetch_plane<A, NT>(D, plane_ptr(blockIdx.x));
  for (int w = blockIdx.x; w < nwork; w += gridDim.x) {
    const int kx = w % g.Hx;
    const int wn = w + (int)gridDim.x;
    l8_plane<A, NT>(plane_ptr(w), kx, Hy, vl8, D, sc, lrow, litem, t, par, lmask, tw,
                    wn < nwork ? plane_ptr(wn) : nullptr);
  }
}

template <int A>
inline size_t pass2_l8_smem(int nt) {
  return sizeof(Cx<float>) * ((size_t)2 * A * 8 + (size_t)(nt / 8) * 2 * A * 8 + (size_t)(8 * A) * l8_pitch<A>());
}

}  // namespace rsx
