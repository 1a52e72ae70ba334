// Pair Poisson solve by pruned, zero-padded FFT convolution: the three passes.
//
// The potential of a pair density rho = f1 f2 on the box (nz, ny, nx) is
//     V = h^3/N_pad * IDFT( ghat * DFT(rho zero-padded to (2nz, 2ny, 2nx)) )
// restricted to the box (Sec. 3.1: Eq. 2's integral as a Poisson problem at
// O(N log N); padding twice the box makes the periodic convolution the isolated one).
// The solve is split so that only one 1-D transform per pass touches HBM:
//
//   pass 1  x forward, real-to-complex (two rows y, y+1 packed as one complex line),
//           output I[q][kx][z][y], kx in [0, Mx/2]       (Mx/2+1) * nz * ny complex
//   pass 2  per (q, kx): y forward on nz rows, z forward + multiply by vhat + z inverse
//           on My columns, y inverse keeping y < ny; in place on I
//   pass 3  per (output p, z, 32 rows): x inverse complex-to-real of every pair of p's
//           list, keeping x < nx, and  out_p -= partner * V  (Eq. 2's sum over j)
//
// Only nz of the 2nz z-planes and ny of the 2ny rows are non-zero, so the x transforms
// run on nz*ny rows and the y transforms on nz rows per kx; I is 4x smaller than a
// padded half spectrum.  A line of length M = 16 A is transformed by 16 lanes:
// lane t holds x[t + 16 a] (a < A), does an A-point DFT, multiplies by the twiddle
// w_M^{t k1}, and after a shared-memory transpose lane k1 does the 16-point DFT over t,
// giving X[k1 + A k2].  The inverse of that split is the same steps in reverse, so in
// pass 2 the z spectrum never leaves registers between forward, multiply and inverse.
#pragma once
#include <cuda_bf16.h>

#include "rsx_internal.cuh"

namespace rsx {

// round-to-nearest-even f32 -> bf16 bit pattern (finite inputs), and back
__device__ __forceinline__ uint32_t f32_to_bf16_bits(float f) {
  const uint32_t u = __float_as_uint(f);
  return (u + 0x7FFFu + ((u >> 16) & 1u)) >> 16;
}
__device__ __forceinline__ float bf16_bits_to_f32(uint32_t b) { return __uint_as_float(b << 16); }

// ---------------------------------------------------------------------------------
// stage helpers (executed by the 16 lanes t of one half-warp on one line)
// stage 1: v holds x[t + 16 a]; DFT over a, twiddle, store scratch[k1][t]
template <int A, int S, typename R, int PITCH = kScrPitch>
__device__ __forceinline__ void stage1_store(Cx<R> (&v)[A], int t, const Cx<R>* __restrict__ tw,
                                             Cx<R>* sc) {
  Dft<A, S>::run(v);
#pragma unroll
  for (int k1 = 1; k1 < A; ++k1) {
    Cx<R> w = tw[t * A + k1];
    if (S > 0) w.y = -w.y;
    v[k1] = cmul(v[k1], w);
  }
#pragma unroll
  for (int k1 = 0; k1 < A; ++k1) sc[k1 * PITCH + t] = v[k1];
}

// stage 1 for a forward transform whose inputs t + 16 a >= 8 A are zero (even A, the
// padded half of a line of length 16 A): only v[0 .. A/2) are used
template <int A, int S, typename R, int PITCH = kScrPitch>
__device__ __forceinline__ void stage1_store_halfin(const Cx<R>* v, int t, const Cx<R>* __restrict__ tw, Cx<R>* sc) {
  Cx<R> x[A];
  DftHalfIn<A, S>::run(v, x);
#pragma unroll
  for (int k1 = 1; k1 < A; ++k1) {
    Cx<R> w = tw[t * A + k1];
    if (S > 0) w.y = -w.y;
    x[k1] = cmul(x[k1], w);
  }
#pragma unroll
  for (int k1 = 0; k1 < A; ++k1) sc[k1 * PITCH + t] = x[k1];
}

// the same with this lane's twiddles already in registers (w[k1] = w_M^{-t k1}, k1 >= 1)
template <int A, typename R, int PITCH = kScrPitch>
__device__ __forceinline__ void stage1_store_halfin_reg(const Cx<R>* v, int t, const Cx<R> (&w)[A], Cx<R>* sc) {
  Cx<R> x[A];
  DftHalfIn<A, -1>::run(v, x);
#pragma unroll
  for (int k1 = 1; k1 < A; ++k1) x[k1] = cmul(x[k1], w[k1]);
#pragma unroll
  for (int k1 = 0; k1 < A; ++k1) sc[k1 * PITCH + t] = x[k1];
}

// stage 2 load: lane s (< A) gathers its 16 values scratch[s][t]; with an even pitch (FP32
// rows on 16-byte boundaries) as eight 16-byte loads
template <typename R, int PITCH = kScrPitch>
__device__ __forceinline__ void stage2_load(Cx<R> (&u)[16], int s, const Cx<R>* sc) {
  if constexpr (sizeof(R) == 4 && PITCH % 2 == 0) {
    const float4* rp = reinterpret_cast<const float4*>(sc + s * PITCH);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const float4 v = rp[j];
      u[2 * j] = cx<R>(v.x, v.y);
      u[2 * j + 1] = cx<R>(v.z, v.w);
    }
  } else {
#pragma unroll
    for (int j = 0; j < 16; ++j) u[j] = sc[s * PITCH + j];
  }
}
// the transposed store: lane s writes its 16 values to scratch row s
template <typename R, int PITCH = kScrPitch>
__device__ __forceinline__ void stage2_store(const Cx<R> (&u)[16], int s, Cx<R>* sc) {
  if constexpr (sizeof(R) == 4 && PITCH % 2 == 0) {
    float4* rp = reinterpret_cast<float4*>(sc + s * PITCH);
#pragma unroll
    for (int j = 0; j < 8; ++j) rp[j] = make_float4(u[2 * j].x, u[2 * j].y, u[2 * j + 1].x, u[2 * j + 1].y);
  } else {
#pragma unroll
    for (int j = 0; j < 16; ++j) sc[s * PITCH + j] = u[j];
  }
}

// line-scratch pitch (complex) of pass 2: 18 for FP32 where the extra bytes fit (rows on
// 16-byte boundaries for the vector loads above, still conflict-free), else 17
template <typename R>
__host__ __device__ constexpr int p2_pitch(int A) { return (sizeof(R) == 4 && A <= 12) ? 18 : kScrPitch; }

// Row-block staging of the x passes, xs[kx][r] (kRowsPerCta = 32 rows per kx): the rows
// are paired into 16 granules (r, r + 1 with r even) and granule g of row kx sits at
// position g ^ (kx & 15), so that the 16 lanes of a line, which read granule `line` of 16
// different kx, hit distinct banks, and granules move with single 16-byte (FP32) accesses.
__device__ __forceinline__ int xs_idx(int kx, int r) {
  return kx * kRowsPerCta + ((((r >> 1) ^ (kx & 15))) << 1) + (r & 1);
}

// two consecutive complex values (one granule) from / to shared memory
template <typename R>
__device__ __forceinline__ void ld_granule(const Cx<R>* p, Cx<R>& a, Cx<R>& b) {
  if constexpr (sizeof(R) == 4) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    a = cx<R>(v.x, v.y);
    b = cx<R>(v.z, v.w);
  } else {
    a = p[0];
    b = p[1];
  }
}
template <typename R>
__device__ __forceinline__ void st_granule(Cx<R>* p, Cx<R> a, Cx<R> b) {
  if constexpr (sizeof(R) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(a.x, a.y, b.x, b.y);
  } else {
    p[0] = a;
    p[1] = b;
  }
}

// ---------------------------------------------------------------------------------
// pass 1: x forward (r2c via row pairs).  One item = (pair q, plane z, 32 rows).
// pass1_item is the body (all threads of the CTA call it with the same item); the
// intermediate of the pair is at `dst_pair` (layout [kx][z][y]).
template <typename R, int AX>
__device__ __forceinline__ void pass1_item(const Geom& g, const R* f1, const R* f2, int z, int yblk,
                                           Cx<R>* __restrict__ dst_pair, const Cx<R>* __restrict__ twx,
                                           unsigned char* smem_raw) {
  constexpr int L = 16 * AX;
  constexpr int SP = AX * kScrPitch;
  constexpr int H = L / 2 + 1;
  Cx<R>* scr = reinterpret_cast<Cx<R>*>(smem_raw);
  Cx<R>* xs = scr;   // [H][kRowsPerCta], see xs_idx: reuses the line scratch once all lines are done with it
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = lane & 15, line = warp * 2 + (lane >> 4);
  const int y0 = yblk * kRowsPerCta;
  const int ya = y0 + 2 * line, yb = ya + 1;
  Cx<R>* sc = scr + line * SP;
  const size_t plane = (size_t)z * g.ny * g.nx;
  f1 += plane;
  f2 += plane;

  constexpr int AIN = (AX % 2 == 0) ? AX / 2 : AX;   // inputs x >= nx = 8 AX are zero
  Cx<R> v[AX];
#pragma unroll
  for (int a = 0; a < AIN; ++a) {
    const int x = t + 16 * a;
    R re = R(0), im = R(0);
    if (x < g.nx) {
      if (ya < g.ny && RSX_IN_RANGE(g, plane + (size_t)ya * g.nx + x, g.N()))
        re = __ldg(f1 + (size_t)ya * g.nx + x) * __ldg(f2 + (size_t)ya * g.nx + x);
      if (yb < g.ny && RSX_IN_RANGE(g, plane + (size_t)yb * g.nx + x, g.N()))
        im = __ldg(f1 + (size_t)yb * g.nx + x) * __ldg(f2 + (size_t)yb * g.nx + x);
    }
    v[a] = cx<R>(re, im);
  }
  if constexpr (AX % 2 == 0) {
    stage1_store_halfin<AX, -1>(v, t, twx, sc);
  } else {
    stage1_store<AX, -1>(v, t, twx, sc);
  }
  __syncwarp();
  Cx<R> u[16];
  if (t < AX) {
    stage2_load(u, t, sc);
    Dft<16, -1>::run(u);
  }
  __syncwarp();
  if (t < AX) {
#pragma unroll
    for (int k2 = 0; k2 < 16; ++k2) sc[t + AX * k2] = u[k2];  // natural order U[k]
  }
  __syncwarp();
  // split the packed line: X_a(k) = (U(k) + conj U(L-k)) / 2,  X_b(k) = (U(k) - conj U(L-k)) / 2i,
  // into registers first: the staging buffer overwrites every line's scratch
  constexpr int NK = (H + 15) / 16;
  Cx<R> xa[NK], xb[NK];
#pragma unroll
  for (int i = 0; i < NK; ++i) {
    const int k = t + 16 * i;
    if (k < H) {
      const Cx<R> U = sc[k];
      const Cx<R> Um = sc[(L - k) % L];
      xa[i] = cx<R>(R(0.5) * (U.x + Um.x), R(0.5) * (U.y - Um.y));
      xb[i] = cx<R>(R(0.5) * (U.y + Um.y), R(-0.5) * (U.x - Um.x));
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NK; ++i) {
    const int k = t + 16 * i;
    if (k < H) st_granule(xs + xs_idx(k, 2 * line), xa[i], xb[i]);
  }
  __syncthreads();
  const int nrow = min(kRowsPerCta, g.ny - y0);   // a multiple of 8 (ny = 8 A)
  Cx<R>* dst = dst_pair + (size_t)z * g.ny + y0;
  const size_t kstride = (size_t)g.nz * g.ny;
  for (int e = threadIdx.x; e < H * (kRowsPerCta / 2); e += kThreads) {
    const int kx = e / (kRowsPerCta / 2), r = 2 * (e - kx * (kRowsPerCta / 2));
    if (r < nrow && RSX_IN_RANGE(g, (size_t)z * g.ny + y0 + (size_t)kx * kstride + r + 1, g.inter_elems())) {
      Cx<R> a, b;
      ld_granule(xs + xs_idx(kx, r), a, b);
      st_granule(dst + (size_t)kx * kstride + r, a, b);
    }
  }
  __syncthreads();
}

// Block order: with g.p1_group == 0 a pair's (z, row block) items are consecutive (long
// contiguous runs of stores per kx); with g.p1_group = G > 0 the pairs are the fastest
// index in groups of G, so that the CTAs in flight share (z, row block) and the orbital
// rows they multiply are read from HBM once per group and then hit in L2.
template <typename R, int AX>
__global__ void __launch_bounds__(kThreads) k_pass1(Geom g, PairMap<R> pm, int q0, int nq, Cx<R>* __restrict__ inter,
                                                    const Cx<R>* __restrict__ twx) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nyb = (g.ny + kRowsPerCta - 1) / kRowsPerCta;
  int b = blockIdx.x;
  int yblk, z, ql;
  if (g.p1_group <= 0) {
    yblk = b % nyb;
    b /= nyb;
    z = b % g.nz;
    ql = b / g.nz;  // local pair slot
  } else {
    const int lo = b % g.p1_group;
    b /= g.p1_group;
    yblk = b % nyb;
    b /= nyb;
    z = b % g.nz;
    ql = (b / g.nz) * g.p1_group + lo;
    if (ql >= nq) return;   // whole CTA: the last group is partial
  }
  if (!RSX_IN_RANGE(g, ql, nq)) return;   // whole CTA
  const R* f1;
  const R* f2;
  pm.pair(q0 + ql, f1, f2);
  pass1_item<R, AX>(g, f1, f2, z, yblk, inter + (size_t)ql * g.inter_elems(), twx, smem_raw);
}

// ---------------------------------------------------------------------------------
// pass 2 pieces.  D is the (nz x My) plane of one (pair, kx), row pitch DP = My + 1.
// Row loops step over pairs of rows per warp so that both half-warps of a warp run
// the same number of iterations (their __syncwarp calls must match).

template <int NT, typename R>
__device__ __forceinline__ void load_plane(Cx<R>* D, int DP, const Cx<R>* P, int nz, int ny) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int z = warp; z < nz; z += NT / 32)
    for (int y = lane; y < ny; y += 32) D[z * DP + y] = P[z * ny + y];
}

template <int NT, typename R>
__device__ __forceinline__ void store_plane(const Cx<R>* D, int DP, Cx<R>* P, int nz, int ny) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int z = warp; z < nz; z += NT / 32)
    for (int y = lane; y < ny; y += 32) P[z * ny + y] = D[z * DP + y];
}

// forward y transform of rows z < nz (input y < ny, output all My)
template <typename R, int AY, int NT, int PITCH = kScrPitch>
__device__ __forceinline__ void y_forward(Cx<R>* D, int DP, int nz, int ny, const Cx<R>* __restrict__ twy,
                                          Cx<R>* sc, int in_off = 0) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, t = lane & 15;
  for (int z0 = 2 * warp; z0 < nz; z0 += NT / 16) {
    const int z = z0 + (lane >> 4);
    const bool ok = z < nz;
    constexpr int AIN = (AY % 2 == 0) ? AY / 2 : AY;   // inputs y >= ny = 8 AY are zero
    Cx<R> v[AY];
#pragma unroll
    for (int a = 0; a < AIN; ++a) {
      const int y = t + 16 * a;
      v[a] = (ok && y < ny) ? D[z * DP + in_off + y] : cx<R>(R(0), R(0));
    }
    if constexpr (AY % 2 == 0) {
      stage1_store_halfin<AY, -1, R, PITCH>(v, t, twy, sc);
    } else {
      stage1_store<AY, -1, R, PITCH>(v, t, twy, sc);
    }
    __syncwarp();
    Cx<R> u[16];
    if (t < AY) {
      stage2_load<R, PITCH>(u, t, sc);
      Dft<16, -1>::run(u);
    }
    __syncwarp();
    if (ok && t < AY) {
#pragma unroll
      for (int k2 = 0; k2 < 16; ++k2) D[z * DP + t + AY * k2] = u[k2];
    }
    __syncwarp();
  }
}

// inverse y transform of rows z < nz (input all My of D's rows, output y < ny written to
// out[z * opitch + y]: back into D, or straight to the plane in global memory)
template <typename R, int AY, int NT, int PITCH = kScrPitch>
__device__ __forceinline__ void y_inverse(Cx<R>* D, int DP, int nz, int ny, const Cx<R>* __restrict__ twy,
                                          Cx<R>* sc, Cx<R>* out = nullptr, int opitch = 0) {
  if (out == nullptr) {
    out = D;
    opitch = DP;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, t = lane & 15;
  // this lane's stage-1 twiddles (conjugated below), the same for every row
  Cx<R> tw[AY];
  if constexpr (AY % 2 == 0) {
#pragma unroll
    for (int k1 = 1; k1 < AY; ++k1) tw[k1] = twy[t * AY + k1];
  }
  for (int z0 = 2 * warp; z0 < nz; z0 += NT / 16) {
    const int z = z0 + (lane >> 4);
    const bool ok = z < nz;
    Cx<R> v[AY];
#pragma unroll
    for (int a = 0; a < AY; ++a) v[a] = ok ? D[z * DP + t + 16 * a] : cx<R>(R(0), R(0));
    if constexpr (AY % 2 == 0) {
      Dft<AY, 1>::run(v);
#pragma unroll
      for (int k1 = 1; k1 < AY; ++k1) v[k1] = cmul(v[k1], conj(tw[k1]));
#pragma unroll
      for (int k1 = 0; k1 < AY; ++k1) sc[k1 * PITCH + t] = v[k1];
    } else {
      stage1_store<AY, 1, R, PITCH>(v, t, twy, sc);
    }
    __syncwarp();
    Cx<R> u[16];
    if (t < AY) {
      stage2_load<R, PITCH>(u, t, sc);
      if constexpr (AY % 2 == 0) {
        Cx<R> o[8];
        DftHalfOut<16, 1>::run(u, o);   // only y = t + AY k2 < ny = 8 AY, i.e. k2 < 8
#pragma unroll
        for (int k2 = 0; k2 < 8; ++k2) u[k2] = o[k2];
      } else {
        Dft<16, 1>::run(u);
      }
    }
    __syncwarp();
    if (ok && t < AY) {
#pragma unroll
      for (int k2 = 0; k2 < ((AY % 2 == 0) ? 8 : 16); ++k2) {
        const int y = t + AY * k2;
        if (y < ny) out[z * opitch + y] = u[k2];
      }
    }
    __syncwarp();
  }
}

// pass 2: per (pair, kx) plane: y forward, z forward * vhat * z inverse, y inverse.
// pass2_plane is the body for one plane P (nz x ny, contiguous) at column kx; D is the
// (nz x My) work plane (row pitch My + 1) and scr the line scratch.
// Input staging: with `prefetched` the plane already sits in the upper half of the D rows
// (columns [ny, 2 ny), copied by cp.async), otherwise it is loaded here into [0, ny).
// With `Pnext` not null, the next plane is cp.async-prefetched into the upper halves
// (dead after the y inverse) while this plane is stored.
template <typename R>
__device__ __forceinline__ void prefetch_plane_upper(Cx<R>* D, int DP, const Cx<R>* P, int nz, int ny, int NT) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int z = warp; z < nz; z += NT / 32)
    for (int y = lane; y < ny; y += 32) {
      Cx<R>* dp = D + z * DP + ny + y;
      const Cx<R>* sp = P + z * ny + y;
      asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(dp)), "l"(sp)
                   : "memory");
      if (sizeof(R) == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(dp) + 8u),
                     "l"(reinterpret_cast<const char*>(sp) + 8)
                     : "memory");
    }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

template <typename R, int AY, int AZ, int NT>
__device__ __forceinline__ void pass2_plane(const Geom& g, Cx<R>* P, int kx, const Cx<R>* __restrict__ twy,
                                            const Cx<R>* __restrict__ twz, const R* __restrict__ vhat,
                                            const float* __restrict__ vlanes, Cx<R>* D, Cx<R>* scr,
                                            bool prefetched = false, const Cx<R>* Pnext = nullptr) {
  constexpr int LY = 16 * AY;
  constexpr int LZ = 16 * AZ;
  constexpr int AMAX = AY > AZ ? AY : AZ;
  constexpr int PITCH = p2_pitch<R>(AMAX);
  constexpr int SP = AMAX * PITCH;
  constexpr int DP = LY + 1;
  constexpr int NZ = 8 * AZ, NY = 8 * AY;   // the box edges (the padded edge M = 16 A is 2n)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = lane & 15, line = warp * 2 + (lane >> 4);
  Cx<R>* sc = scr + line * SP;
  constexpr int Hy = LY / 2 + 1, Hz = LZ / 2 + 1;
  if (prefetched) {
    asm volatile("cp.async.wait_group 0;" ::: "memory");
  } else {
    load_plane<NT>(D, DP, P, NZ, NY);
  }
  __syncthreads();
  y_forward<R, AY, NT, PITCH>(D, DP, NZ, NY, twy, sc, prefetched ? NY : 0);
  __syncthreads();
  // z forward, multiply, z inverse on columns ky (LY is a multiple of 16: uniform trips)
  const R* vrow = vhat + (size_t)kx * Hy * Hz;
  // this lane's forward stage-1 twiddles, the same for every column
  Cx<R> twf[AZ];
  if constexpr (AZ % 2 == 0) {
#pragma unroll
    for (int k1 = 1; k1 < AZ; ++k1) twf[k1] = twz[t * AZ + k1];
  }
  for (int ky = line; ky < LY; ky += NT / 16) {
    const int iy = ky <= LY / 2 ? ky : LY - ky;
    const R* vcol = vrow + (size_t)iy * Hz;
    constexpr int AIN = (AZ % 2 == 0) ? AZ / 2 : AZ;   // inputs z >= nz = 8 AZ are zero
    Cx<R> v[AZ];
#pragma unroll
    for (int a = 0; a < AIN; ++a) {
      const int z = t + 16 * a;
      v[a] = (z < NZ) ? D[z * DP + ky] : cx<R>(R(0), R(0));
    }
    if constexpr (AZ % 2 == 0) {
      stage1_store_halfin_reg<AZ, R, PITCH>(v, t, twf, sc);
    } else {
      stage1_store<AZ, -1, R, PITCH>(v, t, twz, sc);
    }
    __syncwarp();
    Cx<R> u[16];
    if (t < AZ) stage2_load<R, PITCH>(u, t, sc);
    __syncwarp();
    if (t < AZ) {
      Dft<16, -1>::run(u);
      if constexpr (sizeof(R) == 4) {
        // four 16-byte loads per lane from the lane-order table (k_vhat_lanes): the
        // factors of kz = t + AZ k2, k2 = 4 j .. 4 j + 3
        const float4* vq = reinterpret_cast<const float4*>(vlanes + ((size_t)kx * Hy + iy) * LZ) + t;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float4 m = __ldg(vq + j * AZ);
          u[4 * j] = cscale(u[4 * j], m.x);
          u[4 * j + 1] = cscale(u[4 * j + 1], m.y);
          u[4 * j + 2] = cscale(u[4 * j + 2], m.z);
          u[4 * j + 3] = cscale(u[4 * j + 3], m.w);
        }
      } else {
#pragma unroll
        for (int k2 = 0; k2 < 16; ++k2) {
          const int kz = t + AZ * k2;
          const R m = __ldg(vcol + (kz <= LZ / 2 ? kz : LZ - kz));
          u[k2] = cx<R>(u[k2].x * m, u[k2].y * m);
        }
      }
      Dft<16, 1>::run(u);
      if constexpr (AZ % 2 == 0) {
        stage2_store<R, PITCH>(u, t, sc);
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          Cx<R> w = twz[j * AZ + t];
          w.y = -w.y;
          sc[t * PITCH + j] = cmul(u[j], w);
        }
      }
    }
    __syncwarp();
    Cx<R> r[AZ];
#pragma unroll
    for (int k1 = 0; k1 < AZ; ++k1) r[k1] = sc[k1 * PITCH + t];
    if constexpr (AZ % 2 == 0) {
      // the inverse twiddle w_M^{-j k1} (j the 16-point output index) taken after the
      // transpose, where lane t = j holds k1 = 0 .. AZ-1: the conjugates of the forward
      // twiddles this lane already holds, instead of 16 table loads per column
#pragma unroll
      for (int k1 = 1; k1 < AZ; ++k1) r[k1] = cmul(r[k1], conj(twf[k1]));
      Cx<R> o[AZ / 2];
      DftHalfOut<AZ, 1>::run(r, o);   // only z = t + 16 a < nz = 8 AZ, i.e. a < AZ / 2
#pragma unroll
      for (int a = 0; a < AZ / 2; ++a) D[(t + 16 * a) * DP + ky] = o[a];
    } else {
      Dft<AZ, 1>::run(r);
#pragma unroll
      for (int a = 0; a < AZ; ++a) {
        const int z = t + 16 * a;
        if (z < NZ) D[z * DP + ky] = r[a];
      }
    }
    __syncwarp();
  }
  __syncthreads();
  // the inverse rows go straight to the plane in global memory (no copy through D)
  y_inverse<R, AY, NT, PITCH>(D, DP, NZ, NY, twy, sc, P, NY);
  __syncthreads();   // every read of D's upper halves is done
  if (Pnext) prefetch_plane_upper<R>(D, DP, Pnext, NZ, NY, NT);
}

// D lives in shared memory (DSMEM) or, when it does not fit, in a per-CTA slice of
// global scratch.  Persistent grid over the work items (pair, kx).
template <typename R, int AY, int AZ, bool DSMEM, int NT>
__global__ void __launch_bounds__(NT, 1) k_pass2(Geom g, int nq, Cx<R>* __restrict__ inter,
                                                 const Cx<R>* __restrict__ twy, const Cx<R>* __restrict__ twz,
                                                 const R* __restrict__ vhat, const float* __restrict__ vlanes,
                                                 R* gscratch) {
  constexpr int AMAX = AY > AZ ? AY : AZ;
  constexpr int SP = AMAX * p2_pitch<R>(AMAX);
  constexpr int DP = 16 * AY + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Cx<R>* scr = reinterpret_cast<Cx<R>*>(smem_raw);
  Cx<R>* D = DSMEM ? scr + (NT / 16) * SP
                   : reinterpret_cast<Cx<R>*>(gscratch) + (size_t)blockIdx.x * g.nz * DP;
  const int nplane = g.nz * g.ny;
  const int nwork = nq * g.Hx;
  auto plane_ptr = [&](int w) {
    const int ql = w / g.Hx, kx = w - ql * g.Hx;
    return inter + (size_t)ql * g.inter_elems() + (size_t)kx * nplane;
  };
  // in shared memory the next plane is prefetched behind the current one (2 ny <= My + 1)
  const bool pipe = DSMEM;
  if (pipe && (int)blockIdx.x < nwork) prefetch_plane_upper<R>(D, DP, plane_ptr(blockIdx.x), 8 * AZ, 8 * AY, NT);
  for (int w = blockIdx.x; w < nwork; w += gridDim.x) {
    if (!RSX_IN_RANGE(g, (long long)(w / g.Hx) * g.inter_elems() + (long long)(w % g.Hx + 1) * nplane - 1,
                      (long long)nq * g.inter_elems()))
      break;   // whole CTA: its work index decides
    const int kx = w % g.Hx;
    const int wn = w + (int)gridDim.x;
    pass2_plane<R, AY, AZ, NT>(g, plane_ptr(w), kx, twy, twz, vhat, vlanes, D, scr, pipe,
                               (pipe && wn < nwork) ? plane_ptr(wn) : nullptr);
  }
}

// Casida pair spectra (panel tile-major, see below): per (transition q, kx) plane, y forward and z forward, then
// S_q(G) = sqrt(w_kx * ghat(G) * h^6 / N_pad) * (Re, Im) R_q(G) with w = 1 at kx = 0, Mx/2
// and 2 otherwise, split into bf16 hi + lo and written to panel row q at column
// 2 * ((kx * My + ky) * Mz + kz) + {0, 1}.  wsq holds the weights sqrt(w * ghat * h^6 /
// N_pad) on the folded half spectrum [kx][|ky|][|kz|] (k_spectrum_weights).
template <int AY, int AZ, int NT>
__global__ void __launch_bounds__(NT) k_spectrum(Geom g, int nq, const Cx<float>* __restrict__ inter,
                                                       const Cx<float>* __restrict__ twy,
                                                       const Cx<float>* __restrict__ twz,
                                                       const float* __restrict__ wsq,
                                                       uint16_t* __restrict__ hi, uint16_t* __restrict__ lo,
                                                       size_t ld, int nrb) {
  constexpr int LY = 16 * AY;
  constexpr int LZ = 16 * AZ;
  constexpr int AMAX = AY > AZ ? AY : AZ;
  constexpr int SP = AMAX * kScrPitch;
  constexpr int DP = LY + 1;
  constexpr int LPC = NT / 16;   // lines per CTA (one per half-warp)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Cx<float>* scr = reinterpret_cast<Cx<float>*>(smem_raw);
  Cx<float>* D = scr + LPC * SP;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = lane & 15, line = warp * 2 + (lane >> 4);
  Cx<float>* sc = scr + line * SP;
  constexpr int Hy = LY / 2 + 1, Hz = LZ / 2 + 1;
  const int nplane = g.nz * g.ny;
  const int nwork = nq * g.Hx;
  // transitions are the fastest index of the work items: the CTAs in flight fill the same
  // 128 x 64 panel tiles (rows = transitions) instead of scattering 128-byte rows
  auto plane_ptr = [&](int w) {
    const int kx = w / nq, ql = w - kx * nq;
    return inter + (size_t)ql * g.inter_elems() + (size_t)kx * nplane;
  };
  // the plane is staged in the upper halves [ny, 2 ny) of the D rows; the next plane is
  // prefetched there once the z transforms of the upper ky columns are done
  if ((int)blockIdx.x < nwork) prefetch_plane_upper<float>(D, DP, plane_ptr(blockIdx.x), g.nz, g.ny, NT);
  for (int w = blockIdx.x; w < nwork; w += gridDim.x) {
    const int kx = w / nq, ql = w - kx * nq;
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    y_forward<float, AY, NT>(D, DP, g.nz, g.ny, twy, sc, g.ny);
    __syncthreads();
    const float* vrow = wsq + (size_t)kx * Hy * Hz;
    // tile-major panel [ld/64][nrb][128][64]: column g of row ql is at
    // ((g / 64) * nrb + ql / 128) * 8192 + (ql % 128) * 64 + g % 64
    const size_t row_off = (size_t)(ql / 128) * 8192 + (size_t)(ql % 128) * 64;
    const size_t kb_stride = (size_t)nrb * 8192;
    const int wn = w + (int)gridDim.x;
    // this lane's forward stage-1 twiddles, the same for every column
    Cx<float> twf[AZ];
    if constexpr (AZ % 2 == 0) {
#pragma unroll
      for (int k1 = 1; k1 < AZ; ++k1) twf[k1] = twz[t * AZ + k1];
    }
    // columns ky: the upper half [LY/2, LY) first, then the lower half; slot s of line l
    // takes flat position f = s LPC + l (f < LY/2: upper column LY/2 + f, else lower
    // column f - LY/2), so every line runs the same number of columns, and after slot
    // kPre - 1 (when every upper column is done; possibly the last slot) the next plane is
    // prefetched into the upper halves of the D rows
    constexpr int kSlots = (LY + LPC - 1) / LPC;
    constexpr int kPre = (LY / 2 + LPC - 1) / LPC;
    for (int slot = 0; slot < kSlots; ++slot) {
      const int f = slot * LPC + line;
      if (f < LY) {   // uniform in a warp: LPC is even, a warp's two lines are f, f + 1 with LY even
        const int ky = f < LY / 2 ? LY / 2 + f : f - LY / 2;
        const int iy = ky <= LY / 2 ? ky : LY - ky;
        const float* vcol = vrow + (size_t)iy * Hz;
        constexpr int AIN = (AZ % 2 == 0) ? AZ / 2 : AZ;
        Cx<float> v[AZ];
#pragma unroll
        for (int a = 0; a < AIN; ++a) {
          const int z = t + 16 * a;
          v[a] = (z < g.nz) ? D[z * DP + ky] : cx<float>(0.f, 0.f);
        }
        if constexpr (AZ % 2 == 0) {
          stage1_store_halfin_reg<AZ>(v, t, twf, sc);
        } else {
          stage1_store<AZ, -1>(v, t, twz, sc);
        }
        __syncwarp();
        Cx<float> u[16];
        if (t < AZ) {
          stage2_load(u, t, sc);
          Dft<16, -1>::run(u);
        }
        __syncwarp();
        if (t < AZ) {
#pragma unroll
          for (int k2 = 0; k2 < 16; ++k2) {
            const int kz = t + AZ * k2;
            const float m = __ldg(vcol + (kz <= LZ / 2 ? kz : LZ - kz));
            sc[kz] = cx<float>(u[k2].x * m, u[k2].y * m);
          }
        }
        __syncwarp();
        // 16-byte stores: 4 complex -> 8 bf16 of hi and of lo per lane (never straddle a
        // 64-column block: the line starts at a multiple of 32 columns)
        const size_t g0 = ((size_t)kx * LY + ky) * LZ * 2;
        for (int q = t; q < LZ / 4; q += 16) {
          const size_t gq = g0 + 8 * (size_t)q;
          const size_t off = (gq / 64) * kb_stride + row_off + (gq % 64);
          uint32_t hv[4], lv[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            // round-to-nearest-even hardware conversions (re in the low half, im in the high)
            const Cx<float> c = sc[4 * q + j];
            const __nv_bfloat162 h2 = __float22bfloat162_rn(make_float2(c.x, c.y));
            const float2 hf = __bfloat1622float2(h2);
            const __nv_bfloat162 l2 = __float22bfloat162_rn(make_float2(c.x - hf.x, c.y - hf.y));
            hv[j] = *reinterpret_cast<const uint32_t*>(&h2);
            lv[j] = *reinterpret_cast<const uint32_t*>(&l2);
          }
          *reinterpret_cast<uint4*>(hi + off) = make_uint4(hv[0], hv[1], hv[2], hv[3]);
          *reinterpret_cast<uint4*>(lo + off) = make_uint4(lv[0], lv[1], lv[2], lv[3]);
        }
        __syncwarp();
      }
      if (slot == kPre - 1) {
        __syncthreads();   // every read of the upper halves is done
        if (wn < nwork) prefetch_plane_upper<float>(D, DP, plane_ptr(wn), g.nz, g.ny, NT);
      }
    }
  }
}

// ---------------------------------------------------------------------------------
// pass 3: x inverse (c2r via row pairs) of every pair in output p's list, and
// out_p(z, y, x) = - sum_e partner_e(z, y, x) V_e(z, y, x).  One item = (p, z, 32 rows).
// With pot != 0 the output p is the potential V of pair q = p itself (no partner, no sign).
// The next pair's row block and partner tile are copied with cp.async into the second
// of two shared-memory buffers while the current pair is transformed.
// pass3_item is the body; `out_p` is output p's array, `inter` the slot base of q0.

__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// shared-memory bytes of pass 3 for element type R (two buffers of row block + tile)
template <typename R>
__host__ __device__ inline size_t pass3_buffer_elems(int AX, int nx) {
  const int H = 8 * AX + 1;
  return (size_t)H * kRowsPerCta * sizeof(Cx<R>) + (size_t)kRowsPerCta * nx * sizeof(R);
}

template <typename R, int AX>
__device__ __forceinline__ void pass3_prefetch(const Geom& g, const PairMap<R>& pm, int q0, int p, int e, int z,
                                               int y0, int nrow, int pot, const Cx<R>* __restrict__ inter,
                                               Cx<R>* xs, R* tile) {
  constexpr int H = 8 * AX + 1;
  int q = p;
  const R* partner = nullptr;
  if (!pot) pm.entry(p, e, q, partner);
  const Cx<R>* src = inter + (size_t)(q - q0) * g.inter_elems() + (size_t)z * g.ny + y0;
  const size_t kstride = (size_t)g.nz * g.ny;
  const bool slot_ok = RSX_IN_RANGE(g, q - q0, g.dbg_nq > 0 ? g.dbg_nq : 0x7fffffff);
  // one granule (rows r, r + 1) per copy; the intermediate is library-owned and 16-byte
  // aligned, nrow is a multiple of 8
  for (int i = threadIdx.x; i < H * (kRowsPerCta / 2); i += kThreads) {
    const int kx = i / (kRowsPerCta / 2), r = 2 * (i - kx * (kRowsPerCta / 2));
    Cx<R>* dp = xs + xs_idx(kx, r);
    if (r < nrow && slot_ok &&
        RSX_IN_RANGE(g, (size_t)z * g.ny + y0 + (size_t)kx * kstride + r + 1, g.inter_elems())) {
      const Cx<R>* sp = src + (size_t)kx * kstride + r;
      cp_async16(dp, sp);
      if (sizeof(R) == 8) cp_async16(dp + 1, sp + 1);
    } else {
      st_granule(dp, cx<R>(R(0), R(0)), cx<R>(R(0), R(0)));
    }
  }
  if (!pot) {
    const R* prow = partner + (size_t)z * g.ny * g.nx + (size_t)y0 * g.nx;
    const int cnt = RSX_IN_RANGE(g, (size_t)z * g.ny * g.nx + (size_t)(y0 + nrow) * g.nx - 1, g.N()) ? nrow * g.nx : 0;
    if (((reinterpret_cast<uintptr_t>(prow) | (uintptr_t)(cnt * sizeof(R))) & 15u) == 0) {
      constexpr int V = 16 / (int)sizeof(R);
      for (int i = threadIdx.x * V; i < cnt; i += kThreads * V) cp_async16(tile + i, prow + i);
    } else {
      for (int i = threadIdx.x; i < cnt; i += kThreads) {
        if (sizeof(R) == 4)
          cp_async4(tile + i, prow + i);
        else
          cp_async8(tile + i, prow + i);
      }
    }
  }
}

template <typename R, int AX>
__device__ __forceinline__ void pass3_item(const Geom& g, const PairMap<R>& pm, int q0, int p, int z, int yblk,
                                           int pot, const Cx<R>* __restrict__ inter, const Cx<R>* __restrict__ twx,
                                           R* __restrict__ out_p, unsigned char* smem_raw) {
  constexpr int L = 16 * AX;
  constexpr int SP = AX * kScrPitch;
  constexpr int H = L / 2 + 1;
  Cx<R>* scr = reinterpret_cast<Cx<R>*>(smem_raw);
  unsigned char* buf0 = reinterpret_cast<unsigned char*>(scr + kLinesPerCta * SP);
  const size_t bufbytes = pass3_buffer_elems<R>(AX, g.nx);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = lane & 15, line = warp * 2 + (lane >> 4);
  const int y0 = yblk * kRowsPerCta;
  const int nrow = min(kRowsPerCta, g.ny - y0);
  Cx<R>* sc = scr + line * SP;
  const size_t plane = (size_t)z * g.ny * g.nx;
  auto xs_of = [&](int b) { return reinterpret_cast<Cx<R>*>(buf0 + b * bufbytes); };
  auto tile_of = [&](int b) { return reinterpret_cast<R*>(buf0 + b * bufbytes + (size_t)H * kRowsPerCta * sizeof(Cx<R>)); };

  R acc0[16], acc1[16];
#pragma unroll
  for (int k2 = 0; k2 < 16; ++k2) acc0[k2] = acc1[k2] = R(0);

  // this lane's stage-1 twiddles, the same for every entry
  Cx<R> tw[AX];
  if constexpr (AX % 2 == 0) {
#pragma unroll
    for (int k1 = 1; k1 < AX; ++k1) tw[k1] = twx[t * AX + k1];
  }
  const int ne = pot ? 1 : pm.nentries(p);
  __syncthreads();   // the buffers may still be read by a previous item of this CTA
  pass3_prefetch<R, AX>(g, pm, q0, p, 0, z, y0, nrow, pot, inter, xs_of(0), tile_of(0));
  cp_async_commit();
  for (int e = 0; e < ne; ++e) {
    if (e + 1 < ne) {
      pass3_prefetch<R, AX>(g, pm, q0, p, e + 1, z, y0, nrow, pot, inter, xs_of((e + 1) & 1), tile_of((e + 1) & 1));
      cp_async_commit();
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const Cx<R>* xs = xs_of(e & 1);
    const R* tile = tile_of(e & 1);

    // Z(k) = X_a(k) + i X_b(k), Hermitian extension for k > L/2
    Cx<R> v[AX];
#pragma unroll
    for (int a = 0; a < AX; ++a) {
      const int k = t + 16 * a;
      Cx<R> xa, xb;
      if (k < H) {
        ld_granule(xs + xs_idx(k, 2 * line), xa, xb);
      } else {
        ld_granule(xs + xs_idx(L - k, 2 * line), xa, xb);
        xa = conj(xa);
        xb = conj(xb);
      }
      v[a] = cx<R>(xa.x - xb.y, xa.y + xb.x);
    }
    if constexpr (AX % 2 == 0) {
      Dft<AX, 1>::run(v);
#pragma unroll
      for (int k1 = 1; k1 < AX; ++k1) v[k1] = cmul(v[k1], conj(tw[k1]));
#pragma unroll
      for (int k1 = 0; k1 < AX; ++k1) sc[k1 * kScrPitch + t] = v[k1];
    } else {
      stage1_store<AX, 1>(v, t, twx, sc);
    }
    __syncwarp();
    if (t < AX) {
      Cx<R> u[16];
      stage2_load(u, t, sc);
      if constexpr (AX % 2 == 0) {
        Cx<R> o[8];
        DftHalfOut<16, 1>::run(u, o);   // only x = t + AX k2 < nx = 8 AX, i.e. k2 < 8
#pragma unroll
        for (int k2 = 0; k2 < 8; ++k2) u[k2] = o[k2];
      } else {
        Dft<16, 1>::run(u);
      }
      const int ra = 2 * line, rb = ra + 1;
#pragma unroll
      for (int k2 = 0; k2 < ((AX % 2 == 0) ? 8 : 16); ++k2) {
        const int x = t + AX * k2;
        if (x < g.nx) {
          if (pot) {
            acc0[k2] += u[k2].x;
            acc1[k2] += u[k2].y;
          } else {
            if (ra < nrow) acc0[k2] -= tile[ra * g.nx + x] * u[k2].x;
            if (rb < nrow) acc1[k2] -= tile[rb * g.nx + x] * u[k2].y;
          }
        }
      }
    }
    __syncwarp();
    __syncthreads();   // buffer e & 1 is refilled by the prefetch of entry e + 2
  }
  R* tile = tile_of(0);
  if (t < AX) {
    const int ra = 2 * line, rb = ra + 1;
#pragma unroll
    for (int k2 = 0; k2 < ((AX % 2 == 0) ? 8 : 16); ++k2) {   // x = t + AX k2 < nx = 8 AX
      const int x = t + AX * k2;
      if (x < g.nx) {
        if (ra < nrow) tile[ra * g.nx + x] = acc0[k2];
        if (rb < nrow) tile[rb * g.nx + x] = acc1[k2];
      }
    }
  }
  __syncthreads();
  R* orow = out_p + plane + (size_t)y0 * g.nx;
  if (RSX_IN_RANGE(g, plane + (size_t)(y0 + nrow) * g.nx - 1, g.N()))
    for (int i = threadIdx.x; i < nrow * g.nx; i += kThreads) orow[i] = tile[i];
  __syncthreads();
}

template <typename R, int AX>
__global__ void __launch_bounds__(kThreads) k_pass3(Geom g, PairMap<R> pm, int q0, int p0, int pot,
                                                    const Cx<R>* __restrict__ inter,
                                                    const Cx<R>* __restrict__ twx, R* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // outputs are the fastest index: the CTAs in flight share (z, row block), so the partner
  // rows they multiply come from HBM once and then from L2 for the other outputs
  const int nyb = (g.ny + kRowsPerCta - 1) / kRowsPerCta;
  const int np = (int)(gridDim.x / ((unsigned)g.nz * nyb));
  int b = blockIdx.x;
  const int pl = b % np;
  b /= np;
  const int yblk = b % nyb;
  const int z = b / nyb;
  pass3_item<R, AX>(g, pm, q0, p0 + pl, z, yblk, pot, inter, twx, pm.out_row(p0 + pl, out, pl), smem_raw);
}

}  // namespace rsx
