// Register-resident small DFTs used by the line transforms of the pair Poisson solve.
//
// dft<N, S>(v) replaces v[0..N) by X[k] = sum_j v[j] exp(S * 2 pi i j k / N)
// (S = -1 forward, S = +1 inverse, no normalisation).  Supported N: 2, 3, 4, 5, 6, 7,
// 8, 10, 12, 14, 16, 24.  Odd primes use the symmetric real/imaginary split, 8 and 16 are
// radix-2 / radix-4 Cooley-Tukey, and the coprime products 6, 10, 12, 14, 24 use the
// Good-Thomas prime-factor index map, which needs no twiddle factors.  All trig
// constants are exact decimal expansions of cos/sin of rational multiples of pi.
#pragma once
#include <cuda_runtime.h>

#ifndef RSX_HD
#define RSX_HD __host__ __device__ __forceinline__
#endif

namespace rsx {

template <typename R>
struct Cx {
  R x, y;
};

template <typename R>
RSX_HD Cx<R> cx(R a, R b) { Cx<R> c; c.x = a; c.y = b; return c; }
template <typename R>
RSX_HD Cx<R> operator+(Cx<R> a, Cx<R> b) { return cx<R>(a.x + b.x, a.y + b.y); }
template <typename R>
RSX_HD Cx<R> operator-(Cx<R> a, Cx<R> b) { return cx<R>(a.x - b.x, a.y - b.y); }
template <typename R>
RSX_HD Cx<R> cmul(Cx<R> a, Cx<R> b) {
  return cx<R>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename R>
RSX_HD Cx<R> cscale(Cx<R> a, R s) { return cx<R>(a.x * s, a.y * s); }

// FP32 on sm_100-family devices: complex add / subtract / real scaling as packed two-lane
// FP32 instructions (one instruction per complex operation instead of two; the same
// round-to-nearest results as the scalar forms).  The FFT passes are instruction-issue
// bound and these operations are most of their arithmetic.
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
#define RSX_PACKED_F32 1
#endif
template <>
RSX_HD Cx<float> operator+(Cx<float> a, Cx<float> b) {
#ifdef RSX_PACKED_F32
  const float2 r = __fadd2_rn(make_float2(a.x, a.y), make_float2(b.x, b.y));
  return cx<float>(r.x, r.y);
#else
  return cx<float>(a.x + b.x, a.y + b.y);
#endif
}
template <>
RSX_HD Cx<float> operator-(Cx<float> a, Cx<float> b) {
#ifdef RSX_PACKED_F32
  const float2 r = __fadd2_rn(make_float2(a.x, a.y), make_float2(-b.x, -b.y));
  return cx<float>(r.x, r.y);
#else
  return cx<float>(a.x - b.x, a.y - b.y);
#endif
}
template <>
RSX_HD Cx<float> cscale(Cx<float> a, float s) {
#ifdef RSX_PACKED_F32
  const float2 r = __fmul2_rn(make_float2(a.x, a.y), make_float2(s, s));
  return cx<float>(r.x, r.y);
#else
  return cx<float>(a.x * s, a.y * s);
#endif
}
// acc + s * a (real s), fused
template <typename R>
RSX_HD Cx<R> cfma(Cx<R> a, R s, Cx<R> acc) { return cx<R>(fma(s, a.x, acc.x), fma(s, a.y, acc.y)); }
template <>
RSX_HD Cx<float> cfma(Cx<float> a, float s, Cx<float> acc) {
#ifdef RSX_PACKED_F32
  const float2 r = __ffma2_rn(make_float2(a.x, a.y), make_float2(s, s), make_float2(acc.x, acc.y));
  return cx<float>(r.x, r.y);
#else
  return cx<float>(fmaf(s, a.x, acc.x), fmaf(s, a.y, acc.y));
#endif
}
template <typename R>
RSX_HD Cx<R> conj(Cx<R> a) { return cx<R>(a.x, -a.y); }
// S * i * a  for S = +-1
template <int S, typename R>
RSX_HD Cx<R> mul_si(Cx<R> a) {
  return S > 0 ? cx<R>(-a.y, a.x) : cx<R>(a.y, -a.x);
}
// (c + S i s) * a
template <int S, typename R>
RSX_HD Cx<R> rot(Cx<R> a, R c, R s) {
  const R ss = S > 0 ? s : -s;
  return cx<R>(a.x * c - a.y * ss, a.x * ss + a.y * c);
}

// cos(2 pi j / p) and sin(2 pi j / p) for p in {3, 5, 7, 16}, 0 <= j < p (decimal
// expansions of the exact values); constexpr so that unrolled uses fold to immediates.
RSX_HD constexpr double trig_c(int p, int j) {
  return p == 3 ? (j == 0 ? 1.0 : -0.5)
       : p == 5 ? (j == 0 ? 1.0 : (j == 1 || j == 4) ? 0.30901699437494742410 : -0.80901699437494742410)
       : p == 7 ? (j == 0 ? 1.0 : (j == 1 || j == 6) ? 0.62348980185873353053
                           : (j == 2 || j == 5) ? -0.22252093395631440429 : -0.90096886790241912624)
       : /* p == 16 */
         (j == 0 ? 1.0 : j == 1 ? 0.92387953251128675613 : j == 2 ? 0.70710678118654752440
          : j == 3 ? 0.38268343236508977173 : j == 4 ? 0.0 : j == 5 ? -0.38268343236508977173
          : j == 6 ? -0.70710678118654752440 : j == 7 ? -0.92387953251128675613 : j == 8 ? -1.0
          : j == 9 ? -0.92387953251128675613 : j == 10 ? -0.70710678118654752440
          : j == 11 ? -0.38268343236508977173 : j == 12 ? 0.0 : j == 13 ? 0.38268343236508977173
          : j == 14 ? 0.70710678118654752440 : 0.92387953251128675613);
}
RSX_HD constexpr double trig_s(int p, int j) {
  // sin(2 pi j / p) = cos(2 pi j / p - pi / 2); written out per p
  return p == 3 ? (j == 0 ? 0.0 : j == 1 ? 0.86602540378443864676 : -0.86602540378443864676)
       : p == 5 ? (j == 0 ? 0.0 : j == 1 ? 0.95105651629515357212 : j == 2 ? 0.58778525229247312917
                           : j == 3 ? -0.58778525229247312917 : -0.95105651629515357212)
       : p == 7 ? (j == 0 ? 0.0 : j == 1 ? 0.78183148246802980871 : j == 2 ? 0.97492791218182360702
                           : j == 3 ? 0.43388373911755812048 : j == 4 ? -0.43388373911755812048
                           : j == 5 ? -0.97492791218182360702 : -0.78183148246802980871)
       : /* p == 16 */ trig_c(16, (j + 12) % 16);
}

// cos(2 pi a / 24), 0 <= a < 24: multiples of 15 degrees, (sqrt 6 +- sqrt 2) / 4 at 15 and 75
RSX_HD constexpr double trig24_c_q(int a) {   // first quadrant, 0 <= a <= 6
  return a == 0 ? 1.0 : a == 1 ? 0.96592582628906828675 : a == 2 ? 0.86602540378443864676
       : a == 3 ? 0.70710678118654752440 : a == 4 ? 0.5 : a == 5 ? 0.25881904510252076235 : 0.0;
}
RSX_HD constexpr double trig24_c(int a) {
  return a <= 6 ? trig24_c_q(a) : a <= 12 ? -trig24_c_q(12 - a) : a <= 18 ? -trig24_c_q(a - 12) : trig24_c_q(24 - a);
}
RSX_HD constexpr double trig24_s(int a) { return trig24_c((a + 18) % 24); }   // sin x = cos(x - pi / 2)

// cos / sin (2 pi a / A) for even A in {2, ..., 14, 16, 24} and 0 <= a < A / 2 (decimal expansions)
RSX_HD constexpr double trig_even_c(int A, int a) {
  return A == 24 ? trig24_c(a)
       : A == 16 ? trig_c(16, a) : A == 8 ? trig_c(16, 2 * a) : A == 4 ? (a == 0 ? 1.0 : 0.0) : A == 2 ? 1.0
       : A == 6 ? (a == 0 ? 1.0 : a == 1 ? 0.5 : -0.5)
       : A == 10 ? (a == 0 ? 1.0 : a == 1 ? 0.80901699437494742410 : a == 2 ? 0.30901699437494742410
                    : a == 3 ? -0.30901699437494742410 : -0.80901699437494742410)
       : A == 12 ? (a == 0 ? 1.0 : a == 1 ? 0.86602540378443864676 : a == 2 ? 0.5 : a == 3 ? 0.0
                    : a == 4 ? -0.5 : -0.86602540378443864676)
       : /* A == 14 */ (a == 0 ? 1.0 : a == 1 ? 0.90096886790241912624 : a == 2 ? 0.62348980185873353053
                        : a == 3 ? 0.22252093395631440429 : a == 4 ? -0.22252093395631440429
                        : a == 5 ? -0.62348980185873353053 : -0.90096886790241912624);
}
RSX_HD constexpr double trig_even_s(int A, int a) {
  return A == 24 ? trig24_s(a)
       : A == 16 ? trig_s(16, a) : A == 8 ? trig_s(16, 2 * a) : A == 4 ? (a == 0 ? 0.0 : 1.0) : A == 2 ? 0.0
       : A == 6 ? (a == 0 ? 0.0 : 0.86602540378443864676)
       : A == 10 ? (a == 0 ? 0.0 : (a == 1 || a == 4) ? 0.58778525229247312917 : 0.95105651629515357212)
       : A == 12 ? (a == 0 ? 0.0 : (a == 1 || a == 5) ? 0.5 : (a == 2 || a == 4) ? 0.86602540378443864676 : 1.0)
       : /* A == 14 */ (a == 0 ? 0.0 : (a == 1 || a == 6) ? 0.43388373911755812048
                        : (a == 2 || a == 5) ? 0.78183148246802980871 : 0.97492791218182360702);
}

template <int N, int S>
struct Dft;

template <int S>
struct Dft<1, S> {
  template <typename R> RSX_HD static void run(Cx<R>* v) {}
};

template <int S>
struct Dft<2, S> {
  template <typename R>
  RSX_HD static void run(Cx<R>* v) {
    Cx<R> a = v[0], b = v[1];
    v[0] = a + b;
    v[1] = a - b;
  }
};

template <int S>
struct Dft<4, S> {
  template <typename R>
  RSX_HD static void run(Cx<R>* v) {
    Cx<R> a = v[0] + v[2], b = v[0] - v[2], c = v[1] + v[3], d = mul_si<S>(v[1] - v[3]);
    v[0] = a + c;
    v[2] = a - c;
    v[1] = b + d;
    v[3] = b - d;
  }
};

// odd prime p: pairs (k, p-k) split into even (cos) and odd (sin) parts
template <int P, int S>
struct DftOddPrime {
  template <typename R>
  RSX_HD static void run(Cx<R>* v) {
    constexpr int H = (P - 1) / 2;
    Cx<R> a[H], b[H];
    Cx<R> x0 = v[0];
    Cx<R> sum = x0;
#pragma unroll
    for (int k = 1; k <= H; ++k) {
      a[k - 1] = v[k] + v[P - k];
      b[k - 1] = v[k] - v[P - k];
      sum = sum + a[k - 1];
    }
    v[0] = sum;
#pragma unroll
    for (int m = 1; m <= H; ++m) {
      Cx<R> re = x0, im = cx<R>(R(0), R(0));
#pragma unroll
      for (int k = 1; k <= H; ++k) {
        const R c = R(trig_c(P, (m * k) % P));
        const R s = R(trig_s(P, (m * k) % P));
        re = cfma(a[k - 1], c, re);
        im = cfma(b[k - 1], s, im);
      }
      const Cx<R> u = mul_si<S>(im);
      v[m] = re + u;
      v[P - m] = re - u;
    }
  }
};
template <int S> struct Dft<3, S> : DftOddPrime<3, S> {};
template <int S> struct Dft<5, S> : DftOddPrime<5, S> {};
template <int S> struct Dft<7, S> : DftOddPrime<7, S> {};

template <int S>
struct Dft<8, S> {
  template <typename R>
  RSX_HD static void run(Cx<R>* v) {
    Cx<R> e[4] = {v[0], v[2], v[4], v[6]};
    Cx<R> o[4] = {v[1], v[3], v[5], v[7]};
    Dft<4, S>::run(e);
    Dft<4, S>::run(o);
    const R r = R(0.70710678118654752440);
    Cx<R> t1 = rot<S>(o[1], r, r);
    Cx<R> t2 = mul_si<S>(o[2]);
    Cx<R> t3 = rot<S>(o[3], -r, r);
    v[0] = e[0] + o[0];
    v[4] = e[0] - o[0];
    v[1] = e[1] + t1;
    v[5] = e[1] - t1;
    v[2] = e[2] + t2;
    v[6] = e[2] - t2;
    v[3] = e[3] + t3;
    v[7] = e[3] - t3;
  }
};

template <int S>
struct Dft<16, S> {
  template <typename R>
  RSX_HD static void run(Cx<R>* v) {
    Cx<R> y[4][4];
#pragma unroll
    for (int j2 = 0; j2 < 4; ++j2) {
      Cx<R> c[4] = {v[j2], v[j2 + 4], v[j2 + 8], v[j2 + 12]};
      Dft<4, S>::run(c);
#pragma unroll
      for (int k1 = 0; k1 < 4; ++k1) {
        const int e = j2 * k1;   // e = 4 is the rotation by S i: a swap, no multiplies
        y[j2][k1] = (e == 0) ? c[k1] : (e == 4) ? mul_si<S>(c[k1]) : rot<S>(c[k1], R(trig_c(16, e)), R(trig_s(16, e)));
      }
    }
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
      Cx<R> c[4] = {y[0][k1], y[1][k1], y[2][k1], y[3][k1]};
      Dft<4, S>::run(c);
#pragma unroll
      for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = c[k2];
    }
  }
};

RSX_HD constexpr int modinv(int a, int m) {
  int r = 1;
  for (int i = 1; i < m; ++i)
    if ((a * i) % m == 1) r = i;
  return r;
}

// Good-Thomas prime-factor DFT of length P*Q, gcd(P, Q) = 1
template <int P, int Q, int S>
struct DftPfa {
  template <typename R>
  RSX_HD static void run(Cx<R>* v) {
    constexpr int N = P * Q;
    constexpr int qinv = modinv(Q % P, P);
    constexpr int pinv = modinv(P % Q, Q);
    Cx<R> y[P][Q];
#pragma unroll
    for (int n1 = 0; n1 < P; ++n1)
#pragma unroll
      for (int n2 = 0; n2 < Q; ++n2) y[n1][n2] = v[(n1 * Q + n2 * P) % N];
#pragma unroll
    for (int n2 = 0; n2 < Q; ++n2) {
      Cx<R> c[P];
#pragma unroll
      for (int n1 = 0; n1 < P; ++n1) c[n1] = y[n1][n2];
      Dft<P, S>::run(c);
#pragma unroll
      for (int n1 = 0; n1 < P; ++n1) y[n1][n2] = c[n1];
    }
#pragma unroll
    for (int k1 = 0; k1 < P; ++k1) {
      Dft<Q, S>::run(y[k1]);
    }
#pragma unroll
    for (int k1 = 0; k1 < P; ++k1)
#pragma unroll
      for (int k2 = 0; k2 < Q; ++k2) v[(k1 * Q * qinv + k2 * P * pinv) % N] = y[k1][k2];
  }
};
template <int S> struct Dft<6, S> : DftPfa<2, 3, S> {};
template <int S> struct Dft<10, S> : DftPfa<2, 5, S> {};
template <int S> struct Dft<12, S> : DftPfa<3, 4, S> {};
template <int S> struct Dft<14, S> : DftPfa<2, 7, S> {};
template <int S> struct Dft<24, S> : DftPfa<3, 8, S> {};

// DFT of length A (even) whose inputs v[A/2 .. A) are zero: only v[0 .. A/2) are read.
// X[2m] = DFT_{A/2}(v)[m], X[2m+1] = DFT_{A/2}(v[a] w^a)[m], w = exp(S 2 pi i / A).
// Result written to out[0 .. A).
template <int A, int S>
struct DftHalfIn {
  template <typename R>
  RSX_HD static void run(const Cx<R>* v, Cx<R>* out) {
    constexpr int H = A / 2;
    Cx<R> e[H], o[H];
#pragma unroll
    for (int a = 0; a < H; ++a) {
      e[a] = v[a];
      o[a] = (a == 0) ? v[a] : (4 * a == A) ? mul_si<S>(v[a]) : rot<S>(v[a], R(trig_even_c(A, a)), R(trig_even_s(A, a)));
    }
    Dft<H, S>::run(e);
    Dft<H, S>::run(o);
#pragma unroll
    for (int m = 0; m < H; ++m) {
      out[2 * m] = e[m];
      out[2 * m + 1] = o[m];
    }
  }
};

// DFT of length A (even) of which only outputs 0 .. A/2 - 1 are wanted:
// X[a] = DFT_{A/2}(v_even)[a] + w^a DFT_{A/2}(v_odd)[a].  Result written to out[0 .. A/2).
template <int A, int S>
struct DftHalfOut {
  template <typename R>
  RSX_HD static void run(const Cx<R>* v, Cx<R>* out) {
    constexpr int H = A / 2;
    Cx<R> e[H], o[H];
#pragma unroll
    for (int m = 0; m < H; ++m) {
      e[m] = v[2 * m];
      o[m] = v[2 * m + 1];
    }
    Dft<H, S>::run(e);
    Dft<H, S>::run(o);
#pragma unroll
    for (int a = 0; a < H; ++a)
      out[a] = e[a] + ((a == 0) ? o[a] : (4 * a == A) ? mul_si<S>(o[a]) : rot<S>(o[a], R(trig_even_c(A, a)), R(trig_even_s(A, a))));
  }
};


// Pruned 3-point DFTs for the prime-factor codelets below (w = exp(S 2 pi i / 3)):
//   X0 = x0 + a,  X1,2 = x0 - a / 2 +- S i (sqrt 3 / 2) b,   a = x1 + x2,  b = x1 - x2.
// dft3_in<S, N0, N1, N2>: inputs flagged false are zero and never read (all three outputs).
template <int S, bool N0, bool N1, bool N2, typename R>
RSX_HD void dft3_in(Cx<R>& x0, Cx<R>& x1, Cx<R>& x2) {
  const R h = R(-0.5), s3 = R(0.86602540378443864676);
  static_assert(N0 || N1 || N2, "at least one input");
  if constexpr (!N1 && !N2) {   // X_k = x0
    x1 = x0;
    x2 = x0;
  } else if constexpr (!N0 && !N2) {   // only x1: X_k = x1 w^k
    const Cx<R> re = cscale(x1, h), u = mul_si<S>(cscale(x1, s3));
    x0 = x1;
    x2 = re - u;
    x1 = re + u;
  } else if constexpr (!N0 && !N1) {   // only x2: X_k = x2 w^2k
    const Cx<R> re = cscale(x2, h), u = mul_si<S>(cscale(x2, s3));
    x0 = x2;
    x1 = re - u;
    x2 = re + u;
  } else if constexpr (!N2) {   // a = b = x1
    const Cx<R> re = cfma(x1, h, x0), u = mul_si<S>(cscale(x1, s3));
    x0 = x0 + x1;
    x1 = re + u;
    x2 = re - u;
  } else if constexpr (!N1) {   // a = x2, b = -x2
    const Cx<R> re = cfma(x2, h, x0), u = mul_si<S>(cscale(x2, s3));
    x0 = x0 + x2;
    x1 = re - u;
    x2 = re + u;
  } else if constexpr (!N0) {
    const Cx<R> a = x1 + x2, b = x1 - x2;
    const Cx<R> re = cscale(a, h), u = mul_si<S>(cscale(b, s3));
    x0 = a;
    x1 = re + u;
    x2 = re - u;
  } else {
    Cx<R> v[3] = {x0, x1, x2};
    Dft<3, S>::run(v);
    x0 = v[0];
    x1 = v[1];
    x2 = v[2];
  }
}

// dft3_out<S, W0, W1, W2>: all inputs, only the outputs flagged true are formed (in place).
template <int S, bool W0, bool W1, bool W2, typename R>
RSX_HD void dft3_out(Cx<R>& x0, Cx<R>& x1, Cx<R>& x2) {
  const R h = R(-0.5), s3 = R(0.86602540378443864676);
  const Cx<R> a = x1 + x2;
  if constexpr (W0 && !W1 && !W2) {
    x0 = x0 + a;
  } else {
    const Cx<R> b = x1 - x2;
    const Cx<R> re = cfma(a, h, x0), u = mul_si<S>(cscale(b, s3));
    if constexpr (W0) x0 = x0 + a;
    if constexpr (W1) x1 = re + u;
    if constexpr (W2) x2 = re - u;
  }
}

// 4-point DFT forming only outputs 0 and K (K = 1, 3) or 1 and 2 (in place)
template <int S, int W, typename R>
RSX_HD void dft4_two_out(Cx<R>* v) {   // W: 1 -> {0, 1}, 3 -> {0, 3}, 12 -> {1, 2}
  const Cx<R> a = v[0] + v[2], b = v[0] - v[2], c = v[1] + v[3], d = mul_si<S>(v[1] - v[3]);
  if constexpr (W == 1) {
    v[0] = a + c;
    v[1] = b + d;
  } else if constexpr (W == 3) {
    v[0] = a + c;
    v[3] = b - d;
  } else {
    v[1] = b + d;
    v[2] = a - c;
  }
}

// 2-point DFTs with zero inputs skipped / unwanted outputs not formed (in place)
template <bool N0, bool N1, typename R>
RSX_HD void dft2_in(Cx<R>& x0, Cx<R>& x1) {
  static_assert(N0 || N1, "at least one input");
  if constexpr (N0 && N1) {
    const Cx<R> a = x0;
    x0 = a + x1;
    x1 = a - x1;
  } else if constexpr (N0) {
    x1 = x0;
  } else {
    x0 = x1;
    x1 = cx<R>(-x1.x, -x1.y);
  }
}
template <bool W0, bool W1, typename R>
RSX_HD void dft2_out(Cx<R>& x0, Cx<R>& x1) {
  if constexpr (W0 && W1) {
    const Cx<R> a = x0;
    x0 = a + x1;
    x1 = a - x1;
  } else if constexpr (W0) {
    x0 = x0 + x1;
  } else if constexpr (W1) {
    x1 = x0 - x1;
  }
}

// Pruned Good-Thomas DFTs of length N = P Q (P = 2 or 3, gcd(P, Q) = 1), the index maps
// of DftPfa: input (Q n1 + P n2) mod N, output (Q qinv k1 + P pinv k2) mod N.
//   half in  (inputs N/2 .. N zero): per column n2 the P-point DFT over n1 skips the zero
//            inputs, then the Q-point DFTs over n2 are complete;
//   half out (outputs 0 .. N/2 kept): the Q-point DFTs over n2 first, complete, then per
//            column k2 the P-point DFT over n1 forms only the kept outputs.
template <int P, int Q>
struct PfaMap {
  static constexpr int N = P * Q;
  RSX_HD static constexpr int in(int n1, int n2) { return (Q * n1 + P * n2) % N; }
  RSX_HD static constexpr int out(int k1, int k2) { return (Q * modinv(Q % P, P) * k1 + P * modinv(P % Q, Q) * k2) % N; }
  RSX_HD static constexpr bool in_nz(int n1, int n2) { return n1 < P && in(n1, n2) < N / 2; }
  RSX_HD static constexpr bool out_kept(int k1, int k2) { return k1 < P && out(k1, k2) < N / 2; }
};

template <int P, int Q, int S, int C>
struct PfaHalfInCols {   // columns n2 = C .. Q-1
  template <typename R>
  RSX_HD static void run(const Cx<R>* v, Cx<R> (&y)[P][Q]) {
    if constexpr (C < Q) {
      using M = PfaMap<P, Q>;
      constexpr bool m0 = M::in_nz(0, C), m1 = M::in_nz(1, C), m2 = M::in_nz(2, C);
      if constexpr (m0) y[0][C] = v[M::in(0, C)];
      if constexpr (m1) y[1][C] = v[M::in(1, C)];
      if constexpr (P == 2) {
        dft2_in<m0, m1>(y[0][C], y[1][C]);
      } else {
        if constexpr (m2) y[2][C] = v[M::in(2, C)];
        dft3_in<S, m0, m1, m2>(y[0][C], y[1][C], y[2][C]);
      }
      PfaHalfInCols<P, Q, S, C + 1>::run(v, y);
    }
  }
};

template <int P, int Q, int S, int C>
struct PfaHalfOutCols {   // columns k2 = C .. Q-1
  template <typename R>
  RSX_HD static void run(Cx<R> (&y)[P][Q], Cx<R>* out) {
    if constexpr (C < Q) {
      using M = PfaMap<P, Q>;
      constexpr bool w0 = M::out_kept(0, C), w1 = M::out_kept(1, C), w2 = M::out_kept(2, C);
      if constexpr (P == 2) {
        dft2_out<w0, w1>(y[0][C], y[1][C]);
      } else {
        if constexpr (w0 || w1 || w2) dft3_out<S, w0, w1, w2>(y[0][C], y[1][C], y[2][C]);
      }
      if constexpr (w0) out[M::out(0, C)] = y[0][C];
      if constexpr (w1) out[M::out(1, C)] = y[1][C];
      if constexpr (w2) out[M::out(2, C)] = y[2][C];
      PfaHalfOutCols<P, Q, S, C + 1>::run(y, out);
    }
  }
};

template <int P, int Q, int S>
struct DftPfaHalfIn {
  template <typename R>
  RSX_HD static void run(const Cx<R>* v, Cx<R>* out) {
    Cx<R> y[P][Q];
    PfaHalfInCols<P, Q, S, 0>::run(v, y);
#pragma unroll
    for (int k1 = 0; k1 < P; ++k1) {
      Dft<Q, S>::run(y[k1]);
#pragma unroll
      for (int k2 = 0; k2 < Q; ++k2) out[PfaMap<P, Q>::out(k1, k2)] = y[k1][k2];
    }
  }
};

template <int P, int Q, int S>
struct DftPfaHalfOut {
  template <typename R>
  RSX_HD static void run(const Cx<R>* v, Cx<R>* out) {
    Cx<R> y[P][Q];
#pragma unroll
    for (int n1 = 0; n1 < P; ++n1) {
#pragma unroll
      for (int n2 = 0; n2 < Q; ++n2) y[n1][n2] = v[PfaMap<P, Q>::in(n1, n2)];
      Dft<Q, S>::run(y[n1]);
    }
    PfaHalfOutCols<P, Q, S, 0>::run(y, out);
  }
};

template <int S> struct DftHalfIn<6, S> : DftPfaHalfIn<2, 3, S> {};
template <int S> struct DftHalfIn<10, S> : DftPfaHalfIn<2, 5, S> {};
template <int S> struct DftHalfIn<12, S> : DftPfaHalfIn<3, 4, S> {};
template <int S> struct DftHalfIn<14, S> : DftPfaHalfIn<2, 7, S> {};
template <int S> struct DftHalfIn<24, S> : DftPfaHalfIn<3, 8, S> {};
template <int S> struct DftHalfOut<6, S> : DftPfaHalfOut<2, 3, S> {};
template <int S> struct DftHalfOut<10, S> : DftPfaHalfOut<2, 5, S> {};
template <int S> struct DftHalfOut<12, S> : DftPfaHalfOut<3, 4, S> {};
template <int S> struct DftHalfOut<14, S> : DftPfaHalfOut<2, 7, S> {};
template <int S> struct DftHalfOut<24, S> : DftPfaHalfOut<3, 8, S> {};

// The 16-point DFT of which only outputs 0 .. 7 are wanted: Dft<16>'s radix-4 steps with
// the second 4-point DFTs forming outputs k2 = 0, 1 only (k = k1 + 4 k2 < 8).
template <int S>
struct DftHalfOut<16, S> {
  template <typename R>
  RSX_HD static void run(const Cx<R>* v, Cx<R>* out) {
    Cx<R> y[4][4];
#pragma unroll
    for (int j2 = 0; j2 < 4; ++j2) {
      Cx<R> c[4] = {v[j2], v[j2 + 4], v[j2 + 8], v[j2 + 12]};
      Dft<4, S>::run(c);
#pragma unroll
      for (int k1 = 0; k1 < 4; ++k1) {
        const int e = j2 * k1;
        y[k1][j2] = (e == 0) ? c[k1] : (e == 4) ? mul_si<S>(c[k1]) : rot<S>(c[k1], R(trig_c(16, e)), R(trig_s(16, e)));
      }
    }
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
      dft4_two_out<S, 1>(y[k1]);
      out[k1] = y[k1][0];
      out[k1 + 4] = y[k1][1];
    }
  }
};

}  // namespace rsx
