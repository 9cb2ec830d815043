// Per-thread, fully unrolled mixed-radix FFTs held in registers.
//
// A pencil of L complex values lives in two register arrays (re, im).  The
// transform is a decimation-in-frequency recursion with radix-4 / radix-3 /
// radix-2 butterflies; every index, twiddle exponent and the final
// digit-reversal permutation are compile-time constants after unrolling, so
// the permutation costs no instructions and twiddles are constant-bank
// operands.  Twiddles come from the correctly rounded cos/sin(2 pi n / 192)
// tables (192 = lcm of every supported length).
//
// SIGN = -1: forward transform  X_k = sum_j x_j exp(-2 pi i jk / L)
// SIGN = +1: inverse transform  x_j = sum_k X_k exp(+2 pi i jk / L)  (unnormalised)
#pragma once

#include "dfloat.cuh"
#include "twiddles.h"

namespace coll {

template <typename T> struct Tw;
template <> struct Tw<double> {
  static __device__ __forceinline__ double c(int n) { return kTwCosD[n]; }
  static __device__ __forceinline__ double s(int n) { return kTwSinD[n]; }
};
template <> struct Tw<float> {
  static __device__ __forceinline__ float c(int n) { return kTwCosF[n]; }
  static __device__ __forceinline__ float s(int n) { return kTwSinF[n]; }
};
template <> struct Tw<df> {
  static __device__ __forceinline__ df c(int n) { return df{kTwCosF[n], kTwCosL[n]}; }
  static __device__ __forceinline__ df s(int n) { return df{kTwSinF[n], kTwSinL[n]}; }
};

__device__ __forceinline__ double half(double x) { return 0.5 * x; }
__device__ __forceinline__ float half(float x) { return 0.5f * x; }

// first radix applied to a sub-transform of length L
__host__ __device__ constexpr int radix_of(int L) {
  return (L % 4 == 0) ? 4 : (L % 3 == 0 ? 3 : (L % 2 == 0 ? 2 : L));
}

// storage position of output k after the DIF recursion on length L
__host__ __device__ constexpr int dif_pos(int L, int k) {
  int pos = 0, len = L;
  while (len > 1) {
    int r = radix_of(len);
    int m = len / r;
    pos += (k % r) * m;
    k /= r;
    len = m;
  }
  return pos;
}

// multiply (xr, xi) by exp(SIGN * 2 pi i * e / L), e compile-time after unrolling
template <int L, int SIGN, typename T>
__device__ __forceinline__ void twiddle(T& xr, T& xi, int e) {
  const int n = ((e % L) * (192 / L)) % 192;
  if (n == 0) return;
  if (n == 96) { xr = -xr; xi = -xi; return; }
  if (n == 48 || n == 144) {                  // +-i
    const bool pos_i = (n == 48) == (SIGN > 0);
    T t = xr;
    if (pos_i) { xr = -xi; xi = t; } else { xr = xi; xi = -t; }
    return;
  }
  const T c = Tw<T>::c(n);
  const T s = SIGN > 0 ? Tw<T>::s(n) : -Tw<T>::s(n);
  T r = xr * c - xi * s;
  xi = xr * s + xi * c;
  xr = r;
}

template <int R, int SIGN, typename T>
__device__ __forceinline__ void butterfly(T* xr, T* xi) {
  if constexpr (R == 2) {
    T ar = xr[0] + xr[1], ai = xi[0] + xi[1];
    T br = xr[0] - xr[1], bi = xi[0] - xi[1];
    xr[0] = ar; xi[0] = ai; xr[1] = br; xi[1] = bi;
  } else if constexpr (R == 4) {
    T ar = xr[0] + xr[2], ai = xi[0] + xi[2];
    T br = xr[0] - xr[2], bi = xi[0] - xi[2];
    T cr = xr[1] + xr[3], ci = xi[1] + xi[3];
    T er = xr[1] - xr[3], ei = xi[1] - xi[3];
    // d = e * (SIGN i)
    T dr = SIGN > 0 ? -ei : ei;
    T di = SIGN > 0 ? er : -er;
    xr[0] = ar + cr; xi[0] = ai + ci;
    xr[2] = ar - cr; xi[2] = ai - ci;
    xr[1] = br + dr; xi[1] = bi + di;
    xr[3] = br - dr; xi[3] = bi - di;
  } else if constexpr (R == 3) {
    const T h = Tw<T>::s(64);                 // sin(2 pi / 3) = sqrt(3)/2
    T tr = xr[1] + xr[2], ti = xi[1] + xi[2];
    T ur = xr[1] - xr[2], ui = xi[1] - xi[2];
    T mr = xr[0] - half(tr), mi = xi[0] - half(ti);
    // v = SIGN i h u
    T vr = SIGN > 0 ? -h * ui : h * ui;
    T vi = SIGN > 0 ? h * ur : -h * ur;
    xr[0] = xr[0] + tr; xi[0] = xi[0] + ti;
    xr[1] = mr + vr; xi[1] = mi + vi;
    xr[2] = mr - vr; xi[2] = mi - vi;
  }
}

template <int L, int BASE, int SIGN, typename T>
__device__ __forceinline__ void dif(T* re, T* im) {
  if constexpr (L > 1) {
    constexpr int R = radix_of(L);
    constexpr int M = L / R;
#pragma unroll
    for (int j = 0; j < M; ++j) {
      T xr[R], xi[R];
#pragma unroll
      for (int q = 0; q < R; ++q) { xr[q] = re[BASE + j + q * M]; xi[q] = im[BASE + j + q * M]; }
      butterfly<R, SIGN, T>(xr, xi);
#pragma unroll
      for (int p = 1; p < R; ++p) twiddle<L, SIGN, T>(xr[p], xi[p], p * j);
#pragma unroll
      for (int p = 0; p < R; ++p) { re[BASE + j + p * M] = xr[p]; im[BASE + j + p * M] = xi[p]; }
    }
    dif<M, BASE, SIGN, T>(re, im);
    if constexpr (R > 1) dif<M, BASE + M, SIGN, T>(re, im);
    if constexpr (R > 2) dif<M, BASE + 2 * M, SIGN, T>(re, im);
    if constexpr (R > 3) dif<M, BASE + 3 * M, SIGN, T>(re, im);
  }
}

// Undo the digit reversal: out[k] = in[dif_pos(L, k)], one template level per
// k so that every index is a constant expression.
template <int L, int K, typename T>
__device__ __forceinline__ void unscramble(const T* sr, const T* si, T* dr, T* di) {
  if constexpr (K < L) {
    constexpr int P = dif_pos(L, K);
    dr[K] = sr[P];
    di[K] = si[P];
    unscramble<L, K + 1, T>(sr, si, dr, di);
  }
}

// ------------------------------------------------- decimation in time, FMA form
// For FP64 and FP32 the transform is a decimation-in-time
// recursion instead: its butterflies take twiddled INPUTS, so each generic
// twiddle folds into fused multiply-adds.  With w = exp(SIGN 2 pi i n / 192),
//   form 0 (|cos| >= |sin|): w y = m u, m = cos, u = y + i tan * y
//   form 1 (otherwise):      w y = m u, m = sin, u = cot * y + i y
// (|tan|, |cot| <= 1, |m| >= 1/sqrt 2), u costs two FMAs and a +- w y costs two
// more per output instead of a complex multiply and two additions.  In a
// radix-4 butterfly the pair w1 y1 +- w3 y3 is m1 (u1 +- r u3), r = m3 / m1, so
// its outputs a +- m1 (...) are FMAs too: a radix-4 butterfly with three
// generic twiddles costs 22 FP64 instructions instead of 28 (a 32-point
// transform 378 instead of 432).  The twiddles n % 48 == 0 are exact rotations.
template <typename T> struct TwFma;
template <> struct TwFma<double> {
  static __device__ __forceinline__ double m(int n) { return kTwMD[n]; }
  static __device__ __forceinline__ double t(int n) { return kTwTD[n]; }
  static __device__ __forceinline__ double r3(int n) { return kTwR3D[n]; }
  static __device__ __forceinline__ double im(int n) { return kTwIMD[n]; }
};
template <> struct TwFma<float> {
  static __device__ __forceinline__ float m(int n) { return kTwMF[n]; }
  static __device__ __forceinline__ float t(int n) { return kTwTF[n]; }
  static __device__ __forceinline__ float r3(int n) { return kTwR3F[n]; }
  static __device__ __forceinline__ float im(int n) { return kTwIMF[n]; }
};
template <typename T> constexpr bool kFmaFft = false;
template <> constexpr bool kFmaFft<double> = true;
template <> constexpr bool kFmaFft<float> = true;

__host__ __device__ constexpr bool tw_trivial(int n) { return n % 48 == 0; }
__host__ __device__ constexpr int tw_form(int n) { return (n % 96 <= 24 || n % 96 >= 72) ? 0 : 1; }
__host__ __device__ constexpr bool is_pow2(int L) { return L > 0 && (L & (L - 1)) == 0; }

// w y for n % 48 == 0: multiplication by 1, SIGN i, -1, -SIGN i
template <int SIGN, typename T>
__device__ __forceinline__ void tw_exact(T& r, T& i, int n) {
  const int q = (n / 48) % 4;
  const T a = r, b = i;
  if (q == 0) return;
  if (q == 2) { r = -a; i = -b; return; }
  const bool pos_i = (q == 1) == (SIGN > 0);          // multiply by +i or -i
  if (pos_i) { r = -b; i = a; } else { r = b; i = -a; }
}

// (yr, yi) -> (ur, ui) with w y = m u; returns m (generic n only)
template <int SIGN, typename T>
__device__ __forceinline__ T tw_fma(T yr, T yi, int n, T& ur, T& ui) {
  const T t = SIGN > 0 ? TwFma<T>::t(n) : -TwFma<T>::t(n);
  if (tw_form(n) == 0) {
    ur = fma(-t, yi, yr);
    ui = fma(t, yr, yi);
    return TwFma<T>::m(n);
  }
  ur = fma(t, yr, -yi);
  ui = fma(t, yi, yr);
  return SIGN > 0 ? TwFma<T>::m(n) : -TwFma<T>::m(n);
}

// sign of m under SIGN (form 1 scales by sin, which changes sign with SIGN)
template <int SIGN> __host__ __device__ constexpr int tw_msign(int n) { return tw_form(n) == 1 && SIGN < 0 ? -1 : 1; }

// radix-2 combine at (b, b + M): X_0 = y0 + w y1, X_1 = y0 - w y1, w = w_L^j
template <int L, int SIGN, typename T>
__device__ __forceinline__ void dit_comb2(T* yr, T* yi, int b, int M, int j) {
  const int n = (j % L) * (192 / L);
  const T ar = yr[b], ai = yi[b];
  T cr = yr[b + M], ci = yi[b + M];
  if (tw_trivial(n)) {
    tw_exact<SIGN>(cr, ci, n);
    yr[b] = ar + cr; yi[b] = ai + ci;
    yr[b + M] = ar - cr; yi[b + M] = ai - ci;
  } else {
    T ur, ui;
    const T m = tw_fma<SIGN>(cr, ci, n, ur, ui);
    yr[b] = fma(m, ur, ar); yi[b] = fma(m, ui, ai);
    yr[b + M] = fma(-m, ur, ar); yi[b + M] = fma(-m, ui, ai);
  }
}

// radix-4 combine at (b + q M), q < 4: X_p = sum_q (SIGN i)^{pq} w_L^{qj} y_q
template <int L, int SIGN, typename T>
__device__ __forceinline__ void dit_comb4(T* yr, T* yi, int b, int M, int j) {
  const int n1 = (j % L) * (192 / L), n2 = ((2 * j) % L) * (192 / L), n3 = ((3 * j) % L) * (192 / L);
  // A, B = y0 +- w2 y2 (unscaled)
  T Ar, Ai, Br, Bi;
  {
    const T y0r = yr[b], y0i = yi[b];
    T y2r = yr[b + 2 * M], y2i = yi[b + 2 * M];
    if (tw_trivial(n2)) {
      tw_exact<SIGN>(y2r, y2i, n2);
      Ar = y0r + y2r; Ai = y0i + y2i; Br = y0r - y2r; Bi = y0i - y2i;
    } else {
      T ur, ui;
      const T m = tw_fma<SIGN>(y2r, y2i, n2, ur, ui);
      Ar = fma(m, ur, y0r); Ai = fma(m, ui, y0i); Br = fma(-m, ur, y0r); Bi = fma(-m, ui, y0i);
    }
  }
  // C, D = w1 y1 +- w3 y3 = sc (C', D')
  T y1r = yr[b + M], y1i = yi[b + M], y3r = yr[b + 3 * M], y3i = yi[b + 3 * M];
  T Cr, Ci, Dr, Di;
  if (tw_trivial(n1) && tw_trivial(n3)) {
    tw_exact<SIGN>(y1r, y1i, n1);
    tw_exact<SIGN>(y3r, y3i, n3);
    Cr = y1r + y3r; Ci = y1i + y3i; Dr = y1r - y3r; Di = y1i - y3i;
    yr[b] = Ar + Cr; yi[b] = Ai + Ci;
    yr[b + 2 * M] = Ar - Cr; yi[b + 2 * M] = Ai - Ci;
    // (SIGN i) D
    const T er = SIGN > 0 ? -Di : Di, ei = SIGN > 0 ? Dr : -Dr;
    yr[b + M] = Br + er; yi[b + M] = Bi + ei;
    yr[b + 3 * M] = Br - er; yi[b + 3 * M] = Bi - ei;
    return;
  }
  T sc;
  if (!tw_trivial(n1) && !tw_trivial(n3)) {
    T u1r, u1i, u3r, u3i;
    sc = tw_fma<SIGN>(y1r, y1i, n1, u1r, u1i);
    tw_fma<SIGN>(y3r, y3i, n3, u3r, u3i);
    const T r = (tw_msign<SIGN>(n1) * tw_msign<SIGN>(n3) > 0) ? TwFma<T>::r3(n1) : -TwFma<T>::r3(n1);
    Cr = fma(r, u3r, u1r); Ci = fma(r, u3i, u1i); Dr = fma(-r, u3r, u1r); Di = fma(-r, u3i, u1i);
  } else if (!tw_trivial(n1)) {
    T u1r, u1i;
    sc = tw_fma<SIGN>(y1r, y1i, n1, u1r, u1i);
    tw_exact<SIGN>(y3r, y3i, n3);
    const T r = tw_msign<SIGN>(n1) > 0 ? TwFma<T>::im(n1) : -TwFma<T>::im(n1);   // 1 / m1
    Cr = fma(r, y3r, u1r); Ci = fma(r, y3i, u1i); Dr = fma(-r, y3r, u1r); Di = fma(-r, y3i, u1i);
  } else {
    T u3r, u3i;
    sc = tw_fma<SIGN>(y3r, y3i, n3, u3r, u3i);
    tw_exact<SIGN>(y1r, y1i, n1);
    const T r = tw_msign<SIGN>(n3) > 0 ? TwFma<T>::im(n3) : -TwFma<T>::im(n3);   // 1 / m3
    Cr = fma(r, y1r, u3r); Ci = fma(r, y1i, u3i); Dr = fma(r, y1r, -u3r); Di = fma(r, y1i, -u3i);
  }
  yr[b] = fma(sc, Cr, Ar); yi[b] = fma(sc, Ci, Ai);
  yr[b + 2 * M] = fma(-sc, Cr, Ar); yi[b + 2 * M] = fma(-sc, Ci, Ai);
  // B +- sc (SIGN i) D'
  const T ss = SIGN > 0 ? sc : -sc;
  yr[b + M] = fma(-ss, Di, Br); yi[b + M] = fma(ss, Dr, Bi);
  yr[b + 3 * M] = fma(ss, Di, Br); yi[b + 3 * M] = fma(-ss, Dr, Bi);
}

// radix-3 combine at (b + q M), q < 3: X_p = sum_q w3^{pq} w_L^{qj} y_q.  Within the
// supported lengths (radix 4 first, so 3 is always the innermost factor) j = 0 and the
// twiddles are trivial; a generic twiddle is applied as a plain product.
template <int L, int SIGN, typename T>
__device__ __forceinline__ void dit_comb3(T* yr, T* yi, int b, int M, int j) {
  T a0r = yr[b], a0i = yi[b], a1r = yr[b + M], a1i = yi[b + M], a2r = yr[b + 2 * M], a2i = yi[b + 2 * M];
#pragma unroll
  for (int q = 1; q < 3; ++q) {
    const int n = ((q * j) % L) * (192 / L);
    T& r = q == 1 ? a1r : a2r;
    T& i = q == 1 ? a1i : a2i;
    if (tw_trivial(n)) {
      tw_exact<SIGN>(r, i, n);
    } else {
      T ur, ui;
      const T m = tw_fma<SIGN>(r, i, n, ur, ui);
      r = m * ur;
      i = m * ui;
    }
  }
  const T h = Tw<T>::s(64);                 // sin(2 pi / 3) = sqrt(3)/2
  const T tr = a1r + a2r, ti = a1i + a2i, dr = a1r - a2r, di = a1i - a2i;
  const T mr = fma(T(-0.5), tr, a0r), mi = fma(T(-0.5), ti, a0i);
  const T vr = SIGN > 0 ? -h * di : h * di, vi = SIGN > 0 ? h * dr : -h * dr;   // SIGN i h d
  yr[b] = a0r + tr; yi[b] = a0i + ti;
  yr[b + M] = mr + vr; yi[b + M] = mi + vi;
  yr[b + 2 * M] = mr - vr; yi[b + 2 * M] = mi - vi;
}

template <int L, int OFF, int STRIDE, int OB, int SIGN, typename T>
__device__ __forceinline__ void dit(const T* xr, const T* xi, T* yr, T* yi);

template <int L, int OFF, int STRIDE, int OB, int SIGN, typename T, int Q>
__device__ __forceinline__ void dit_subs(const T* xr, const T* xi, T* yr, T* yi) {
  constexpr int R = radix_of(L), M = L / R;
  if constexpr (Q < R) {
    dit<M, OFF + STRIDE * Q, STRIDE * R, OB + Q * M, SIGN, T>(xr, xi, yr, yi);
    dit_subs<L, OFF, STRIDE, OB, SIGN, T, Q + 1>(xr, xi, yr, yi);
  }
}

// DFT of x[OFF + STRIDE m], m < L, into y[OB + k], k < L (natural order)
template <int L, int OFF, int STRIDE, int OB, int SIGN, typename T>
__device__ __forceinline__ void dit(const T* xr, const T* xi, T* yr, T* yi) {
  if constexpr (L == 1) {
    yr[OB] = xr[OFF];
    yi[OB] = xi[OFF];
  } else {
    constexpr int R = radix_of(L), M = L / R;
    static_assert(R == 2 || R == 3 || R == 4, "lengths 2^a 3^b");
    dit_subs<L, OFF, STRIDE, OB, SIGN, T, 0>(xr, xi, yr, yi);
#pragma unroll
    for (int j = 0; j < M; ++j) {
      if constexpr (R == 4) dit_comb4<L, SIGN, T>(yr, yi, OB + j, M, j);
      else if constexpr (R == 3) dit_comb3<L, SIGN, T>(yr, yi, OB + j, M, j);
      else dit_comb2<L, SIGN, T>(yr, yi, OB + j, M, j);
    }
  }
}

// In-place length-L transform of (re, im), natural order in and out.
template <int L, int SIGN, typename T>
__device__ __forceinline__ void fft(T* re, T* im) {
  if constexpr (kFmaFft<T>) {
    T tr[L], ti[L];
    dit<L, 0, 1, 0, SIGN, T>(re, im, tr, ti);
#pragma unroll
    for (int k = 0; k < L; ++k) { re[k] = tr[k]; im[k] = ti[k]; }
  } else {
    dif<L, 0, SIGN, T>(re, im);
    T tr[L], ti[L];
    unscramble<L, 0, T>(re, im, tr, ti);
#pragma unroll
    for (int k = 0; k < L; ++k) { re[k] = tr[k]; im[k] = ti[k]; }
  }
}

}  // namespace coll
