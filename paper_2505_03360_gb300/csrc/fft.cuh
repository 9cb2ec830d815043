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

// In-place length-L transform of (re, im), natural order in and out.
template <int L, int SIGN, typename T>
__device__ __forceinline__ void fft(T* re, T* im) {
  dif<L, 0, SIGN, T>(re, im);
  T tr[L], ti[L];
  unscramble<L, 0, T>(re, im, tr, ti);
#pragma unroll
  for (int k = 0; k < L; ++k) { re[k] = tr[k]; im[k] = ti[k]; }
}

}  // namespace coll
