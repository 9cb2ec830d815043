// Galerkin mode of the collision operator (plan dealias = 1; the oracle's
// zero-padded products, reading g8 of the aliasing question in sec. 4.4.1).
//
// The quadratic products are formed on the 3N/2 grid, where the product of
// two functions with modes |k_d| < N/2 has no aliased modes below N/2, and
// the result is projected back onto the modes |k_d| < N/2:
//   f_pad = IDFT_Np( pad( DFT_N(f) / N^3 ) )            (spectral interpolation)
//   Q_pad = the collision kernel on the Np grid, whose tables carry the
//           multipliers of the base modes and zeros elsewhere
//   Q     = IDFT_N( trunc( DFT_Np(Q_pad) / Np^3 ) )    (projection)
// with every mode of some |k_d| >= N/2 dropped.  The operator is translation
// invariant (a bilinear Fourier multiplier), so the grids need no phase
// factors as long as both resamplings use the same convention.
//
// Both resamplings are separable: per axis, pencils of NI values go through a
// forward NI-point transform, a 1/NI scale, the mode map (signed k kept when
// |k| < min(NI, NO)/2, moved from index k mod NI to k mod NO) and an inverse
// NO-point transform.  One thread per pencil, register FFTs (fft.cuh); a 3D
// resampling is three passes over the cell batch.
#include <cuda_runtime.h>

#include "coll_internal.h"
#include "fft.cuh"

namespace coll {

namespace {

constexpr int kRsThreads = 128;

// Resample along the middle axis of per-cell arrays [A][NI][B] -> [A][NO][B].
template <int NI, int NO, typename T, typename Tin, typename Tout, bool kRealIn, bool kRealOut>
__global__ void __launch_bounds__(kRsThreads) resample_kernel(const Tin* __restrict__ in, Tout* __restrict__ out,
                                                              long long n_cells, int A, int B) {
  constexpr int KB = NI < NO ? NI : NO;              // base grid: modes |k| < KB/2 are kept
  const long long pencils = n_cells * A * B;
  const size_t in_cell = size_t(A) * NI * B, out_cell = size_t(A) * NO * B;
  const T inv = T(1) / T(NI);
  for (long long id = blockIdx.x * (long long)kRsThreads + threadIdx.x; id < pencils;
       id += (long long)gridDim.x * kRsThreads) {
    const long long c = id / (A * B);
    const int rem = int(id % (A * B));
    const int a = rem / B, b = rem % B;
    T xr[NI], xi[NI];
    const size_t ib = size_t(c) * in_cell + size_t(a) * NI * B + b;
#pragma unroll
    for (int j = 0; j < NI; ++j) {
      if constexpr (kRealIn) {
        xr[j] = T(in[ib + size_t(j) * B]);
        xi[j] = T(0);
      } else {
        const Tin v = in[ib + size_t(j) * B];
        xr[j] = T(v.x);
        xi[j] = T(v.y);
      }
    }
    fft<NI, -1, T>(xr, xi);
    T yr[NO], yi[NO];
#pragma unroll
    for (int k = 0; k < NO; ++k) { yr[k] = T(0); yi[k] = T(0); }
#pragma unroll
    for (int k = 0; k < KB / 2; ++k) {                 // k = 0 .. KB/2 - 1
      yr[k] = xr[k] * inv;
      yi[k] = xi[k] * inv;
    }
#pragma unroll
    for (int m = 1; m < KB / 2; ++m) {                 // k = -m
      yr[NO - m] = xr[NI - m] * inv;
      yi[NO - m] = xi[NI - m] * inv;
    }
    fft<NO, +1, T>(yr, yi);
    const size_t ob = size_t(c) * out_cell + size_t(a) * NO * B + b;
#pragma unroll
    for (int j = 0; j < NO; ++j) {
      if constexpr (kRealOut) {
        out[ob + size_t(j) * B] = Tout(yr[j]);
      } else {
        Tout v;
        v.x = decltype(v.x)(yr[j]);
        v.y = decltype(v.y)(yi[j]);
        out[ob + size_t(j) * B] = v;
      }
    }
  }
}

template <typename T> struct Cplx;
template <> struct Cplx<double> { using type = double2; };
template <> struct Cplx<float> { using type = float2; };

int grid_of(const void* k, long long pencils) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, kRsThreads, 0);
  if (per < 1) per = 1;
  const long long want = (pencils + kRsThreads - 1) / kRsThreads;
  const long long cap = static_cast<long long>(sms) * per;
  return int(want < cap ? (want < 1 ? 1 : want) : cap);
}

template <int NI, int NO, typename T, typename Tin, typename Tout, bool RI, bool RO>
int pass(const void* in, void* out, long long n_cells, int A, int B, cudaStream_t st) {
  auto k = resample_kernel<NI, NO, T, Tin, Tout, RI, RO>;
  const int grid = grid_of(reinterpret_cast<const void*>(k), n_cells * A * B);
  k<<<grid, kRsThreads, 0, st>>>(static_cast<const Tin*>(in), static_cast<Tout*>(out), n_cells, A, B);
  return int(cudaGetLastError());
}

// f [n][N][N][N] (Tio) -> f_pad [n][Np][Np][Np] (Tio), through complex scratch sa, sb
template <int N, typename T, typename Tio>
int up(const Tio* f, Tio* fpad, void* sa, void* sb, long long n, cudaStream_t st) {
  constexpr int Np = 3 * N / 2;
  using C = typename Cplx<T>::type;
  int e = pass<N, Np, T, Tio, C, true, false>(f, sa, n, N * N, 1, st);             // [N][N][Np]
  if (e == 0) e = pass<N, Np, T, C, C, false, false>(sa, sb, n, N, Np, st);      // [N][Np][Np]
  if (e == 0) e = pass<N, Np, T, C, Tio, false, true>(sb, fpad, n, 1, Np * Np, st);   // [Np][Np][Np]
  return e;
}

// Q_pad [n][Np]^3 (Tio) -> Q [n][N]^3 (Tio)
template <int N, typename T, typename Tio>
int down(const Tio* qpad, Tio* Q, void* sa, void* sb, long long n, cudaStream_t st) {
  constexpr int Np = 3 * N / 2;
  using C = typename Cplx<T>::type;
  int e = pass<Np, N, T, Tio, C, true, false>(qpad, sa, n, Np * Np, 1, st);        // [Np][Np][N]
  if (e == 0) e = pass<Np, N, T, C, C, false, false>(sa, sb, n, Np, N, st);      // [Np][N][N]
  if (e == 0) e = pass<Np, N, T, C, Tio, false, true>(sb, Q, n, 1, N * N, st);   // [N][N][N]
  return e;
}

}  // namespace

// Complex scratch per cell of each of the two resampling buffers (elements).
size_t galerkin_scratch_elems(int N) {
  const size_t Np = size_t(3) * N / 2;
  return size_t(N) * Np * Np;                          // the larger intermediate, N x Np x Np
}

int launch_galerkin_resample(bool to_pad, int N, bool compute_f64, bool io_f64, const void* in, void* out,
                             void* sa, void* sb, long long n_cells, void* stream) {
  count_launches(3);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (N == 16) {
    if (compute_f64) {
      if (io_f64) return to_pad ? up<16, double, double>((const double*)in, (double*)out, sa, sb, n_cells, st)
                                : down<16, double, double>((const double*)in, (double*)out, sa, sb, n_cells, st);
      return to_pad ? up<16, double, float>((const float*)in, (float*)out, sa, sb, n_cells, st)
                    : down<16, double, float>((const float*)in, (float*)out, sa, sb, n_cells, st);
    }
    if (io_f64) return int(cudaErrorInvalidValue);
    return to_pad ? up<16, float, float>((const float*)in, (float*)out, sa, sb, n_cells, st)
                  : down<16, float, float>((const float*)in, (float*)out, sa, sb, n_cells, st);
  }
  if (N == 32 && !compute_f64 && !io_f64)
    return to_pad ? up<32, float, float>((const float*)in, (float*)out, sa, sb, n_cells, st)
                  : down<32, float, float>((const float*)in, (float*)out, sa, sb, n_cells, st);
  return int(cudaErrorInvalidValue);
}

}  // namespace coll
