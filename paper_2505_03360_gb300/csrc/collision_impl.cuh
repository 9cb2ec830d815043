// Fused batched evaluation of the Carleman collision operator Q^R(f,f)
// (arxiv 2505.03360, sec. 4.4.1): one CTA per cell, persistent over cells.
//
// Per cell, in index space (the grid offset v_0 = -L cancels because every
// multiplier is real and even):
//   F      = DFT3(f)                         real-to-complex, half spectrum
//   z_t    = IDFT3((A_t + i B_t) F)          one complex inverse 3D FFT per term
//   Q     += Re(z_t) * Im(z_t)               summed over the terms t
// with A_t = c_t alpha_t / N^3 and B_t = alpha'_t / N^3 for the gain terms and
// A = -Lambda / N^3, B = 1 / N^3 for the last (loss) term, all zero on every
// |k_d| = N/2 mode.  Packing the two real inverse transforms of a term into
// one complex transform (a + i b) makes every pass a plain complex FFT.
//
// Passes (each pencil is one thread's register FFT, fft.cuh):
//   F1  rows along axis 2: two real rows packed per complex FFT, split into
//       their half spectra                                   -> Fh
//   F2  axis 1, F3 axis 0 (complex, in place on Fh)
//   per term t, per v0-slab s:
//   P1  axis 0 inverse for every (k1, k2) pencil of the full spectrum, built on
//       the fly from Fh (Hermitian partner for k2 > N/2) times (A + iB); only
//       the outputs v0 = s mod S0 are formed (decimation in frequency)  -> W
//   P2  axis 1 inverse on the slab (in place)
//   P3  axis 2 inverse per (v0, v1) row; G += Re * Im; the loss term writes
//       Q = G + Re * Im and clears G for the next cell
#pragma once
#include <cuda_runtime.h>

#include "coll_internal.h"
#include "collision_layout.cuh"
#include "fft.cuh"

namespace coll {

template <typename Tio, typename T> __device__ __forceinline__ T ld_io(const Tio* p) { return T(*p); }

// ------------------------------------------------------------ per-cell body
// smem: dynamic shared memory base; wsc: this CTA's workspace slice.
template <int N, typename T, typename Tio>
__device__ __forceinline__ void process_cell(const Tio* __restrict__ f, Tio* __restrict__ Q,
                                             const typename C2<T>::type* __restrict__ tab, int n_terms,
                                             unsigned char* smem, unsigned char* wsc, bool& bad) {
  using Ly = Lay<N, T>;
  using Cf = Cfg<N, T>;
  using V2 = typename C2<T>::type;
  constexpr int H = Ly::H, FR = Ly::FH_ROW, WR = Ly::W_ROW, S0 = Ly::S0, NS = Ly::NS;
  const int tid = threadIdx.x;

  unsigned char* sp = smem;
  unsigned char* gp = wsc;
  V2* W = reinterpret_cast<V2*>(Cf::W ? sp : gp);
  if (Cf::W) sp += Ly::round16(Ly::W_BYTES); else gp += Ly::round16(Ly::W_BYTES);
  V2* Fh = reinterpret_cast<V2*>(Cf::FH ? sp : gp);
  if (Cf::FH) sp += Ly::round16(Ly::FH_BYTES); else gp += Ly::round16(Ly::FH_BYTES);
  T* G = reinterpret_cast<T*>(Cf::G ? sp : gp);

  // ---- F1: real rows along axis 2, two per complex FFT -> half spectra
  for (int pid = tid; pid < N * N / 2; pid += kThreads) {
    const int r0 = 2 * pid, r1 = 2 * pid + 1;
    T zr[N], zi[N];
#pragma unroll
    for (int j = 0; j < N; ++j) {
      zr[j] = ld_io<Tio, T>(f + size_t(r0) * N + j);
      zi[j] = ld_io<Tio, T>(f + size_t(r1) * N + j);
    }
    fft<N, -1, T>(zr, zi);
    V2* o0 = Fh + size_t(r0) * FR;
    V2* o1 = Fh + size_t(r1) * FR;
#pragma unroll
    for (int k = 0; k < H; ++k) {
      const int kn = (N - k) % N;
      const T hr = T(0.5) * (zr[k] + zr[kn]), hi = T(0.5) * (zi[k] - zi[kn]);
      const T gr = T(0.5) * (zi[k] + zi[kn]), gi = T(0.5) * (zr[kn] - zr[k]);
      o0[k] = V2{hr, hi};
      o1[k] = V2{gr, gi};
    }
  }
  __syncthreads();
  // ---- F2: axis 1 (stride FR), pencils (j0, k2)
  for (int pid = tid; pid < N * H; pid += kThreads) {
    const int j0 = pid / H, k2 = pid % H;
    V2* p = Fh + size_t(j0) * N * FR + k2;
    T xr[N], xi[N];
#pragma unroll
    for (int j = 0; j < N; ++j) { V2 v = p[size_t(j) * FR]; xr[j] = v.x; xi[j] = v.y; }
    fft<N, -1, T>(xr, xi);
#pragma unroll
    for (int j = 0; j < N; ++j) p[size_t(j) * FR] = V2{xr[j], xi[j]};
  }
  __syncthreads();
  // ---- F3: axis 0 (stride N*FR), pencils (k1, k2)
  for (int pid = tid; pid < N * H; pid += kThreads) {
    const int k1 = pid / H, k2 = pid % H;
    V2* p = Fh + size_t(k1) * FR + k2;
    T xr[N], xi[N];
#pragma unroll
    for (int j = 0; j < N; ++j) { V2 v = p[size_t(j) * N * FR]; xr[j] = v.x; xi[j] = v.y; }
    fft<N, -1, T>(xr, xi);
#pragma unroll
    for (int j = 0; j < N; ++j) p[size_t(j) * N * FR] = V2{xr[j], xi[j]};
  }
  __syncthreads();

  for (int t = 0; t < n_terms; ++t) {
    const V2* __restrict__ tb = tab + size_t(t) * N * N * H;
    const bool last = (t == n_terms - 1);
    for (int s = 0; s < S0; ++s) {
      // ---- P1: axis-0 inverse of (A + iB) F for every full-spectrum pencil
      for (int pid = tid; pid < N * N; pid += kThreads) {
        const int k1 = pid / N, k2 = pid % N;
        T yr[NS], yi[NS];
        if (k2 == H || k1 == H) {
#pragma unroll
          for (int m = 0; m < NS; ++m) { yr[m] = T(0); yi[m] = T(0); }
        } else {
          const bool up = k2 > H;
          const int k2s = up ? N - k2 : k2;
          const int k1s = up ? (N - k1) % N : k1;
          const T cs = up ? T(-1) : T(1);          // conj for the Hermitian partner
#pragma unroll
          for (int kp = 0; kp < NS; ++kp) {
            T ar = T(0), ai = T(0);
#pragma unroll
            for (int q = 0; q < S0; ++q) {
              const int k0 = kp + q * NS;
              const int k0s = up ? (N - k0) % N : k0;
              const size_t idx = (size_t(k0s) * N + k1s);
              const V2 F = Fh[idx * FR + k2s];
              const V2 AB = tb[idx * H + k2s];
              const T fr = F.x, fi = cs * F.y;
              T xr = AB.x * fr - AB.y * fi;
              T xi = AB.x * fi + AB.y * fr;
              if (S0 > 1 && q > 0) {
                const int n = (s * q * (192 / S0)) % 192;
                const T c = Tw<T>::c(n), sn = Tw<T>::s(n);
                const T rr = xr * c - xi * sn;
                xi = xr * sn + xi * c;
                xr = rr;
              }
              ar += xr;
              ai += xi;
            }
            if (S0 > 1) {
              const int n = (s * kp * (192 / N)) % 192;
              const T c = Tw<T>::c(n), sn = Tw<T>::s(n);
              const T rr = ar * c - ai * sn;
              ai = ar * sn + ai * c;
              ar = rr;
            }
            yr[kp] = ar;
            yi[kp] = ai;
          }
          fft<NS, +1, T>(yr, yi);
        }
#pragma unroll
        for (int m = 0; m < NS; ++m) W[(size_t(m) * N + k1) * WR + k2] = V2{yr[m], yi[m]};
      }
      __syncthreads();
      // ---- P2: axis-1 inverse within the slab, pencils (m, k2)
      for (int pid = tid; pid < NS * N; pid += kThreads) {
        const int m = pid / N, k2 = pid % N;
        if (k2 == H) continue;                      // Nyquist plane stays zero
        V2* p = W + size_t(m) * N * WR + k2;
        T xr[N], xi[N];
#pragma unroll
        for (int j = 0; j < N; ++j) { V2 v = p[size_t(j) * WR]; xr[j] = v.x; xi[j] = v.y; }
        fft<N, +1, T>(xr, xi);
#pragma unroll
        for (int j = 0; j < N; ++j) p[size_t(j) * WR] = V2{xr[j], xi[j]};
      }
      __syncthreads();
      // ---- P3: axis-2 inverse per row; accumulate Re * Im
      for (int pid = tid; pid < NS * N; pid += kThreads) {
        const int m = pid / N, v1 = pid % N;
        const V2* p = W + (size_t(m) * N + v1) * WR;
        T xr[N], xi[N];
#pragma unroll
        for (int j = 0; j < N; ++j) { V2 v = p[j]; xr[j] = v.x; xi[j] = v.y; }
        fft<N, +1, T>(xr, xi);
        const int v0 = s + S0 * m;
        T* g = G + (size_t(v0) * N + v1) * N;
        if (!last) {
#pragma unroll
          for (int j = 0; j < N; ++j) g[j] += xr[j] * xi[j];
        } else {
          Tio* q = Q + (size_t(v0) * N + v1) * N;
#pragma unroll
          for (int j = 0; j < N; ++j) {
            const T val = g[j] + xr[j] * xi[j];
            bad |= !isfinite(val);
            q[j] = Tio(val);
            g[j] = T(0);
          }
        }
      }
      __syncthreads();
    }
  }
}

template <int N, typename T>
__device__ __forceinline__ void zero_gain(unsigned char* smem, unsigned char* wsc) {
  using Ly = Lay<N, T>;
  using Cf = Cfg<N, T>;
  unsigned char* sp = smem;
  unsigned char* gp = wsc;
  if (Cf::W) sp += Ly::round16(Ly::W_BYTES); else gp += Ly::round16(Ly::W_BYTES);
  if (Cf::FH) sp += Ly::round16(Ly::FH_BYTES); else gp += Ly::round16(Ly::FH_BYTES);
  T* G = reinterpret_cast<T*>(Cf::G ? sp : gp);
  for (int i = threadIdx.x; i < N * N * N; i += kThreads) G[i] = T(0);
}

template <int N, typename T, typename Tio>
__global__ void __launch_bounds__(kThreads, 1) collision_kernel(CollArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned char* wsc = static_cast<unsigned char*>(a.ws) + size_t(blockIdx.x) * a.ws_per_cta;
  zero_gain<N, T>(smem, wsc);
  __syncthreads();
  bool bad = false;
  const auto* tab = static_cast<const typename C2<T>::type*>(a.tab);
  for (long long c = blockIdx.x; c < a.n_cells; c += gridDim.x) {
    const Tio* f = static_cast<const Tio*>(a.f) + size_t(c) * N * N * N;
    Tio* Q = static_cast<Tio*>(a.Q) + size_t(c) * N * N * N;
    process_cell<N, T, Tio>(f, Q, tab, a.n_terms, smem, wsc, bad);
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(a.status, kStatusNonFinite);
}

template <int N, typename T, typename Tio>
int launch_one(const CollArgs& a, int grid, cudaStream_t st) {
  constexpr size_t smem = Lay<N, T>::SMEM;
  auto k = collision_kernel<N, T, Tio>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return int(e);
  k<<<grid, kThreads, smem, st>>>(a);
  return int(cudaGetLastError());
}

template <int N, typename T, typename Tio>
int occupancy_one(int* ctas) {
  constexpr size_t smem = Lay<N, T>::SMEM;
  auto k = collision_kernel<N, T, Tio>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return int(e);
  return int(cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, k, kThreads, smem));
}

}  // namespace coll
