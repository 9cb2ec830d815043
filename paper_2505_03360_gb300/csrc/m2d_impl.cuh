// Fast spectral collision operator for Maxwell molecules in two velocity
// dimensions (arxiv 2505.03360, sec. 4.4.1, "The 2d case"): the Carleman
// weight is constant, so K(l, m) = sum_p c alpha_p(l) alpha'_p(m) with
// alpha_p(xi) = phi(xi . e_p), alpha'_p(xi) = phi(xi . e_p^perp),
// phi(s) = 2R sinc(R s), theta_p = p pi / A and c = 2 b0 pi / A.
//
// Per cell (one CTA, persistent over cells), in index space:
//   F    = DFT2(f)                      half spectrum k1 < N/2, |k_d| = N/2 dropped
//   z_t  = IDFT2((A_t + i B_t) F)       one complex inverse 2D FFT per term
//   Q    = sum_t Re(z_t) Im(z_t)
// with (A_t, B_t) = (c alpha_p / N^2, alpha'_p / N^2) for the A gain terms and
// (-Lambda / N^2, 1 / N^2) for the loss term (the plan's table).  The grid
// offset v_0 = -L cancels because every multiplier is real and even.
//
// A 2D cell has only N pencils per axis, too few for a CTA, so TB terms run
// side by side (TB N threads; 128 threads for N <= 32, so that two CTAs share
// an SM and one's barriers and partial batches overlap the other's work): pass A (thread = term, column k1) forms the
// column of (A + iB) F from the half spectrum and transforms it along k0;
// pass B (thread = term, row v0) transforms the row along k1 and writes
// Re * Im over the row it has just read; a reduction over the TB terms adds
// the products into the gain accumulator, which lives in registers (N^2 / (TB N)
// values per thread).  Every array is in shared memory: nothing but f, Q and
// the table touches global memory.
#pragma once
#include <cuda_runtime.h>

#include "coll_internal.h"
#include "collision_layout.cuh"
#include "fft.cuh"

namespace coll {

template <int N, typename T> struct M2Lay {
  using V2 = typename C2<T>::type;
  static constexpr int H = N / 2;
  static constexpr int TB = N == 64 ? 4 : 128 / N;    // terms side by side
  static constexpr int THREADS = TB * N;
  static constexpr int WR = N + 1;                     // W row pitch (complex), conflict-free rows
  static constexpr int FR = H + 1;                     // Fh row pitch (complex)
  static constexpr int E = N * N / THREADS;            // accumulator values per thread
  static constexpr size_t W_BYTES = size_t(TB) * N * WR * sizeof(V2);
  static constexpr size_t FH_BYTES = size_t(N) * FR * sizeof(V2);
  static constexpr size_t SMEM = W_BYTES + FH_BYTES;
  static_assert(N == 16 || N == 32 || N == 64, "N in {16, 32, 64}");
  static_assert(SMEM <= 227 * 1024, "shared memory");
};

template <typename Tio, typename T> __device__ __forceinline__ T m2_ld(Tio v) { return T(v); }
template <> __device__ __forceinline__ df m2_ld<double, df>(double v) { return df_from_double(v); }
template <> __device__ __forceinline__ df m2_ld<float, df>(float v) { return df_from_float(v); }
template <typename Tio, typename T> __device__ __forceinline__ Tio m2_st(T v) { return Tio(v); }
template <> __device__ __forceinline__ double m2_st<double, df>(df v) { return df_to_double(v); }
template <> __device__ __forceinline__ float m2_st<float, df>(df v) { return __fadd_rn(v.h, v.l); }
__device__ __forceinline__ bool m2_finite(double x) { return ::isfinite(x); }
__device__ __forceinline__ bool m2_finite(float x) { return ::isfinite(x); }

template <int N, typename T, typename Tio>
__global__ void __launch_bounds__(M2Lay<N, T>::THREADS, 1) m2d_kernel(M2Args a) {
  using Ly = M2Lay<N, T>;
  using V2 = typename Ly::V2;
  constexpr int H = Ly::H, TB = Ly::TB, WR = Ly::WR, FR = Ly::FR, E = Ly::E, NT = Ly::THREADS;
  extern __shared__ __align__(16) unsigned char smem[];
  V2* W = reinterpret_cast<V2*>(smem);
  V2* Fh = reinterpret_cast<V2*>(smem + Ly::W_BYTES);
  Tio* fs = reinterpret_cast<Tio*>(smem);                 // staged f, rows of pitch N + 1 (in W)
  const V2* tab = static_cast<const V2*>(a.tab);
  const int tid = threadIdx.x;
  bool bad = false;

  for (long long c = blockIdx.x; c < a.n_cells; c += gridDim.x) {
    const Tio* f = static_cast<const Tio*>(a.f) + size_t(c) * N * N;
    __syncthreads();                                     // the previous cell is done with W
    for (int i = tid; i < N * N; i += NT) fs[(i / N) * (N + 1) + i % N] = f[i];
    __syncthreads();

    // forward, axis 1: rows p and p + N/2 packed into one complex transform,
    // split into their half spectra (conj in and out: forward by the inverse kernel)
    if (tid < H) {
      T xr[N], xi[N];
      const Tio* r0 = fs + tid * (N + 1);
      const Tio* r1 = fs + (tid + H) * (N + 1);
#pragma unroll
      for (int j = 0; j < N; ++j) {
        xr[j] = m2_ld<Tio, T>(r0[j]);
        xi[j] = -m2_ld<Tio, T>(r1[j]);
      }
      fft<N, +1, T>(xr, xi);
      V2* o0 = Fh + tid * FR;
      V2* o1 = Fh + (tid + H) * FR;
#pragma unroll
      for (int k = 0; k < H; ++k) {
        const int kn = (N - k) % N;
        const T zrk = xr[k], zik = -xi[k], zrn = xr[kn], zin = -xi[kn];
        o0[k] = V2{half(zrk + zrn), half(zik - zin)};
        o1[k] = V2{half(zik + zin), half(zrn - zrk)};
      }
    }
    __syncthreads();
    // forward, axis 0, per column k1 < N/2; the Nyquist row k0 = N/2 is dropped
    if (tid < H) {
      T xr[N], xi[N];
#pragma unroll
      for (int j = 0; j < N; ++j) {
        const V2 v = Fh[j * FR + tid];
        xr[j] = v.x;
        xi[j] = -v.y;
      }
      fft<N, +1, T>(xr, xi);
#pragma unroll
      for (int k = 0; k < N; ++k) Fh[k * FR + tid] = k == H ? V2{T{}, T{}} : V2{xr[k], -xi[k]};
    }
    __syncthreads();

    T G[E];
#pragma unroll
    for (int e = 0; e < E; ++e) G[e] = T{};
    const int tb = tid / N, ln = tid % N;
    for (int t0 = 0; t0 < a.n_terms; t0 += TB) {
      const int t = t0 + tb;
      V2* Wt = W + size_t(tb) * N * WR;
      // pass A: column k1 = ln of (A + iB) F (Hermitian partner for k1 > N/2), inverse along k0
      if (t < a.n_terms && ln != H) {
        const bool up = ln > H;
        const int k1s = up ? N - ln : ln;
        const V2* tt = tab + size_t(t) * N * H;
        T xr[N], xi[N];
#pragma unroll
        for (int k0 = 0; k0 < N; ++k0) {
          const int k0s = up ? (N - k0) % N : k0;
          const V2 F = Fh[k0s * FR + k1s];
          const V2 AB = tt[k0s * H + k1s];
          const T fr = F.x, fi = up ? -F.y : F.y;
          xr[k0] = AB.x * fr - AB.y * fi;
          xi[k0] = AB.x * fi + AB.y * fr;
        }
        fft<N, +1, T>(xr, xi);
#pragma unroll
        for (int v0 = 0; v0 < N; ++v0) Wt[v0 * WR + ln] = V2{xr[v0], xi[v0]};
      }
      __syncthreads();
      // pass B: row v0 = ln, inverse along k1 (column N/2 is zero), Re * Im over the row
      if (t < a.n_terms) {
        V2* row = Wt + ln * WR;
        T xr[N], xi[N];
#pragma unroll
        for (int k1 = 0; k1 < N; ++k1) {
          if (k1 == H) {
            xr[k1] = T{};
            xi[k1] = T{};
          } else {
            const V2 v = row[k1];
            xr[k1] = v.x;
            xi[k1] = v.y;
          }
        }
        fft<N, +1, T>(xr, xi);
        T* prow = reinterpret_cast<T*>(row);
#pragma unroll
        for (int v1 = 0; v1 < N; ++v1) prow[v1] = xr[v1] * xi[v1];
      }
      __syncthreads();
      const int nb = a.n_terms - t0 < TB ? a.n_terms - t0 : TB;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int idx = tid + e * NT, v0 = idx / N, v1 = idx % N;
        T s = G[e];
        for (int b = 0; b < nb; ++b) s = s + reinterpret_cast<const T*>(W + (size_t(b) * N + v0) * WR)[v1];
        G[e] = s;
      }
      __syncthreads();
    }
    Tio* Q = static_cast<Tio*>(a.Q) + size_t(c) * N * N;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const Tio q = m2_st<Tio, T>(G[e]);
      bad |= !m2_finite(q);
      Q[tid + e * NT] = q;
    }
  }
  if (__syncthreads_or(bad) && tid == 0) atomicOr(a.status, kStatusNonFinite);
}

template <int N, typename T, typename Tio>
int m2d_launch_t(const M2Args& a, int grid, cudaStream_t st) {
  auto k = m2d_kernel<N, T, Tio>;
  constexpr size_t smem = M2Lay<N, T>::SMEM;
  const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return int(e);
  k<<<grid, M2Lay<N, T>::THREADS, smem, st>>>(a);
  return int(cudaGetLastError());
}

template <int N, typename T, typename Tio>
int m2d_occupancy_t(int* ctas) {
  auto k = m2d_kernel<N, T, Tio>;
  constexpr size_t smem = M2Lay<N, T>::SMEM;
  const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return int(e);
  return int(cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, k, M2Lay<N, T>::THREADS, smem));
}


// Dispatch over N and the io type for one compute type T (m2d_d.cu, m2d_f.cu, m2d_x.cu).
template <typename T, int... Ns> struct M2Dispatch;
template <typename T> struct M2Dispatch<T> {
  static int launch(int, bool, const M2Args&, int, cudaStream_t) { return int(cudaErrorInvalidValue); }
  static int occupancy(int, bool, int*) { return int(cudaErrorInvalidValue); }
};
template <typename T, int N0, int... Ns> struct M2Dispatch<T, N0, Ns...> {
  static int launch(int N, bool io_f64, const M2Args& a, int grid, cudaStream_t st) {
    if (N != N0) return M2Dispatch<T, Ns...>::launch(N, io_f64, a, grid, st);
    return io_f64 ? m2d_launch_t<N0, T, double>(a, grid, st) : m2d_launch_t<N0, T, float>(a, grid, st);
  }
  static int occupancy(int N, bool io_f64, int* ctas) {
    if (N != N0) return M2Dispatch<T, Ns...>::occupancy(N, io_f64, ctas);
    return io_f64 ? m2d_occupancy_t<N0, T, double>(ctas) : m2d_occupancy_t<N0, T, float>(ctas);
  }
};

}  // namespace coll
