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
//   per v0-slab s (planes v0 = s mod S0), per term t:
//   P1  axis 0 inverse for every (k1, k2) pencil of the full spectrum, built on
//       the fly from Fh (Hermitian partner for k2 > N/2) times (A + iB); only
//       the outputs of slab s are formed (decimation in frequency)   -> W
//   P2  axis 1 inverse on the slab (in place)
//   P3  axis 2 inverse per (v0, v1) row; G_s += Re * Im; the loss term
//       writes Q = G_s + Re * Im for the slab's planes
// Slabs outermost keep only one slab of the gain accumulator live, so it
// stays in shared memory.  F1, F2, F3, P2 and P3 share one FFT body (a
// non-inlined pass function; forward transforms by conjugation) to keep the
// instruction footprint small.
#pragma once
#include <cuda_runtime.h>

#include <initializer_list>

#include "coll_internal.h"
#include "collision_layout.cuh"
#include "fft.cuh"
#include "tcgen05.cuh"

namespace coll {

template <typename Tio, typename T> __device__ __forceinline__ T ld_io(const Tio* p) { return T(*p); }
template <> __device__ __forceinline__ df ld_io<double, df>(const double* p) { return df_from_double(*p); }
template <> __device__ __forceinline__ df ld_io<float, df>(const float* p) { return df_from_float(*p); }
template <typename Tio, typename T> __device__ __forceinline__ Tio to_io(T v) { return Tio(v); }
template <> __device__ __forceinline__ double to_io<double, df>(df v) { return df_to_double(v); }
template <> __device__ __forceinline__ float to_io<float, df>(df v) { return __fadd_rn(v.h, v.l); }
__device__ __forceinline__ bool finite_v(double x) { return ::isfinite(x); }
__device__ __forceinline__ bool finite_v(float x) { return ::isfinite(x); }
__device__ __forceinline__ bool finite_v(df x) { return isfinite(x); }

// The term tables are read by every CTA for every cell and are read-only for
// the kernel's lifetime.  At N >= 48, where the per-CTA workspaces exceed L2,
// their loads carry an L2 evict_last policy so that the tables stay (measured
// 2.5-3 % faster at N = 48 and 64; at N = 32, where the workspaces fit, plain
// loads are as fast or faster).  A hint only: the values are those of plain loads.
template <int N> constexpr bool kKeepTables = N >= 48;
__device__ __forceinline__ unsigned long long l2_keep() {
  unsigned long long p;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
// read-only (non-coherent path) global load of an 8- or 16-byte table element under an L2 policy
template <typename V>
__device__ __forceinline__ V ldg_pol(const V* p, unsigned long long pol) {
  static_assert(sizeof(V) == 8 || sizeof(V) == 16, "complex element of 8 or 16 bytes");
  if constexpr (sizeof(V) == 8) {
    union { uint2 u; V v; } r;
    asm("ld.global.nc.L2::cache_hint.v2.u32 {%0, %1}, [%2], %3;" : "=r"(r.u.x), "=r"(r.u.y) : "l"(p), "l"(pol));
    return r.v;
  } else {
    union { uint4 u; V v; } r;
    asm("ld.global.nc.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
        : "=r"(r.u.x), "=r"(r.u.y), "=r"(r.u.z), "=r"(r.u.w) : "l"(p), "l"(pol));
    return r.v;
  }
}

enum PassMode : int { kPassF1 = 0, kPassFwd = 1, kPassInv = 2, kPassP3 = 3 };

// One pass of length-N register FFTs over a set of pencils (this thread's: p0,
// p0 + pstep, ...; by default threadIdx.x in steps of the CTA).  Pencil pid maps to
// (a, b) = (pid / inner, pid % inner) and starts at base + a*s_outer + b*s_inner;
// its elements are s_elem apart.  Modes:
//   kPassF1   two real rows of f packed into one complex FFT, split into the
//             two half spectra (rows 2 pid, 2 pid + 1 of Fh = base)
//   kPassFwd  forward transform in place (as conj(IFFT(conj x)))
//   kPassInv  inverse transform in place; pencils with b == skip_b are zero
//   kPassP3   inverse transform of W rows, then G += Re*Im (or, on the last
//             term, Q = G + Re*Im for the planes v0 = s + S0 m)
// Returns true if a non-finite output was written.
template <int N, typename T, typename Tio>
__device__ __noinline__ bool run_pass(int mode, typename C2<T>::type* base, int count, int inner, int s_outer,
                                      int s_inner, int s_elem, int skip_b, const Tio* __restrict__ f, Tio* Q,
                                      T* G, int s, int S0, int fh_row, bool last, int p0 = -1, int pstep = kThreads) {
  using V2 = typename C2<T>::type;
  constexpr int H = N / 2;
  bool bad = false;
  for (int pid = p0 < 0 ? int(threadIdx.x) : p0; pid < count; pid += pstep) {
    const int a = pid / inner, b = pid % inner;
    if (mode == kPassInv && b == skip_b) continue;
    T xr[N], xi[N];
    V2* p = base + size_t(a) * s_outer + size_t(b) * s_inner;
    if (mode == kPassF1) {
      const Tio* r0 = f + size_t(2 * pid) * N;
#pragma unroll
      for (int j = 0; j < N; ++j) {
        xr[j] = ld_io<Tio, T>(r0 + j);
        xi[j] = -ld_io<Tio, T>(r0 + N + j);     // conj for the forward transform
      }
    } else {
#pragma unroll
      for (int j = 0; j < N; ++j) {
        const V2 v = p[size_t(j) * s_elem];
        xr[j] = v.x;
        xi[j] = (mode == kPassFwd) ? -v.y : v.y;
      }
    }
    fft<N, +1, T>(xr, xi);
    if (mode == kPassF1) {
      // Z = conj(xi) is the forward transform of row0 + i row1; split
      V2* o0 = base + size_t(2 * pid) * fh_row;
      V2* o1 = o0 + fh_row;
#pragma unroll
      for (int k = 0; k < H; ++k) {
        const int kn = (N - k) % N;
        const T zrk = xr[k], zik = -xi[k], zrn = xr[kn], zin = -xi[kn];
        o0[k] = V2{half(zrk + zrn), half(zik - zin)};
        o1[k] = V2{half(zik + zin), half(zrn - zrk)};
      }
    } else if (mode == kPassFwd || mode == kPassInv) {
#pragma unroll
      for (int j = 0; j < N; ++j) p[size_t(j) * s_elem] = V2{xr[j], (mode == kPassFwd) ? -xi[j] : xi[j]};
    } else {
      T* g = G + (size_t(a) * N + b) * (N + 1);          // padded rows: conflict-free row access
      if (!last) {
#pragma unroll
        for (int j = 0; j < N; ++j) g[j] += xr[j] * xi[j];
      } else {
        const int v0 = s + S0 * a;
        Tio* q = Q + (size_t(v0) * N + b) * N;
#pragma unroll
        for (int j = 0; j < N; ++j) {
          const T val = g[j] + xr[j] * xi[j];
          bad |= !finite_v(val);
          q[j] = to_io<Tio, T>(val);
        }
      }
    }
  }
  return bad;
}

// (xr, xi) times i^m, m in 0..3, by selects (the slab index is a runtime
// value, so these exact rotations would otherwise cost a complex multiply).
// Used for FP64, whose pipe bounds the kernel; for the FP32-pipe types the
// extra branches and selects cost more than the multiplies they save.
template <typename T> constexpr bool kQuarterBySelect = false;
template <> constexpr bool kQuarterBySelect<double> = true;
template <typename T>
__device__ __forceinline__ void rotate_quarter(T& xr, T& xi, int m) {
  const T r = xr, i = xi;
  const T nr = -r, ni = -i;
  xr = m == 0 ? r : (m == 1 ? ni : (m == 2 ? nr : i));
  xi = m == 0 ? i : (m == 1 ? r : (m == 2 ? ni : nr));
}

// P1: axis-0 inverse of (A + iB) F for every full-spectrum pencil (k1, k2),
// forming only the outputs v0 = s + S0 m (decimation in frequency):
//   y[k'] = w_N^{s k'} sum_q x[k' + q NS] e^{2 pi i s q / S0},  then an NS-point IFFT.
template <int N, typename T, int V>
__device__ __noinline__ void run_p1(const typename C2<T>::type* __restrict__ tb, const typename C2<T>::type* Fh,
                                    typename C2<T>::type* W, int s) {
  using Ly = Lay<N, T, V>;
  using V2 = typename C2<T>::type;
  constexpr int H = Ly::H, FR = Ly::FH_ROW, WR = Ly::W_ROW, S0 = Ly::S0, NS = Ly::NS;
  const unsigned long long keep = l2_keep();
  for (int pid = threadIdx.x; pid < N * N; pid += kThreads) {
    const int k1 = pid / N, k2 = pid % N;
    T yr[NS], yi[NS];
    if (k2 == H || k1 == H) {
#pragma unroll
      for (int m = 0; m < NS; ++m) { yr[m] = T{}; yi[m] = T{}; }
    } else {
      const bool up = k2 > H;
      const int k2s = up ? N - k2 : k2;
      const int k1s = up ? (N - k1) % N : k1;
#pragma unroll
      for (int kp = 0; kp < NS; ++kp) {
        T ar = T{}, ai = T{};
#pragma unroll
        for (int q = 0; q < S0; ++q) {
          const int k0 = kp + q * NS;
          const int k0s = up ? (N - k0) % N : k0;
          const size_t idx = (size_t(k0s) * N + k1s);
          const V2 F = Fh[idx * FR + k2s];
          V2 AB;
          if constexpr (kKeepTables<N>) AB = ldg_pol(tb + idx * H + k2s, keep);
          else AB = tb[idx * H + k2s];
          const T fr = F.x, fi = up ? -F.y : F.y;   // conj for the Hermitian partner
          T xr = AB.x * fr - AB.y * fi;
          T xi = AB.x * fi + AB.y * fr;
          if (S0 > 1 && q > 0) {
            const int n = (s * q * (192 / S0)) % 192;
            if (kQuarterBySelect<T> && n % 48 == 0) {
              rotate_quarter(xr, xi, n / 48);             // +-1, +-i: no multiplies (uniform branch)
            } else {
              const T c = Tw<T>::c(n), sn = Tw<T>::s(n);
              const T rr = xr * c - xi * sn;
              xi = xr * sn + xi * c;
              xr = rr;
            }
          }
          ar = ar + xr;
          ai = ai + xi;
        }
        if (S0 > 1) {
          const int n = (s * kp * (192 / N)) % 192;
          if (kQuarterBySelect<T> && n % 48 == 0) {
            rotate_quarter(ar, ai, n / 48);
          } else {
            const T c = Tw<T>::c(n), sn = Tw<T>::s(n);
            const T rr = ar * c - ai * sn;
            ai = ar * sn + ai * c;
            ar = rr;
          }
        }
        yr[kp] = ar;
        yi[kp] = ai;
      }
      fft<NS, +1, T>(yr, yi);
    }
#pragma unroll
    for (int m = 0; m < NS; ++m) W[(size_t(m) * N + k1) * WR + k2] = V2{yr[m], yi[m]};
  }
}

// P1F: full axis-0 inverse of (A + iB) F for every full-spectrum pencil
// (k1, k2) (no slab split; this thread's pencils as in run_pass), into the term
// buffer Wg[v0][k1][k2] (global).
template <int N, typename T, int V>
__device__ __noinline__ void run_p1f(const typename C2<T>::type* __restrict__ tb, const typename C2<T>::type* Fh,
                                     typename C2<T>::type* Wg, int p0 = -1, int pstep = kThreads) {
  using Ly = Lay<N, T, V>;
  using V2 = typename C2<T>::type;
  constexpr int H = Ly::H, FR = Ly::FH_ROW;
  const unsigned long long keep = l2_keep();
  for (int pid = p0 < 0 ? int(threadIdx.x) : p0; pid < N * N; pid += pstep) {
    const int k1 = pid / N, k2 = pid % N;
    T xr[N], xi[N];
    if (k2 == H || k1 == H) {
#pragma unroll
      for (int k0 = 0; k0 < N; ++k0) { xr[k0] = T{}; xi[k0] = T{}; }
    } else {
      const bool up = k2 > H;
      const int k2s = up ? N - k2 : k2;
      const int k1s = up ? (N - k1) % N : k1;
#pragma unroll
      for (int k0 = 0; k0 < N; ++k0) {
        const int k0s = up ? (N - k0) % N : k0;
        const size_t idx = (size_t(k0s) * N + k1s);
        const V2 F = Fh[idx * FR + k2s];
        V2 AB;
        if constexpr (kKeepTables<N>) AB = ldg_pol(tb + idx * H + k2s, keep);
        else AB = tb[idx * H + k2s];
        const T fr = F.x, fi = up ? -F.y : F.y;   // conj for the Hermitian partner
        xr[k0] = AB.x * fr - AB.y * fi;
        xi[k0] = AB.x * fi + AB.y * fr;
      }
      fft<N, +1, T>(xr, xi);
    }
#pragma unroll
    for (int v0 = 0; v0 < N; ++v0) Wg[(size_t(v0) * N + k1) * N + k2] = V2{xr[v0], xi[v0]};
  }
}

// asynchronous global -> shared copies of 16 or 8 bytes (and their completion);
// both addresses aligned to the copy size
__device__ __forceinline__ void cp16(void* dst_smem, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(static_cast<unsigned>(__cvta_generic_to_shared(dst_smem))),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp8(void* dst_smem, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(static_cast<unsigned>(__cvta_generic_to_shared(dst_smem))),
               "l"(src)
               : "memory");
}
template <typename V2> __device__ __forceinline__ void cp_elem(V2* dst_smem, const V2* src) {
  static_assert(sizeof(V2) == 16 || sizeof(V2) == 8, "complex element of 8 or 16 bytes");
  if constexpr (sizeof(V2) == 16) cp16(dst_smem, src); else cp8(dst_smem, src);
}
__device__ __forceinline__ void cp16_wait() { asm volatile("cp.async.commit_group;\n cp.async.wait_group 0;" ::: "memory"); }


// ------------------------------------------------------------ per-cell body
// smem: dynamic shared memory base; wsc: this CTA's workspace slice.
template <int N, typename T, typename Tio, int V = 0>
__device__ __forceinline__ void process_cell(const Tio* __restrict__ f, Tio* __restrict__ Q,
                                             const typename C2<T>::type* __restrict__ tab, int n_terms,
                                             unsigned char* smem, unsigned char* wsc, bool& bad) {
  using Ly = Lay<N, T, V>;
  using Cf = Cfg<N, T, V>;
  using V2 = typename C2<T>::type;
  constexpr int H = Ly::H, FR = Ly::FH_ROW, WR = Ly::W_ROW, S0 = Ly::S0, NS = Ly::NS;

  unsigned char* sp = smem;
  unsigned char* gp = wsc;
  V2* W = reinterpret_cast<V2*>(Cf::W ? sp : gp);
  if (Cf::W) sp += Ly::round16(Ly::W_BYTES); else gp += Ly::round16(Ly::W_BYTES);
  V2* Fh = reinterpret_cast<V2*>(Cf::FH ? sp : gp);
  if (Cf::FH) sp += Ly::round16(Ly::FH_BYTES); else gp += Ly::round16(Ly::FH_BYTES);
  T* G = reinterpret_cast<T*>(Cf::G ? sp : gp);

  // forward half spectrum: rows (F1), axis 1 (F2), axis 0 (F3)
  run_pass<N, T, Tio>(kPassF1, Fh, N * N / 2, 1, 0, 0, 1, -1, f, Q, G, 0, S0, FR, false);
  __syncthreads();
  run_pass<N, T, Tio>(kPassFwd, Fh, N * H, H, N * FR, 1, FR, -1, f, Q, G, 0, S0, FR, false);
  __syncthreads();
  run_pass<N, T, Tio>(kPassFwd, Fh, N * H, H, FR, 1, N * FR, -1, f, Q, G, 0, S0, FR, false);
  __syncthreads();

  if constexpr (Cf::P1F) {
    // terms outer: one full axis-0 pass per term into Wg, then per slab (planes
    // v0 = s NS .. s NS + NS - 1): copy the slab into W, restore the slab's
    // gain accumulator, axis 1, axis 2 with G += Re*Im (Q on the last term),
    // save the accumulator.
    V2* Wg = reinterpret_cast<V2*>(gp);
    gp += Ly::round16(Ly::WG_BYTES);
    T* Gg = reinterpret_cast<T*>(gp);
    constexpr int GSLAB = NS * N * (N + 1);                 // doubles of one slab of G
    for (int t = 0; t < n_terms; ++t) {
      run_p1f<N, T, V>(tab + size_t(t) * N * N * H, Fh, Wg);
      __syncthreads();
      for (int s = 0; s < S0; ++s) {
        const V2* src = Wg + size_t(s) * NS * N * N;
        for (int i = threadIdx.x; i < NS * N * N; i += kThreads) {
          const int m = i / (N * N), rem = i % (N * N);
          cp_elem(W + (size_t(m) * N + rem / N) * WR + rem % N, src + i);
        }
        if (t == 0) {
          for (int i = threadIdx.x; i < GSLAB; i += kThreads) G[i] = T{};
        } else {
          static_assert((GSLAB * sizeof(T)) % 16 == 0, "G slab copy in 16-byte pieces");
          const unsigned char* gsrc = reinterpret_cast<const unsigned char*>(Gg + size_t(s) * GSLAB);
          for (int i = threadIdx.x; i < GSLAB * int(sizeof(T)) / 16; i += kThreads)
            cp16(reinterpret_cast<unsigned char*>(G) + 16 * i, gsrc + 16 * i);
        }
        cp16_wait();
        __syncthreads();
        run_pass<N, T, Tio>(kPassInv, W, NS * N, N, N * WR, 1, WR, H, f, Q, G, s * NS, 1, FR, false);
        __syncthreads();
        const bool last = t == n_terms - 1;
        bad |= run_pass<N, T, Tio>(kPassP3, W, NS * N, N, N * WR, WR, 1, -1, f, Q, G, s * NS, 1, FR, last);
        __syncthreads();
        if (!last) {
          uint4* gdst = reinterpret_cast<uint4*>(Gg + size_t(s) * GSLAB);
          const uint4* gs = reinterpret_cast<const uint4*>(G);
          for (int i = threadIdx.x; i < GSLAB * int(sizeof(T)) / 16; i += kThreads) gdst[i] = gs[i];
          __syncthreads();
        }
      }
    }
  } else {
    for (int s = 0; s < S0; ++s) {
      for (int i = threadIdx.x; i < NS * N * (N + 1); i += kThreads) G[i] = T{};
      __syncthreads();
      for (int t = 0; t < n_terms; ++t) {
        run_p1<N, T, V>(tab + size_t(t) * N * N * H, Fh, W, s);
        __syncthreads();
        run_pass<N, T, Tio>(kPassInv, W, NS * N, N, N * WR, 1, WR, H, f, Q, G, s, S0, FR, false);
        __syncthreads();
        bad |= run_pass<N, T, Tio>(kPassP3, W, NS * N, N, N * WR, WR, 1, -1, f, Q, G, s, S0, FR,
                                   t == n_terms - 1);
        __syncthreads();
      }
    }
  }
}

template <int N, typename T, typename Tio, int V>
__global__ void __launch_bounds__(kThreads, 1) collision_kernel(CollArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned char* wsc = static_cast<unsigned char*>(a.ws) + size_t(blockIdx.x) * a.ws_per_cta;
  bool bad = false;
  const auto* tab = static_cast<const typename C2<T>::type*>(a.tab);
  for (long long c = blockIdx.x; c < a.n_cells; c += gridDim.x) {
    const Tio* f = static_cast<const Tio*>(a.f) + size_t(c) * N * N * N;
    Tio* Q = static_cast<Tio*>(a.Q) + size_t(c) * N * N * N;
    process_cell<N, T, Tio, V>(f, Q, tab, a.n_terms, smem, wsc, bad);
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(a.status, kStatusNonFinite);
}

// Persistent kernel over a ragged table of cell groups (mixed N): CTAs take
// cells from a global counter in schedule order (the host sorts the groups by
// decreasing N, largest work first); each cell runs the per-N body above.
template <typename T, typename Tio, int... Ns>
struct RaggedDispatch;

template <typename T, typename Tio>
struct RaggedDispatch<T, Tio> {
  static __device__ __forceinline__ void run(int, int, const Tio*, Tio*, const typename C2<T>::type*, int,
                                             unsigned char*, unsigned char*, bool&) {}
};

// One cell in one (N, slab shape) as a separate function: each body gets its own
// register allocation instead of the union of all of them inside the ragged kernel.
template <int N, typename T, typename Tio, int V>
__device__ __noinline__ bool ragged_cell(const Tio* f, Tio* Q, const typename C2<T>::type* tab, int nt,
                                         unsigned char* smem, unsigned char* wsc) {
  bool bad = false;
  process_cell<N, T, Tio, V>(f, Q, tab, nt, smem, wsc, bad);
  return bad;
}

// per-N body in the slab shape the group's plan uses (so that a ragged launch
// equals coll_eval_batch of each group alone, whichever shape the autotuner chose)
template <typename T, typename Tio, int N0, int... Ns>
struct RaggedDispatch<T, Tio, N0, Ns...> {
  static __device__ __forceinline__ void run(int N, int V, const Tio* f, Tio* Q, const typename C2<T>::type* tab,
                                             int nt, unsigned char* smem, unsigned char* wsc, bool& bad) {
    if (N == N0) {
      if (V == 1) bad |= ragged_cell<N0, T, Tio, RaggedBody<N0, T, 1>::v>(f, Q, tab, nt, smem, wsc);
      else bad |= ragged_cell<N0, T, Tio, RaggedBody<N0, T, 0>::v>(f, Q, tab, nt, smem, wsc);
    } else {
      RaggedDispatch<T, Tio, Ns...>::run(N, V, f, Q, tab, nt, smem, wsc, bad);
    }
  }
};

template <typename T, typename Tio, int... Ns>
__global__ void __launch_bounds__(kThreads, 1) ragged_kernel(RaggedTable tbl, void* ws, size_t ws_per_cta) {
  extern __shared__ __align__(16) unsigned char smem[];
  // the whole dynamic shared memory may be in use by the largest N, so the
  // work-unit broadcast goes through a 256-byte header of the CTA's workspace
  unsigned long long* counter = static_cast<unsigned long long*>(ws);
  unsigned char* slice = static_cast<unsigned char*>(ws) + 256 + size_t(blockIdx.x) * ws_per_cta;
  volatile long long* unit_slot = reinterpret_cast<volatile long long*>(slice);
  unsigned char* wsc = slice + 256;
  for (;;) {
    if (threadIdx.x == 0) *unit_slot = (long long)atomicAdd(counter, 1ull);
    __syncthreads();
    const long long u = *unit_slot;
    __syncthreads();
    if (u >= tbl.total_units) break;
    int g = 0;
    while (g + 1 < tbl.n_items && u >= tbl.items[g + 1].first_unit) ++g;
    const RaggedItem& it = tbl.items[g];
    const long long c = u - it.first_unit;
    const size_t n3 = size_t(it.N) * it.N * it.N;
    bool bad = false;
    RaggedDispatch<T, Tio, Ns...>::run(it.N, it.variant, static_cast<const Tio*>(it.f) + c * n3,
                                       static_cast<Tio*>(it.Q) + c * n3,
                                       static_cast<const typename C2<T>::type*>(it.tab), it.n_terms, smem, wsc, bad);
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(it.status, kStatusNonFinite);
  }
}

template <typename T, typename Tio, int... Ns>
struct RaggedLaunch {
  static constexpr size_t smem() {      // the largest of every N's two slab shapes
    size_t m = 0;
    for (size_t v : {Lay<Ns, T, RaggedBody<Ns, T, 0>::v>::SMEM..., Lay<Ns, T, RaggedBody<Ns, T, 1>::v>::SMEM...}) m = v > m ? v : m;
    return m;
  }
  static constexpr size_t ws() {        // per CTA: 256-byte header + the largest scratch
    size_t m = 0;
    for (size_t v : {Lay<Ns, T, RaggedBody<Ns, T, 0>::v>::WS..., Lay<Ns, T, RaggedBody<Ns, T, 1>::v>::WS...}) m = v > m ? v : m;
    return 256 + (m + 255) / 256 * 256;
  }
  // dynamic shared memory of the launch: that of the largest body it runs
  // (t.smem_bytes), not of the largest it could run, so that the L1 keeps the rest
  static int launch(const RaggedTable& t, void* wsp, size_t ws_per_cta, int grid, cudaStream_t st) {
    auto k = ragged_kernel<T, Tio, Ns...>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem()));
    if (e != cudaSuccess) return int(e);
    const size_t sm = t.smem_bytes > 0 && t.smem_bytes <= smem() ? t.smem_bytes : smem();
    k<<<grid, kThreads, sm, st>>>(t, wsp, ws_per_cta);
    return int(cudaGetLastError());
  }
  static int occupancy(int* ctas) {
    auto k = ragged_kernel<T, Tio, Ns...>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem()));
    if (e != cudaSuccess) return int(e);
    return int(cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, k, kThreads, smem()));
  }
};

// ------------------------------------------------------------ cluster form
// C CTAs of a thread-block cluster evaluate one cell together (Cfg::CLUSTER):
// the full first pass with its global arrays shared by the cluster.  The
// cluster's workspace holds the forward spectrum Fh and two term buffers Wg
// (term t uses Wg[t mod 2]); every pass over Fh or Wg splits its pencils over
// the C CTAs (CTA r takes pencils r T + i, r T + i + C T, ..., T threads per CTA),
// and CTA r owns the slabs r SPC .. r SPC + SPC - 1 (SPC = S0 / C), whose gain
// accumulators stay in its shared memory over all terms (no save and restore).
// Per cell: F1, F2, F3 with a cluster barrier after each; per term P1F into
// Wg[t mod 2], cluster barrier, then per own slab: copy the slab into shared
// memory, axis 1, axis 2 with G += Re*Im (Q on the last term).
// Ordering: P1F(t + 2) rewrites Wg[t mod 2] only after the barrier that follows
// P1F(t + 1), which every CTA reaches after its slab copies of term t; the next
// cell's F1 rewrites Fh only after the barrier that follows the last P1F.  Each
// (pencil, slab) is computed by the same code as in the one-CTA full first pass,
// so the results equal that form's bit for bit.
template <int N, typename T, typename Tio, int V>
__device__ __forceinline__ void process_cell_cluster(const Tio* __restrict__ f, Tio* __restrict__ Q,
                                                     const typename C2<T>::type* __restrict__ tab, int n_terms,
                                                     unsigned char* smem, unsigned char* wcl, int r, bool& bad) {
  using Ly = Lay<N, T, V>;
  using V2 = typename C2<T>::type;
  constexpr int C = Cfg<N, T, V>::CLUSTER;
  constexpr int H = Ly::H, FR = Ly::FH_ROW, WR = Ly::W_ROW, NS = Ly::NS, SPC = Ly::SLABS_PER_CTA;
  constexpr int GSLAB = NS * N * (N + 1);                 // elements of one slab of G
  V2* W = reinterpret_cast<V2*>(smem);
  T* G = reinterpret_cast<T*>(smem + Ly::round16(Ly::W_BYTES));
  V2* Fh = reinterpret_cast<V2*>(wcl);
  V2* Wg[2] = {reinterpret_cast<V2*>(wcl + Ly::round16(Ly::FH_BYTES)),
               reinterpret_cast<V2*>(wcl + Ly::round16(Ly::FH_BYTES) + Ly::round16(Ly::WG_BYTES))};
  const int p0 = r * kThreads + int(threadIdx.x), ps = C * kThreads;

  run_pass<N, T, Tio>(kPassF1, Fh, N * N / 2, 1, 0, 0, 1, -1, f, Q, G, 0, 1, FR, false, p0, ps);
  cluster_sync();
  run_pass<N, T, Tio>(kPassFwd, Fh, N * H, H, N * FR, 1, FR, -1, f, Q, G, 0, 1, FR, false, p0, ps);
  cluster_sync();
  run_pass<N, T, Tio>(kPassFwd, Fh, N * H, H, FR, 1, N * FR, -1, f, Q, G, 0, 1, FR, false, p0, ps);
  for (int i = threadIdx.x; i < SPC * GSLAB; i += kThreads) G[i] = T{};
  cluster_sync();
  for (int t = 0; t < n_terms; ++t) {
    V2* Wt = Wg[t & 1];
    run_p1f<N, T, V>(tab + size_t(t) * N * N * H, Fh, Wt, p0, ps);
    cluster_sync();
    const bool last = t == n_terms - 1;
    for (int j = 0; j < SPC; ++j) {
      const int s = r * SPC + j;                          // planes v0 = s NS .. s NS + NS - 1
      const V2* src = Wt + size_t(s) * NS * N * N;
      for (int i = threadIdx.x; i < NS * N * N; i += kThreads) {
        const int m = i / (N * N), rem = i % (N * N);
        cp_elem(W + (size_t(m) * N + rem / N) * WR + rem % N, src + i);
      }
      cp16_wait();
      __syncthreads();
      T* Gs = G + j * GSLAB;
      run_pass<N, T, Tio>(kPassInv, W, NS * N, N, N * WR, 1, WR, H, f, Q, Gs, s * NS, 1, FR, false);
      __syncthreads();
      bad |= run_pass<N, T, Tio>(kPassP3, W, NS * N, N, N * WR, WR, 1, -1, f, Q, Gs, s * NS, 1, FR, last);
      __syncthreads();
    }
  }
}

template <int N, typename T, typename Tio, int V>
__global__ void __launch_bounds__(kThreads, 1) collision_cluster_kernel(CollArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int C = Cfg<N, T, V>::CLUSTER;
  const int r = int(cluster_ctarank());
  const long long first = blockIdx.x / C, step = gridDim.x / C;
  // the cluster's workspace: its C consecutive per-CTA slices
  unsigned char* wcl = static_cast<unsigned char*>(a.ws) + size_t(first) * C * a.ws_per_cta;
  const auto* tab = static_cast<const typename C2<T>::type*>(a.tab);
  bool bad = false;
  for (long long c = first; c < a.n_cells; c += step) {       // the same cells for every CTA of a cluster
    const Tio* f = static_cast<const Tio*>(a.f) + size_t(c) * N * N * N;
    Tio* Q = static_cast<Tio*>(a.Q) + size_t(c) * N * N * N;
    process_cell_cluster<N, T, Tio, V>(f, Q, tab, a.n_terms, smem, wcl, r, bad);
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(a.status, kStatusNonFinite);
}

// Launch in clusters of C CTAs (one cell per cluster at a time).  `grid` is the
// number of CTAs the caller's workspace covers (a.ws_per_cta each); the kernel
// runs max(1, grid / C) clusters, capped at the cell count and at the number of
// clusters that can be resident at once.
template <int N, typename T, typename Tio, int V>
int launch_cluster(const CollArgs& a, int grid, cudaStream_t st) {
  constexpr int C = Cfg<N, T, V>::CLUSTER;
  constexpr size_t smem = Lay<N, T, V>::SMEM;
  auto k = collision_cluster_kernel<N, T, Tio, V>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return int(e);
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  long long clusters = grid / C < 1 ? 1 : grid / C;
  if (clusters > a.n_cells) clusters = a.n_cells;
  cfg.gridDim = dim3(C);
  int resident = 0;
  e = cudaOccupancyMaxActiveClusters(&resident, k, &cfg);
  if (e != cudaSuccess) return int(e);
  if (resident >= 1 && clusters > resident) clusters = resident;
  cfg.gridDim = dim3(unsigned(C * clusters));
  e = cudaLaunchKernelEx(&cfg, k, a);
  if (e != cudaSuccess) return int(e);
  return int(cudaGetLastError());
}

template <int N, typename T, typename Tio, int V>
int launch_one(const CollArgs& a, int grid, cudaStream_t st) {
  if constexpr (Cfg<N, T, V>::CLUSTER > 0) {
    return launch_cluster<N, T, Tio, V>(a, grid, st);
  } else {
    constexpr size_t smem = Lay<N, T, V>::SMEM;
    auto k = collision_kernel<N, T, Tio, V>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return int(e);
    k<<<grid, kThreads, smem, st>>>(a);
    return int(cudaGetLastError());
  }
}

template <int N, typename T, typename Tio, int V>
int occupancy_one(int* ctas) {
  constexpr size_t smem = Lay<N, T, V>::SMEM;
  auto k = [] {
    if constexpr (Cfg<N, T, V>::CLUSTER > 0) return collision_cluster_kernel<N, T, Tio, V>;
    else return collision_kernel<N, T, Tio, V>;
  }();
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return int(e);
  return int(cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, k, kThreads, smem));
}

}  // namespace coll
