// Penalised IMEX time stepping of the space-homogeneous Boltzmann equation
// df/dt = Q(f)/eps (arxiv 2505.03360, sec. 4.4: the BGK-like penalisation
// P(f) = beta (M - f) with beta = 2 pi rho, the first-order scheme eq. 1002;
// sec. 4.3: the PR(2,2,2) IMEX Runge-Kutta tableaux, g = 1 - 1/sqrt 2).
//
// Every stage is elementwise given the cell's Maxwellian, so one kernel
// streams the cell once: one CTA per cell (persistent over cells) computes the
// stage's per-cell coefficients and the Maxwellian's three 1D factors
// exp(-(v_j - u_d)^2 / (2T)) (scaled by the coefficient) in shared memory from
// the cell's moment record, then walks the N^3 values four at a time along a
// row (coherent streaming loads: out may be f, each value is read and then
// written by the same thread).  GB300's FP64 pipe is narrow, so each value
// costs only FMAs (no division): about four FP64 operations per value.
// Stages (P keeps the moments, so M is the Maxwellian of f throughout):
//   0  eq. 1002:  out = eps/(eps + b1 dt) (f - dt tr) + dt (Q1 - b0 (M0 - f))/(eps + b1 dt)
//                       + b1 dt/(eps + b1 dt) M1     (M1, b1 from mom1, the moments of f - dt tr)
//   1  Y1 = (eps f + dt g b M) / (eps + dt g b)
//   2  Y2 = (eps f + dt Q1 - 2 g dt b (M - Y) + dt g b M) / (eps + dt g b)
//   3  out = f + dt / (2 eps) (Q1 + Q2)
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "coll_internal.h"

namespace coll {

namespace {

constexpr int kImexThreads = 256;
constexpr double kTwoPi = 6.283185307179586476925286766559;

struct ImexArgs {
  int stage;
  const void* f;
  const void* Y;
  const void* Q1;
  const void* Q2;
  const void* tr;
  const coll_moments* mom0;
  const coll_moments* mom1;
  void* out;
  long long n_cells;
  int N;
  double L, dt, eps;
};

// four consecutive values (one row segment) of a cell array, as doubles
template <typename T> struct Quad;
template <> struct Quad<double> {
  static __device__ __forceinline__ void ld(const void* p, size_t q, double (&v)[4]) {
    const double2* b = reinterpret_cast<const double2*>(p) + 2 * q;
    const double2 x = __ldcs(b), y = __ldcs(b + 1);
    v[0] = x.x; v[1] = x.y; v[2] = y.x; v[3] = y.y;
  }
  static __device__ __forceinline__ void st(void* p, size_t q, const double (&v)[4]) {
    double2* b = reinterpret_cast<double2*>(p) + 2 * q;
    b[0] = make_double2(v[0], v[1]);
    b[1] = make_double2(v[2], v[3]);
  }
};
template <> struct Quad<float> {
  static __device__ __forceinline__ void ld(const void* p, size_t q, double (&v)[4]) {
    const float4 x = __ldcs(reinterpret_cast<const float4*>(p) + q);
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
  }
  static __device__ __forceinline__ void st(void* p, size_t q, const double (&v)[4]) {
    reinterpret_cast<float4*>(p)[q] = make_float4(float(v[0]), float(v[1]), float(v[2]), float(v[3]));
  }
};

// Factors of c M, M = rho (2 pi T)^{-3/2} prod_d exp(-(v_j - u_d)^2 / (2T)):
// gx = rho (2 pi T)^{-3/2} e0, gy = e1, gz = c e2, so c M = gx[j0] gy[j1] gz[j2].
// Returns beta = 2 pi rho.
__device__ __forceinline__ double maxwell_factors(const coll_moments& m, int N, double L, double c, double* g) {
  const double h = 2.0 * L / N, T = m.T, s = kTwoPi * T;
  const double amp = m.rho / (s * sqrt(s));
  for (int i = threadIdx.x; i < 3 * N; i += blockDim.x) {
    const int d = i / N, j = i % N;
    const double x = -L + j * h - m.u[d];
    const double e = exp(-(x * x) / (2.0 * T));
    g[i] = d == 0 ? amp * e : (d == 1 ? e : c * e);
  }
  return kTwoPi * m.rho;
}

// The stages as linear combinations with per-cell coefficients (eq. 1002 and
// the PR(2,2,2) stages rearranged; g = 1 - 1/sqrt 2):
//   0: cf f + ct tr + cq Q1 + cM0 M0 + cM1 M1, den = eps + b1 dt:
//      cf = (eps + dt b0)/den, ct = -eps dt/den, cq = dt/den, cM0 = -dt b0/den, cM1 = b1 dt/den
//   1: cf f + cM M,  cf = eps/den, cM = dt g b/den, den = eps + dt g b
//   2: cf f + cq Q1 + cy Y + cM M,  cf = eps/den, cq = dt/den, cy = 2 g dt b/den, cM = -dt g b/den
//   3: f + c (Q1 + Q2),  c = dt/(2 eps)
template <int N, typename Tio>
__global__ void __launch_bounds__(kImexThreads) imex_kernel(ImexArgs a) {
  using V = Quad<Tio>;
  extern __shared__ double g[];                 // [2][3N]: factors of cM0 M0 and (stage 0) cM1 M1
  constexpr int n3 = N * N * N, nq = n3 / 4;
  static_assert(N % 4 == 0, "row segments of four");
  const double gam = 1.0 - 1.0 / sqrt(2.0);
  const bool with_tr = a.stage == 0 && a.tr != nullptr;
  for (long long c = blockIdx.x; c < a.n_cells; c += gridDim.x) {
    __syncthreads();                            // the previous cell is done with g
    double cf = 1.0, cq = 0.0, cy = 0.0, ct = 0.0;
    if (a.stage == 0) {
      const double b0 = kTwoPi * a.mom0[c].rho;
      const double b1 = with_tr ? kTwoPi * a.mom1[c].rho : b0;
      const double den = a.eps + b1 * a.dt;
      cf = (a.eps + a.dt * b0) / den;
      ct = -a.eps * a.dt / den;
      cq = a.dt / den;
      maxwell_factors(a.mom0[c], N, a.L, -a.dt * b0 / den, g);
      maxwell_factors(with_tr ? a.mom1[c] : a.mom0[c], N, a.L, b1 * a.dt / den, g + 3 * N);
    } else if (a.stage == 1 || a.stage == 2) {
      const double b = kTwoPi * a.mom0[c].rho;
      const double den = a.eps + a.dt * gam * b;
      cf = a.eps / den;
      cq = a.dt / den;
      cy = 2.0 * gam * a.dt * b / den;
      maxwell_factors(a.mom0[c], N, a.L, (a.stage == 1 ? 1.0 : -1.0) * a.dt * gam * b / den, g);
    } else {
      cq = a.dt / (2.0 * a.eps);
    }
    __syncthreads();
    const size_t base = size_t(c) * nq;
    for (int q = threadIdx.x; q < nq; q += blockDim.x) {
      const int e = 4 * q, j0 = e / (N * N), j1 = (e / N) % N, j2 = e % N;
      double f[4], o[4];
      V::ld(a.f, base + q, f);
      if (a.stage == 3) {
        double q1[4], q2[4];
        V::ld(a.Q1, base + q, q1);
        V::ld(a.Q2, base + q, q2);
#pragma unroll
        for (int k = 0; k < 4; ++k) o[k] = fma(cq, q1[k] + q2[k], f[k]);
      } else {
        const double R = g[j0] * g[N + j1];
#pragma unroll
        for (int k = 0; k < 4; ++k) o[k] = fma(R, g[2 * N + j2 + k], cf * f[k]);
        if (a.stage != 1) {
          double q1[4];
          V::ld(a.Q1, base + q, q1);
#pragma unroll
          for (int k = 0; k < 4; ++k) o[k] = fma(cq, q1[k], o[k]);
        }
        if (a.stage == 2) {
          double y[4];
          V::ld(a.Y, base + q, y);
#pragma unroll
          for (int k = 0; k < 4; ++k) o[k] = fma(cy, y[k], o[k]);
        }
        if (a.stage == 0) {
          const double* h = g + 3 * N;
          const double R1 = h[j0] * h[N + j1];
#pragma unroll
          for (int k = 0; k < 4; ++k) o[k] = fma(R1, h[2 * N + j2 + k], o[k]);
          if (with_tr) {
            double t[4];
            V::ld(a.tr, base + q, t);
#pragma unroll
            for (int k = 0; k < 4; ++k) o[k] = fma(ct, t[k], o[k]);
          }
        }
      }
      V::st(a.out, base + q, o);
    }
  }
}

template <int N>
void launch_imex_n(const ImexArgs& a, bool io_f64, unsigned grid, size_t smem, cudaStream_t st) {
  if (io_f64) imex_kernel<N, double><<<grid, kImexThreads, smem, st>>>(a);
  else imex_kernel<N, float><<<grid, kImexThreads, smem, st>>>(a);
}

}  // namespace

int launch_imex(int stage, const void* f, const void* Y, const void* Q1, const void* Q2, const void* tr,
                const coll_moments* mom0, const coll_moments* mom1, bool io_f64, int N, double L, long long n_cells,
                double dt, double eps, void* out, void* stream) {
  ImexArgs a;
  a.stage = stage;
  a.f = f;
  a.Y = Y;
  a.Q1 = Q1;
  a.Q2 = Q2;
  a.tr = tr;
  a.mom0 = mom0;
  a.mom1 = mom1;
  a.out = out;
  a.n_cells = n_cells;
  a.N = N;
  a.L = L;
  a.dt = dt;
  a.eps = eps;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  long long grid = static_cast<long long>(sms) * 8;
  if (grid > n_cells) grid = n_cells;
  const size_t smem = size_t(6) * N * sizeof(double);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  switch (N) {
    case 16: launch_imex_n<16>(a, io_f64, unsigned(grid), smem, st); break;
    case 24: launch_imex_n<24>(a, io_f64, unsigned(grid), smem, st); break;
    case 32: launch_imex_n<32>(a, io_f64, unsigned(grid), smem, st); break;
    case 48: launch_imex_n<48>(a, io_f64, unsigned(grid), smem, st); break;
    case 64: launch_imex_n<64>(a, io_f64, unsigned(grid), smem, st); break;
    default: return int(cudaErrorInvalidValue);
  }
  return int(cudaGetLastError());
}

}  // namespace coll
