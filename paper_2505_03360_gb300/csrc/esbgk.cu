// ES-BGK relaxation step (arxiv 2505.03360, sec. 2.2: corrected tensor
// Tau = (1 - beta) T I + beta Theta, Gaussian G[f] and Q_ES = nu (G[f] - f);
// sec. 4.3: the first-order IMEX scheme eq. 1000, space homogeneous).
//
// Per cell, from its moment record: nu = rho sqrt(T) / ((1 - beta) mu0),
// Theta^{n+1} = (eps Theta + (1 - beta) nu dt T I) / (eps + (1 - beta) nu dt),
// Tau^{n+1} = (1 - beta) T I + beta Theta^{n+1}, and
//   out = eps/(eps + nu dt) f + nu dt/(eps + nu dt) G[f^{n+1}],
//   G = rho / sqrt(det(2 pi Tau)) exp(-(v - u)^T Tau^{-1} (v - u) / 2).
// One CTA per cell (persistent over cells); thread 0 forms Tau^{-1} and the
// coefficients.  Every thread streams eight consecutive values of a row (v2
// varies), where the exponent is quadratic in the index: one exponential for
// the first value and a multiplicative step whose ratio factors are tabulated
// per cell (v2) and per row (N + N^2 exponentials per cell, in shared memory),
// which spares GB300's narrow FP64 pipe without any factor that could
// overflow.  out may be f.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "coll_internal.h"

namespace coll {

namespace {

constexpr int kEsThreads = 256;
constexpr double kTwoPiE = 6.283185307179586476925286766559;

struct EsArgs {
  const void* f;
  const coll_moments* mom;
  void* out;
  long long n_cells;
  double L, dt, eps, beta, mu0;
};

struct EsCell {
  double Li[6];        // Tau^{-1}, packed xx, yy, zz, xy, xz, yz
  double u[3];
  double cf, cg;       // eps/(eps + nu dt), nu dt/(eps + nu dt) rho / sqrt(det(2 pi Tau))
};

template <typename T> struct Quad4;
template <> struct Quad4<double> {
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
template <> struct Quad4<float> {
  static __device__ __forceinline__ void ld(const void* p, size_t q, double (&v)[4]) {
    const float4 x = __ldcs(reinterpret_cast<const float4*>(p) + q);
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
  }
  static __device__ __forceinline__ void st(void* p, size_t q, const double (&v)[4]) {
    reinterpret_cast<float4*>(p)[q] = make_float4(float(v[0]), float(v[1]), float(v[2]), float(v[3]));
  }
};

__device__ void cell_setup(const coll_moments& m, const EsArgs& a, EsCell& c) {
  const double rho = m.rho, T = m.T, b = a.beta;
  const double nu = rho * sqrt(T) / ((1.0 - b) * a.mu0);
  const double s = (1.0 - b) * nu * a.dt;
  double Tau[6];
  for (int k = 0; k < 6; ++k) {
    const double iso = k < 3 ? s * T : 0.0;
    const double th1 = (a.eps * m.Theta[k] + iso) / (a.eps + s);        // Theta^{n+1}
    Tau[k] = b * th1 + (k < 3 ? (1.0 - b) * T : 0.0);
  }
  const double xx = Tau[0], yy = Tau[1], zz = Tau[2], xy = Tau[3], xz = Tau[4], yz = Tau[5];
  const double c00 = yy * zz - yz * yz, c11 = xx * zz - xz * xz, c22 = xx * yy - xy * xy;
  const double c01 = xz * yz - xy * zz, c02 = xy * yz - xz * yy, c12 = xy * xz - xx * yz;
  const double det = xx * c00 + xy * c01 + xz * c02;
  const double inv = 1.0 / det;
  c.Li[0] = c00 * inv;
  c.Li[1] = c11 * inv;
  c.Li[2] = c22 * inv;
  c.Li[3] = c01 * inv;
  c.Li[4] = c02 * inv;
  c.Li[5] = c12 * inv;
  for (int d = 0; d < 3; ++d) c.u[d] = m.u[d];
  const double den = a.eps + nu * a.dt;
  c.cf = a.eps / den;
  c.cg = nu * a.dt / den * rho / sqrt(kTwoPiE * kTwoPiE * kTwoPiE * det);
}

template <int N, typename Tio>
__global__ void __launch_bounds__(kEsThreads) esbgk_kernel(EsArgs a) {
  using V = Quad4<Tio>;
  __shared__ EsCell sc;
  // Along a row (w0, w1 fixed) the exponent is q(w2) = A w2^2 + 2 B w2 + C, A = Tinv_zz,
  // B = Tinv_xz w0 + Tinv_yz w1.  Each group of eight starts from E = exp(-q/2) (<= 1) and steps
  // with E_{j+1} = E_j U[j] W[row]: U[j] = exp(-A h w2_j) (per cell), W = exp(-(A h^2 + 2 B h)/2)
  // (per row).  Every factor is a bounded exponential (|A h w2| <= A h L, |B h| <= 2 A' h L), so
  // nothing overflows however far the grid reaches into the Gaussian's tails.  Groups of eight
  // values per exponential: seven steps add at most seven roundings to E.  A group whose first
  // value is below 1e-280 (a narrow Gaussian whose peak lies further along the group) takes one
  // exponential per value, like a group with a ratio outside (1e-300, 1e300).
  extern __shared__ double tabs[];
  double* U = tabs;
  double* Wr = tabs + N;
  constexpr int n3 = N * N * N, nq = n3 / 4;
  static_assert(N % 8 == 0, "row segments of eight");
  const double h = 2.0 * a.L / N;
  for (long long c = blockIdx.x; c < a.n_cells; c += gridDim.x) {
    __syncthreads();
    if (threadIdx.x == 0) cell_setup(a.mom[c], a, sc);
    __syncthreads();
    const EsCell e = sc;
    const double A = e.Li[2];
    // a ratio factor whose exponent reaches 690 in modulus (an extremely cold or stretched
    // Gaussian on a wide box) is stored as 0; a group whose step ratios leave (1e-300, 1e300)
    // takes one exponential per value
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      const double lu = -A * h * (-a.L + i * h - e.u[2]);
      U[i] = fabs(lu) < 690.0 ? exp(lu) : 0.0;
    }
    for (int r = threadIdx.x; r < N * N; r += blockDim.x) {
      const double w0 = -a.L + (r / N) * h - e.u[0], w1 = -a.L + (r % N) * h - e.u[1];
      const double B = e.Li[4] * w0 + e.Li[5] * w1;
      const double lw = -0.5 * (A * h * h + 2.0 * B * h);
      Wr[r] = fabs(lw) < 690.0 ? exp(lw) : 0.0;
    }
    __syncthreads();
    const size_t base = size_t(c) * nq;
    for (int q2 = threadIdx.x; q2 < nq / 2; q2 += blockDim.x) {
      const int idx = 8 * q2, row = idx / N, j0 = row / N, j1 = row % N, j2 = idx % N;
      const double w0 = -a.L + j0 * h - e.u[0], w1 = -a.L + j1 * h - e.u[1], w2 = -a.L + j2 * h - e.u[2];
      const double B = e.Li[4] * w0 + e.Li[5] * w1;
      const double C = e.Li[0] * w0 * w0 + 2.0 * e.Li[3] * w0 * w1 + e.Li[1] * w1 * w1;
      double E = exp(-0.5 * ((A * w2 + 2.0 * B) * w2 + C));
      const double wr = Wr[row];
      double rs[7];
      bool step = E > 1e-280;                 // a subnormal start would lose the group's precision
#pragma unroll
      for (int k = 0; k < 7; ++k) {
        rs[k] = U[j2 + k] * wr;
        step &= rs[k] > 1e-300 && rs[k] < 1e300;
      }
      double f[8], o[8];
      V::ld(a.f, base + 2 * q2, *reinterpret_cast<double(*)[4]>(f));
      V::ld(a.f, base + 2 * q2 + 1, *reinterpret_cast<double(*)[4]>(f + 4));
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        if (k > 0) {
          if (step) {
            E *= rs[k - 1];
          } else {
            const double wk = w2 + k * h;
            E = exp(-0.5 * ((A * wk + 2.0 * B) * wk + C));
          }
        }
        o[k] = fma(e.cg, E, e.cf * f[k]);
      }
      V::st(a.out, base + 2 * q2, *reinterpret_cast<const double(*)[4]>(o));
      V::st(a.out, base + 2 * q2 + 1, *reinterpret_cast<const double(*)[4]>(o + 4));
    }
  }
}

template <int N, typename Tio>
int launch_es_t(const EsArgs& a, unsigned grid, cudaStream_t st) {
  constexpr size_t smem = size_t(N + N * N) * sizeof(double);
  auto k = esbgk_kernel<N, Tio>;
  const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return int(e);
  k<<<grid, kEsThreads, smem, st>>>(a);
  return int(cudaGetLastError());
}

template <int N>
int launch_es_n(const EsArgs& a, bool io_f64, unsigned grid, cudaStream_t st) {
  return io_f64 ? launch_es_t<N, double>(a, grid, st) : launch_es_t<N, float>(a, grid, st);
}

}  // namespace

int launch_esbgk(const void* f, const coll_moments* mom, bool io_f64, int N, double L, long long n_cells, double dt,
                 double eps, double beta, double mu0, void* out, void* stream) {
  EsArgs a;
  a.f = f;
  a.mom = mom;
  a.out = out;
  a.n_cells = n_cells;
  a.L = L;
  a.dt = dt;
  a.eps = eps;
  a.beta = beta;
  a.mu0 = mu0;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  long long grid = static_cast<long long>(sms) * 8;
  if (grid > n_cells) grid = n_cells;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  switch (N) {
    case 16: return launch_es_n<16>(a, io_f64, unsigned(grid), st);
    case 24: return launch_es_n<24>(a, io_f64, unsigned(grid), st);
    case 32: return launch_es_n<32>(a, io_f64, unsigned(grid), st);
    case 48: return launch_es_n<48>(a, io_f64, unsigned(grid), st);
    case 64: return launch_es_n<64>(a, io_f64, unsigned(grid), st);
    default: return int(cudaErrorInvalidValue);
  }
}

}  // namespace coll
