// Regime indicator on the 2D spatial grid and the regime update of
// Algorithm 1 (arxiv 2505.03360, sec. 4.5; V_eps^1 and its closed-form
// eigenvalues, sec. 3.3 and 4.5; lambda_B, sec. 3.3; mu = mu0 sqrt(T),
// kappa = kappa0 sqrt(T) for hard spheres, sec. 3.1).
//
// One thread per cell.  The fields rho, u_x, u_y, T come as four planes of
// (ny + 2) x (nx + 2) doubles with a one-cell halo filled by the caller, so the
// one-cell stencil needs no boundary logic.  Every indicator is one fixed
// sequence of correctly rounded double operations (__d*_rn, no contraction),
// with the reciprocals 1/(2 dx), 1/(2 dy), 1/(dx dy) and 1/3 rounded once on
// the host: the regime, an integer decided by floating point, is then
// reproducible on any machine that follows the same sequence.  Delta u is the
// vector (Delta u_x, Delta u_y), |Delta u|^2 the sum of the squares.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "coll_internal.h"

namespace coll {

namespace {

__device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double dvd(double a, double b) { return __ddiv_rn(a, b); }

struct RegimeArgs {
  const double* fields;   // [4][ny + 2][nx + 2]
  const double* l1;       // [ny][nx]
  const uint8_t* r_in;    // [ny][nx]
  uint8_t* r_out;         // [ny][nx]
  double* ind;            // [4][ny][nx] or null
  int nx, ny;
  double eps, mu0, kappa0, i2dx, i2dy, ilap, third, eta0, eta1, delta0;
};

constexpr uint8_t kInvalid = 0x80;

__global__ void __launch_bounds__(256) regime_kernel(RegimeArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= a.nx || j >= a.ny) return;
  const size_t W = size_t(a.nx) + 2, plane = W * (size_t(a.ny) + 2);
  const size_t cc = (size_t(j) + 1) * W + (size_t(i) + 1);
  // centre, east (i+1), west (i-1), north (j+1), south (j-1) of plane q
  double v[4][5];
  bool fin = true;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const double* F = a.fields + size_t(q) * plane;
    v[q][0] = __ldg(F + cc);
    v[q][1] = __ldg(F + cc + 1);
    v[q][2] = __ldg(F + cc - 1);
    v[q][3] = __ldg(F + cc + W);
    v[q][4] = __ldg(F + cc - W);
#pragma unroll
    for (int k = 0; k < 5; ++k) fin &= isfinite(v[q][k]);
  }
  const size_t cell = size_t(j) * a.nx + i;
  const uint8_t r = a.r_in[cell];
  const double l1 = r == 1 ? __ldg(a.l1 + cell) : 0.0;

  auto ddx = [&](int q) { return mul(sub(v[q][1], v[q][2]), a.i2dx); };
  auto ddy = [&](int q) { return mul(sub(v[q][3], v[q][4]), a.i2dy); };
  auto lap = [&](int q) {
    return mul(sub(add(add(add(v[q][2], v[q][1]), v[q][4]), v[q][3]), mul(4.0, v[q][0])), a.ilap);
  };
  const double ux_x = ddx(1), ux_y = ddy(1), uy_x = ddx(2), uy_y = ddy(2);
  const double T_x = ddx(3), T_y = ddy(3);
  const double rho = v[0][0], T = v[3][0];
  const double lux = lap(1), luy = lap(2);
  const double rr = dvd(lap(0), rho);
  const double gT2 = add(mul(T_x, T_x), mul(T_y, T_y));
  const double gu2 = add(add(add(mul(ux_x, ux_x), mul(ux_y, ux_y)), mul(uy_x, uy_x)), mul(uy_y, uy_y));
  const double eps2 = mul(a.eps, a.eps);
  const double inner = mul(add(add(mul(lux, lux), mul(luy, luy)), mul(rr, rr)), add(1.0, mul(T, T)));
  const double lamB = mul(eps2, add(add(dvd(gT2, T), gu2), __dsqrt_rn(inner)));

  const double sT = __dsqrt_rn(T);
  const double mu = mul(a.mu0, sT), kap = mul(a.kappa0, sT);
  const double xi1 = dvd(mul(a.eps, mu), mul(rho, T));
  const double xi2 = mul(eps2, dvd(mul(2.0, mul(kap, kap)), mul(3.0, mul(mul(rho, rho), mul(mul(T, T), T)))));
  const double a1 = mul(sub(mul(4.0, ux_x), mul(2.0, uy_y)), a.third);
  const double c1 = mul(sub(mul(4.0, uy_y), mul(2.0, ux_x)), a.third);
  const double h1 = -mul(mul(2.0, add(ux_x, uy_y)), a.third);
  const double a2 = mul(T_x, T_x), b1 = add(ux_y, uy_x), b2 = mul(T_x, T_y), c2 = mul(T_y, T_y);
  const double d = add(mul(xi1, b1), mul(xi2, b2));
  const double P = add(mul(xi1, sub(a1, c1)), mul(xi2, sub(a2, c2)));
  const double S = add(add(add(mul(xi1, a1), mul(xi2, a2)), mul(xi1, c1)), mul(xi2, c2));
  const double root = __dsqrt_rn(add(mul(P, P), mul(4.0, mul(d, d))));
  const double lam_a = mul(add(sub(root, S), 2.0), 0.5);
  const double lam_b = mul(add(sub(-root, S), 2.0), 0.5);
  const double lam_c = sub(1.0, mul(xi1, h1));

  // Algorithm 1
  const bool close = fabs(sub(lam_a, 1.0)) <= a.eta0 && fabs(sub(lam_b, 1.0)) <= a.eta0 &&
                     fabs(sub(lam_c, 1.0)) <= a.eta0;
  const bool burnett = fabs(lamB) > a.eta1;
  const bool valid = fin && rho > 0.0 && T > 0.0 && r <= 2 && (r != 1 || isfinite(l1));
  uint8_t out;
  if (!valid) out = uint8_t(r | kInvalid);
  else if (r == 2) out = burnett ? 2 : 1;
  else if (r == 1) out = burnett ? 2 : ((close && l1 <= a.delta0) ? 0 : 1);
  else out = close ? 0 : 1;
  a.r_out[cell] = out;
  if (a.ind) {
    const size_t pl = size_t(a.nx) * a.ny;
    a.ind[cell] = lam_a;
    a.ind[pl + cell] = lam_b;
    a.ind[2 * pl + cell] = lam_c;
    a.ind[3 * pl + cell] = lamB;
  }
}

}  // namespace

int launch_regime(const double* fields, const double* l1, const uint8_t* r_in, int nx, int ny,
                  const coll_regime_params& p, uint8_t* r_out, double* ind, void* stream) {
  RegimeArgs a;
  a.fields = fields;
  a.l1 = l1;
  a.r_in = r_in;
  a.r_out = r_out;
  a.ind = ind;
  a.nx = nx;
  a.ny = ny;
  a.eps = p.eps;
  a.mu0 = p.mu0;
  a.kappa0 = p.kappa0;
  a.i2dx = 1.0 / (2.0 * p.dx);
  a.i2dy = 1.0 / (2.0 * p.dy);
  a.ilap = 1.0 / (p.dx * p.dy);
  a.third = 1.0 / 3.0;
  a.eta0 = p.eta0;
  a.eta1 = p.eta1;
  a.delta0 = p.delta0;
  const dim3 block(32, 8);
  const dim3 grid(unsigned((nx + 31) / 32), unsigned((ny + 7) / 8));
  regime_kernel<<<grid, block, 0, static_cast<cudaStream_t>(stream)>>>(a);
  return int(cudaGetLastError());
}

}  // namespace coll
