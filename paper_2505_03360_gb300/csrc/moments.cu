// Per-cell moments, realizability matrices, L1 distance and regime bits
// (arxiv 2505.03360: sec. 2 hypothesis H3 for rho, u, T; sec. 2.2 stress
// tensor; sec. 3.1 eq. for Abar, Bbar; sec. 3.2 eq. for V_eps; App. A for tau,
// q, Cbar and the general-Cbar Schur form; sec. 3.3 L1 criterion).
//
// Reproducibility: every grid sum is an exact integer.  f is converted to
// fixed point F = trunc(f 2^P) with a per-cell scale P = 61 - e (max|f| < 2^e),
// multiplied by integer grid monomials (v = dv k, k_d = j_d - N/2) and summed
// in 128-bit integers, so the result does not depend on the order of the
// reduction or on the launch shape.  Each sum is rounded once to double, and
// the scalar algebra is a fixed sequence of correctly rounded double
// operations without contraction (__dadd_rn / __dmul_rn / __ddiv_rn /
// __dsqrt_rn).  The Maxwellian of the L1 test is separable; its 1D factors use
// our own exp (Cody-Waite reduction by ln 2, degree-13 Horner Taylor
// polynomial) and are rounded to 31-bit fixed point; f and the Maxwellian are
// resolved to 2^-30 of the larger peak, so |F2 - M_fix| is again an exact
// integer sum in 32-bit arithmetic.  Only the eigenvalues of V_eps (cyclic
// Jacobi) are not bit-reproducible.
//
// Streaming work per cell: one CTA.  Pass 0 takes max|f|; pass 1 walks rows
// (j0, j1) and forms the five row sums sum_j2 F k2^c with 32x32->64-bit
// multiply-adds on a 31-bit split of F, then folds them into the 14 global sums
// with the row's k0, k1 weights; pass 2 (re-read from L2) accumulates
// |F2 - M_fix|.  The scalar algebra runs afterwards, one thread per cell.
#include <cuda_runtime.h>

#include "coll_internal.h"

namespace coll {

namespace {

constexpr int kMThreads = 128;   // several cells per SM in flight: one cell's serial
                                  // scalar section overlaps the others' streaming
constexpr int kFixTop = 61;   // moment sums: |F| < 2^61
constexpr int kL1Top = 30;    // L1 test: |F2|, M < 2^30 (32-bit arithmetic)
constexpr int kEBits = 31;

typedef __int128 i128;
typedef unsigned __int128 u128;

__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double ddiv(double a, double b) { return __ddiv_rn(a, b); }

// trunc(x * 2^P) (toward zero) for a finite value m * 2^(ex_field - bias_shift),
// exact integer arithmetic on the bit pattern.  The caller guarantees
// |x| 2^P < 2^62.
__device__ __forceinline__ long long fix_bits(unsigned long long m, int ex_field, int bias_shift, int P,
                                              bool neg) {
  const int sh = ex_field - bias_shift + P;
  const unsigned long long r = sh >= 0 ? (m << sh) : (sh < -63 ? 0ull : (m >> -sh));
  return neg ? -static_cast<long long>(r) : static_cast<long long>(r);
}

__device__ __forceinline__ long long fix_val(double x, int P) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
  int ex = int((b >> 52) & 0x7ffull);
  unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  if (ex == 0) ex = 1; else m |= (1ull << 52);
  return fix_bits(m, ex, 1075, P, (b >> 63) != 0);
}

__device__ __forceinline__ long long fix_val(float x, int P) {
  const unsigned int b = __float_as_uint(x);
  int ex = int((b >> 23) & 0xffu);
  unsigned long long m = b & 0x7fffffu;
  if (ex == 0) ex = 1; else m |= (1ull << 23);
  return fix_bits(m, ex, 150, P, (b >> 31) != 0);
}

__device__ __forceinline__ double absval(double x) { return fabs(x); }
__device__ __forceinline__ float absval(float x) { return fabsf(x); }
__device__ __forceinline__ bool finite_val(double x) { return isfinite(x); }
__device__ __forceinline__ bool finite_val(float x) { return isfinite(x); }

// correctly rounded (half to even) conversion of a 128-bit integer to double
__device__ double i128_to_double(i128 x) {
  const bool neg = x < 0;
  u128 u = neg ? static_cast<u128>(-x) : static_cast<u128>(x);
  if (u == 0) return 0.0;
  const unsigned long long hi = static_cast<unsigned long long>(u >> 64);
  const unsigned long long lo = static_cast<unsigned long long>(u);
  const int nbits = hi ? 128 - __clzll(static_cast<long long>(hi)) : 64 - __clzll(static_cast<long long>(lo));
  double d;
  if (nbits <= 53) {
    d = static_cast<double>(lo);
  } else {
    int sh = nbits - 53;
    u128 q = u >> sh;
    const u128 rem = u - (q << sh);
    const u128 half = static_cast<u128>(1) << (sh - 1);
    if (rem > half || (rem == half && (q & 1))) {
      q += 1;
      if (q >> 53) { q >>= 1; sh += 1; }
    }
    d = ldexp(static_cast<double>(static_cast<unsigned long long>(q)), sh);
  }
  return neg ? -d : d;
}

// exp(x), x <= 0 (Cody & Waite range reduction by ln 2, Taylor-Horner degree
// 13, no fused multiply-add).  ln 2 = LN2_HI + LN2_LO with a 32-bit head so
// that k * LN2_HI is exact; 1/k! rounded once to double.
__device__ double own_exp(double x) {
  if (x < -700.0) return 0.0;
  const double kInvLn2 = 0x1.71547652b82fep+0;
  const double kLn2Hi = 0x1.62e42ff0p-1;
  const double kLn2Lo = -0x1.718432a1b0e26p-35;
  const double c[14] = {1.0,
                        1.0,
                        1.0 / 2.0,
                        1.0 / 6.0,
                        1.0 / 24.0,
                        1.0 / 120.0,
                        1.0 / 720.0,
                        1.0 / 5040.0,
                        1.0 / 40320.0,
                        1.0 / 362880.0,
                        1.0 / 3628800.0,
                        1.0 / 39916800.0,
                        1.0 / 479001600.0,
                        1.0 / 6227020800.0};
  const double k = rint(dmul(x, kInvLn2));
  const double t1 = dmul(k, kLn2Hi);
  const double t2 = dsub(x, t1);
  const double t3 = dmul(k, kLn2Lo);
  const double r = dsub(t2, t3);
  double p = c[13];
#pragma unroll
  for (int n = 12; n >= 0; --n) {
    p = dmul(p, r);
    p = dadd(p, c[n]);
  }
  const long long ki = static_cast<long long>(k);
  const double scale = __longlong_as_double((ki + 1023) << 52);   // k >= -1010 here
  return dmul(p, scale);
}

__device__ __forceinline__ bool psd3(const double* S) {
  const double a = S[0], b = S[1], c = S[2], d = S[3], e = S[4], f = S[5];
  if (!(a >= 0.0 && b >= 0.0 && c >= 0.0)) return false;
  const double m01 = dsub(dmul(a, b), dmul(d, d));
  const double m02 = dsub(dmul(a, c), dmul(e, e));
  const double m12 = dsub(dmul(b, c), dmul(f, f));
  if (!(m01 >= 0.0 && m02 >= 0.0 && m12 >= 0.0)) return false;
  // det = (a (bc - f^2) - d (dc - fe)) + e (df - be)
  const double det = dadd(dsub(dmul(a, m12), dmul(d, dsub(dmul(d, c), dmul(f, e)))),
                          dmul(e, dsub(dmul(d, f), dmul(b, e))));
  return det >= 0.0;
}

// eigenvalues of a symmetric 3x3 matrix, ascending: cyclic Jacobi rotations
// (accurate to a few ulps of the matrix norm, also for clustered eigenvalues).
// An off-diagonal entry below 2^-60 (|a_pp| + |a_qq|) is set to zero instead of
// rotated: it moves the eigenvalues by O(a_pq^2), far below one ulp, and the
// sweeps stop after quadratic convergence instead of waiting for underflow.
__device__ void eig3(const double* S, double* ev) {
  double a[3][3] = {{S[0], S[3], S[4]}, {S[3], S[1], S[5]}, {S[4], S[5], S[2]}};
  for (int sweep = 0; sweep < 16; ++sweep) {
    const double off = fabs(a[0][1]) + fabs(a[0][2]) + fabs(a[1][2]);
    if (off == 0.0) break;
#pragma unroll
    for (int pq = 0; pq < 3; ++pq) {
      const int p = pq == 2 ? 1 : 0, q = pq == 0 ? 1 : 2;
      const double apq = a[p][q];
      if (fabs(apq) <= 0x1p-60 * (fabs(a[p][p]) + fabs(a[q][q]))) {
        a[p][q] = a[q][p] = 0.0;
        continue;
      }
      const double theta = (a[q][q] - a[p][p]) / (2.0 * apq);
      const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
      const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
      a[p][p] -= t * apq;
      a[q][q] += t * apq;
      a[p][q] = a[q][p] = 0.0;
      const int r = 3 - p - q;
      const double arp = a[r][p], arq = a[r][q];
      a[r][p] = a[p][r] = c * arp - s * arq;
      a[r][q] = a[q][r] = s * arp + c * arq;
    }
  }
  double x = a[0][0], y = a[1][1], z = a[2][2], tt;
  if (x > y) { tt = x; x = y; y = tt; }
  if (y > z) { tt = y; y = z; z = tt; }
  if (x > y) { tt = x; x = y; y = tt; }
  ev[0] = x; ev[1] = y; ev[2] = z;
}

__device__ __forceinline__ i128 warp_sum(i128 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long lo = static_cast<unsigned long long>(v);
    const long long hi = static_cast<long long>(v >> 64);
    const unsigned long long olo = __shfl_down_sync(0xffffffffu, lo, o);
    const long long ohi = __shfl_down_sync(0xffffffffu, hi, o);
    const u128 other = (static_cast<u128>(static_cast<unsigned long long>(ohi)) << 64) | static_cast<u128>(olo);
    v = static_cast<i128>(static_cast<u128>(v) + other);
  }
  return v;
}

// block-wide exact sum of K 128-bit values; the totals land in red[0..K-1]
// (shared memory), valid after the call for every thread
template <int K>
__device__ __forceinline__ void block_sum(i128 (&v)[K], i128* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < K; ++i) v[i] = warp_sum(v[i]);
  __syncthreads();                                  // red may still be read from a previous use
  if (lane == 0) {
#pragma unroll
    for (int i = 0; i < K; ++i) red[K + warp * K + i] = v[i];
  }
  __syncthreads();
  if (threadIdx.x < K) {
    i128 s = 0;
    for (int w = 0; w < kMThreads / 32; ++w) s += red[K + w * K + threadIdx.x];
    red[threadIdx.x] = s;
  }
  __syncthreads();
}


// fold the five row sums R_c = sum_j2 F k2^c of row (k0, k1) into the 14
// moment sums: sum F, sum F k_d, sum F k_d k_e, sum F k_d |k|^2, sum F |k|^4
__device__ __forceinline__ void fold_row(i128 (&acc)[14], const i128 (&R)[5], long long k0, long long k1) {
  const long long r2 = k0 * k0 + k1 * k1;
  acc[0] += R[0];
  acc[1] += R[0] * k0;
  acc[2] += R[0] * k1;
  acc[3] += R[1];
  acc[4] += R[0] * (k0 * k0);
  acc[5] += R[0] * (k1 * k1);
  acc[6] += R[2];
  acc[7] += R[0] * (k0 * k1);
  acc[8] += R[1] * k0;
  acc[9] += R[1] * k1;
  acc[10] += R[0] * (k0 * r2) + R[2] * k0;
  acc[11] += R[0] * (k1 * r2) + R[2] * k1;
  acc[12] += R[1] * r2 + R[3];
  acc[13] += R[0] * (r2 * r2) + R[2] * (2 * r2) + R[4];
}

template <typename Tio> struct Bits;
// trunc(t * 2^(-k)) for t < 2^62 and k >= 1 (t >> 63 is already 0)
__device__ __forceinline__ unsigned long long rshift_trunc(unsigned long long t, int k) {
  return t >> (k > 63 ? 63 : k);
}

template <> struct Bits<double> {
  using U = unsigned long long;
  static constexpr U kAbs = 0x7FFFFFFFFFFFFFFFull, kExp = 0x7FF0000000000000ull;
  // trunc(x 2^P), with |x| 2^P < 2^61 guaranteed by the per-cell scale
  static __device__ __forceinline__ long long fix(U b, int P) {
    const int ex = int((b >> 52) & 0x7ffull);
    const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (ex ? (1ull << 52) : 0ull);
    // value = m 2^(max(ex,1) - 1075); scaled: m 2^(max(ex,1) - 1075 + P) = (m << 9) 2^-k
    const int k = 1075 + 9 - P - (ex ? ex : 1);
    const unsigned long long r = rshift_trunc(m << 9, k);
    return (b >> 63) ? -(long long)r : (long long)r;
  }
  static __device__ __forceinline__ double value(U a) { return __longlong_as_double((long long)a); }
  // trunc(x 2^P) for a result below 2^30 in magnitude, from the top 32 mantissa bits
  // (truncating the low bits first does not change a truncated result)
  static __device__ __forceinline__ int fix32(U b, int P) {
    const unsigned int hi = (unsigned int)(b >> 32), lo = (unsigned int)b;
    const int ex = int((hi >> 20) & 0x7ffu);
    const unsigned int top = __funnelshift_l(lo, hi, 11) | 0x80000000u;   // 1.m as a 32-bit integer
    // value = top 2^(ex - 1023 - 31); scaled by 2^P: top >> (1054 - P - ex)
    const int k = 1054 - P - ex;
    const unsigned int r = (ex == 0) ? 0u : (top >> (k > 31 ? 31 : k)) >> (k > 31 ? 1 : 0);
    return (hi >> 31) ? -(int)r : (int)r;
  }
  static __device__ __forceinline__ U shfl_max(U v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const U w = __shfl_down_sync(0xffffffffu, v, o);
      v = w > v ? w : v;
    }
    return v;
  }
};
template <> struct Bits<float> {
  using U = unsigned int;
  static constexpr U kAbs = 0x7FFFFFFFu, kExp = 0x7F800000u;
  static __device__ __forceinline__ long long fix(U b, int P) {
    const int ex = int((b >> 23) & 0xffu);
    const unsigned long long m = (b & 0x7fffffu) | (ex ? (1u << 23) : 0u);
    const int k = 150 + 38 - P - (ex ? ex : 1);
    const unsigned long long r = rshift_trunc(m << 38, k);
    return (b >> 31) ? -(long long)r : (long long)r;
  }
  static __device__ __forceinline__ double value(U a) { return double(__uint_as_float(a)); }
  static __device__ __forceinline__ int fix32(U b, int P) {
    const int ex = int((b >> 23) & 0xffu);
    const unsigned int m = (b & 0x7fffffu) | (ex ? 0x800000u : 0u);
    // value = m 2^(max(ex,1) - 150); scaled: m 2^(max(ex,1) - 150 + P), below 2^30
    const int sh = (ex ? ex : 1) - 150 + P;
    const unsigned int r = sh >= 0 ? (m << sh) : (sh < -31 ? 0u : (m >> -sh));
    return (b >> 31) ? -(int)r : (int)r;
  }
  static __device__ __forceinline__ U shfl_max(U v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const U w = __shfl_down_sync(0xffffffffu, v, o);
      v = w > v ? w : v;
    }
    return v;
  }
};

// 16-byte load through the read-only path with an L2 eviction priority: kL2Keep
// (evict_last) where a later pass reads the cell again, kL2Drop (evict_first)
// on its last read, so that the lines of finished cells leave L2 before those of
// cells still in flight.
enum : int { kL2Normal = 0, kL2Keep = 1, kL2Drop = 2 };
template <int H>
__device__ __forceinline__ uint4 ldg_l2(const uint4* p) {
  uint4 v;
  if constexpr (H == kL2Normal) {
    v = __ldg(p);
  } else {
    unsigned long long pol;
    if constexpr (H == kL2Keep)
      asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    else
      asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    asm("ld.global.nc.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
        : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p), "l"(pol));
  }
  return v;
}

// 8 consecutive elements of a row as bit patterns (two 16-byte loads)
template <typename Tio, int H = kL2Normal>
__device__ __forceinline__ void load8(const Tio* p, typename Bits<Tio>::U* b) {
  const uint4* q = reinterpret_cast<const uint4*>(p);
  const uint4 a = ldg_l2<H>(q), c = ldg_l2<H>(q + 1);
  if constexpr (sizeof(Tio) == 8) {
    b[0] = (unsigned long long)a.x | ((unsigned long long)a.y << 32);
    b[1] = (unsigned long long)a.z | ((unsigned long long)a.w << 32);
    b[2] = (unsigned long long)c.x | ((unsigned long long)c.y << 32);
    b[3] = (unsigned long long)c.z | ((unsigned long long)c.w << 32);
    const uint4 d = ldg_l2<H>(q + 2), e = ldg_l2<H>(q + 3);
    b[4] = (unsigned long long)d.x | ((unsigned long long)d.y << 32);
    b[5] = (unsigned long long)d.z | ((unsigned long long)d.w << 32);
    b[6] = (unsigned long long)e.x | ((unsigned long long)e.y << 32);
    b[7] = (unsigned long long)e.z | ((unsigned long long)e.w << 32);
  } else {
    b[0] = a.x; b[1] = a.y; b[2] = a.z; b[3] = a.w;
    b[4] = c.x; b[5] = c.y; b[6] = c.z; b[7] = c.w;
  }
}

// ---------------------------------------------------------------------------
// Two launches per batch.
//
//   K1 (one CTA per cell, persistent over cells): pass 0 (max |f|, finiteness),
//      pass 1 (the 14 exact moment sums), the Maxwellian parameters rho, u, T
//      (a short serial section), pass 2 (the exact L1 sum).  It leaves the
//      integer results in the cell's output record, used as scratch.
//   K2 (one thread per cell): the scalar algebra of the record (tensors,
//      realizability and Euler-breakdown tests, eigenvalues) from those
//      integers, overwriting the scratch with the final record and mask.
//
// FP64 runs at a small fraction of the integer rate on this GPU, so the long
// dependent chain of correctly rounded divisions and square roots per cell is
// taken off the streaming CTAs and run for all cells side by side.
// ---------------------------------------------------------------------------

// scratch words in the 40-double record written by K1 and read by K2
enum : int {
  kWSums = 0,      // 14 sums as (low, high) 64-bit words: words 0..27
  kWState = 28,    // 0: finite, non-zero cell; 1: non-finite value; 2: all zero
  kWP1 = 29,       // scale of the moment sums
  kWL1Lo = 30,     // exact L1 sum (unsigned 128-bit), valid when kWHasL1 = 1
  kWL1Hi = 31,
  kWP2 = 32,       // scale of the L1 sum
  kWHasL1 = 33,
};

struct CellShared {
  i128 red[(kMThreads / 32 + 1) * 14];
  double e[3][64];
  unsigned long long E2[64];
  double dsum[7];
  double bc[8];          // broadcast: CM, 1/(2T), h, u[3]
  int ibc[4];            // broadcast: Maxwellian valid, P2
  unsigned int anybad;
  double fmax_d;
};

// rho, u, T and the quantities they are built from, from the first 7 sums
// rounded to double (D[0] = sum F, D[1..3] = sum F k_d, D[4..6] = sum F k_d^2).
// The same sequence of operations serves K1 (Maxwellian of the L1 test) and K2
// (the record), so both see bitwise identical values.
struct Basic {
  double h, vol, h2, rho, inv0, kap[3], u[3], m2d[3], C[3], trC, Tg, T;
};
__device__ __forceinline__ void basic_moments(const double* D, int P1, int N, double L, Basic& b) {
  b.h = ddiv(dmul(2.0, L), double(N));
  b.vol = dmul(dmul(b.h, b.h), b.h);
  b.rho = dmul(ldexp(D[0], -P1), b.vol);
  b.h2 = dmul(b.h, b.h);
  if (!(D[0] > 0.0)) return;
  b.inv0 = ddiv(1.0, D[0]);
  for (int d = 0; d < 3; ++d) {
    b.kap[d] = dmul(D[1 + d], b.inv0);
    b.u[d] = dmul(b.kap[d], b.h);
  }
  for (int d = 0; d < 3; ++d) {
    b.m2d[d] = dmul(D[4 + d], b.inv0);
    b.C[d] = dsub(b.m2d[d], dmul(b.kap[d], b.kap[d]));
  }
  b.trC = dadd(dadd(b.C[0], b.C[1]), b.C[2]);
  b.Tg = ddiv(b.trC, 3.0);
  b.T = dmul(b.Tg, b.h2);
}

// Scalar algebra of one cell from its exact integer sums: the record o[0..38]
// and the realizability / Euler-breakdown bits, in the oracle's order of
// operations.  Returns false (mask 0x07) for a cell without positive density
// or temperature.
__device__ bool scalar_part(const i128* acc, int P1, int N, double L, double eta0, double* o, uint8_t& mbits) {
  double D[7];
  for (int i = 0; i < 7; ++i) D[i] = i128_to_double(acc[i]);
  Basic b;
  basic_moments(D, P1, N, L, b);
  o[0] = b.rho;
  if (!(D[0] > 0.0)) { mbits = 0x07; return false; }
  for (int d = 0; d < 3; ++d) o[1 + d] = b.u[d];
  o[4] = b.T;
  if (!(b.Tg > 0.0)) { mbits = 0x07; return false; }
  const double* kap = b.kap;
  const double inv0 = b.inv0, Tg = b.Tg, h2 = b.h2, rho = b.rho, trC = b.trC;
  double m2[6], C[6];
  for (int d = 0; d < 3; ++d) { m2[d] = b.m2d[d]; C[d] = b.C[d]; }
  const int pd[6] = {0, 1, 2, 0, 0, 1}, pe[6] = {0, 1, 2, 1, 2, 2};
  for (int i = 3; i < 6; ++i) {
    m2[i] = dmul(i128_to_double(acc[4 + i]), inv0);
    C[i] = dsub(m2[i], dmul(kap[pd[i]], kap[pe[i]]));
  }
  double Theta[6], tau[6];
  for (int i = 0; i < 6; ++i) Theta[i] = dmul(C[i], h2);
  const double p = dmul(rho, b.T);
  for (int i = 0; i < 6; ++i) tau[i] = i < 3 ? dsub(dmul(rho, Theta[i]), p) : dmul(rho, Theta[i]);
  double E3[3];
  for (int d = 0; d < 3; ++d) E3[d] = dmul(i128_to_double(acc[10 + d]), inv0);
  const double kk = dadd(dadd(dmul(kap[0], kap[0]), dmul(kap[1], kap[1])), dmul(kap[2], kap[2]));
  auto Cs = [&](int d, int e) -> double {       // symmetric access C(d, e)
    if (d == e) return C[d];
    const int lo = d < e ? d : e, hi = d < e ? e : d;
    return lo == 0 ? (hi == 1 ? C[3] : C[4]) : C[5];
  };
  double m3[3], q[3];
  const double rv = dmul(rho, b.vol);
  for (int d = 0; d < 3; ++d) {
    const double sC = dadd(dadd(dmul(kap[0], Cs(d, 0)), dmul(kap[1], Cs(d, 1))), dmul(kap[2], Cs(d, 2)));
    m3[d] = dsub(dsub(dsub(E3[d], dmul(2.0, sC)), dmul(kap[d], trC)), dmul(kap[d], kk));
    q[d] = dmul(0.5, dmul(rv, m3[d]));
  }
  const double E4 = dmul(i128_to_double(acc[13]), inv0);
  const double kE3 = dadd(dadd(dmul(kap[0], E3[0]), dmul(kap[1], E3[1])), dmul(kap[2], E3[2]));
  const double trm2 = dadd(dadd(m2[0], m2[1]), m2[2]);
  const double km2k =
      dadd(dadd(dadd(dmul(dmul(kap[0], kap[0]), m2[0]), dmul(dmul(kap[1], kap[1]), m2[1])),
                dmul(dmul(kap[2], kap[2]), m2[2])),
           dmul(2.0, dadd(dadd(dmul(dmul(kap[0], kap[1]), m2[3]), dmul(dmul(kap[0], kap[2]), m2[4])),
                          dmul(dmul(kap[1], kap[2]), m2[5]))));
  const double m4 = dsub(dadd(dadd(dsub(E4, dmul(4.0, kE3)), dmul(dmul(2.0, kk), trm2)), dmul(4.0, km2k)),
                         dmul(3.0, dmul(kk, kk)));
  const double Cbar = dsub(ddiv(m4, dmul(10.0, dmul(Tg, Tg))), 0.5);
  double Abar[6];
  for (int i = 0; i < 6; ++i) Abar[i] = i < 3 ? dsub(ddiv(C[i], Tg), 1.0) : ddiv(C[i], Tg);
  const double sq = dmul(Tg, __dsqrt_rn(Tg));
  double Bbar[3];
  for (int d = 0; d < 3; ++d) Bbar[d] = ddiv(dmul(0.5, m3[d]), sq);
  const double c23 = 2.0 / 3.0;
  double V[6];
  for (int i = 0; i < 6; ++i) {
    const double bb = dmul(Bbar[pd[i]], Bbar[pe[i]]);
    V[i] = i < 3 ? dsub(dadd(1.0, Abar[i]), dmul(c23, bb)) : dsub(Abar[i], dmul(c23, bb));
  }
  bool realizable = false;
  if (Cbar > 0.4) {
    const double gam = ddiv(2.0, dmul(5.0, Cbar));
    const double coef = ddiv(gam, dsub(1.0, gam));
    double Vg[6];
    for (int i = 0; i < 6; ++i) {
      const double bb = dmul(Bbar[pd[i]], Bbar[pe[i]]);
      Vg[i] = i < 3 ? dsub(dadd(1.0, Abar[i]), dmul(coef, bb)) : dsub(Abar[i], dmul(coef, bb));
    }
    realizable = psd3(Vg);
  }
  double up[6], dn[6];
  for (int i = 0; i < 6; ++i) {
    up[i] = i < 3 ? dsub(dadd(1.0, eta0), V[i]) : -V[i];
    dn[i] = i < 3 ? dsub(V[i], dsub(1.0, eta0)) : V[i];
  }
  const bool near_euler = psd3(up) && psd3(dn);
  mbits = (realizable ? 0 : 1) | (near_euler ? 0 : 2);
  double ev[3];
  eig3(V, ev);
  for (int i = 0; i < 6; ++i) { o[5 + i] = Theta[i]; o[11 + i] = tau[i]; o[20 + i] = Abar[i]; o[30 + i] = V[i]; }
  for (int d = 0; d < 3; ++d) { o[17 + d] = q[d]; o[26 + d] = Bbar[d]; o[36 + d] = ev[d]; }
  o[29] = Cbar;
  return true;
}

// ---- K1 pieces shared by the runtime-N and compile-time-N cell functions

// Pass-0 epilogue: block max / finiteness; writes the scratch state of an
// invalid or all-zero cell and returns false for it.
__device__ __forceinline__ bool cell_state(unsigned long long mx_bits, bool bad, unsigned long long* w, CellShared& sh,
                                           double* fmaxv) {
  const int tid = threadIdx.x;
  if (tid == 0) { sh.fmax_d = 0.0; sh.anybad = 0u; }
  __syncthreads();
  if ((tid & 31) == 0) atomicMax(reinterpret_cast<unsigned long long*>(&sh.fmax_d), mx_bits);
  if (bad) atomicOr(&sh.anybad, 1u);
  __syncthreads();
  *fmaxv = sh.fmax_d;
  const bool invalid = sh.anybad != 0u;
  if (invalid || *fmaxv == 0.0) {
    if (tid == 0) w[kWState] = invalid ? 1ull : 2ull;
    __syncthreads();
    return false;
  }
  return true;
}

// After pass 1: store the sums and P1, then the Maxwellian of the L1 test
// (serial part, thread 0) into sh.bc / sh.ibc.  Returns whether pass 2 runs.
__device__ __forceinline__ bool after_sums(i128 (&acc)[14], int P1, int ef, int N, double L, unsigned long long* w,
                                           CellShared& sh) {
  const int tid = threadIdx.x;
  block_sum<14>(acc, sh.red);
  if (tid < 28) {
    const u128 v = static_cast<u128>(sh.red[tid >> 1]);
    w[kWSums + tid] = (tid & 1) ? static_cast<unsigned long long>(v >> 64) : static_cast<unsigned long long>(v);
  } else if (tid < 35) {
    sh.dsum[tid - 28] = i128_to_double(sh.red[tid - 28]);
  }
  __syncthreads();
  if (tid == 0) {
    w[kWState] = 0;
    w[kWP1] = static_cast<unsigned long long>(static_cast<long long>(P1));
    Basic b;
    basic_moments(sh.dsum, P1, N, L, b);
    const bool ok = sh.dsum[0] > 0.0 && b.Tg > 0.0;
    sh.ibc[0] = ok;
    w[kWHasL1] = ok;
    if (ok) {
      const double s = dmul(2.0 * 3.141592653589793, b.T);
      const double CM = ddiv(b.rho, dmul(s, __dsqrt_rn(s)));
      int eM;
      frexp(CM, &eM);
      const int P2 = kL1Top - (ef > eM ? ef : eM);
      sh.bc[0] = CM;
      sh.bc[1] = ddiv(1.0, dmul(2.0, b.T));
      sh.bc[2] = b.h;
      for (int d = 0; d < 3; ++d) sh.bc[3 + d] = b.u[d];
      sh.ibc[1] = P2;
      w[kWP2] = static_cast<unsigned long long>(static_cast<long long>(P2));
    }
  }
  __syncthreads();
  return sh.ibc[0] != 0;
}

// 1D factors of the separable Maxwellian: e_d[j] = exp(-(h (j - N/2) - u_d)^2 / (2T)),
// and the k2 factor in 31-bit fixed point.
__device__ __forceinline__ void maxwell_factors(int N, CellShared& sh) {
  const int tid = threadIdx.x, half = N / 2;
  const double inv2T = sh.bc[1], h = sh.bc[2];
  for (int i = tid; i < 3 * N; i += kMThreads) {
    const int d = i / N, j = i % N;
    const double x = dsub(dmul(h, double(j - half)), sh.bc[3 + d]);
    sh.e[d][j] = own_exp(-dmul(dmul(x, x), inv2T));
  }
  __syncthreads();
  if (tid < N) sh.E2[tid] = static_cast<unsigned long long>(__double2ll_rn(ldexp(sh.e[2][tid], kEBits)));
  __syncthreads();
}

__device__ __forceinline__ void store_l1(u128 l1acc, unsigned long long* w, CellShared& sh) {
  i128 l1v[1] = {static_cast<i128>(l1acc)};
  block_sum<1>(l1v, sh.red);
  if (threadIdx.x == 0) {
    const u128 v = static_cast<u128>(sh.red[0]);
    w[kWL1Lo] = static_cast<unsigned long long>(v);
    w[kWL1Hi] = static_cast<unsigned long long>(v >> 64);
  }
  __syncthreads();
}

// ---- K1, runtime N (any even N <= 64, any alignment)
template <typename Tio>
__device__ void sums_cell(const Tio* __restrict__ f, int N, double L, unsigned long long* w, CellShared& sh) {
  const int tid = threadIdx.x;
  const int n3 = N * N * N;
  const int half = N / 2;

  double mx = 0.0;
  bool bad = false;
  for (int i = tid; i < n3; i += kMThreads) {
    const Tio x = f[i];
    bad |= !finite_val(x);
    const double ax = double(absval(x));
    mx = ax > mx ? ax : mx;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
  double fmaxv;      // mx >= 0: the bit patterns order like the values
  if (!cell_state(static_cast<unsigned long long>(__double_as_longlong(mx)), bad, w, sh, &fmaxv)) return;
  int ef;
  frexp(fmaxv, &ef);
  const int P1 = kFixTop - ef;

  i128 acc[14];
#pragma unroll
  for (int i = 0; i < 14; ++i) acc[i] = 0;
  for (int row = tid; row < N * N; row += kMThreads) {
    const int j0 = row / N, j1 = row % N;
    const long long k0 = j0 - half, k1 = j1 - half;
    long long rl[5] = {0, 0, 0, 0, 0}, rh[5] = {0, 0, 0, 0, 0};
    const Tio* fr = f + size_t(row) * N;
    for (int j2 = 0; j2 < N; ++j2) {
      const long long F = fix_val(fr[j2], P1);
      const int flo = int(F & 0x7fffffffll);
      const int fhi = int(F >> 31);
      const int k2 = j2 - half;
      int kp = 1;
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        rl[c] += static_cast<long long>(flo) * kp;
        rh[c] += static_cast<long long>(fhi) * kp;
        kp *= k2;
      }
    }
    i128 R[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) R[c] = static_cast<i128>(rh[c]) * (static_cast<i128>(1) << 31) + static_cast<i128>(rl[c]);
    fold_row(acc, R, k0, k1);
  }
  if (!after_sums(acc, P1, ef, N, L, w, sh)) return;

  maxwell_factors(N, sh);
  const double CM = sh.bc[0];
  const int P2 = sh.ibc[1];
  u128 l1acc = 0;
  for (int row = tid; row < N * N; row += kMThreads) {
    const int j0 = row / N, j1 = row % N;
    const double A = dmul(dmul(CM, sh.e[0][j0]), sh.e[1][j1]);
    const unsigned long long Af = static_cast<unsigned long long>(__double2ll_rn(ldexp(A, P2)));   // < 2^30
    const Tio* fr = f + size_t(row) * N;
    for (int j2 = 0; j2 < N; ++j2) {
      const long long F2 = fix_val(fr[j2], P2);
      const long long M = static_cast<long long>((Af * sh.E2[j2] + (1ull << (kEBits - 1))) >> kEBits);
      const long long dlt = F2 - M;
      l1acc += static_cast<u128>(dlt < 0 ? -dlt : dlt);
    }
  }
  store_l1(l1acc, w, sh);
}

// ---- K1, compile-time N over bit patterns (16-byte aligned f)
template <int N, typename Tio>
__device__ void sums_cell_fast(const Tio* __restrict__ f, double L, unsigned long long* w, CellShared& sh) {
  using B = Bits<Tio>;
  using U = typename B::U;
  constexpr int half = N / 2;
  constexpr int n3 = N * N * N;
  constexpr int VEC = 16 / int(sizeof(Tio));
  const int tid = threadIdx.x;

  // pass 0: max |f| as an integer max of the magnitude bits, finiteness
  U mx = 0;
  bool bad = false;
  const uint4* f4 = reinterpret_cast<const uint4*>(f);
  for (int i = tid; i < n3 / VEC; i += kMThreads) {
    const uint4 v = ldg_l2<kL2Keep>(f4 + i);
    U e[VEC];
    if constexpr (sizeof(Tio) == 8) {
      e[0] = (unsigned long long)v.x | ((unsigned long long)v.y << 32);
      e[1] = (unsigned long long)v.z | ((unsigned long long)v.w << 32);
    } else {
      e[0] = v.x; e[1] = v.y; e[2] = v.z; e[3] = v.w;
    }
#pragma unroll
    for (int k = 0; k < VEC; ++k) {
      const U a = e[k] & B::kAbs;
      bad |= a >= B::kExp;
      mx = a > mx ? a : mx;
    }
  }
  mx = B::shfl_max(mx);
  double fmaxv;
  const unsigned long long mxd = static_cast<unsigned long long>(__double_as_longlong(B::value(mx)));
  if (!cell_state(mxd, bad, w, sh, &fmaxv)) return;
  int ef;
  frexp(fmaxv, &ef);
  // The bit-pattern conversions below assume a cell maximum well above the
  // subnormal range (shift counts stay non-negative, subnormal entries of the
  // L1 pass truncate to 0); a cell of tinier values takes the general path.
  if (ef < (sizeof(Tio) == 8 ? -990 : -100)) {
    sums_cell<Tio>(f, N, L, w, sh);
    return;
  }
  const int P1 = kFixTop - ef;

  // pass 1: rows of N with immediate k2 powers
  i128 acc[14];
#pragma unroll
  for (int i = 0; i < 14; ++i) acc[i] = 0;
  for (int row = tid; row < N * N; row += kMThreads) {
    const long long k0 = row / N - half, k1 = row % N - half;
    long long rl[5] = {0, 0, 0, 0, 0}, rh[5] = {0, 0, 0, 0, 0};
    const Tio* fr = f + size_t(row) * N;
#pragma unroll
    for (int c0 = 0; c0 < N; c0 += 8) {
      U b[8];
      load8<Tio, kL2Keep>(fr + c0, b);
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int k2 = c0 + e - half;                 // compile-time after unrolling
        const long long F = B::fix(b[e], P1);
        const int flo = int(F & 0x7fffffffll);         // 31-bit split: 32x32 -> 64-bit products
        const int fhi = int(F >> 31);
        const int p1 = k2, p2 = k2 * k2, p3 = p2 * k2, p4 = p2 * p2;
        rl[0] += flo; rh[0] += fhi;
        rl[1] += (long long)flo * p1; rh[1] += (long long)fhi * p1;
        rl[2] += (long long)flo * p2; rh[2] += (long long)fhi * p2;
        rl[3] += (long long)flo * p3; rh[3] += (long long)fhi * p3;
        rl[4] += (long long)flo * p4; rh[4] += (long long)fhi * p4;
      }
    }
    i128 R[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) R[c] = static_cast<i128>(rh[c]) * (static_cast<i128>(1) << 31) + static_cast<i128>(rl[c]);
    fold_row(acc, R, k0, k1);
  }
  if (!after_sums(acc, P1, ef, N, L, w, sh)) return;

  // pass 2: L1 distance to the Maxwellian in 32-bit fixed point
  maxwell_factors(N, sh);
  const double CM = sh.bc[0];
  const int P2 = sh.ibc[1];
  unsigned long long l1acc = 0;                      // < 2^18 values of < 2^31 each
  for (int row = tid; row < N * N; row += kMThreads) {
    const int j0 = row / N, j1 = row % N;
    const double A = dmul(dmul(CM, sh.e[0][j0]), sh.e[1][j1]);
    const unsigned int Af = static_cast<unsigned int>(__double2ll_rn(ldexp(A, P2)));   // < 2^30
    const Tio* fr = f + size_t(row) * N;
#pragma unroll
    for (int c0 = 0; c0 < N; c0 += 8) {
      U b[8];
      load8<Tio, kL2Drop>(fr + c0, b);
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int F2 = B::fix32(b[e], P2);
        const unsigned int E = (unsigned int)sh.E2[c0 + e];                 // < 2^31
        const int M = (int)(((unsigned long long)Af * E + (1ull << 30)) >> 31);
        const int dlt = F2 - M;
        l1acc += (unsigned int)(dlt < 0 ? -dlt : dlt);
      }
    }
  }
  store_l1(l1acc, w, sh);
}

template <typename Tio>
__global__ void __launch_bounds__(kMThreads, 4) sums_kernel(const Tio* __restrict__ f, int N, double L,
                                                         long long n_cells, coll_moments* mom) {
  __shared__ CellShared sh;
  const size_t n3 = size_t(N) * N * N;
  for (long long c = blockIdx.x; c < n_cells; c += gridDim.x)
    sums_cell<Tio>(f + size_t(c) * n3, N, L, reinterpret_cast<unsigned long long*>(mom + c), sh);
}

template <int N, typename Tio>
__global__ void __launch_bounds__(kMThreads, 4) sums_kernel_fast(const Tio* __restrict__ f, double L,
                                                              long long n_cells, coll_moments* mom) {
  __shared__ CellShared sh;
  constexpr size_t n3 = size_t(N) * N * N;
  for (long long c = blockIdx.x; c < n_cells; c += gridDim.x)
    sums_cell_fast<N, Tio>(f + size_t(c) * n3, L, reinterpret_cast<unsigned long long*>(mom + c), sh);
}

// ---- K2: one thread per cell
constexpr int kFinishThreads = 32;

__global__ void __launch_bounds__(kFinishThreads) finish_kernel(int N, double L, long long n_cells, double eta0,
                                                                double delta0, coll_moments* mom, uint8_t* mask) {
  const long long c = static_cast<long long>(blockIdx.x) * kFinishThreads + threadIdx.x;
  if (c >= n_cells) return;
  unsigned long long* w = reinterpret_cast<unsigned long long*>(mom + c);
  double* out = reinterpret_cast<double*>(mom + c);
  const double qnan = __longlong_as_double(0x7ff8000000000000ll);
  double o[40];
  for (int i = 0; i < 40; ++i) o[i] = qnan;
  uint8_t mbits;
  const unsigned long long state = w[kWState];
  if (state != 0) {
    if (state == 2) o[0] = 0.0;
    mbits = state == 1 ? 0x87 : 0x07;
  } else {
    i128 acc[14];
    for (int i = 0; i < 14; ++i)
      acc[i] = static_cast<i128>((static_cast<u128>(w[kWSums + 2 * i + 1]) << 64) | static_cast<u128>(w[kWSums + 2 * i]));
    const int P1 = static_cast<int>(static_cast<long long>(w[kWP1]));
    const bool has_l1 = w[kWHasL1] != 0;
    const u128 l1s = (static_cast<u128>(w[kWL1Hi]) << 64) | static_cast<u128>(w[kWL1Lo]);
    const int P2 = static_cast<int>(static_cast<long long>(w[kWP2]));
    if (scalar_part(acc, P1, N, L, eta0, o, mbits) && has_l1) {
      const double h = ddiv(dmul(2.0, L), double(N));
      const double vol = dmul(dmul(h, h), h);
      const double l1 = dmul(ldexp(i128_to_double(static_cast<i128>(l1s)), -P2), vol);
      o[39] = l1;
      if (l1 > delta0) mbits |= 4;
    }
  }
  for (int i = 0; i < 40; ++i) out[i] = o[i];
  mask[c] = mbits;
}

template <typename Tio>
__device__ __forceinline__ void unpack16(const uint4 v, typename Bits<Tio>::U* b) {
  if constexpr (sizeof(Tio) == 8) {
    b[0] = (unsigned long long)v.x | ((unsigned long long)v.y << 32);
    b[1] = (unsigned long long)v.z | ((unsigned long long)v.w << 32);
  } else {
    b[0] = v.x; b[1] = v.y; b[2] = v.z; b[3] = v.w;
  }
}

// ---------------------------------------------------------------------------
// Collision invariants of Q (hypothesis H1, sec. 2): per cell the exact
// fixed-point sums of F = trunc(Q 2^P) times 1, k_d, |k|^2 and of |F| times
// 1, |k_0| + |k_1| + |k_2|, |k|^2 (v = h k), each rounded once to double and
// scaled by 2^-P h^3 (times h or h^2).  The same scale rule as the moment
// sums: P = 61 - e with max |Q| < 2^e.  One CTA per cell, persistent: pass 0
// takes max |Q| and finiteness, pass 1 (from L2) the eight sums.
// ---------------------------------------------------------------------------
struct ConsShared {
  i128 red[(kMThreads / 32 + 1) * 8];
  unsigned long long wmx[kMThreads / 32];
  unsigned int wbad[kMThreads / 32];
};

// rows [row0, row0 + nrows) of a cell at base (global memory; the cell's last read)
template <int N, typename Tio>
__device__ __forceinline__ void cons_rows(const unsigned char* base, int row0, int nrows, int P, bool general,
                                          i128 (&acc)[8]) {
  using B = Bits<Tio>;
  using U = typename B::U;
  constexpr int half = N / 2;
  constexpr int RB = N * int(sizeof(Tio)), NCH = RB / 16, EPC = 16 / int(sizeof(Tio));
  constexpr int ROT = NCH < 8 ? NCH : 8;
  const int s = threadIdx.x % ROT;
  for (int lr = threadIdx.x; lr < nrows; lr += kMThreads) {
    const int row = row0 + lr;
    const long long k0 = row / N - half, k1 = row % N - half;
    long long rl[3] = {0, 0, 0}, rh[3] = {0, 0, 0}, al[3] = {0, 0, 0}, ah[3] = {0, 0, 0};
    const unsigned char* rp = base + size_t(lr) * RB;
    auto add = [&](long long F, int k2) {
      const long long aF = F < 0 ? -F : F;
      const int flo = int(F & 0x7fffffffll), fhi = int(F >> 31);
      const int alo = int(aF & 0x7fffffffll), ahi = int(aF >> 31);
      const int ak = k2 < 0 ? -k2 : k2, k22 = k2 * k2;
      rl[0] += flo; rh[0] += fhi;
      rl[1] += (long long)flo * k2; rh[1] += (long long)fhi * k2;
      rl[2] += (long long)flo * k22; rh[2] += (long long)fhi * k22;
      al[0] += alo; ah[0] += ahi;
      al[1] += (long long)alo * ak; ah[1] += (long long)ahi * ak;
      al[2] += (long long)alo * k22; ah[2] += (long long)ahi * k22;
    };
    if (!general) {
#pragma unroll
      for (int i = 0; i < NCH; ++i) {
        int j = i + s;
        if (j >= NCH) j -= NCH;
        U b[EPC];
        unpack16<Tio>(ldg_l2<kL2Drop>(reinterpret_cast<const uint4*>(rp + 16 * j)), b);
#pragma unroll
        for (int e = 0; e < EPC; ++e) add(B::fix(b[e], P), j * EPC + e - half);
      }
    } else {
      const Tio* fr = reinterpret_cast<const Tio*>(rp);
      for (int j2 = 0; j2 < N; ++j2) add(fix_val(fr[j2], P), j2 - half);
    }
    i128 R[3], A[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      R[c] = static_cast<i128>(rh[c]) * (static_cast<i128>(1) << 31) + static_cast<i128>(rl[c]);
      A[c] = static_cast<i128>(ah[c]) * (static_cast<i128>(1) << 31) + static_cast<i128>(al[c]);
    }
    const long long r2 = k0 * k0 + k1 * k1, r1 = (k0 < 0 ? -k0 : k0) + (k1 < 0 ? -k1 : k1);
    acc[0] += R[0];
    acc[1] += R[0] * k0;
    acc[2] += R[0] * k1;
    acc[3] += R[1];
    acc[4] += R[0] * r2 + R[2];
    acc[5] += A[0];
    acc[6] += A[0] * r1 + A[1];
    acc[7] += A[0] * r2 + A[2];
  }
}

int grid_for(const void* kernel, long long n_cells) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, kMThreads, 0);
  if (per < 1) per = 1;
  long long grid = static_cast<long long>(sms) * per;
  return int(grid > n_cells ? n_cells : grid);
}

template <int N, typename Tio>
__global__ void __launch_bounds__(kMThreads, 4) cons_kernel(const Tio* __restrict__ Q, double L, long long n_cells,
                                                           double* __restrict__ out) {
  using B = Bits<Tio>;
  using U = typename B::U;
  constexpr int EPC = 16 / int(sizeof(Tio));
  constexpr int BYTES = N * N * N * int(sizeof(Tio));
  __shared__ ConsShared x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const double qnan = __longlong_as_double(0x7ff8000000000000ll);
  for (long long c = blockIdx.x; c < n_cells; c += gridDim.x) {
    const unsigned char* base = reinterpret_cast<const unsigned char*>(Q + size_t(c) * N * N * N);
    double* o = out + size_t(c) * 8;
    // ---- pass 0: max |Q| (magnitude bits), finiteness
    U mx = 0;
    bool bad = false;
    const uint4* s4 = reinterpret_cast<const uint4*>(base);
    for (int i = tid; i < BYTES / 16; i += kMThreads) {
      U e[EPC];
      unpack16<Tio>(ldg_l2<kL2Keep>(s4 + i), e);
#pragma unroll
      for (int k = 0; k < EPC; ++k) {
        const U a = e[k] & B::kAbs;
        bad |= a >= B::kExp;
        mx = a > mx ? a : mx;
      }
    }
    mx = B::shfl_max(mx);
    bad = __any_sync(0xffffffffu, bad);
    __syncthreads();                                        // x.wmx may still be read for the previous cell
    if (lane == 0) {
      x.wmx[warp] = static_cast<unsigned long long>(__double_as_longlong(B::value(mx)));
      x.wbad[warp] = bad ? 1u : 0u;
    }
    __syncthreads();
    unsigned long long mxd = 0;
    unsigned int fl = 0;
#pragma unroll
    for (int k = 0; k < kMThreads / 32; ++k) {
      mxd = x.wmx[k] > mxd ? x.wmx[k] : mxd;
      fl |= x.wbad[k];
    }
    const double qmax = __longlong_as_double(static_cast<long long>(mxd));
    if (fl || qmax == 0.0) {                                // non-finite or all-zero cell
      if (tid < 8) o[tid] = fl ? qnan : 0.0;
      continue;
    }
    int e;
    frexp(qmax, &e);
    const bool general = e < (sizeof(Tio) == 8 ? -990 : -100);
    const int P = kFixTop - e;
    // ---- pass 1: the eight exact sums
    i128 acc[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[i] = 0;
    cons_rows<N, Tio>(base, 0, N * N, P, general, acc);
    block_sum<8>(acc, x.red);
    if (tid < 8) {
      const double h = ddiv(dmul(2.0, L), double(N));
      const double vol = dmul(dmul(h, h), h);
      double v = dmul(ldexp(i128_to_double(x.red[tid]), -P), vol);
      const int pw = (tid == 4 || tid == 7) ? 2 : (tid == 0 || tid == 5) ? 0 : 1;
      if (pw == 1) v = dmul(v, h);
      if (pw == 2) v = dmul(v, dmul(h, h));
      o[tid] = v;
    }
  }
}

template <int N, typename Tio>
int launch_cons_n(const Tio* Q, double L, long long n_cells, double* out, cudaStream_t st) {
  const int grid = grid_for(reinterpret_cast<const void*>(cons_kernel<N, Tio>), n_cells);
  cons_kernel<N, Tio><<<grid, kMThreads, 0, st>>>(Q, L, n_cells, out);
  return int(cudaGetLastError());
}

template <typename Tio>
int launch_cons(const Tio* Q, int N, double L, long long n_cells, double* out, cudaStream_t st) {
  switch (N) {
    case 16: return launch_cons_n<16, Tio>(Q, L, n_cells, out, st);
    case 24: return launch_cons_n<24, Tio>(Q, L, n_cells, out, st);
    case 32: return launch_cons_n<32, Tio>(Q, L, n_cells, out, st);
    case 48: return launch_cons_n<48, Tio>(Q, L, n_cells, out, st);
    case 64: return launch_cons_n<64, Tio>(Q, L, n_cells, out, st);
    default: return int(cudaErrorInvalidValue);
  }
}

template <int N, typename Tio>
int launch_fast(const Tio* f, double L, long long n_cells, coll_moments* mom, cudaStream_t st) {
  const int grid = grid_for(reinterpret_cast<const void*>(sums_kernel_fast<N, Tio>), n_cells);
  sums_kernel_fast<N, Tio><<<grid, kMThreads, 0, st>>>(f, L, n_cells, mom);
  return int(cudaGetLastError());
}

template <typename Tio>
int launch_sums(const Tio* f, int N, double L, long long n_cells, coll_moments* mom, cudaStream_t st) {
  if ((reinterpret_cast<uintptr_t>(f) & 15u) == 0) {
    switch (N) {
      case 16: return launch_fast<16, Tio>(f, L, n_cells, mom, st);
      case 24: return launch_fast<24, Tio>(f, L, n_cells, mom, st);
      case 32: return launch_fast<32, Tio>(f, L, n_cells, mom, st);
      case 48: return launch_fast<48, Tio>(f, L, n_cells, mom, st);
      case 64: return launch_fast<64, Tio>(f, L, n_cells, mom, st);
      default: break;
    }
  }
  const int grid = grid_for(reinterpret_cast<const void*>(sums_kernel<Tio>), n_cells);
  sums_kernel<Tio><<<grid, kMThreads, 0, st>>>(f, N, L, n_cells, mom);
  return int(cudaGetLastError());
}

}  // namespace

int launch_conservation(const void* Q, int io_f64, int N, double L, long long n_cells, double* out, void* stream) {
  count_launches(1);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return io_f64 ? launch_cons<double>(static_cast<const double*>(Q), N, L, n_cells, out, st)
                : launch_cons<float>(static_cast<const float*>(Q), N, L, n_cells, out, st);
}

int launch_moments(const void* f, int io_f64, int N, double L, long long n_cells, double eta0, double delta0,
                   coll_moments* mom, uint8_t* mask, void* stream) {
  count_launches(2);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int r = io_f64 ? launch_sums<double>(static_cast<const double*>(f), N, L, n_cells, mom, st)
                       : launch_sums<float>(static_cast<const float*>(f), N, L, n_cells, mom, st);
  if (r != 0) return r;
  const long long blocks = (n_cells + kFinishThreads - 1) / kFinishThreads;
  finish_kernel<<<static_cast<unsigned int>(blocks), kFinishThreads, 0, st>>>(N, L, n_cells, eta0, delta0, mom, mask);
  return int(cudaGetLastError());
}

}  // namespace coll
