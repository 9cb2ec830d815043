// Float-pair ("double-float") arithmetic on the FP32 pipe.
//
// A value is h + l with two floats, |l| <= ulp(h) / 2, about 48 significant
// bits.  GB300 runs FP32 at 64 times its FP64 rate, so a float-pair operation
// (7 to 11 FP32 instructions) is still several times faster than one FP64
// instruction.  Algorithms (error-free transformations): Knuth's two-sum,
// Dekker's fast two-sum, and the FMA-based exact product; additions use the
// cheap variant whose error is relative to |a| + |b| (enough for FFT
// butterflies, whose error analysis is in those terms).
//
// Conversions to and from double are done on the bit patterns with integer
// instructions only, so that loading f64 inputs and storing f64 outputs does
// not touch the FP64 pipe.  Values below 2^-126 in magnitude flush to zero.
#pragma once

#include <cstdint>

namespace coll {

struct df {
  float h, l;
};

struct __align__(16) cdf {
  df x, y;   // real part, imaginary part
};

__device__ __forceinline__ df quick_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float e = __fsub_rn(b, __fsub_rn(s, a));
  return df{s, e};
}

__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return df{s, e};
}

__device__ __forceinline__ df operator+(df a, df b) {
  df s = two_sum(a.h, b.h);
  s.l = __fadd_rn(s.l, __fadd_rn(a.l, b.l));
  return quick_two_sum(s.h, s.l);
}
__device__ __forceinline__ df operator-(df a) { return df{-a.h, -a.l}; }
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }
__device__ __forceinline__ df operator*(df a, df b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return quick_two_sum(p, e);
}
__device__ __forceinline__ df& operator+=(df& a, df b) { a = a + b; return a; }
__device__ __forceinline__ df half(df a) { return df{0.5f * a.h, 0.5f * a.l}; }
__device__ __forceinline__ bool isfinite(df a) { return ::isfinite(a.h) && ::isfinite(a.l); }

// ---- conversions (integer bit manipulation, no FP64 instructions)

// float with the value m * 2^e2 for an integer 0 < m < 2^32 (mantissa truncated
// to 24 bits); 0 if below the float normal range
__device__ __forceinline__ float float_from_int_scaled(unsigned int m, int e2) {
  if (m == 0u) return 0.0f;
  const int lz = __clz(m);
  const int top = 31 - lz;                    // position of the leading bit
  unsigned int mant = top >= 23 ? (m >> (top - 23)) : (m << (23 - top));
  const int exp = e2 + top;                   // value = 1.mant * 2^exp
  if (exp < -126) return 0.0f;
  if (exp > 127) return __uint_as_float(0x7f800000u);
  return __uint_as_float((unsigned int)(exp + 127) << 23 | (mant & 0x7fffffu));
}

__device__ __forceinline__ df df_from_double(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned int sgn = (unsigned int)(b >> 63) << 31;
  const int e = int((b >> 52) & 0x7ffull);
  const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  if (e == 0x7ff) {                                            // inf / nan
    return df{__uint_as_float(sgn | 0x7f800000u | ((b & 0xFFFFFFFFFFFFFull) ? 0x400000u : 0u)), 0.0f};
  }
  const int ex = e - 1023;                                     // x = 1.m * 2^ex
  if (ex < -126) return df{__uint_as_float(sgn), 0.0f};
  if (ex > 127) return df{__uint_as_float(sgn | 0x7f800000u), 0.0f};
  const unsigned int mh = (unsigned int)(m >> 29);             // 24 leading bits
  const unsigned int ml = (unsigned int)(m & 0x1fffffffull);   // 29 trailing bits
  const float h = __uint_as_float(sgn | (unsigned int)(ex + 127) << 23 | (mh & 0x7fffffu));
  float l = float_from_int_scaled(ml, ex - 52);
  l = __uint_as_float(__float_as_uint(l) | sgn);
  return df{h, l};
}

__device__ __forceinline__ df df_from_float(float x) { return df{x, 0.0f}; }

// nearest double to h + l (ties to even), |l| <= ulp(h)
__device__ __forceinline__ double df_to_double(df v) {
  const unsigned int bh = __float_as_uint(v.h), bl = __float_as_uint(v.l);
  const int eh = int((bh >> 23) & 0xffu), el = int((bl >> 23) & 0xffu);
  if (eh == 0xff || eh == 0) {
    // inf/nan, or zero/subnormal head (flushed): the head alone
    if (eh == 0) return __longlong_as_double((long long)((unsigned long long)(bh >> 31) << 63));
    const unsigned long long s = (unsigned long long)(bh >> 31) << 63;
    return __longlong_as_double((long long)(s | 0x7ff0000000000000ull | ((bh & 0x7fffffu) ? 1ull << 51 : 0ull)));
  }
  // head as (sign, 24-bit integer, exponent of its lsb)
  const long long mh = (long long)((bh & 0x7fffffu) | 0x800000u);
  const int qh = eh - 127 - 23;
  long long acc = (bh >> 31) ? -mh : mh;
  int q = qh - 30;                                              // work at 30 extra bits
  acc <<= 30;                                                   // |acc| < 2^54
  if (el != 0 && el != 0xff) {
    const long long ml = (long long)((bl & 0x7fffffu) | 0x800000u);
    const int ql = el - 127 - 23;
    const int sh = ql - q;                                      // shift of the tail onto the grid 2^q
    long long t = (bl >> 31) ? -ml : ml;
    if (sh >= 0) {
      acc += t << sh;                                           // sh <= 6 when |l| <= ulp(h)
    } else if (sh > -62) {
      // arithmetic shift rounds toward -inf; the dropped part is below 2^(q-1),
      // far below the double's last bit (q is 30 bits under the head's lsb)
      acc += t >> (-sh);
    }
  }
  if (acc == 0) return 0.0;
  const bool neg = acc < 0;
  unsigned long long u = neg ? (unsigned long long)(-acc) : (unsigned long long)acc;
  const int top = 63 - __clzll((long long)u);                   // leading bit position
  int exp = q + top;                                            // value = 1.x * 2^exp
  unsigned long long mant;
  if (top > 52) {
    const int drop = top - 52;
    const unsigned long long rem = u & ((1ull << drop) - 1ull);
    const unsigned long long halfu = 1ull << (drop - 1);
    mant = u >> drop;
    if (rem > halfu || (rem == halfu && (mant & 1ull))) {
      mant += 1ull;
      if (mant >> 53) { mant >>= 1; exp += 1; }
    }
  } else {
    mant = u << (52 - top);
  }
  const unsigned long long bits = ((unsigned long long)neg << 63) | ((unsigned long long)(exp + 1023) << 52) |
                                  (mant & 0xFFFFFFFFFFFFFull);
  return __longlong_as_double((long long)bits);
}

}  // namespace coll
