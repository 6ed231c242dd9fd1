// Exact fixed-point sums of FP64 values for stencils with integer weights.
//
// On this part the FP64 pipe issues about two lanes per clock per SM, some
// 32 times fewer than the integer ALU.  The finite differences of the Z4c
// right-hand side (Sec. II.B.1-2: 6th-order central first and second
// derivatives, the 6th-order lopsided advection stencil, 8th-order
// Kreiss-Oliger dissipation) are sums of a few values with small integer
// weights, scaled at the end by 1/(60 dx), 1/(180 dx^2) and the like.  Such a
// sum is formed exactly in 64-bit integers: the values of one stencil set are
// put on the fixed-point grid 2^(E - 1076), E the largest exponent field among
// them (one guard bit), so every value within a factor of two of the largest
// is represented exactly and smaller ones lose only bits below half an ulp of
// the largest.  The integer sum has no rounding at all; converting it to FP64
// and applying the scale are the only two roundings of the result.
#pragma once

namespace sacra {
namespace fx {

constexpr long long kFrac = (1ll << 52) - 1;
constexpr int kGrid = 1076;                 // grid unit 2^(E - kGrid): 1075 + one guard bit

__device__ __forceinline__ long long bits(double v) { return __double_as_longlong(v); }
__device__ __forceinline__ int expo(long long b) { return (int)((unsigned long long)b >> 52) & 0x7FF; }

// The finite value with bits b as an integer multiple of 2^(E - kGrid), for
// E >= its exponent field: |result| < 2^54, exact when the exponent field is
// E or E - 1, truncated towards zero below that.
__device__ __forceinline__ long long fix(long long b, int E) {
  const int e = expo(b);
  const long long m = ((b & kFrac) | (e ? (1ll << 52) : 0ll)) << 1;
  const int d = E - (e ? e : 1);
  const long long v = d < 63 ? (m >> d) : 0ll;
  return b < 0 ? -v : v;
}

// c * 2^(E - kGrid) for a finite c: exact (an exponent shift) while the result
// is a normal number; 0 for c = 0 or a subnormal c.
__device__ __forceinline__ double unit(double c, int E) {
  const long long cb = bits(c);
  const int ec = expo(cb);
  if (ec == 0) return 0.0;
  const int k = E - kGrid;
  const int er = ec + k;
  if (er >= 1 && er <= 2046) return __longlong_as_double(cb + (long long)k * (1ll << 52));
  return ldexp(c, k);
}

// |x| rounded down to a bound usable in overflow checks (x ^ sign: |x| or |x| - 1)
__device__ __forceinline__ long long mag(long long x) { return x ^ (x >> 63); }

// x / 2^k rounded towards minus infinity, for any k >= 0
__device__ __forceinline__ long long shr(long long x, int k) { return k < 63 ? (x >> k) : (x >> 63); }

// The 6th-order central first-difference numerator 45 (u_1 - u_-1) - 9 (u_2 -
// u_-2) + (u_3 - u_-3) of the six values u[n s], n = +-1..+-3, exactly on the
// grid 2^(E - kGrid) of their largest exponent field (E >= 1); E = -1 when a
// value is not finite.  diff6_of takes the bit patterns of u_1, u_-1, u_2,
// u_-2, u_3, u_-3; diff6_bits reads them from the patterns c[n s].
__device__ __forceinline__ void diff6_of(const long long b[6], long long &num, int &E) {
  int e = 1;
#pragma unroll
  for (int n = 0; n < 6; ++n) e = max(e, expo(b[n]));
  if (e == 2047) {
    num = 0;
    E = -1;
    return;
  }
  long long v[6];
#pragma unroll
  for (int n = 0; n < 6; ++n) v[n] = fix(b[n], e);
  num = 45 * (v[0] - v[1]) - 9 * (v[2] - v[3]) + (v[4] - v[5]);
  E = e;
}

__device__ __forceinline__ void diff6_bits(const long long *c, int s, long long &num, int &E) {
  long long b[6];
#pragma unroll
  for (int n = 0; n < 3; ++n) {
    b[2 * n] = c[(n + 1) * s];
    b[2 * n + 1] = c[-(n + 1) * s];
  }
  diff6_of(b, num, E);
}

}  // namespace fx
}  // namespace sacra
