// Double-float arithmetic: a value is the unevaluated sum hi + lo of two FP32
// numbers (a 48-bit significand), multiplied and added with the error-free
// transformations of Dekker (products, through the fused multiply-add) and
// Knuth (sums). This GPU runs FP32 multiply-adds about 70 times faster than
// FP64 ones, so products whose accumulation must be FP64-accurate run here on
// the FP32 units: a product-and-add costs about twelve FP32 operations and no
// FP64 one.
//
// Error: a product carries the rounding error of hi*hi exactly and the cross
// terms hi*lo + lo*hi in FP32 (lo*lo, below 2^-48 relative, is dropped); a sum
// keeps the error of its hi parts exactly and adds the lo parts in FP32. Over
// a sum of m terms the result is within about m 2^-47 of the sum of the
// magnitudes of the terms.
#pragma once

#include <cuda_runtime.h>

namespace sghsc {

struct __align__(8) df64 {
  float hi, lo;
  __host__ __device__ df64() : hi(0.f), lo(0.f) {}
  __host__ __device__ explicit df64(float h, float l = 0.f) : hi(h), lo(l) {}
};

// a * b as (rounded product, its error plus the cross terms); not renormalised
__device__ __forceinline__ df64 operator*(const df64& a, const df64& b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return df64(p, e);
}

// x += y: the hi parts by Knuth's two-sum (exact), the lo parts in FP32; the
// pair is left unnormalised (normalise before converting or scaling)
__device__ __forceinline__ df64& operator+=(df64& x, const df64& y) {
  const float s = x.hi + y.hi;
  const float bb = s - x.hi;
  const float e = (x.hi - (s - bb)) + (y.hi - bb);
  x.hi = s;
  x.lo = x.lo + y.lo + e;
  return x;
}

// |lo| <= ulp(hi) / 2 again (fast two-sum)
__device__ __forceinline__ df64 df_norm(const df64& x) {
  const float s = x.hi + x.lo;
  return df64(s, x.lo - (s - x.hi));
}

// FP64 -> double-float on the host (setup): round-to-nearest hi, then the rest
inline df64 df_split_host(double v) {
  const float h = (float)v;
  return df64(h, (float)(v - (double)h));
}

// FP32 -> double-float: exact
__device__ __forceinline__ df64 df_from_float(float x) { return df64(x, 0.f); }

// FP64 -> double-float with integer operations only (the FP64 pipe is the
// narrow one): hi takes the sign, exponent and top 23 fraction bits of x
// (truncation, so hi is exact), lo the remaining 29 fraction bits, normalised
// from their leading one and truncated to 24 bits: the pair is within
// 2^-47 |x| + 2^-125 of x (a lo that would fall under the normal FP32 range
// is dropped; from |x| >= 2^-79 on the error is below 2^-47 |x|). Zeros give
// zeros; magnitudes outside the normal FP32 range of hi (below 2^-126 or
// above 2^127) take the rounded FP32 conversion with a zero lo.
__device__ __forceinline__ df64 df_from_double(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7ff);
  if (E == 0) return df64(0.f, 0.f);
  const int eh = E - 1023 + 127;
  if (eh < 1 || eh > 254) return df64(__double2float_rn(x), 0.f);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const float hi = __uint_as_float(sign | ((unsigned)eh << 23) | (unsigned)((b >> 29) & 0x7fffffu));
  const unsigned m29 = (unsigned)(b & 0x1fffffffu);
  if (m29 == 0u) return df64(hi, 0.f);
  // m29 * 2^(E - 1075): leading one of m29 at bit t, value 1.f * 2^(t + E - 1075)
  const int t = 31 - __clz(m29);
  const int el = t + E - 1075 + 127;
  if (el < 1) return df64(hi, 0.f);   // lo below the normal FP32 range: dropped
  const unsigned frac = t >= 23 ? (m29 >> (t - 23)) & 0x7fffffu : (m29 << (23 - t)) & 0x7fffffu;
  return df64(hi, __uint_as_float(sign | ((unsigned)el << 23) | frac));
}

}  // namespace sghsc
