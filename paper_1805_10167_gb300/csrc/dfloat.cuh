// Double-float arithmetic: a value is an unevaluated sum hi + lo of two
// floats with |lo| <= ulp(hi) / 2 (Dekker 1971, "A floating-point technique
// for extending the available precision"; Knuth, TAOCP vol. 2, 4.2.2).
// About 48 significant bits; every operation runs on the FP32 pipes.
//
//   two_sum      error-free a + b = s + e (Knuth, 6 flops)
//   fast_two_sum error-free a + b = s + e for |a| >= |b| (Dekker, 3 flops)
//   df_add       "sloppy" double-float addition: absolute error about
//                2^-47 (|x| + |y|)
//   df_mul       product with the FMA-based exact two-product
//
// Conversions to and from double use integer bit operations only, so that
// they do not occupy the (narrow) FP64 pipe, except one FP64 addition in
// to_double; d2f_rn and f2d_bits are the plain binary64 <-> binary32
// conversions done the same way.  Magnitudes below 2^-126 are flushed to zero; the low word is
// dropped below 2^-74 (relative error 2^-24 of such tiny values).
#pragma once

#include <cstdint>
#include <cmath>
#include <cstring>

#ifdef __CUDACC__
#define HHG_HD __host__ __device__ __forceinline__
#else
#define HHG_HD inline
#endif

namespace hhg {

struct dfl {
  float hi, lo;
};

HHG_HD uint64_t dbits(double d) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(d);
#else
  uint64_t u;
  std::memcpy(&u, &d, 8);
  return u;
#endif
}
HHG_HD double bitsd(uint64_t u) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)u);
#else
  double d;
  std::memcpy(&d, &u, 8);
  return d;
#endif
}
HHG_HD uint32_t fbits(float f) {
#ifdef __CUDA_ARCH__
  return (uint32_t)__float_as_uint(f);
#else
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return u;
#endif
}
HHG_HD float bitsf(uint32_t u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float f;
  std::memcpy(&f, &u, 4);
  return f;
#endif
}

HHG_HD dfl two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return {s, e};
}

HHG_HD dfl fast_two_sum(float a, float b) {
  const float s = a + b;
  return {s, b - (s - a)};
}

HHG_HD dfl df_add(dfl x, dfl y) {
  const dfl s = two_sum(x.hi, y.hi);
  const float e = s.lo + (x.lo + y.lo);
  return fast_two_sum(s.hi, e);
}

HHG_HD dfl df_mul(dfl x, dfl y) {
  const float p = x.hi * y.hi;
  float e = fmaf(x.hi, y.hi, -p);
  e = fmaf(x.hi, y.lo, e);
  e = fmaf(x.lo, y.hi, e);
  return fast_two_sum(p, e);
}

// acc + w * s
HHG_HD dfl df_fma(dfl w, dfl s, dfl acc) { return df_add(df_mul(w, s), acc); }

// double -> (hi, lo): hi = the top 24 significand bits (truncated), lo = the
// next 29 bits rounded to a float.
HHG_HD dfl from_double(double d) {
  const uint64_t u = dbits(d);
  const uint32_t sign = (uint32_t)(u >> 32) & 0x80000000u;
  const int e = (int)((u >> 52) & 0x7FF) - 1023;
  if (e < -126) return {0.f, 0.f};
  if (e > 127) return {bitsf(sign | 0x7F800000u), 0.f};
  const uint64_t m = u & 0x000FFFFFFFFFFFFFull;
  const float hi = bitsf(sign | ((uint32_t)(e + 127) << 23) | (uint32_t)(m >> 29));
  const uint32_t r = (uint32_t)(m & 0x1FFFFFFFull);
  float lo = 0.f;
  if (r != 0 && e - 52 >= -126) {
    const float scale = bitsf((uint32_t)(e - 52 + 127) << 23);
    lo = (float)r * scale;
    if (sign) lo = -lo;
  }
  return {hi, lo};
}

// float -> double by bit construction (exact; float denormals -> 0)
HHG_HD double f2d_bits(float f) {
  const uint32_t u = fbits(f);
  const uint32_t e8 = (u >> 23) & 0xFF;
  if (e8 == 0) return 0.0;
  const uint64_t sign = (uint64_t)(u & 0x80000000u) << 32;
  const uint64_t e11 = (uint64_t)(e8 - 127 + 1023) << 52;
  const uint64_t m = (uint64_t)(u & 0x7FFFFFu) << 29;
  return bitsd(sign | e11 | m);
}

HHG_HD double to_double(dfl x) { return f2d_bits(x.hi) + f2d_bits(x.lo); }

// double -> float rounded to nearest, ties to even (IEEE 754 binary64 to
// binary32), by integer operations only: the 52-bit significand keeps its
// top 23 bits and the 29 dropped bits decide the rounding; a carry out of
// the significand moves into the exponent (and to infinity past the largest
// float).  Magnitudes below 2^-126 are flushed to zero; NaN stays NaN.
HHG_HD float d2f_rn(double d) {
  const uint64_t u = dbits(d);
  const uint32_t sign = (uint32_t)(u >> 32) & 0x80000000u;
  const int e = (int)((u >> 52) & 0x7FF) - 1023;
  const uint64_t m = u & 0x000FFFFFFFFFFFFFull;
  if (e == 1024) return bitsf(sign | (m ? 0x7FC00000u : 0x7F800000u));
  if (e > 127) return bitsf(sign | 0x7F800000u);
  if (e < -126) return bitsf(sign);
  uint32_t bits = ((uint32_t)(e + 127) << 23) | (uint32_t)(m >> 29);
  const uint32_t rest = (uint32_t)(m & 0x1FFFFFFFull);
  if (rest > 0x10000000u || (rest == 0x10000000u && (bits & 1u))) bits += 1u;
  return bitsf(sign | bits);
}

}  // namespace hhg
