// Arithmetic of the face kernels on FP64 data: IEEE FP64 (V = the storage
// type) or double-float (V = dfl, a pair of floats on the FP32 pipes, about
// 47 significant bits; values must lie in [2^-74, 2^127] in magnitude for
// full precision, smaller ones keep 24 bits).  On a GPU whose FP64 rate is
// 1/64 of its FP32 rate the double-float form moves the stencil arithmetic
// off the narrow FP64 pipe; it is an opt-in mode (hhg_set_fp64_arith).
#pragma once

#include "dfloat.cuh"

namespace hhg {

// a / b in double-float: one float quotient, its residual a - b q1 in
// double-float, and a float correction (error about 2^-44 relative)
HHG_HD dfl df_div(dfl a, dfl b) {
  const float q1 = a.hi / b.hi;
  const dfl p = df_mul(b, dfl{q1, 0.f});
  const dfl r = df_add(a, dfl{-p.hi, -p.lo});
  const float q2 = r.hi / b.hi;
  return fast_two_sum(q1, q2);
}

template <typename T, bool DF>
struct Arith {
  using V = T;
  static __device__ __forceinline__ V in(T x) { return x; }
  static __device__ __forceinline__ T out(V v) { return v; }
  static __device__ __forceinline__ V add(V a, V b) { return a + b; }
  static __device__ __forceinline__ V sub(V a, V b) { return a - b; }
  static __device__ __forceinline__ V mul(V a, V b) { return a * b; }
  static __device__ __forceinline__ V fma(V a, V b, V c) { return ::fma(a, b, c); }   // a b + c
  static __device__ __forceinline__ V div(V a, V b) { return a / b; }
  static __device__ __forceinline__ V shfl_up(V v) { return __shfl_up_sync(0xffffffffu, v, 1); }
  static __device__ __forceinline__ V shfl_down(V v) { return __shfl_down_sync(0xffffffffu, v, 1); }
  static __device__ __forceinline__ double sq(V v) { return (double)v * (double)v; }
  static __device__ __forceinline__ float to_f32(V v) { return (float)v; }
};

template <>
struct Arith<double, true> {
  using V = dfl;
  static __device__ __forceinline__ V in(double x) { return from_double(x); }
  static __device__ __forceinline__ double out(V v) { return to_double(v); }
  static __device__ __forceinline__ V add(V a, V b) { return df_add(a, b); }
  static __device__ __forceinline__ V sub(V a, V b) { return df_add(a, dfl{-b.hi, -b.lo}); }
  static __device__ __forceinline__ V mul(V a, V b) { return df_mul(a, b); }
  static __device__ __forceinline__ V fma(V a, V b, V c) { return df_add(df_mul(a, b), c); }
  static __device__ __forceinline__ V div(V a, V b) { return df_div(a, b); }
  static __device__ __forceinline__ V shfl_up(V v) {
    return dfl{__shfl_up_sync(0xffffffffu, v.hi, 1), __shfl_up_sync(0xffffffffu, v.lo, 1)};
  }
  static __device__ __forceinline__ V shfl_down(V v) {
    return dfl{__shfl_down_sync(0xffffffffu, v.hi, 1), __shfl_down_sync(0xffffffffu, v.lo, 1)};
  }
  static __device__ __forceinline__ double sq(V v) {
    const double d = to_double(v);
    return d * d;
  }
  // the float nearest the pair (|lo| <= ulp(hi) / 2, so one rounded add)
  static __device__ __forceinline__ float to_f32(V v) { return v.hi + v.lo; }
};

}  // namespace hhg
