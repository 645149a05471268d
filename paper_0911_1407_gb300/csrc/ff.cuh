// ff.cuh -- float-float ("double-word") arithmetic on the FP32 pipes.
//
// A real is held as the unevaluated sum hi + lo of two floats with
// |lo| <= ulp(hi) / 2: about 48 significant bits, for transforms that need
// more than FP32 at a fraction of the cost of GB300's FP64 rate (1/64 of
// FP32).  Built from the error-free transforms TwoSum (Knuth, The Art of
// Computer Programming vol. 2, Sec. 4.2.2), Fast2Sum (Dekker, Numer. Math.
// 18, 1971) and the exact product by FMA (a*b - fl(a*b) = fma(a, b,
// -fl(a*b))), as analysed for double-word numbers by Joldes, Muller &
// Popescu (ACM TOMS 44, 2017):
//   - sum: the high parts added exactly, the low parts added to the error
//     term, one renormalisation (the error is a few 2^-48 of |a| + |b|,
//     which is what the butterflies of an FFT need);
//   - product: exact product of the high parts, the cross terms added by
//     FMA, one renormalisation.
// The compiler must not reassociate these expressions (nvcc does not without
// fast-math flags) nor contract the high product into an FMA (__fmul_rn).
#pragma once

#include "common.cuh"

namespace plc {

struct __align__(8) ff {
  float hi, lo;
  ff() = default;
  __host__ __device__ constexpr ff(float h, float l) : hi(h), lo(l) {}
  // the float-float nearest a double: hi = fl(d), lo = fl(d - hi)
  __host__ __device__ explicit ff(double d)
      : hi((float)d), lo((float)(d - (double)(float)d)) {}
};

struct __align__(16) ffc {
  ff x, y;
};
template <> struct CplxOf<ff> { using type = ffc; };

__device__ __forceinline__ ff operator+(ff a, ff b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  const float e = (a.hi - (s - bb)) + (b.hi - bb);   // TwoSum error of the high parts
  const float t = e + (a.lo + b.lo);
  const float h = s + t;                              // Fast2Sum renormalisation
  return ff(h, t - (h - s));
}
__device__ __forceinline__ ff operator-(ff a) { return ff(-a.hi, -a.lo); }
__device__ __forceinline__ ff operator-(ff a, ff b) { return a + (-b); }
__device__ __forceinline__ ff operator*(ff a, ff b) {
  const float p = __fmul_rn(a.hi, b.hi);              // never contracted into an FMA
  float e = fmaf(a.hi, b.hi, -p);                     // exact error of the product
  e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
  const float h = p + e;
  return ff(h, e - (h - p));
}
// sign factors of the small DFTs (+-1)
__device__ __forceinline__ ff operator*(int s, ff a) {
  return s == 1 ? a : (s == -1 ? -a : ff((double)s) * a);
}

// exact halving
__device__ __forceinline__ float halve(float a) { return 0.5f * a; }
__device__ __forceinline__ ff halve(ff a) { return ff(0.5f * a.hi, 0.5f * a.lo); }

__device__ __forceinline__ double to_double(ff a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ double to_double(float a) { return (double)a; }

}  // namespace plc
