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

// double -> float-float by integer operations on the IEEE-754 bit fields, so
// that the FP64 pipe (1/64 of the FP32 rate on GB300) is not used for it.
// (The other direction, hi + lo in FP64, measured faster with the FP64
// conversions than with integer widening.)
//
// ff_split(d): hi = d with its significand cut to 24 bits, lo = the remaining
// 29 bits rounded to a float (exact scaling by a power of two), then one
// Fast2Sum so that |lo| <= ulp(hi) / 2.  hi + lo equals d to 2^-48 relative.
// |d| < 2^-149 gives 0; the narrow bands where hi or lo would leave the normal
// float range (2^-149 <= |d| < 2^-70, |d| >= 2^128, inf, NaN) take the
// FP64 conversion.
__device__ __forceinline__ ff ff_split(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned top = (unsigned)(b >> 32);
  const int e = (int)((top >> 20) & 0x7ffu) - 1023;
  if (e < -149) return ff(0.f, 0.f);
  if (e < -70 || e > 127) return ff(d);
  const unsigned sign = top & 0x80000000u;
  const unsigned long long mant = b & 0xFFFFFFFFFFFFFull;             // 52 bits
  const float h = __uint_as_float(sign | ((unsigned)(e + 127) << 23) | (unsigned)(mant >> 29));
  const float scale = __uint_as_float((unsigned)(e - 52 + 127) << 23);  // 2^(e - 52), normal
  float l = __uint2float_rn((unsigned)(mant & 0x1FFFFFFFull)) * scale;
  if (sign) l = -l;
  const float s = h + l;                                                // Fast2Sum, |h| >= |l|
  return ff(s, l - (s - h));
}

__device__ __forceinline__ ff ff_abs(ff a) { return a.hi < 0.f ? -a : a; }

// exp(x) of a float-float argument, by the table-driven method of
// Tang (ACM TOMS 15, 1989) with 64 table points: x = (64 m + j) ln2/64 + r,
// |r| <= ln2/128, exp(x) = 2^m 2^(j/64) (1 + p(r)), p the Taylor polynomial
// of exp(r) - 1 to degree 5 (remainder below 4e-17).  The reduction is done
// in float-float, so the relative error is a few 2^-48 of max(|x|, 1).
// tab[j] = 2^(j/64) in float-float (device memory, read through L1).
// For |x| < 80.
__device__ __forceinline__ ff exp_ff(ff xf, const ff* __restrict__ tab) {
  const float nf = rintf(xf.hi * 92.332482616893657f);     // 64 / ln 2
  const int nn = (int)nf;
  const int j = nn & 63, m = (nn - j) / 64;
  // ln2 / 64 as a float-float; nf is an integer below 2^13, exact in float
  const ff l64(1.083042473e-02f, -2.976022206e-11f);
  const ff r = xf - ff(nf, 0.f) * l64;
  // p(r) = r + r^2 (1/2 + r (1/6 + r (1/24 + r / 120))): the inner part to
  // float accuracy suffices (it carries r^3 / 6 < 3e-8)
  const float q = fmaf(fmaf(r.hi, 1.f / 120.f, 1.f / 24.f), r.hi, 1.f / 6.f);
  const float rq = r.hi * q;
  const float t_hi = 0.5f + rq;
  const ff t(t_hi, rq - (t_hi - 0.5f));                    // Fast2Sum, |rq| < 0.5
  const ff p = r + (r * r) * t;
  const float2 tj = __ldg(reinterpret_cast<const float2*>(tab) + j);
  const ff sj(tj.x, tj.y);
  const ff e = sj + sj * p;
  return ff(ldexpf(e.hi, m), ldexpf(e.lo, m));
}

// Sum accumulator in float-float (for sums that must carry FP64-level
// accuracy out of float-float arithmetic).
struct AccFF {
  ff s;
  __device__ void init(bool) { s = ff(0.f, 0.f); }
  __device__ void add(ff x) { s = s + x; }
  __device__ double get() const { return to_double(s); }
  __device__ void merge(const AccFF& o, bool) { s = s + o.s; }
  __device__ AccFF shfl_down(int o) const {
    return AccFF{ff(__shfl_down_sync(0xffffffffu, s.hi, o), __shfl_down_sync(0xffffffffu, s.lo, o))};
  }
};

}  // namespace plc
