// Double-float arithmetic: a value is the unevaluated sum hi + lo of two
// floats with |lo| <= ulp(hi)/2, about 48 significant bits. Built from the
// error-free transformations of Knuth (two-sum: the rounding error of a + b
// is itself a float) and of Dekker with a fused multiply-add (two-product:
// the rounding error of a * b is fma(a, b, -fl(a*b))). Addition is the short
// form (error bounded by about 2^-44 times |a| + |b|, not |a + b|), which is
// what a residual b - A x needs: its error must be small next to the operand
// scale |b|, not next to the small result.
//
// On this GPU FP64 runs at 1/58 of the FP32 rate, so an operator pass in
// double-float, about ten FP32 operations per FP64 one, is several times
// faster than the same pass in FP64 and far more accurate than an FP32 one.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

namespace heat {

// Bit patterns of IEEE-754 binary32 / binary64 values.
__host__ __device__ __forceinline__ uint32_t df_fbits(float f) {
#ifdef __CUDA_ARCH__
  return (uint32_t)__float_as_uint(f);
#else
  uint32_t b;
  std::memcpy(&b, &f, 4);
  return b;
#endif
}
__host__ __device__ __forceinline__ float df_ffrom(uint32_t b) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(b);
#else
  float f;
  std::memcpy(&f, &b, 4);
  return f;
#endif
}
__host__ __device__ __forceinline__ uint64_t df_dbits(double d) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(d);
#else
  uint64_t b;
  std::memcpy(&b, &d, 8);
  return b;
#endif
}
__host__ __device__ __forceinline__ double df_dfrom(uint64_t b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double d;
  std::memcpy(&d, &b, 8);
  return d;
#endif
}

// float -> double by rewriting the fields (exact): the exponent is rebiased
// from 127 to 1023 and the 23 fraction bits move to the top of the 52. Zeros
// keep their sign; subnormal, infinite and NaN inputs (never met by the
// solver's values) take the hardware conversion. On this GPU the hardware
// conversion runs on the FP64 unit, at 1/58 of the FP32 rate (measured); this
// form runs on the integer unit.
__host__ __device__ __forceinline__ double df_f2d(float f) {
  const uint32_t b = df_fbits(f);
  const uint32_t e = (b >> 23) & 0xFFu;
  const uint64_t sgn = (uint64_t)(b >> 31) << 63;
  if (e == 0u && (b << 1) == 0u) return df_dfrom(sgn);
  if (e == 0u || e == 0xFFu) return (double)f;
  return df_dfrom(sgn | ((uint64_t)(e + 896u) << 52) | ((uint64_t)(b & 0x7FFFFFu) << 29));
}

// double -> (hi, lo): hi is d rounded to the nearest float (ties to even),
// lo the remainder d - hi rounded to the nearest float, from the fields of d:
// of the 53-bit significand m, hi keeps the top 24 bits (rounded) and lo is
// the signed remainder of the low 29 bits scaled by 2^(e-52). This is the
// value pair the FP64 conversions (float)d, (float)(d - (double)(float)d)
// give, for 2^-74 <= |d| < 2^127. Below 2^-74 the remainder is dropped
// (below 2^-126 both halves), an absolute error under 2^-98 that the
// solver's sums cannot see; above, and for infinities and NaNs, the
// hardware conversions run.
__host__ __device__ __forceinline__ void df_split(double d, float& hi, float& lo) {
  const uint64_t u = df_dbits(d);
  const int e = (int)((u >> 52) & 0x7FFu) - 1023;
  const uint32_t sgn = (uint32_t)(u >> 63) << 31;
  if (e >= -74 && e <= 126) {
    uint32_t mh = (uint32_t)(((u & 0xFFFFFFFFFFFFFull) | (1ull << 52)) >> 29);  // 24 bits
    int32_t r = (int32_t)(u & 0x1FFFFFFFull);                                    // 29 bits
    if (r > (1 << 28) || (r == (1 << 28) && (mh & 1u))) {
      mh += 1u;
      r -= (1 << 29);
    }
    int eh = e;
    if (mh == (1u << 24)) {
      mh >>= 1;
      eh += 1;
    }
    hi = df_ffrom(sgn | ((uint32_t)(eh + 127) << 23) | (mh & 0x7FFFFFu));
    // r * 2^(e-52): the power of two is a normal float for e >= -74
    lo = (float)r * df_ffrom(sgn | ((uint32_t)(e - 52 + 127) << 23));
    return;
  }
  if (e < -74 && e >= -126) {
    uint32_t mh = (uint32_t)(((u & 0xFFFFFFFFFFFFFull) | (1ull << 52)) >> 29);
    const uint32_t r = (uint32_t)(u & 0x1FFFFFFFull);
    if (r > (1u << 28) || (r == (1u << 28) && (mh & 1u))) mh += 1u;
    int eh = e;
    if (mh == (1u << 24)) {
      mh >>= 1;
      eh += 1;
    }
    hi = df_ffrom(sgn | ((uint32_t)(eh + 127) << 23) | (mh & 0x7FFFFFu));
    lo = 0.f;
    return;
  }
  if (e < -126) {
    hi = df_ffrom(sgn);
    lo = 0.f;
    return;
  }
  hi = (float)d;
  lo = (float)(d - (double)hi);
}

struct DF {
  float hi, lo;
  DF() = default;
  __host__ __device__ __forceinline__ DF(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ __forceinline__ DF(int v) : hi((float)v), lo(0.f) {}
  __host__ __device__ __forceinline__ DF(double d) { df_split(d, hi, lo); }
  // exact: both halves convert exactly, and |lo| <= ulp(hi)/2 makes the sum exact
  __host__ __device__ __forceinline__ double to_double() const { return df_f2d(hi) + df_f2d(lo); }
};

// s + e == a + b exactly (Knuth)
__host__ __device__ __forceinline__ void df_two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
// s + e == a + b exactly when |a| >= |b| (Dekker)
__host__ __device__ __forceinline__ void df_fast_two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  e = b - (s - a);
}

__host__ __device__ __forceinline__ DF operator+(const DF& a, const DF& b) {
  float s, e;
  df_two_sum(a.hi, b.hi, s, e);
  e += a.lo + b.lo;
  float h, l;
  df_fast_two_sum(s, e, h, l);
  return DF(h, l);
}
__host__ __device__ __forceinline__ DF operator-(const DF& a) { return DF(-a.hi, -a.lo); }
__host__ __device__ __forceinline__ DF operator-(const DF& a, const DF& b) { return a + (-b); }
__host__ __device__ __forceinline__ DF operator*(const DF& a, const DF& b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);  // the product's rounding error, exactly
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  float h, l;
  df_fast_two_sum(p, e, h, l);
  return DF(h, l);
}
__host__ __device__ __forceinline__ DF& operator+=(DF& a, const DF& b) {
  a = a + b;
  return a;
}

// d rounded to the nearest float (the hi half of df_split), without the FP64 unit
__host__ __device__ __forceinline__ float df_d2f(double d) {
  float hi, lo;
  df_split(d, hi, lo);
  return hi;
}

__host__ __device__ __forceinline__ double to_d(double v) { return v; }
__host__ __device__ __forceinline__ double to_d(const DF& v) { return v.to_double(); }

struct DF2 {
  DF x, y;
};

}  // namespace heat

#ifdef __CUDACC__
// Segment shuffles of a double-float (both halves); at global scope beside
// the built-in overloads so that unqualified calls keep finding those.
__device__ __forceinline__ heat::DF __shfl_down_sync(unsigned mask, const heat::DF& v, unsigned delta, int width) {
  return heat::DF(__shfl_down_sync(mask, v.hi, delta, width), __shfl_down_sync(mask, v.lo, delta, width));
}
__device__ __forceinline__ heat::DF __shfl_up_sync(unsigned mask, const heat::DF& v, unsigned delta, int width) {
  return heat::DF(__shfl_up_sync(mask, v.hi, delta, width), __shfl_up_sync(mask, v.lo, delta, width));
}
#endif
