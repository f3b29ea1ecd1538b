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

namespace heat {

struct DF {
  float hi, lo;
  DF() = default;
  __host__ __device__ __forceinline__ DF(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ __forceinline__ DF(int v) : hi((float)v), lo(0.f) {}
  __host__ __device__ __forceinline__ DF(double d) {
    hi = (float)d;
    lo = (float)(d - (double)hi);
  }
  __host__ __device__ __forceinline__ double to_double() const { return (double)hi + (double)lo; }
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
