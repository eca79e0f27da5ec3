// Double-float ("df64") arithmetic on the FP32 pipe.
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2
// after normalisation, i.e. a 48-bit significand with the FP32 exponent range.
// Error-free transformations (Dekker 1971; Knuth, TAOCP vol. 2, 4.2.2):
//   product  a*b:   p = fl(a.hi b.hi), e = fma(a.hi, b.hi, -p) is exact, and
//                   the cross terms a.hi b.lo + a.lo b.hi are added into e
//                   (a.lo b.lo, of relative size 2^-48, is dropped);
//   sum      a+b:   two-sum of the high parts (s = a.hi + b.hi, and the exact
//                   rounding error of s by six additions), low parts added;
//   normalise:      fast two-sum (s = hi + lo, lo' = lo - (s - hi)).
// A multiply-add therefore costs 12 FP32 instructions; on GB300 the FP32 pipe
// issues 64x the FP64 rate, so df64 contractions run several times faster
// than native FP64 while staying within about 2^-47 relative per operation.
// Valid while magnitudes stay inside the normal FP32 range (about 1e-30 ..
// 1e30 for the low parts to stay normal).
#pragma once

#include <cuda_runtime.h>

struct __align__(8) df64 {
  float hi, lo;
  __host__ __device__ df64() {}
  __host__ __device__ df64(int z) : hi((float)z), lo(0.0f) {}
  __host__ __device__ df64(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ explicit df64(double d) {
    hi = (float)d;
    lo = (float)(d - (double)hi);
  }
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ df64 operator*(const df64 a, const df64 b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return df64(p, e);
}

__device__ __forceinline__ df64 operator+(const df64 a, const df64 b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  const float err = (a.hi - (s - bb)) + (b.hi - bb);
  return df64(s, err + (a.lo + b.lo));
}

__device__ __forceinline__ df64 operator-(const df64 a) { return df64(-a.hi, -a.lo); }
__device__ __forceinline__ df64 operator-(const df64 a, const df64 b) { return a + (-b); }

__device__ __forceinline__ df64& operator+=(df64& a, const df64 b) {
  a = a + b;
  return a;
}

// Normalise (fast two-sum): afterwards |lo| <= ulp(hi) / 2.
__device__ __forceinline__ df64 df_norm(const df64 a) {
  const float s = a.hi + a.lo;
  return df64(s, a.lo - (s - a.hi));
}

// Identity for the native types; normalisation for df64. Called where a
// finished sum becomes a factor of later products.
__device__ __forceinline__ double fe_norm(double v) { return v; }
__device__ __forceinline__ float fe_norm(float v) { return v; }
__device__ __forceinline__ df64 fe_norm(df64 v) { return df_norm(v); }

// Read-only loads of the element data.
__device__ __forceinline__ double fe_ldg(const double* p) { return __ldg(p); }
__device__ __forceinline__ float fe_ldg(const float* p) { return __ldg(p); }
__device__ __forceinline__ df64 fe_ldg(const df64* p) {
  const float2 v = __ldg(reinterpret_cast<const float2*>(p));
  return df64(v.x, v.y);
}

// Conversions between the compute type T and the vector type TX.
template <typename T>
__device__ __forceinline__ T fe_from(double v) { return (T)v; }
template <typename T>
__device__ __forceinline__ T fe_from(float v) { return (T)v; }
template <>
__device__ __forceinline__ df64 fe_from<df64>(double v) { return df64(v); }
__device__ __forceinline__ void fe_store(double* p, double v) { *p = v; }
__device__ __forceinline__ void fe_store(float* p, float v) { *p = v; }
__device__ __forceinline__ void fe_store(double* p, df64 v) { *p = (double)v; }
