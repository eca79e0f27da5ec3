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

// double -> df64 and df64 -> double by bit manipulation on the integer
// pipe, keeping the conversions of every gathered input and every output off
// GB300's FP64 pipe (1/64 of the FP32 rate; four FP64-pipe instructions per
// input and three per output in the plain form).
//   in:  v = s 2^E (1.m), 52-bit m. hi = v with its 29 lowest mantissa bits
//        cleared (exactly a float), lo = those 29 bits times 2^(E - 52)
//        (one integer-to-float conversion, rounded to 24 bits), then a fast
//        two-sum normalises the pair. Error below 2^-48 |v|, as for the
//        rounded split. Taken for 2^-74 <= |v| < 2^127, where hi and the
//        scale of lo are normal floats; other inputs take the FP64 path.
//   out: each float widened to double by rebiasing its exponent and
//        shifting its mantissa (exact; zero handled, subnormal and
//        non-finite floats take the FP64 conversion), then one FP64 add, as
//        (double)hi + (double)lo computes it.
__device__ __forceinline__ df64 df64_from_double_bits(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const unsigned hw = (unsigned)(b >> 32), lw = (unsigned)b;
  const int e = (int)((hw >> 20) & 0x7ffu);
  if (e < 949 || e > 1149) return df64(v);
  const unsigned sign = hw & 0x80000000u;
  const unsigned m_hi = ((hw & 0xfffffu) << 3) | (lw >> 29);
  const float hi = __uint_as_float(sign | ((unsigned)(e - 1023 + 127) << 23) | m_hi);
  const float scale = __uint_as_float((unsigned)(e - 1075 + 127) << 23);  // 2^(E - 52)
  float lo = __uint2float_rn(lw & 0x1fffffffu) * scale;
  lo = __uint_as_float(__float_as_uint(lo) | sign);
  return df_norm(df64(hi, lo));
}

__device__ __forceinline__ double double_of_float_bits(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned e = (b >> 23) & 0xffu;
  if ((b & 0x7fffffffu) == 0) return __hiloint2double((int)(b & 0x80000000u), 0);
  if (e == 0 || e == 255) return (double)f;
  const unsigned m = b & 0x7fffffu;
  const unsigned hw = (b & 0x80000000u) | ((e - 127 + 1023) << 20) | (m >> 3);
  return __hiloint2double((int)hw, (int)(m << 29));
}

// Conversions between the compute type T and the vector type TX.
template <typename T>
__device__ __forceinline__ T fe_from(double v) { return (T)v; }
template <typename T>
__device__ __forceinline__ T fe_from(float v) { return (T)v; }
template <>
__device__ __forceinline__ df64 fe_from<df64>(double v) { return df64_from_double_bits(v); }
__device__ __forceinline__ void fe_store(double* p, double v) { *p = v; }
__device__ __forceinline__ void fe_store(float* p, float v) { *p = v; }
__device__ __forceinline__ void fe_store(double* p, df64 v) {
  *p = double_of_float_bits(v.hi) + double_of_float_bits(v.lo);
}
