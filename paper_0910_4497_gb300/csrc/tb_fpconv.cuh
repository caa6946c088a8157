// IEEE-754 binary64 <-> binary32 conversions by integer operations on the
// bit patterns (sign kept, exponent rebiased between the two formats, the
// 52-bit fraction cut to 23 bits and rounded on its first dropped bit, ties
// away from zero).  On this GPU the conversion instructions run on the FP64
// pipe; kernels whose FP64 arithmetic already keeps that pipe busy (the
// density blocks) convert their FP64 records with these instead.
// Results below the binary32 normal range flush to (signed) zero; infinities
// and NaNs map to infinities and NaNs.  Within the normal range d2f is within
// half a binary32 ulp of the value and f2d is exact.
#pragma once
#include <cstring>

namespace tbconv {

__host__ __device__ __forceinline__ unsigned long long bits64(double x) {
#ifdef __CUDA_ARCH__
  return (unsigned long long)__double_as_longlong(x);
#else
  unsigned long long b;
  std::memcpy(&b, &x, sizeof(b));
  return b;
#endif
}

__host__ __device__ __forceinline__ float from_bits32(unsigned u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float f;
  std::memcpy(&f, &u, sizeof(f));
  return f;
#endif
}

__host__ __device__ __forceinline__ unsigned bits32(float x) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(x);
#else
  unsigned u;
  std::memcpy(&u, &x, sizeof(u));
  return u;
#endif
}

__host__ __device__ __forceinline__ double from_bits64(unsigned long long b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double x;
  std::memcpy(&x, &b, sizeof(x));
  return x;
#endif
}

__host__ __device__ __forceinline__ float d2f(double x) {
  const unsigned long long b = bits64(x);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned sign = hi & 0x80000000u;
  const int ed = (int)((hi >> 20) & 0x7ffu);
  if (ed == 0x7ff)                                   // infinity or NaN
    return from_bits32(sign | 0x7f800000u | ((((hi & 0xfffffu) | lo) != 0u) ? 0x400000u : 0u));
  const int ef = ed - 1023 + 127;
  if (ef <= 0) return from_bits32(sign);             // below the normal range
  if (ef >= 255) return from_bits32(sign | 0x7f800000u);
  const unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);
  // a carry out of the fraction moves into the exponent (to infinity at the top)
  return from_bits32(sign | (((unsigned)ef << 23) + m + ((lo >> 28) & 1u)));
}

__host__ __device__ __forceinline__ double f2d(float x) {
  const unsigned u = bits32(x);
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  const unsigned ef = (u >> 23) & 0xffu;
  const unsigned long long m = u & 0x7fffffu;
  if (ef == 0u) return from_bits64(sign);            // zero (subnormals flushed)
  const unsigned long long ed = ef == 0xffu ? 0x7ffull : (unsigned long long)(ef - 127u + 1023u);
  return from_bits64(sign | (ed << 52) | (m << 29));
}

}  // namespace tbconv
