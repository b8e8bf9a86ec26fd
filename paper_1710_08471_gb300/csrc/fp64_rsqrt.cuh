// 1/sqrt(d) and sqrt(d) for the Cholesky pivots, in few FP64 operations.
//
// The pivots of a right-looking Cholesky are a serial chain (each waits for
// the previous column), and on GB300 every dependent FP64 operation costs 64
// clocks (a conversion between FP32 and FP64 as much), while integer and FP32
// operations take a few. The library's correctly rounded sqrt and division
// take many FP64 operations each. Here instead:
//   d = f 2^(2k) with f in [1, 4) (exponent split by integer operations),
//   y0 = single-precision 1/sqrt(f) of f's leading 24 bits (the operand and
//        the result moved between the formats by bit operations, not by
//        conversion instructions; about 22 correct bits),
//   one third-order step for the root of 1/y^2 - f:
//     e = 1 - f y0^2,  y = y0 (1 + e/2 + 3 e^2/8),
//   whose error term 5 e^3 / 16 is below 2^-60 (four dependent FP64
//   operations against six for two Newton-Raphson steps), then
//   1/sqrt(d) = y 2^(-k) (exact exponent shift) and sqrt(d) = d * (1/sqrt(d)).
// Both results are within a few ulps, which the factorization's rounding
// analysis absorbs. Zero, subnormal, negative and non-finite pivots take the
// library functions (a breakdown is reported from the pivot value anyway).
// Host-compilable, so the error bound is checked on the CPU.
#pragma once

#include <math.h>
#include <stdint.h>
#include <string.h>

#if defined(__CUDACC__)
#define RS_HD __host__ __device__ __forceinline__
#else
#define RS_HD inline
#endif

namespace cqr2 {

RS_HD unsigned long long rs_bits(double x) {
#if defined(__CUDA_ARCH__)
  return (unsigned long long)__double_as_longlong(x);
#else
  unsigned long long b;
  memcpy(&b, &x, sizeof b);
  return b;
#endif
}

RS_HD double rs_from_bits(unsigned long long b) {
#if defined(__CUDA_ARCH__)
  return __longlong_as_double((long long)b);
#else
  double x;
  memcpy(&x, &b, sizeof x);
  return x;
#endif
}

RS_HD unsigned rs_f32_bits(float x) {
#if defined(__CUDA_ARCH__)
  return (unsigned)__float_as_uint(x);
#else
  unsigned b;
  memcpy(&b, &x, sizeof b);
  return b;
#endif
}

RS_HD float rs_f32_from_bits(unsigned b) {
#if defined(__CUDA_ARCH__)
  return __uint_as_float(b);
#else
  float x;
  memcpy(&x, &b, sizeof x);
  return x;
#endif
}

// Single-precision seed of 1/sqrt(f), f in [1, 4).
RS_HD float rs_seed(float f) {
#if defined(__CUDA_ARCH__)
  return rsqrtf(f);
#else
  return 1.0f / sqrtf(f);
#endif
}

// One third-order step from a seed y0 ~ 1/sqrt(f), f in [1, 4):
// y = y0 (1 + e/2 + 3 e^2/8) with e = 1 - f y0^2.
RS_HD double rs_refine3(double f, double y0) {
  const double t = f * y0;
  const double e = fma(-t, y0, 1.0);
  const double p = fma(e, 0.375, 0.5);
  const double ye = y0 * e;
  return fma(ye, p, y0);
}

// The FP64 value of a positive normal float, by bit operations.
RS_HD double rs_f32_to_f64(float x) {
  const unsigned b = rs_f32_bits(x);
  return rs_from_bits(((unsigned long long)((b >> 23) - 127 + 1023) << 52) | ((unsigned long long)(b & 0x7FFFFF) << 29));
}

// r = 1/sqrt(d) for a positive normal d; returns false (and fills r and l
// from the library functions) otherwise. l is left to the caller on success
// (l = d * r, which a kernel can fold into its column scaling).
RS_HD bool chol_rsqrt_r(double d, double* r, double* l) {
  const unsigned long long b = rs_bits(d);
  const int ex = (int)((b >> 52) & 0x7FF);
  if ((b >> 63) != 0 || ex == 0 || ex == 0x7FF) {
    *l = sqrt(d);
    *r = 1.0 / *l;
    return false;
  }
  const int e = ex - 1023;                 // d = 1.m 2^e
  const int k = (e >= 0 ? e : e - 1) / 2;  // floor(e / 2)
  const int fe = e - 2 * k;                // 0 or 1: f = 1.m 2^fe in [1, 4)
  const unsigned long long m = b & ((1ull << 52) - 1);
  const double f = rs_from_bits(m | ((unsigned long long)(1023 + fe) << 52));
  const float ff = rs_f32_from_bits(((unsigned)(127 + fe) << 23) | (unsigned)(m >> 29));  // f truncated
  const double y = rs_refine3(f, rs_f32_to_f64(rs_seed(ff)));
  // 1/sqrt(d) = y 2^-k: y is in (1/2, 1], so the shifted exponent stays normal
  *r = rs_from_bits(rs_bits(y) - ((unsigned long long)(long long)k << 52));
  return true;
}

// r = 1/sqrt(d) and l = sqrt(d) for a positive normal d; returns false (and
// fills both from the library functions) otherwise.
RS_HD bool chol_rsqrt(double d, double* r, double* l) {
  if (!chol_rsqrt_r(d, r, l)) return false;
  *l = d * *r;
  return true;
}

}  // namespace cqr2
