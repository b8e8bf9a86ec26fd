// 1/sqrt(d) and sqrt(d) for the Cholesky pivots, in few FP64 operations.
//
// GB300 issues an FP64 warp instruction at a small fraction of the FP32 rate,
// and the pivots of a right-looking Cholesky are a serial chain: each one
// waits for the previous column. The library's correctly rounded sqrt and
// division take many FP64 operations each. Here instead:
//   d = f 2^(2k) with f in [1, 4) (exponent split by integer operations),
//   y0 = single-precision 1/sqrt(f) (about 23 correct bits),
//   two Newton-Raphson steps for the root of 1/y^2 - f:
//     y <- y + y (1 - f y^2) / 2,
//   each doubling the correct bits (to the FP64 rounding level), then
//   1/sqrt(d) = y 2^(-k) (exact exponent shift) and sqrt(d) = d / sqrt(d)
//   taken as d * (1/sqrt(d)).
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

// Single-precision seed of 1/sqrt(f), f in [1, 4).
RS_HD float rs_seed(float f) {
#if defined(__CUDA_ARCH__)
  return rsqrtf(f);
#else
  return 1.0f / sqrtf(f);
#endif
}

// Newton-Raphson from a given seed y0 ~ 1/sqrt(f), f in [1, 4): two steps,
// three FP64 operations each (f / 2 is exact).
RS_HD double rs_newton2(double f, double y) {
  const double hf = 0.5 * f;
#if defined(__CUDA_ARCH__)
#pragma unroll
#endif
  for (int it = 0; it < 2; ++it) {
    const double h = hf * y;
    const double e = fma(-h, y, 0.5);  // (1 - f y^2) / 2
    y = fma(y, e, y);
  }
  return y;
}

// r = 1/sqrt(d) and l = sqrt(d) for a positive normal d; returns false (and
// fills both from the library functions) otherwise.
RS_HD bool chol_rsqrt(double d, double* r, double* l) {
  const unsigned long long b = rs_bits(d);
  const int ex = (int)((b >> 52) & 0x7FF);
  if ((b >> 63) != 0 || ex == 0 || ex == 0x7FF) {
    *l = sqrt(d);
    *r = 1.0 / *l;
    return false;
  }
  const int e = ex - 1023;              // d = 1.m 2^e
  const int k = (e >= 0 ? e : e - 1) / 2;  // floor(e / 2)
  const int fe = e - 2 * k;             // 0 or 1: f = 1.m 2^fe in [1, 4)
  const double f = rs_from_bits((b & ((1ull << 52) - 1)) | ((unsigned long long)(1023 + fe) << 52));
  const double y = rs_newton2(f, (double)rs_seed((float)f));
  // 1/sqrt(d) = y 2^-k: y is in (1/2, 1], so the shifted exponent stays normal
  const double rr = rs_from_bits(rs_bits(y) - ((unsigned long long)(long long)k << 52));
  *r = rr;
  *l = d * rr;
  return true;
}

}  // namespace cqr2
