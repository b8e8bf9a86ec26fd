// Integer arithmetic of the split-precision path, host-compilable so that it
// can be checked on the CPU against exact rational arithmetic:
// - slicing: an FP64 entry x with shared exponent e (|x| < 2^e) becomes the
//   fixed-point integer v = round(x 2^(7 + 8 (S - 1) - e)) and then S
//   balanced base-256 digits, v = sum_s d_s 256^(S - 1 - s);
// - recombination: the fixed-point accumulators back to FP64, with integer
//   operations only (GB300's FP64 pipe is far too slow even for conversions).
#pragma once

#include <stdint.h>
#include <string.h>

#if defined(__CUDACC__)
#define OZ_HD __host__ __device__ __forceinline__
#else
#define OZ_HD inline
#endif

namespace cqr2 {

constexpr int OZ_EXP_NONFINITE = 1 << 20;  // exponent sentinel: a non-finite entry was seen

OZ_HD long long oz_double_bits(double x) {
#if defined(__CUDA_ARCH__)
  return __double_as_longlong(x);
#else
  long long b;
  memcpy(&b, &x, sizeof b);
  return b;
#endif
}

// v = x 2^(7 + 8 (S - 1) - e), rounded half away from zero, for |x| < 2^e:
// |v| < 2^(7 + 8 (S - 1)). Zero for a non-finite x or exponent.
OZ_HD long long oz_to_fixed(double x, int e, int S) {
  const unsigned long long b = (unsigned long long)oz_double_bits(x);
  int ex = (int)((b >> 52) & 0x7FF);
  unsigned long long mant = b & ((1ull << 52) - 1);
  if (ex == 0) {
    if (mant == 0) return 0;
    ex = 1;
  } else {
    mant |= 1ull << 52;
  }
  if (e >= OZ_EXP_NONFINITE || ex == 0x7FF) return 0;
  const int sh = ex - 1075 + 7 + 8 * (S - 1) - e;  // < 8S - 53 because |x| < 2^e
  long long v;
  if (sh >= 0) {
    v = (long long)(mant << sh);
  } else if (sh > -63) {
    v = (long long)((mant + (1ull << (-sh - 1))) >> (-sh));
  } else {
    v = 0;
  }
  return (b >> 63) ? -v : v;
}

// Balanced base-256 digits of v, most significant first: d[1..S-1] in
// [-128, 127] and v = sum_s d[s] 256^(S - 1 - s). With B = 128 in each of the
// S - 1 low bytes, the low digits are the bytes of v + B minus 128 and the
// top digit is v + B shifted down arithmetically -- the same digits as
// peeling the signed low byte off one at a time (d = sext(v mod 256), v =
// (v - d) / 256), without that serial chain.
template <int S>
OZ_HD void oz_balanced_digits(long long v, int (&d)[S]) {
  constexpr unsigned long long B = ((1ull << (8 * (S - 1))) - 1) / 255 * 128;
  const unsigned long long u = (unsigned long long)v + B;
  const unsigned lo = (unsigned)u, hi = (unsigned)(u >> 32);
#if defined(__CUDA_ARCH__)
#pragma unroll
#endif
  for (int i = 0; i < S - 1; ++i) {
    const unsigned byte = ((i < 4 ? lo : hi) >> (8 * (i & 3))) & 0xFFu;
    d[S - 1 - i] = (int)byte - 128;
  }
  d[0] = (int)((long long)u >> (8 * (S - 1)));
}

OZ_HD int oz_clz64(unsigned long long x) {
#if defined(__CUDA_ARCH__)
  return __clzll((long long)x);
#else
  return x ? __builtin_clzll(x) : 64;
#endif
}

OZ_HD double oz_bits_to_double(unsigned long long b) {
#if defined(__CUDA_ARCH__)
  return __longlong_as_double((long long)b);
#else
  double d;
  memcpy(&d, &b, sizeof d);
  return d;
#endif
}

// Exact value m 2^e (m < 2^53) rounded into the subnormal range (or zero),
// for the rare results below the normal range. Round to nearest, ties to even.
OZ_HD double oz_scale_small(unsigned long long mant53, unsigned long long sticky_in, int e) {
  // result bits = round(mant53 2^(e + 1074)); e + 1074 < 0 here
  const int sh = -(e + 1074);
  if (sh >= 64) return 0.0;
  const unsigned long long q = mant53 >> sh;
  const unsigned long long r = mant53 & ((1ull << sh) - 1ull);
  const unsigned long long halfv = 1ull << (sh - 1);
  const bool up = r > halfv || (r == halfv && (sticky_in || (q & 1ull)));
  return oz_bits_to_double(q + (up ? 1ull : 0ull));
}

// (hi 2^32 + lo) 2^E rounded to the nearest double, ties to even, for
// |hi|, |lo| < 2^62 (the accumulators of 2^20 rows stay far below that).
OZ_HD double oz_fixed_to_double(long long hi, long long lo, int E) {
  // T = H 2^32 + L with 0 <= L < 2^32
  const long long H = hi + (lo >> 32);
  const unsigned L = (unsigned)(unsigned long long)lo;
  const bool neg = H < 0;
  // |T| = W 2^32 + w0
  const unsigned w0 = neg ? 0u - L : L;
  const unsigned long long W = neg ? ~(unsigned long long)H + (L == 0u ? 1ull : 0ull) : (unsigned long long)H;
  unsigned long long hw = W, lw = (unsigned long long)w0 << 32;
  int top = 95;  // bit of |T| that bit 63 of hw holds
  if (hw == 0) {
    hw = lw;
    lw = 0;
    top = 31;
  }
  if (hw == 0) return 0.0;
  const int lz = oz_clz64(hw);
  const unsigned long long N = (hw << lz) | (lw >> 1 >> (63 - lz));  // top 64 bits, bit 63 set
  const unsigned long long rest = lw << lz;                           // bits below N
  const int msb = top - lz;                                            // |T| in [2^msb, 2^(msb+1))
  unsigned long long mant = N >> 11;                                   // 53 bits, bit 52 set
  const unsigned long long halfbit = (N >> 10) & 1ull;
  const unsigned long long sticky = ((N & 0x3FFull) | rest) != 0 ? 1ull : 0ull;
  const int biased = msb + E + 1023;
  if (biased < 1) {
    const double mag = oz_scale_small(mant, halfbit | sticky, msb + E - 52);
    return neg ? -mag : mag;
  }
  mant += halfbit & (sticky | (mant & 1ull));
  // the implicit bit adds one to the exponent field; a rounding carry to
  // 2^53 moves it one further, as it must
  unsigned long long bits = ((unsigned long long)(biased - 1) << 52) + mant;
  if (biased > 2046) bits = 0x7FF0000000000000ull;  // overflow to infinity
  return oz_bits_to_double(bits | (neg ? 1ull << 63 : 0ull));
}

// The accumulators as kept by the kernel: T = X 2^24 + Y with X holding
// groups 0-3 and Y groups 4-6. Exact conversion through (hi, lo).
OZ_HD double oz_xy_to_double(long long X, long long Y, int E) {
  const long long hi = X >> 8;  // T = hi 2^32 + ((X mod 2^8) 2^24 + Y)
  const long long lo = (long long)((unsigned long long)(X & 0xFF) << 24) + Y;
  return oz_fixed_to_double(hi, lo, E);
}

#if defined(__CUDA_ARCH__)
// The exact routine as an out-of-line call for the fast routine's rare
// subnormal case: inlined at every output it would crowd the instruction
// cache of the epilogue loop with code that almost never runs.
static __device__ __noinline__ double oz_xy_to_double_cold(long long X, long long Y, int E) {
  return oz_xy_to_double(X, Y, E);
}
#define OZ_XY_COLD oz_xy_to_double_cold
#else
#define OZ_XY_COLD oz_xy_to_double
#endif

// Faster conversion of T = X 2^24 + Y (|X| < 2^61, |Y| < 2^55) to within one
// ulp of T 2^E: scale T by 2^-sh so that it fits 62 bits (the bits of Y that
// fall off are below 2^-61 of it), then round that int64 to nearest.
OZ_HD double oz_xy_to_double_fast(long long X, long long Y, int E) {
  const unsigned long long ax = X < 0 ? 0ull - (unsigned long long)X : (unsigned long long)X;
  const int bl = 64 - oz_clz64(ax);  // bit length of |X|
  const int sh = bl > 38 ? bl - 38 : 0;
  const long long Z = (long long)((unsigned long long)X << (24 - sh)) + (Y >> sh);
  const bool neg = Z < 0;
  unsigned long long u = neg ? 0ull - (unsigned long long)Z : (unsigned long long)Z;
  if (u == 0) return 0.0;
  const int lz = oz_clz64(u);
  u <<= lz;
  unsigned long long mant = u >> 11;
  const unsigned long long rb = (u >> 10) & 1ull, st = (u & 0x3FFull) != 0 ? 1ull : 0ull;
  const int biased = 63 - lz + E + sh + 1023;
  if (biased < 1) return OZ_XY_COLD(X, Y, E);  // subnormal: rare, exact path
  mant += rb & (st | (mant & 1ull));
  unsigned long long bits = ((unsigned long long)(biased - 1) << 52) + mant;
  if (biased > 2046) bits = 0x7FF0000000000000ull;
  return oz_bits_to_double(bits | (neg ? 1ull << 63 : 0ull));
}

}  // namespace cqr2
