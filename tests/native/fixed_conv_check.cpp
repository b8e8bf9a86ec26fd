// Reads "mode a b E" lines (decimal) from stdin and prints the bit pattern of
// the split-precision accumulator conversion for each, one hex word a line.
// mode 0: (hi, lo) = (a, b), exact; mode 1: (X, Y) = (a, b), exact;
// mode 2: (X, Y) = (a, b), the faster conversion.
// mode 3: slicing of the double with bit pattern a, exponent E, b = S slices
// (6 or 7): prints the fixed-point value and the S digits, decimal, one line.
#include <cinttypes>
#include <cstdio>

#include "oz_fixed.cuh"

template <int S>
static void slice(long long bits, int e) {
  double x;
  memcpy(&x, &bits, sizeof x);
  const long long v = cqr2::oz_to_fixed(x, e, S);
  int d[S];
  cqr2::oz_balanced_digits<S>(v, d);
  std::printf("%lld", v);
  for (int s = 0; s < S; ++s) std::printf(" %d", d[s]);
  std::printf("\n");
}

int main() {
  long long a, b;
  int mode, e;
  while (std::scanf("%d %lld %lld %d", &mode, &a, &b, &e) == 4) {
    if (mode == 3) {
      if (b == 7) slice<7>(a, e);
      else slice<6>(a, e);
      continue;
    }
    const double d = mode == 0   ? cqr2::oz_fixed_to_double(a, b, e)
                     : mode == 1 ? cqr2::oz_xy_to_double(a, b, e)
                                 : cqr2::oz_xy_to_double_fast(a, b, e);
    unsigned long long u;
    memcpy(&u, &d, sizeof u);
    std::printf("%016llx\n", u);
  }
  return 0;
}
