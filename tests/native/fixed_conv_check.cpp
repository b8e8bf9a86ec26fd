// Reads "mode a b E" lines (decimal) from stdin and prints the bit pattern of
// the split-precision accumulator conversion for each, one hex word a line.
// mode 0: (hi, lo) = (a, b), exact; mode 1: (X, Y) = (a, b), exact;
// mode 2: (X, Y) = (a, b), the faster conversion.
#include <cinttypes>
#include <cstdio>

#include "oz_fixed.cuh"

int main() {
  long long a, b;
  int mode, e;
  while (std::scanf("%d %lld %lld %d", &mode, &a, &b, &e) == 4) {
    const double d = mode == 0   ? cqr2::oz_fixed_to_double(a, b, e)
                     : mode == 1 ? cqr2::oz_xy_to_double(a, b, e)
                                 : cqr2::oz_xy_to_double_fast(a, b, e);
    unsigned long long u;
    memcpy(&u, &d, sizeof u);
    std::printf("%016llx\n", u);
  }
  return 0;
}
