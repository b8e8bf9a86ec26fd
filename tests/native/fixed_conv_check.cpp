// Reads "hi lo E" triples (decimal) from stdin and prints the bit pattern of
// the split-precision accumulator conversion for each, one hex word a line.
#include <cinttypes>
#include <cstdio>

#include "oz_fixed.cuh"

int main() {
  long long hi, lo;
  int e;
  while (std::scanf("%lld %lld %d", &hi, &lo, &e) == 3) {
    const double d = cqr2::oz_fixed_to_double(hi, lo, e);
    unsigned long long b;
    memcpy(&b, &d, sizeof b);
    std::printf("%016llx\n", b);
  }
  return 0;
}
