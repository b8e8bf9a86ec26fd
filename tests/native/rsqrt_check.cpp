// Reads "mode bits pert" lines from stdin (bits: an FP64 bit pattern as a
// signed decimal; pert: a seed perturbation in float ulps) and prints hex bit
// patterns of the pivot routine's results.
// mode 0: chol_rsqrt(d) -> "r l"; mode 1: rs_refine3(f, seed perturbed by
// pert float ulps) for f = d in [1, 4) -> "y".
#include <cstdio>
#include <cstring>

#include "fp64_rsqrt.cuh"

static unsigned long long bits_of(double x) {
  unsigned long long u;
  memcpy(&u, &x, sizeof u);
  return u;
}

int main() {
  int mode, pert;
  long long b;
  while (std::scanf("%d %lld %d", &mode, &b, &pert) == 3) {
    double d;
    memcpy(&d, &b, sizeof d);
    if (mode == 0) {
      double r, l;
      cqr2::chol_rsqrt(d, &r, &l);
      std::printf("%016llx %016llx\n", bits_of(r), bits_of(l));
    } else {
      float s = 1.0f / sqrtf((float)d);
      unsigned u;
      memcpy(&u, &s, sizeof u);
      u += (unsigned)pert;
      memcpy(&s, &u, sizeof s);
      std::printf("%016llx\n", bits_of(cqr2::rs_refine3(d, (double)s)));
    }
  }
  return 0;
}
