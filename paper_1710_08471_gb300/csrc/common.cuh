// Internal helpers shared by the CholeskyQR2 kernels (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace cqr2 {

// Device-side outcome of a factorization, written by the CholInv base-case
// kernel on the first non-positive or non-finite pivot. `lock` makes the
// first reporter win; later breakdowns (which see NaNs) are ignored.
struct DevStatus {
  int status;  // 0 = ok, 2 = not SPD
  int pass;    // CholeskyQR pass (1 or 2)
  long long pivot;
  double value;
  int lock;
  int pad;
};

__device__ __forceinline__ void report_pivot(DevStatus* st, int pass, long long pivot, double v) {
  if (atomicCAS(&st->lock, 0, 1) == 0) {
    st->status = 2;
    st->pass = pass;
    st->pivot = pivot;
    st->value = v;
  }
}

// 8-byte asynchronous global->shared copy; src_bytes = 0 zero-fills the
// destination without reading `src` (which must still be a valid address).
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem, int src_bytes) {
  unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace cqr2
