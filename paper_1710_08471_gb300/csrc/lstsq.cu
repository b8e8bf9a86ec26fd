// Least-squares tail x = R^-1 (Q^T b). The paper uses QR for least squares
// (Section I) but gives no solve; this library forms c = Q^T b with split-m
// partial sums (summed in a fixed order) and solves R x = c by back
// substitution in one CTA.
#include <algorithm>

#include "kernels.h"

namespace cqr2 {
namespace {

constexpr int GT = 256;

__global__ void __launch_bounds__(GT) k_gemv_t_partial(const double* __restrict__ Q, int64_t ldq, int64_t m, int n,
                                                       const double* __restrict__ b, int64_t rows_per,
                                                       double* __restrict__ partial) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t r0 = (int64_t)blockIdx.x * rows_per;
  const int64_t r1 = min(m, r0 + rows_per);
  for (int j = warp; j < n; j += GT / 32) {
    const double* q = Q + (int64_t)j * ldq;
    double s = 0.0;
    for (int64_t r = r0 + lane; r < r1; r += 32) s = fma(q[r], b[r], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) partial[(int64_t)blockIdx.x * n + j] = s;
  }
}

__global__ void __launch_bounds__(1024) k_lstsq_solve(const double* __restrict__ partial, int64_t nsplit, int n,
                                                      const double* __restrict__ R, int64_t ldr,
                                                      double* __restrict__ x) {
  extern __shared__ double c[];
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    double s = 0.0;
    for (int64_t b = 0; b < nsplit; ++b) s += partial[b * n + j];
    c[j] = s;
  }
  __syncthreads();
  for (int j = n - 1; j >= 0; --j) {
    if (threadIdx.x == 0) c[j] = c[j] / R[j + (int64_t)j * ldr];
    __syncthreads();
    const double xj = c[j];
    for (int i = threadIdx.x; i < j; i += blockDim.x) c[i] = fma(-R[i + (int64_t)j * ldr], xj, c[i]);
    __syncthreads();
  }
  for (int j = threadIdx.x; j < n; j += blockDim.x) x[j] = c[j];
}

}  // namespace

int64_t gemv_splits(int64_t m, int n) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return std::max<int64_t>(1, std::min<int64_t>(ceil_div(m, 1024), (int64_t)2 * sms));
}

cudaError_t gemv_t_partials(const double* Q, int64_t ldq, int64_t m, int n, const double* b, int64_t nsplit,
                            double* partial, cudaStream_t s) {
  const int64_t rows_per = ceil_div(m, nsplit);
  k_gemv_t_partial<<<(unsigned)nsplit, GT, 0, s>>>(Q, ldq, m, n, b, rows_per, partial);
  count_launch();
  return cudaGetLastError();
}

cudaError_t lstsq_solve(const double* partial, int64_t nsplit, int n, const double* R, int64_t ldr, double* x,
                        cudaStream_t s) {
  const size_t sm = (size_t)n * sizeof(double);
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_lstsq_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  k_lstsq_solve<<<1, 1024, sm, s>>>(partial, nsplit, n, R, ldr, x);
  count_launch();
  return cudaGetLastError();
}

}  // namespace cqr2
