// Small device helpers of CholeskyQR2 on column panels (the subpanel variant
// the paper's conclusion names as future work, Section V): the sum of the two
// block projections' coefficients, and the merge of a panel's breakdown into
// the whole factorization's status word.
#include <algorithm>

#include "kernels.h"

namespace cqr2 {
namespace {

// B(0:rows, 0:cols) += A(0:rows, 0:cols), column-major.
__global__ void k_add_block(const double* __restrict__ A, int64_t lda, double* __restrict__ B, int64_t ldb,
                            int64_t rows, int64_t cols) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t j = blockIdx.y;
  for (int64_t jj = j; jj < cols; jj += gridDim.y)
    if (i < rows) B[i + jj * ldb] += A[i + jj * lda];
}

// The first breakdown of a panel's CholeskyQR2 becomes the factorization's,
// its pivot index shifted to the whole matrix's columns.
__global__ void k_status_merge(DevStatus* __restrict__ outer, const DevStatus* __restrict__ inner,
                               long long col0) {
  if (inner->status != 0 && outer->status == 0) {
    outer->pass = inner->pass;
    outer->pivot = inner->pivot >= 0 ? inner->pivot + col0 : inner->pivot;
    outer->value = inner->value;
    outer->lock = 1;
    __threadfence();
    outer->status = inner->status;
  }
}

}  // namespace

cudaError_t add_block(const double* A, int64_t lda, double* B, int64_t ldb, int64_t rows, int64_t cols,
                      cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  dim3 grid((unsigned)ceil_div(rows, 256), (unsigned)std::min<int64_t>(cols, 65535));
  k_add_block<<<grid, 256, 0, s>>>(A, lda, B, ldb, rows, cols);
  count_launch();
  return cudaGetLastError();
}

cudaError_t status_merge(DevStatus* outer, const DevStatus* inner, int64_t col0, cudaStream_t s) {
  k_status_merge<<<1, 1, 0, s>>>(outer, inner, (long long)col0);
  count_launch();
  return cudaGetLastError();
}

}  // namespace cqr2
