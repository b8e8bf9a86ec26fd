// General FP64 GEMM C = alpha op(A) op(B) + beta C (the MM of Section II-A)
// with triangular-structure flags, used for the CholInv recursion
// (Algorithm 1), R = R2 R1, and the Q-forming multiply when n > 256.
//
// 64 x 64 x 16 tiles, 256 threads, 4 x 4 register micro-tiles, register
// double buffering of the next k-slice. GB300's FP64 pipe (about 2 FMA per
// clock per SM) is the bound, so the structure flags matter more than the
// load path: a tile's k range is clipped to the blocks that the triangles of
// op(A) and op(B) leave nonzero, output tiles outside the requested triangle
// are skipped, and elements inside the zero triangle are never read (they are
// masked to zero at load), so callers may leave garbage there.
#include <algorithm>

#include "kernels.h"

namespace cqr2 {
namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

template <bool TA, bool TB>
__global__ void __launch_bounds__(NT) k_gemm_f64(int64_t M, int64_t N, int64_t K, double alpha,
                                                 const double* __restrict__ A, int64_t lda,
                                                 const double* __restrict__ B, int64_t ldb, double beta,
                                                 double* __restrict__ C, int64_t ldc, unsigned flags, int ksplit,
                                                 double* __restrict__ P) {
  __shared__ double As[2][BK][BM + 1];
  __shared__ double Bs[2][BK][BN + 1];
  const int64_t i0 = (int64_t)blockIdx.x * BM, j0 = (int64_t)blockIdx.y * BN;
  const int t = threadIdx.x, tx = t & 15, ty = t >> 4;

  if ((flags & GEMM_C_LOWER) && j0 > i0 + BM - 1) return;
  if ((flags & GEMM_C_UPPER) && i0 > j0 + BN - 1) {
    if (ksplit > 1) return;  // the reduction writes the zeros
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int64_t gi = i0 + tx + 16 * r, gj = j0 + ty + 16 * c;
        if (gi < M && gj < N) C[gi + gj * ldc] = 0.0;
      }
    return;
  }
  int64_t kb = 0, ke = K;
  if (flags & GEMM_A_LOWER) ke = min(ke, i0 + BM);
  if (flags & GEMM_A_UPPER) kb = max(kb, i0);
  if (flags & GEMM_B_LOWER) kb = max(kb, j0);
  if (flags & GEMM_B_UPPER) ke = min(ke, j0 + BN);
  kb = (kb / BK) * BK;
  if (ksplit > 1) {  // this CTA's share of the k range, in whole k-slices
    const int64_t per = ((ke - kb + BK - 1) / BK + ksplit - 1) / ksplit * BK;
    const int64_t z0 = kb + (int64_t)blockIdx.z * per;
    ke = min(ke, z0 + per);
    kb = z0;
  }

  double acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = 0.0;

  double ra[4], rb[4];
  auto load = [&](int64_t k0) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = t + q * NT;
      int i, k;
      if (!TA) { i = e % BM; k = e / BM; } else { k = e % BK; i = e / BK; }
      const int64_t gi = i0 + i, gk = k0 + k;
      bool ok = gi < M && gk < K;
      if (flags & GEMM_A_LOWER) ok = ok && gk <= gi;
      if (flags & GEMM_A_UPPER) ok = ok && gk >= gi;
      ra[q] = ok ? (TA ? A[gk + gi * lda] : A[gi + gk * lda]) : 0.0;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = t + q * NT;
      int j, k;
      if (!TB) { k = e % BK; j = e / BK; } else { j = e % BN; k = e / BN; }
      const int64_t gj = j0 + j, gk = k0 + k;
      bool ok = gj < N && gk < K;
      if (flags & GEMM_B_LOWER) ok = ok && gk >= gj;
      if (flags & GEMM_B_UPPER) ok = ok && gk <= gj;
      rb[q] = ok ? (TB ? B[gj + gk * ldb] : B[gk + gj * ldb]) : 0.0;
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = t + q * NT;
      int i, k;
      if (!TA) { i = e % BM; k = e / BM; } else { k = e % BK; i = e / BK; }
      As[buf][k][i] = ra[q];
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = t + q * NT;
      int j, k;
      if (!TB) { k = e % BK; j = e / BK; } else { j = e % BN; k = e / BN; }
      Bs[buf][k][j] = rb[q];
    }
  };

  if (kb < ke) {
    load(kb);
    store(0);
    __syncthreads();
    int buf = 0;
    for (int64_t k0 = kb; k0 < ke; k0 += BK) {
      const bool more = k0 + BK < ke;
      if (more) load(k0 + BK);
#pragma unroll
      for (int k = 0; k < BK; ++k) {
        double a[4], b[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) a[r] = As[buf][k][tx + 16 * r];
#pragma unroll
        for (int c = 0; c < 4; ++c) b[c] = Bs[buf][k][ty + 16 * c];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
      }
      if (more) store(buf ^ 1);
      __syncthreads();
      buf ^= 1;
    }
  }

  if (ksplit > 1) {  // partial of split z: P[z][j][i] = alpha * sum over its k range
    double* Pz = P + (int64_t)blockIdx.z * M * N;
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int64_t gi = i0 + tx + 16 * r, gj = j0 + ty + 16 * c;
        if (gi < M && gj < N) Pz[gi + gj * M] = alpha * acc[r][c];
      }
    return;
  }
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int64_t gi = i0 + tx + 16 * r, gj = j0 + ty + 16 * c;
      if (gi >= M || gj >= N) continue;
      if ((flags & GEMM_C_LOWER) && gi < gj) continue;
      if ((flags & GEMM_C_UPPER) && gi > gj) {
        C[gi + gj * ldc] = 0.0;
        continue;
      }
      double v = alpha * acc[r][c];
      if (!(flags & GEMM_BETA0)) v = fma(beta, C[gi + gj * ldc], v);
      C[gi + gj * ldc] = v;
    }
}

// C = sum of the k-split partials in split order (deterministic), then beta C
// and the output-triangle rules as in the unsplit kernel.
__global__ void k_gemm_splitk_reduce(int64_t M, int64_t N, int ksplit, const double* __restrict__ P, double beta,
                                     double* __restrict__ C, int64_t ldc, unsigned flags) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= M * N) return;
  const int64_t gi = e % M, gj = e / M;
  if ((flags & GEMM_C_LOWER) && gi < gj) return;
  if ((flags & GEMM_C_UPPER) && gi > gj) {
    C[gi + gj * ldc] = 0.0;
    return;
  }
  double v = 0.0;
  for (int z = 0; z < ksplit; ++z) v += P[(int64_t)z * M * N + e];
  if (!(flags & GEMM_BETA0)) v = fma(beta, C[gi + gj * ldc], v);
  C[gi + gj * ldc] = v;
}

}  // namespace

cudaError_t gemm_f64(int64_t M, int64_t N, int64_t K, double alpha, const double* A, int64_t lda, const double* B,
                     int64_t ldb, double beta, double* C, int64_t ldc, unsigned flags, cudaStream_t s, double* ws,
                     size_t ws_doubles) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  const int64_t gx = ceil_div(M, BM), gy = ceil_div(N, BN);
  if (gy > 65535) return cudaErrorInvalidValue;
  // Small products fill few SMs, each doing about 2 FP64 FMA per clock: with
  // scratch, split k over up to 8 CTAs per tile (whole k-slices each).
  int ks = 1;
  if (ws && K >= 2 * BK) {
    int sms = 148, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = std::max<int64_t>(1, sms / (gx * gy));
    ks = (int)std::min<int64_t>({want, 8, K / BK});
    while (ks > 1 && (size_t)ks * M * N > ws_doubles) --ks;
  }
  dim3 grid((unsigned)gx, (unsigned)gy, (unsigned)ks);
  const bool ta = flags & GEMM_TA, tb = flags & GEMM_TB;
  if (!ta && !tb)
    k_gemm_f64<false, false><<<grid, NT, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, flags, ks, ws);
  else if (!ta && tb)
    k_gemm_f64<false, true><<<grid, NT, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, flags, ks, ws);
  else if (ta && !tb)
    k_gemm_f64<true, false><<<grid, NT, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, flags, ks, ws);
  else
    k_gemm_f64<true, true><<<grid, NT, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, flags, ks, ws);
  count_launch();
  if (ks > 1) {
    const int64_t total = M * N;
    k_gemm_splitk_reduce<<<(unsigned)ceil_div(total, 256), 256, 0, s>>>(M, N, ks, ws, beta, C, ldc, flags);
    count_launch();
  }
  return cudaGetLastError();
}

// R = op(A) B of two upper-triangular n x n factors (the R2 R1 of Algorithm
// CQR2), n <= TRMM_SMALL_MAX, in one launch: CTA j forms column j; four
// threads share each element, thread q summing op(A)(i, k) B(k, j) over
// k = i + q, i + q + 4, ... <= j in order, and the four partial sums are
// added in a fixed order through two shuffles (a chain of at most 32 FMAs
// where one thread per element would hold 128). C below the diagonal is
// written as 0. op(A)(i, k) = A(k, i) when a_trans (A holds the lower
// transpose, as the Cholesky factor L2 does), else A(i, k). The general GEMM
// needs a split-k launch and its reduction for this 2 n^3 / 6 flop product.
constexpr int TRMM_PARTS = 4;
__global__ void __launch_bounds__(TRMM_PARTS * TRMM_SMALL_MAX)
    k_trmm_upper_small(int n, const double* __restrict__ A, int64_t lda, bool a_trans, const double* __restrict__ B,
                       int64_t ldb, double* __restrict__ C, int64_t ldc) {
  __shared__ double bj[TRMM_SMALL_MAX];
  const int j = blockIdx.x, t = threadIdx.x, i = t / TRMM_PARTS, q = t % TRMM_PARTS;
  for (int k = t; k <= j; k += blockDim.x) bj[k] = B[k + (int64_t)j * ldb];
  __syncthreads();
  double acc = 0.0;
  if (i <= j) {  // i < n since j < n
    if (a_trans) {
      const double* a = A + (int64_t)i * lda;  // column i of the lower factor
#pragma unroll 4
      for (int k = i + q; k <= j; k += TRMM_PARTS) acc = fma(a[k], bj[k], acc);
    } else {
#pragma unroll 4
      for (int k = i + q; k <= j; k += TRMM_PARTS) acc = fma(A[i + (int64_t)k * lda], bj[k], acc);
    }
  }
  // (p0 + p1) + (p2 + p3): the four threads of an element are adjacent lanes
  acc += __shfl_xor_sync(0xffffffffu, acc, 1);
  acc += __shfl_xor_sync(0xffffffffu, acc, 2);
  if (q == 0 && i < n) C[i + (int64_t)j * ldc] = acc;
}

cudaError_t trmm_upper_small(int n, const double* A, int64_t lda, bool a_trans, const double* B, int64_t ldb,
                             double* C, int64_t ldc, cudaStream_t s) {
  if (n < 1 || n > TRMM_SMALL_MAX) return cudaErrorInvalidValue;
  const int threads = (TRMM_PARTS * n + 31) / 32 * 32;
  k_trmm_upper_small<<<n, threads, 0, s>>>(n, A, lda, a_trans, B, ldb, C, ldc);
  count_launch();
  return cudaGetLastError();
}

}  // namespace cqr2
