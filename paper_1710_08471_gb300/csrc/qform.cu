// Q-forming multiply Q = A R^-1 (Algorithm CQR step 3) for n <= 256, and its
// fusion with the next pass's Gram (Algorithm CQR2 steps 1-2: the Q1 panel
// that pass 1 produces is accumulated into pass 2's Gram while it is still on
// chip, so Q1 is not read back from memory for the Gram).
//
// R^-1 is upper triangular, so column j of Q needs only k <= j. One lane
// owns one row of a 32-row panel; a warp owns a group of w = n/16 adjacent
// columns, so every lane of a warp runs the same k range and no FP64 lane is
// spent on the zero triangle. Warp v takes column groups v and 15 - v, which
// gives all eight warps the same amount of work. R^-1 is pre-packed per group
// ([group][k][c], contiguous in c) and read through the read-only path as a
// warp-wide broadcast; the A panel is staged in shared memory as [k][row],
// which makes both the global loads and the shared loads conflict-free.
#include <algorithm>

#include "kernels.h"

namespace cqr2 {
namespace {

constexpr int PANEL = 32;   // rows per panel (one per lane)
constexpr int NGROUP = 16;  // column groups
constexpr int QT = 256;     // threads per CTA

__global__ void k_pack_rinv(const double* __restrict__ X, int64_t ldx, int n, int w, bool from_lower,
                            double* __restrict__ Rp) {
  const int64_t total = (int64_t)NGROUP * n * w;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e % w);
    const int k = (int)((e / w) % n);
    const int g = (int)(e / ((int64_t)w * n));
    const int col = g * w + c;
    double v = 0.0;
    if (col < n && k <= col) v = from_lower ? X[col + (int64_t)k * ldx] : X[k + (int64_t)col * ldx];
    Rp[e] = v;
  }
}

template <int W>
__device__ __forceinline__ void load_w(const double* __restrict__ p, double (&r)[W]) {
  if constexpr (W >= 2) {
#pragma unroll
    for (int c = 0; c < W; c += 2) {
      const double2 v = __ldg(reinterpret_cast<const double2*>(p + c));
      r[c] = v.x;
      r[c + 1] = v.y;
    }
  } else {
    r[0] = __ldg(p);
  }
}

// Computes the W columns of group g for the lane's row of the staged panel.
template <int W>
__device__ __forceinline__ void qform_group(const double* As, int lane, int n, int g,
                                            const double* __restrict__ Rp, double (&acc)[W]) {
  const int c0 = g * W;
  const double* rp = Rp + (int64_t)g * n * W;
#pragma unroll
  for (int c = 0; c < W; ++c) acc[c] = 0.0;
#pragma unroll 4
  for (int k = 0; k < c0; ++k) {
    const double a = As[k * PANEL + lane];
    double r[W];
    load_w<W>(rp + (int64_t)k * W, r);
#pragma unroll
    for (int c = 0; c < W; ++c) acc[c] = fma(a, r[c], acc[c]);
  }
#pragma unroll
  for (int kk = 0; kk < W; ++kk) {
    const int k = c0 + kk;
    if (k < n) {
      const double a = As[k * PANEL + lane];
      double r[W];
      load_w<W>(rp + (int64_t)k * W, r);
#pragma unroll
      for (int c = kk; c < W; ++c) acc[c] = fma(a, r[c], acc[c]);
    }
  }
}

__device__ __forceinline__ void stage_panel(const double* A, int64_t lda, int64_t m, int n, int64_t row0,
                                            double* As) {
  for (int e = threadIdx.x; e < n * PANEL; e += QT) {
    const int r = e & (PANEL - 1), k = e >> 5;
    const int64_t row = row0 + r;
    As[e] = row < m ? A[row + (int64_t)k * lda] : 0.0;
  }
}

// A is deliberately not __restrict__: Q may alias A.
template <int W>
__global__ void __launch_bounds__(QT) k_qform_small(const double* A, int64_t lda, int64_t m, int n,
                                                    const double* __restrict__ Rp, double* Q, int64_t ldq,
                                                    int64_t npanels) {
  extern __shared__ double As[];  // [n][PANEL]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t panel = blockIdx.x; panel < npanels; panel += gridDim.x) {
    const int64_t row0 = panel * PANEL;
    stage_panel(A, lda, m, n, row0, As);
    __syncthreads();
    const int64_t row = row0 + lane;
#pragma unroll 1
    for (int half = 0; half < 2; ++half) {
      const int g = half ? (NGROUP - 1 - warp) : warp;
      if (g * W >= n) continue;
      double acc[W];
      qform_group<W>(As, lane, n, g, Rp, acc);
      if (row < m) {
#pragma unroll
        for (int c = 0; c < W; ++c)
          if (g * W + c < n) Q[row + (int64_t)(g * W + c) * ldq] = acc[c];
      }
    }
    __syncthreads();
  }
}

// Fused Q-form + Gram for n <= T (one diagonal Gram tile of width T). The
// Gram part is the flattened-upper-pair scheme of the Gram kernel, reading
// the freshly formed Q panel from shared memory ([row][col], padded).
template <int W, int T>
__global__ void __launch_bounds__(QT) k_qform_gram_small(const double* A, int64_t lda, int64_t m, int n,
                                                         const double* __restrict__ Rp, double* Q, int64_t ldq,
                                                         int64_t rows_per_split, int ntiles_total,
                                                         double* __restrict__ partial) {
  constexpr int LDQ = T + 1;
  constexpr int P = T * (T + 1) / 2;
  constexpr int S = (P + QT - 1) / QT;
  extern __shared__ double smem[];
  double* As = smem;                       // [n][PANEL]
  double* Qs = smem + (size_t)T * PANEL;   // [PANEL][LDQ]
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;

  int oi[S], oj[S];
  bool last_ok = true;
  {
    int i = 0, start = 0;
#pragma unroll
    for (int s = 0; s < S; ++s) {
      int p = t + s * QT;
      if (p >= P) {
        p = P - 1;
        last_ok = false;
      }
      while (p >= start + (T - i)) {
        start += T - i;
        ++i;
      }
      oi[s] = i;
      oj[s] = i + (p - start);
    }
  }
  double gacc[S];
#pragma unroll
  for (int s = 0; s < S; ++s) gacc[s] = 0.0;
  // Columns n..T-1 of the staged Q panel stay zero.
  for (int e = t; e < PANEL * LDQ; e += QT) Qs[e] = 0.0;
  __syncthreads();

  const int64_t r_begin = (int64_t)blockIdx.x * rows_per_split;
  const int64_t r_end = min(m, r_begin + rows_per_split);
  for (int64_t row0 = r_begin; row0 < r_end; row0 += PANEL) {
    stage_panel(A, lda, r_end, n, row0, As);
    __syncthreads();
    const int64_t row = row0 + lane;
#pragma unroll 1
    for (int half = 0; half < 2; ++half) {
      const int g = half ? (NGROUP - 1 - warp) : warp;
      if (g * W >= n) continue;
      double acc[W];
      qform_group<W>(As, lane, n, g, Rp, acc);
#pragma unroll
      for (int c = 0; c < W; ++c) {
        const int col = g * W + c;
        if (col < n) {
          Qs[lane * LDQ + col] = acc[c];
          if (row < r_end) Q[row + (int64_t)col * ldq] = acc[c];
        }
      }
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < PANEL; ++kk) {
      const double* qrow = Qs + kk * LDQ;
#pragma unroll
      for (int s = 0; s < S; ++s) gacc[s] = fma(qrow[oi[s]], qrow[oj[s]], gacc[s]);
    }
    __syncthreads();
  }
  double* out = partial + (int64_t)blockIdx.x * ntiles_total * (int64_t)(T * T);
#pragma unroll
  for (int s = 0; s < S; ++s)
    if (s < S - 1 || last_ok) out[oi[s] + oj[s] * T] = gacc[s];
}

int sm_count() {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

template <int W>
cudaError_t launch_qform(const double* A, int64_t lda, int64_t m, int n, const double* Rp, double* Q, int64_t ldq,
                         cudaStream_t s) {
  const size_t sm = (size_t)n * PANEL * sizeof(double);
  auto kern = k_qform_small<W>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  const int64_t npanels = ceil_div(m, PANEL);
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, QT, sm);
  const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(npanels, (int64_t)sm_count() * std::max(1, per_sm)));
  kern<<<(unsigned)grid, QT, sm, s>>>(A, lda, m, n, Rp, Q, ldq, npanels);
  count_launch();
  return cudaGetLastError();
}

template <int W, int T>
cudaError_t launch_fused(const double* A, int64_t lda, int64_t m, int n, const double* Rp, double* Q, int64_t ldq,
                         const GramGeom& g, double* partial, cudaStream_t s) {
  const size_t sm = ((size_t)T * PANEL + (size_t)PANEL * (T + 1)) * sizeof(double);
  auto kern = k_qform_gram_small<W, T>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)g.nsplit, QT, sm, s>>>(A, lda, m, n, Rp, Q, ldq, g.rows_per_split, g.ntiles_total, partial);
  count_launch();
  return cudaGetLastError();
}

}  // namespace

int qform_group_width(int n) {
  if (n > 256) return 0;
  const int w = (int)ceil_div(n, NGROUP);
  int p = 1;
  while (p < w) p *= 2;
  return p;
}

size_t rpack_doubles(int n) {
  const int w = qform_group_width(n);
  return (size_t)NGROUP * n * (w ? w : 0);
}

static cudaError_t pack(const double* X, int64_t ldx, int n, bool lower, double* Rp, cudaStream_t s) {
  const int w = qform_group_width(n);
  if (!w) return cudaErrorInvalidValue;
  const int64_t total = (int64_t)NGROUP * n * w;
  const int grid = (int)std::min<int64_t>(ceil_div(total, 256), 4096);
  k_pack_rinv<<<grid, 256, 0, s>>>(X, ldx, n, w, lower, Rp);
  count_launch();
  return cudaGetLastError();
}

cudaError_t pack_rinv_from_lower(const double* Y, int64_t ldy, int n, double* Rp, cudaStream_t s) {
  return pack(Y, ldy, n, true, Rp, s);
}

cudaError_t pack_rinv_from_upper(const double* Rinv, int64_t ld, int n, double* Rp, cudaStream_t s) {
  return pack(Rinv, ld, n, false, Rp, s);
}

cudaError_t qform_small(const double* A, int64_t lda, int64_t m, int n, const double* Rp, double* Q, int64_t ldq,
                        cudaStream_t s) {
  switch (qform_group_width(n)) {
    case 1: return launch_qform<1>(A, lda, m, n, Rp, Q, ldq, s);
    case 2: return launch_qform<2>(A, lda, m, n, Rp, Q, ldq, s);
    case 4: return launch_qform<4>(A, lda, m, n, Rp, Q, ldq, s);
    case 8: return launch_qform<8>(A, lda, m, n, Rp, Q, ldq, s);
    case 16: return launch_qform<16>(A, lda, m, n, Rp, Q, ldq, s);
    default: return cudaErrorInvalidValue;
  }
}

bool qform_gram_fusable(int n) { return n >= 1 && n <= 128; }

cudaError_t qform_gram_small(const double* A, int64_t lda, int64_t m, int n, const double* Rp, double* Q,
                             int64_t ldq, const GramGeom& g, double* partial, cudaStream_t s) {
  if (!qform_gram_fusable(n) || g.ntile != 1 || g.T < n) return cudaErrorInvalidValue;
  const int w = qform_group_width(n);
  switch (g.T) {
    case 32:
      if (w == 1) return launch_fused<1, 32>(A, lda, m, n, Rp, Q, ldq, g, partial, s);
      return launch_fused<2, 32>(A, lda, m, n, Rp, Q, ldq, g, partial, s);
    case 64:
      return launch_fused<4, 64>(A, lda, m, n, Rp, Q, ldq, g, partial, s);
    case 128:
      return launch_fused<8, 128>(A, lda, m, n, Rp, Q, ldq, g, partial, s);
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace cqr2
