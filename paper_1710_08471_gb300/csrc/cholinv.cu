// CholInv (Algorithm 1, Section II-D): [L, Y] = CholInv(W) with W = L L^T and
// Y = L^-1, by the paper's halving recursion
//     [L11, Y11] = CholInv(W11)
//     L21 = W21 Y11^T
//     [L22, Y22] = CholInv(W22 - L21 L21^T)
//     Y21 = -Y22 (L21 Y11)            (association of Algorithm CFR3D)
// run as FP64 GEMM launches on one stream. The recursion stops at a base case
// of at most 64 (the paper's base case is n = 1; CFR3D stops at n_o and
// factors the block redundantly, which is what the one-CTA base kernel does).
// The split point is a multiple of 64 near n/2 instead of floor(n/2): the
// result is the same factorization, rounded in a different order.
//
// The base case holds the block in shared memory, runs a right-looking
// Cholesky with the right-looking triangular inverse interleaved, and reports the first
// non-positive or non-finite pivot in the device status word (it keeps going
// with NaNs instead of trapping, so the context stays usable).
#include <algorithm>

#include "fp64_rsqrt.cuh"
#include "kernels.h"

namespace cqr2 {
namespace {

constexpr int NB = CHOLINV_BASE;
constexpr int LD = NB + 1;

__global__ void __launch_bounds__(256) k_cholinv_base(const double* __restrict__ Wk, int64_t ldk, int nb,
                                                      double* __restrict__ L, int64_t ldl, double* __restrict__ Y,
                                                      int64_t ldy, DevStatus* st, int pass, long long off) {
  extern __shared__ double smem[];
  double* S = smem;            // S(i, j) = S[j * LD + i], lower part
  double* T = smem + NB * LD;  // right-looking inverse workspace / result
  const int t = threadIdx.x;
  for (int e = t; e < nb * nb; e += 256) {
    const int i = e % nb, j = e / nb;
    S[j * LD + i] = (i >= j) ? Wk[i + (int64_t)j * ldk] : 0.0;
    T[j * LD + i] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  // Right-looking Cholesky with the right-looking inverse interleaved, and a
  // look-ahead of one pivot. GB300 issues an FP64 warp instruction at a small
  // fraction of the FP32 rate, and the pivots are a serial chain, so in step k
  // (column k of L and row k of Y = L^-1 already final)
  //   - warp 0 applies step k to column k+1 of L and row k+1 of Y, forms pivot
  //     k+1 (its square root and reciprocal from a short Newton sequence) and
  //     scales that column and row by 1/l_(k+1,k+1);
  //   - the other warps apply step k to the rest of the trailing matrix and to
  //     the rows of Y below k+1, numbered consecutively (the triangle's part
  //     through a table of its elements, column by column) so that nearly
  //     every FP64 warp instruction updates 32 of them -- the FP64 pipe
  //     charges an instruction in full whatever its active lanes;
  // with one block barrier per step. Every element sees the same operations in
  // the same order as the plain factorization followed by the plain inverse.
  __shared__ double rdiag[NB];
  auto pivot = [&](int k) {
    const double d = S[k * LD + k];
    if (!(d > 0.0) || !isfinite(d)) report_pivot(st, pass, off + k, d);
    double l, rl;
    chol_rsqrt(d, &rl, &l);
    S[k * LD + k] = l;
    rdiag[k] = rl;
  };
  const int warp = t >> 5, lane = t & 31;
  if (warp == 0) {
    if (lane == 0) pivot(0);
    __syncwarp();
    const double rl = rdiag[0];
    for (int i = 1 + lane; i < nb; i += 32) S[i] *= rl;
    if (lane == 0) T[0] *= rl;
  }
  __syncthreads();
  const int u = t - 32;  // warps 1..7 share the packed trailing elements
  // the lower triangle column by column, (j << 8) | i: the trailing part of
  // step k is the suffix from column k+2 on
  __shared__ unsigned short tab[NB * (NB + 1) / 2];
  if (t < nb) {
    const int st = t * nb - t * (t - 1) / 2;
    for (int i = t; i < nb; ++i) tab[st + i - t] = (unsigned short)((t << 8) | i);
  }
  __syncthreads();
  const int ntri = nb * (nb + 1) / 2;
  for (int k = 0; k < nb; ++k) {
    if (warp == 0) {
      if (k + 1 < nb) {
        const double lk1 = S[k * LD + k + 1];
        for (int i = k + 1 + lane; i < nb; i += 32)
          S[(k + 1) * LD + i] = fma(-S[k * LD + i], lk1, S[(k + 1) * LD + i]);
        for (int j = lane; j <= k; j += 32) T[j * LD + k + 1] = fma(-lk1, T[j * LD + k], T[j * LD + k + 1]);
        __syncwarp();
        if (lane == 0) pivot(k + 1);
        __syncwarp();
        const double rl = rdiag[k + 1];
        for (int i = k + 2 + lane; i < nb; i += 32) S[(k + 1) * LD + i] *= rl;
        for (int j = lane; j <= k + 1; j += 32) T[j * LD + k + 1] *= rl;
      }
    } else {
      const int s0 = (k + 2) * nb - (k + 2) * (k + 1) / 2;  // start of column k+2
      const int cS = k + 2 < nb ? ntri - s0 : 0;
      const int h = nb - k - 2;
      const int cT = h > 0 ? (k + 1) * h : 0;
      const float rh = h > 0 ? 1.0f / (float)h : 0.0f;
      for (int e = u; e < cS + cT; e += 224) {
        if (e < cS) {
          const int ji = tab[s0 + e], j = ji >> 8, i = ji & 255;
          S[j * LD + i] = fma(-S[k * LD + i], S[k * LD + j], S[j * LD + i]);
        } else {
          const int e2 = e - cS, j = __float2int_rz(((float)e2 + 0.5f) * rh), i = k + 2 + (e2 - j * h);
          T[j * LD + i] = fma(-S[k * LD + i], T[j * LD + k], T[j * LD + i]);
        }
      }
    }
    __syncthreads();
  }
  for (int e = t; e < nb * nb; e += 256) {
    const int i = e % nb, j = e / nb;
    if (i >= j) {
      L[i + (int64_t)j * ldl] = S[j * LD + i];
      Y[i + (int64_t)j * ldy] = T[j * LD + i];
    }
  }
}

// The 64 x 64 base case (every leaf of a recursion on n = 64 2^p). FP64 on
// GB300 issues under three rules that decide this design: a dependent FP64
// operation takes 64 clocks; the SM starts at most one FP64 warp instruction
// per 16 clocks; and an instruction whose lanes are all predicated off still
// takes its slot. The runtime kernel above spends about 25 instructions of
// index arithmetic and shared-memory traffic on each trailing update, as a
// dependency chain per warp. Here:
//  - warp 0 applies step k to column k+1 of L (from the diagonal down) and to
//    row k+1 of Y = L^-1 (left of the diagonal), 64 elements in two warp
//    instructions, forms the pivot from lane 0's element and scales both; the
//    diagonal of L is lane 0's own product d / sqrt(d);
//  - five bulk warps keep the trailing part of L in registers: element
//    (i, j), 2 <= j <= i < 64, at position e' = u + 160 s of the column-major
//    packed order read backwards, so that the elements still active at step
//    k (j >= k + 2) fill the first slots; a fall-through switch on the count
//    of active slots issues exactly those; each step they write out column
//    k+2, which warp 0 takes over next;
//  - the bulk warps update Y's trailing block (rows k+2.., columns 0..k) in
//    shared memory, numbered column by column (division by a multiply-shift
//    from a table), two elements per pass with both loads ahead of the FMAs.
// The step loop stays a loop: compiled step by step the kernel ran 8% faster
// while its code was hot but was 16 times larger (410 KB) and, after large
// kernels had refilled L2, took 1.6 times as long.
// Every element sees the same operations in the same order as in the runtime
// kernel, so the two agree bit for bit.
constexpr int B64_BW = 5;                       // bulk warps
constexpr int B64_P = 32 * B64_BW;              // bulk threads
constexpr int B64_NL = (NB - 2) * (NB - 1) / 2;  // trailing elements of L
constexpr int B64_NS = (B64_NL + B64_P - 1) / B64_P;  // register slots per bulk thread
static_assert(B64_NS <= 16, "the slot switch has 16 cases");

// Writes the whole 64 x 64 blocks of L and Y (zeros above the diagonal) and,
// when given, R = L^T (zeros below) and the Q-form's packed R^-1 (column
// groups of rpw, see k_pack_rinv). W is read completely before anything is
// written, so it may share storage with an output.
__global__ void __launch_bounds__(32 * (B64_BW + 1), 1)
    k_cholinv_base64(const double* Wk, int64_t ldk, double* L, int64_t ldl, double* Y, int64_t ldy, double* Rt,
                     int64_t ldrt, double* Rp, int rpw, DevStatus* st, int pass, long long off) {
  constexpr int NT = 32 * (B64_BW + 1), P = B64_P, NS = B64_NS;
  extern __shared__ double smem[];
  double* S = smem;            // S(i, j) = S[j * LD + i], lower part
  double* T = smem + NB * LD;  // Y
  __shared__ unsigned mdiv[NB];  // floor(e / h) = (e * mdiv[h]) >> 16 for e < 1024, h < 64
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  for (int e = t; e < NB * NB; e += NT) {
    const int i = e % NB, j = e / NB;
    S[j * LD + i] = (i >= j) ? Wk[i + (int64_t)j * ldk] : 0.0;
    T[j * LD + i] = (i == j) ? 1.0 : 0.0;
  }
  if (t < NB) mdiv[t] = t > 0 ? (1u << 16) / (unsigned)t + 1 : 0;
  __syncthreads();
  double z[NS];
  int row[NS], col[NS], cmax[NS];  // cmax: the slot's largest column (lane 0's)
  const int u = t - 32;
  if (warp == 0) {
    double rl = 0.0, l = 0.0;
    if (lane == 0) {
      const double d = S[0];
      if (!(d > 0.0) || !isfinite(d)) report_pivot(st, pass, off, d);
      chol_rsqrt(d, &rl, &l);
      S[0] = l;
      T[0] = rl;
    }
    rl = __shfl_sync(0xffffffffu, rl, 0);
    for (int i = 1 + lane; i < NB; i += 32) S[i] *= rl;
  } else {
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      const int ep = u + P * s;
      int i = 0, j = 0;
      if (ep < B64_NL) {
        int p = B64_NL - 1 - ep;  // position in the forward column-major order of columns 2..
        j = 2;
        while (p >= NB - j) {
          p -= NB - j;
          ++j;
        }
        i = j + p;
      }
      row[s] = i;
      col[s] = j;
      z[s] = (j >= 2) ? S[j * LD + i] : 0.0;
      cmax[s] = __shfl_sync(0xffffffffu, j, 0);
    }
  }
  __syncthreads();
  for (int k = 0; k < NB - 1; ++k) {
    const int k1 = k + 1, kb = k * LD;
    if (warp == 0) {
      const int ns = NB - k1;
      const double lk1 = S[kb + k1];
      int od[2];
      double v[2];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int e = lane + 32 * q;
        int ox = 0;
        od[q] = -1;
        if (e < ns) {
          od[q] = k1 * LD + k1 + e;
          ox = kb + k1 + e;
        } else if (e < NB) {
          od[q] = NB * LD + (e - ns) * LD + k1;
          ox = NB * LD + (e - ns) * LD + k;
        }
        v[q] = od[q] >= 0 ? fma(-smem[ox], lk1, smem[od[q]]) : 0.0;
      }
      double rl = 0.0, l = 0.0;
      bool fast = true;
      if (lane == 0) {
        const double d = v[0];
        // d <= 0, NaN or infinite, tested on the bits (no FP64 compare on the chain)
        const unsigned long long db = (unsigned long long)__double_as_longlong(d);
        if ((db >> 63) != 0 || db == 0 || ((db >> 52) & 0x7FF) == 0x7FF) report_pivot(st, pass, off + k1, d);
        fast = chol_rsqrt_r(d, &rl, &l);
        T[k1 * LD + k1] = rl;  // Y's diagonal: 1 / l
      }
      rl = __shfl_sync(0xffffffffu, rl, 0);
#pragma unroll
      for (int q = 0; q < 2; ++q)
        if (od[q] >= 0) smem[od[q]] = v[q] * rl;  // lane 0: the diagonal d / sqrt(d)
      if (!fast) S[k1 * LD + k1] = l;
    } else {
      int na = NS;  // slots with an active lane: a prefix
#pragma unroll
      for (int s = NS - 1; s >= 0; --s)
        if (cmax[s] < k + 2) na = s;
#define CQ2_SLOT(s)                                                   \
  case (s) + 1:                                                       \
    if constexpr ((s) < NS) {                                         \
      const double r = fma(-S[kb + row[s]], S[kb + col[s]], z[s]);    \
      z[s] = col[s] >= k + 2 ? r : z[s];                              \
    }
      switch (na) {
        CQ2_SLOT(15) CQ2_SLOT(14) CQ2_SLOT(13) CQ2_SLOT(12) CQ2_SLOT(11) CQ2_SLOT(10) CQ2_SLOT(9) CQ2_SLOT(8)
        CQ2_SLOT(7) CQ2_SLOT(6) CQ2_SLOT(5) CQ2_SLOT(4) CQ2_SLOT(3) CQ2_SLOT(2) CQ2_SLOT(1) CQ2_SLOT(0)
        default:
          break;
      }
#undef CQ2_SLOT
      // Y rows k+2.., columns 0..k, numbered column by column, two per pass
      const int h = NB - 2 - k, cY = h > 0 ? h * k1 : 0;
      const unsigned m = mdiv[h > 0 ? h : 1];
      for (int e0 = u; e0 < cY; e0 += 2 * P) {
        const int e1 = e0 + P;
        const bool in1 = e1 < cY;
        const int j0 = (int)(((unsigned)e0 * m) >> 16), i0 = k + 2 + (e0 - j0 * h);
        const int j1 = (int)(((unsigned)e1 * m) >> 16), i1 = k + 2 + (e1 - j1 * h);
        const double x0 = S[kb + i0], y0 = T[j0 * LD + k], z0 = T[j0 * LD + i0];
        double x1 = 0.0, y1 = 0.0, z1 = 0.0;
        if (in1) {
          x1 = S[kb + i1];
          y1 = T[j1 * LD + k];
          z1 = T[j1 * LD + i1];
        }
        const double r0 = fma(-x0, y0, z0);
        const double r1 = fma(-x1, y1, z1);
        T[j0 * LD + i0] = r0;
        if (in1) T[j1 * LD + i1] = r1;
      }
#pragma unroll
      for (int s = 0; s < NS; ++s)
        if (col[s] == k + 2) S[(k + 2) * LD + row[s]] = z[s];
    }
    __syncthreads();
  }
  for (int e = t; e < NB * NB; e += NT) {
    const int i = e % NB, j = e / NB;
    L[i + (int64_t)j * ldl] = i >= j ? S[j * LD + i] : 0.0;
    Y[i + (int64_t)j * ldy] = i >= j ? T[j * LD + i] : 0.0;
    if (Rt != nullptr) Rt[i + (int64_t)j * ldrt] = i <= j ? S[i * LD + j] : 0.0;  // R(i, j) = L(j, i)
  }
  if (Rp != nullptr) {
    // element e of the packing: group g, row k, column c within the group
    for (int e = t; e < RP_GROUPS * NB * rpw; e += NT) {
      const int c = e % rpw, k = (e / rpw) % NB, col = (e / (rpw * NB)) * rpw + c;
      Rp[e] = (col < NB && k <= col) ? T[k * LD + col] : 0.0;  // R^-1(k, col) = Y(col, k)
    }
  }
}

__global__ void k_transpose_lower(const double* __restrict__ L, int64_t ldl, int n, double* __restrict__ R,
                                  int64_t ldr) {
  __shared__ double tile[32][33];
  const int bi = blockIdx.x * 32, bj = blockIdx.y * 32;  // R block (rows bi.., cols bj..)
  // read L block (rows bj.., cols bi..) coalesced along its rows
  for (int y = threadIdx.y; y < 32; y += 8) {
    const int li = bj + threadIdx.x, lj = bi + y;
    tile[y][threadIdx.x] = (li < n && lj < n) ? L[li + (int64_t)lj * ldl] : 0.0;
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += 8) {
    const int ri = bi + threadIdx.x, rj = bj + y;
    if (ri < n && rj < n) R[ri + (int64_t)rj * ldr] = (ri <= rj) ? tile[threadIdx.x][y] : 0.0;
  }
}

__global__ void k_copy_upper(const double* __restrict__ X, int64_t ldx, int n, double* __restrict__ R, int64_t ldr) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i < n) R[i + (int64_t)j * ldr] = (i <= j) ? X[i + (int64_t)j * ldx] : 0.0;
}

constexpr size_t BASE_SMEM = 2 * NB * LD * sizeof(double);

cudaError_t set_base_smem() {
  cudaError_t e = cudaFuncSetAttribute(k_cholinv_base, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BASE_SMEM);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_cholinv_base64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BASE_SMEM);
}

cudaError_t rec(int n, double* Wk, int64_t ldk, double* L, int64_t ldl, double* Y, int64_t ldy, double* U,
                int64_t ldu, DevStatus* st, int pass, long long off, cudaStream_t s, double* ws, size_t wsn) {
  if (n == NB) {
    k_cholinv_base64<<<1, 32 * (B64_BW + 1), BASE_SMEM, s>>>(Wk, ldk, L, ldl, Y, ldy, nullptr, 0, nullptr, 0, st,
                                                                 pass, off);
    count_launch();
    return cudaGetLastError();
  }
  if (n < NB) {
    k_cholinv_base<<<1, 256, BASE_SMEM, s>>>(Wk, ldk, n, L, ldl, Y, ldy, st, pass, off);
    count_launch();
    return cudaGetLastError();
  }
  const int n1 = NB * (int)ceil_div(n, 2 * NB);
  const int n2 = n - n1;
  cudaError_t e;
  // [L11, Y11] = CholInv(W11)
  if ((e = rec(n1, Wk, ldk, L, ldl, Y, ldy, U, ldu, st, pass, off, s, ws, wsn)) != cudaSuccess) return e;
  // L21 = W21 Y11^T
  if ((e = gemm_f64(n2, n1, n1, 1.0, Wk + n1, ldk, Y, ldy, 0.0, L + n1, ldl, GEMM_TB | GEMM_B_UPPER | GEMM_BETA0,
                    s, ws, wsn)) != cudaSuccess)
    return e;
  // W22 <- W22 - L21 L21^T (lower triangle)
  double* W22 = Wk + n1 + (int64_t)n1 * ldk;
  if ((e = gemm_f64(n2, n2, n1, -1.0, L + n1, ldl, L + n1, ldl, 1.0, W22, ldk, GEMM_TB | GEMM_C_LOWER, s, ws,
                    wsn)) != cudaSuccess)
    return e;
  // [L22, Y22] = CholInv(W22 - L21 L21^T)
  double* L22 = L + n1 + (int64_t)n1 * ldl;
  double* Y22 = Y + n1 + (int64_t)n1 * ldy;
  if ((e = rec(n2, W22, ldk, L22, ldl, Y22, ldy, U, ldu, st, pass, off + n1, s, ws, wsn)) != cudaSuccess) return e;
  // U = L21 Y11
  if ((e = gemm_f64(n2, n1, n1, 1.0, L + n1, ldl, Y, ldy, 0.0, U, ldu, GEMM_B_LOWER | GEMM_BETA0, s, ws, wsn)) !=
      cudaSuccess)
    return e;
  // Y21 = -Y22 U
  return gemm_f64(n2, n1, n2, -1.0, Y22, ldy, U, ldu, 0.0, Y + n1, ldy, GEMM_A_LOWER | GEMM_BETA0, s, ws, wsn);
}

// Depth-limited recursion: the top `depth` levels form L21 by block forward
// substitution through the diagonal blocks' inverses and leave Y21 zero.
cudaError_t rec_depth(int n, double* Wk, int64_t ldk, double* L, int64_t ldl, double* Y, int64_t ldy, double* U,
                      int64_t ldu, double* T, int64_t ldt, DevStatus* st, int pass, long long off, int depth,
                      cudaStream_t s, double* ws, size_t wsn) {
  if (depth <= 0 || n <= NB) return rec(n, Wk, ldk, L, ldl, Y, ldy, U, ldu, st, pass, off, s, ws, wsn);
  const int n1 = NB * (int)ceil_div(n, 2 * NB);
  const int n2 = n - n1;
  cudaError_t e;
  // [L11, Y11] with Y11 known on its leaf blocks only
  if ((e = rec_depth(n1, Wk, ldk, L, ldl, Y, ldy, U, ldu, T, ldt, st, pass, off, depth - 1, s, ws, wsn)) !=
      cudaSuccess)
    return e;
  // L21 = W21 L11^-T
  if ((e = right_solve(n2, n1, Wk + n1, ldk, L + n1, ldl, L, ldl, Y, ldy, depth - 1, T, ldt, s)) != cudaSuccess)
    return e;
  // W22 <- W22 - L21 L21^T (lower triangle)
  double* W22 = Wk + n1 + (int64_t)n1 * ldk;
  if ((e = gemm_f64(n2, n2, n1, -1.0, L + n1, ldl, L + n1, ldl, 1.0, W22, ldk, GEMM_TB | GEMM_C_LOWER, s, ws,
                    wsn)) != cudaSuccess)
    return e;
  return rec_depth(n2, W22, ldk, L + n1 + (int64_t)n1 * ldl, ldl, Y + n1 + (int64_t)n1 * ldy, ldy, U, ldu, T, ldt,
                   st, pass, off + n1, depth - 1, s, ws, wsn);
}

}  // namespace

cudaError_t right_solve(int64_t M, int N, const double* B, int64_t ldb, double* X, int64_t ldx, const double* L,
                        int64_t ldl, const double* Y, int64_t ldy, int depth, double* T, int64_t ldt,
                        cudaStream_t s) {
  cudaError_t e;
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (depth <= 0 || N <= NB) {
    // X = B Y^T with Y the inverse of this diagonal block (Y^T upper triangular)
    if ((const double*)X != B)
      return gemm_f64(M, N, N, 1.0, B, ldb, Y, ldy, 0.0, X, ldx, GEMM_TB | GEMM_B_UPPER | GEMM_BETA0, s);
    if ((e = gemm_f64(M, N, N, 1.0, B, ldb, Y, ldy, 0.0, T, ldt, GEMM_TB | GEMM_B_UPPER | GEMM_BETA0, s)) !=
        cudaSuccess)
      return e;
    return cudaMemcpy2DAsync(X, (size_t)ldx * sizeof(double), T, (size_t)ldt * sizeof(double),
                             (size_t)M * sizeof(double), (size_t)N, cudaMemcpyDeviceToDevice, s);
  }
  // the split of the recursion that formed Y, so the leaves are its inverted blocks
  const int n1 = NB * (int)ceil_div(N, 2 * NB);
  const int n2 = N - n1;
  // X1 = B1 L11^-T
  if ((e = right_solve(M, n1, B, ldb, X, ldx, L, ldl, Y, ldy, depth - 1, T, ldt, s)) != cudaSuccess) return e;
  // X2 = (B2 - X1 L21^T) L22^-T, the bracket formed in X2
  double* X2 = X + (int64_t)n1 * ldx;
  if ((const double*)X != B &&
      (e = cudaMemcpy2DAsync(X2, (size_t)ldx * sizeof(double), B + (int64_t)n1 * ldb, (size_t)ldb * sizeof(double),
                             (size_t)M * sizeof(double), (size_t)n2, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
    return e;
  if ((e = gemm_f64(M, n2, n1, -1.0, X, ldx, L + n1, ldl, 1.0, X2, ldx, GEMM_TB, s)) != cudaSuccess) return e;
  return right_solve(M, n2, X2, ldx, X2, ldx, L + n1 + (int64_t)n1 * ldl, ldl, Y + n1 + (int64_t)n1 * ldy, ldy,
                     depth - 1, T, ldt, s);
}

// Split-k partials of one product: ks * M * N with ks * tiles <= SMs, so 256
// SMs' worth of 64 x 64 tiles is enough for any size (the GEMM lowers ks
// further if the scratch is short).
size_t cholinv_splitk_doubles() { return (size_t)256 * 64 * 64; }

int right_solve_temp_cols(int n) { return n <= NB ? n : NB * (int)ceil_div(n, 2 * NB); }

cudaError_t cholinv_depth(int n, const double* W, int64_t ldw, double* L, int64_t ldl, double* Y, int64_t ldy,
                          double* work, double* U, double* T, int64_t ldt, DevStatus* st, int pass, int depth,
                          cudaStream_t s, double* ws, size_t wsn) {
  if (depth <= 0) return cholinv(n, W, ldw, L, ldl, Y, ldy, work, U, st, pass, s, ws, wsn);
  cudaError_t e;
  if ((e = set_base_smem()) != cudaSuccess) return e;
  if ((e = cudaMemcpy2DAsync(work, (size_t)n * sizeof(double), W, (size_t)ldw * sizeof(double),
                             (size_t)n * sizeof(double), (size_t)n, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
    return e;
  if ((e = cudaMemset2DAsync(L, (size_t)ldl * sizeof(double), 0, (size_t)n * sizeof(double), (size_t)n, s)) !=
      cudaSuccess)
    return e;
  if ((e = cudaMemset2DAsync(Y, (size_t)ldy * sizeof(double), 0, (size_t)n * sizeof(double), (size_t)n, s)) !=
      cudaSuccess)
    return e;
  return rec_depth(n, work, n, L, ldl, Y, ldy, U, n, T, ldt, st, pass, 0, depth, s, ws, wsn);
}

cudaError_t cholinv(int n, const double* W, int64_t ldw, double* L, int64_t ldl, double* Y, int64_t ldy,
                    double* work, double* U, DevStatus* st, int pass, cudaStream_t s, double* ws, size_t wsn,
                    double* Rt, int64_t ldrt, double* Rp) {
  cudaError_t e;
  if ((e = set_base_smem()) != cudaSuccess) return e;
  if (n == NB) {
    // one base case: straight from W, with R and the packed R^-1 when asked
    const int rpw = Rp != nullptr ? qform_group_width(n) : 0;
    // the packing's layout is the Q-form's: the same number of column groups
    if (Rp != nullptr && rpack_doubles(n) != (size_t)RP_GROUPS * n * rpw) return cudaErrorInvalidValue;
    k_cholinv_base64<<<1, 32 * (B64_BW + 1), BASE_SMEM, s>>>(W, ldw, L, ldl, Y, ldy, Rt, ldrt, Rp, rpw, st, pass, 0);
    count_launch();
    return cudaGetLastError();
  }
  if ((e = cudaMemcpy2DAsync(work, (size_t)n * sizeof(double), W, (size_t)ldw * sizeof(double),
                             (size_t)n * sizeof(double), (size_t)n, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
    return e;
  if ((e = cudaMemset2DAsync(L, (size_t)ldl * sizeof(double), 0, (size_t)n * sizeof(double), (size_t)n, s)) !=
      cudaSuccess)
    return e;
  if ((e = cudaMemset2DAsync(Y, (size_t)ldy * sizeof(double), 0, (size_t)n * sizeof(double), (size_t)n, s)) !=
      cudaSuccess)
    return e;
  if ((e = rec(n, work, n, L, ldl, Y, ldy, U, n, st, pass, 0, s, ws, wsn)) != cudaSuccess) return e;
  if (Rt != nullptr && (e = transpose_lower(L, ldl, n, Rt, ldrt, s)) != cudaSuccess) return e;
  if (Rp != nullptr) return pack_rinv_from_lower(Y, ldy, n, Rp, s);
  return cudaSuccess;
}

// Shift of the shifted CholeskyQR pass: W += s I with
// s = 11 (m n + n (n+1)) u trace(W), u = 2^-53 (||A||_F^2 = trace(A^T A)).
// One CTA; the trace is summed in a fixed order.
__global__ void __launch_bounds__(256) k_add_shift(double* __restrict__ W, int64_t ldw, int n, int64_t m) {
  __shared__ double part[256];
  double t = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) t += W[i + (int64_t)i * ldw];
  part[threadIdx.x] = t;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) part[threadIdx.x] += part[threadIdx.x + h];
    __syncthreads();
  }
  const double s = 11.0 * ((double)m * n + (double)n * (n + 1)) * 0x1p-53 * part[0];
  for (int i = threadIdx.x; i < n; i += 256) W[i + (int64_t)i * ldw] += s;
}

cudaError_t add_shift(double* W, int64_t ldw, int n, int64_t m, cudaStream_t s) {
  k_add_shift<<<1, 256, 0, s>>>(W, ldw, n, m);
  count_launch();
  return cudaGetLastError();
}

cudaError_t transpose_lower(const double* L, int64_t ldl, int n, double* R, int64_t ldr, cudaStream_t s) {
  dim3 grid((unsigned)ceil_div(n, 32), (unsigned)ceil_div(n, 32));
  k_transpose_lower<<<grid, dim3(32, 8), 0, s>>>(L, ldl, n, R, ldr);
  count_launch();
  return cudaGetLastError();
}

cudaError_t copy_upper(const double* X, int64_t ldx, int n, double* R, int64_t ldr, cudaStream_t s) {
  dim3 grid((unsigned)ceil_div(n, 128), (unsigned)n);
  k_copy_upper<<<grid, 128, 0, s>>>(X, ldx, n, R, ldr);
  count_launch();
  return cudaGetLastError();
}

}  // namespace cqr2
