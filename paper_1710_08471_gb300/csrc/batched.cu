// Persistent grouped CholeskyQR2 for many small problems (n <= 64) in one
// launch. Every CTA takes whole problems from a device work queue (an atomic
// counter over a list sorted by decreasing work) and runs all of Algorithm
// CQR2 for each one on chip:
//   W1 = A^T A over all rows (flattened upper pairs, as in the Gram kernel),
//   [L1, Y1] = CholInv(W1) in shared memory (right-looking Cholesky and
//   triangular inverse, the base case of Algorithm 1),
//   Q1 = A Y1^T panel by panel, its Gram W2 accumulated on the fly (the fused
//   pass-1 Q-form / pass-2 Gram), Q1 staged in the output Q,
//   [L2, Y2] = CholInv(W2), Q = Q1 Y2^T in place, R = L2^T L1^T,
//   and, for a least-squares problem (b given), c = Q^T b accumulated while
//   the final Q is formed and x from R x = c by back substitution (one warp).
// One launch replaces the ~40 launches a planned factorization issues, which
// dominate for small m n^2. A breakdown is recorded per problem (pass, pivot)
// and never traps.
#include <algorithm>

#include "fp64_rsqrt.cuh"
#include "kernels.h"

namespace cqr2 {
namespace {

constexpr int BT = 256;   // threads
constexpr int BNMAX = 64; // largest n
constexpr int BLD = BNMAX + 1;
constexpr int BPANEL = 32;
constexpr int BP = BNMAX * (BNMAX + 1) / 2;  // 2080 upper pairs
constexpr int BS = (BP + BT - 1) / BT;       // 9 slots per thread

struct SmallSmem {
  double S[BNMAX * BLD];   // W, then L (column-major, lower), S(i,j) = S[j*BLD + i]
  double T[BNMAX * BLD];   // Y = L^-1 (lower)
  double R1[BNMAX * BLD];  // R1 = L1^T (upper) kept for R = R2 R1
  double P[BPANEL * BLD];  // row panel of A or Q1, [row][col]
  double rd[BNMAX];        // reciprocals of L's diagonal
  int fail_pivot;
};

// acc[s] += sum over the 32 rows of the panel of P(r, oi[s]) P(r, oj[s]) for
// the first NS slots. A slot whose 32 pairs all lie beyond the P pairs of
// this n is skipped by the whole warp: the FP64 pipe issues a warp
// instruction at full cost whatever its lane mask or predicate, so the
// branch sits outside the row loop and idle slots issue nothing.
template <int NS>
__device__ __forceinline__ void gram_panel_ns(const double* __restrict__ Pn, const int* oi, const int* oj,
                                              const bool* wact, double* acc) {
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    if (wact[s]) {
      double a = acc[s];
#pragma unroll 8
      for (int kk = 0; kk < BPANEL; ++kk) a = fma(Pn[kk * BLD + oi[s]], Pn[kk * BLD + oj[s]], a);
      acc[s] = a;
    }
  }
}

__device__ __forceinline__ void gram_panel(int nslots, const double* Pn, const int* oi, const int* oj,
                                           const bool* wact, double* acc) {
  switch (nslots) {
    case 1: gram_panel_ns<1>(Pn, oi, oj, wact, acc); break;
    case 2: gram_panel_ns<2>(Pn, oi, oj, wact, acc); break;
    case 3: gram_panel_ns<3>(Pn, oi, oj, wact, acc); break;
    case 4: gram_panel_ns<4>(Pn, oi, oj, wact, acc); break;
    case 5: gram_panel_ns<5>(Pn, oi, oj, wact, acc); break;
    case 6: gram_panel_ns<6>(Pn, oi, oj, wact, acc); break;
    case 7: gram_panel_ns<7>(Pn, oi, oj, wact, acc); break;
    case 8: gram_panel_ns<8>(Pn, oi, oj, wact, acc); break;
    default: gram_panel_ns<BS>(Pn, oi, oj, wact, acc); break;
  }
}

// Register prefetch of a 32-row panel (all n columns): thread t holds the
// elements e = t + BT i of the panel, e = r + 32 c. Issued before the current
// panel's arithmetic, so the global load latency overlaps it.
constexpr int PF = BPANEL * BNMAX / BT;  // 8
__device__ __forceinline__ void panel_load(const double* X, int64_t ldx, int64_t m, int n, int64_t r0, double* pf) {
#pragma unroll
  for (int i = 0; i < PF; ++i) {
    const int e = threadIdx.x + BT * i;
    const int r = e % BPANEL, c = e / BPANEL;
    pf[i] = (c < n && r0 + r < m) ? X[r0 + r + (int64_t)c * ldx] : 0.0;
  }
}
__device__ __forceinline__ void panel_store(const double* pf, int n, double* P) {
#pragma unroll
  for (int i = 0; i < PF; ++i) {
    const int e = threadIdx.x + BT * i;
    const int r = e % BPANEL, c = e / BPANEL;
    if (c < n) P[r * BLD + c] = pf[i];
  }
}

// Right-looking Cholesky of S (n x n, lower) and inverse into T; returns the
// first bad pivot index or -1. All threads participate.
__device__ int cholinv_smem(SmallSmem& sm, int n) {
  const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
  if (t == 0) sm.fail_pivot = -1;
  for (int e = t; e < n * n; e += BT) {
    const int i = e % n, j = e / n;
    sm.T[j * BLD + i] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  // One reciprocal square root per pivot (a short Newton sequence); the
  // column and the inverse's row are then scaled by multiplication: on GB300
  // an FP64 division or square root costs many times a multiply, and the n
  // pivots are a serial chain.
  for (int k = 0; k < n; ++k) {
    if (t == 0) {
      const double d = sm.S[k * BLD + k];
      if ((!(d > 0.0) || !isfinite(d)) && sm.fail_pivot < 0) sm.fail_pivot = k;
      double l, rl;
      chol_rsqrt(d, &rl, &l);
      sm.S[k * BLD + k] = l;
      sm.rd[k] = rl;
    }
    __syncthreads();
    const double rl = sm.rd[k];
    for (int i = k + 1 + t; i < n; i += BT) sm.S[k * BLD + i] *= rl;
    __syncthreads();
    for (int j = k + 1 + tx; j < n; j += 16)
      for (int i = j + ty; i < n; i += 16) sm.S[j * BLD + i] = fma(-sm.S[k * BLD + i], sm.S[k * BLD + j], sm.S[j * BLD + i]);
    __syncthreads();
  }
  for (int k = 0; k < n; ++k) {
    const double rkk = sm.rd[k];
    for (int j = t; j <= k; j += BT) sm.T[j * BLD + k] *= rkk;
    __syncthreads();
    for (int j = tx; j <= k; j += 16)
      for (int i = k + 1 + ty; i < n; i += 16) sm.T[j * BLD + i] = fma(-sm.S[k * BLD + i], sm.T[j * BLD + k], sm.T[j * BLD + i]);
    __syncthreads();
  }
  return sm.fail_pivot;
}

__global__ void __launch_bounds__(BT, 1) k_cqr2_small_batched(const BatchProblem* __restrict__ probs, int count,
                                                           int* __restrict__ next, BatchStatus* __restrict__ status) {
  extern __shared__ double smem_raw[];
  SmallSmem& sm = *reinterpret_cast<SmallSmem*>(smem_raw);
  __shared__ int s_job;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  for (;;) {
    if (t == 0) s_job = atomicAdd(next, 1);
    __syncthreads();
    const int job = s_job;
    __syncthreads();
    if (job >= count) break;
    const BatchProblem pb = probs[job];
    const int n = (int)pb.n;
    const int64_t m = pb.m;
    const int P = n * (n + 1) / 2;
    // flattened upper pairs of this n
    int oi[BS], oj[BS];
    {
      int i = 0, start = 0;
#pragma unroll
      for (int s = 0; s < BS; ++s) {
        int p = t + s * BT;
        if (p >= P) p = P - 1;
        while (p >= start + (n - i)) {
          start += n - i;
          ++i;
        }
        oi[s] = i;
        oj[s] = i + (p - start);
      }
    }
    const int nslots = (P + BT - 1) / BT;
    bool wact[BS];  // slot s of this warp holds at least one real pair
#pragma unroll
    for (int s = 0; s < BS; ++s) wact[s] = (t & ~31) + s * BT < P;
    int fail_pass = 0, fail_pivot = -1;
    for (int pass = 1; pass <= 2; ++pass) {
      const double* X = pass == 1 ? pb.A : pb.Q;
      const int64_t ldx = pass == 1 ? pb.lda : pb.ldq;
      double acc[BS];
#pragma unroll
      for (int s = 0; s < BS; ++s) acc[s] = 0.0;
      if (pass == 1) {
        // W1 = A^T A
        double pf[PF];
        panel_load(X, ldx, m, n, 0, pf);
        for (int64_t r0 = 0; r0 < m; r0 += BPANEL) {
          panel_store(pf, n, sm.P);
          __syncthreads();
          if (r0 + BPANEL < m) panel_load(X, ldx, m, n, r0 + BPANEL, pf);
          gram_panel(nslots, sm.P, oi, oj, wact, acc);
          __syncthreads();
        }
      }
      // (pass 2's Gram was accumulated while Q1 was formed, see below)
      if (pass == 2) {
#pragma unroll
        for (int s = 0; s < BS; ++s) acc[s] = 0.0;
      }
      if (pass == 1) {
#pragma unroll
        for (int s = 0; s < BS; ++s)
          if (s < nslots && t + s * BT < P) {
            sm.S[oi[s] * BLD + oj[s]] = acc[s];  // S(j, i) = W(i, j): the lower triangle
          }
        __syncthreads();
      }
      const int piv = cholinv_smem(sm, n);
      if (piv >= 0 && fail_pass == 0) {
        fail_pass = pass;
        fail_pivot = piv;
      }
      if (pass == 1) {
        // R1 = L1^T kept in shared memory
        for (int e = t; e < n * n; e += BT) {
          const int i = e % n, j = e / n;
          sm.R1[j * BLD + i] = (i <= j) ? sm.S[i * BLD + j] : 0.0;
        }
        __syncthreads();
      }
      // Q-form: Qout = X Y^T (R^-1 = Y^T), one lane per row, warps over column groups.
      // Pass 1 also accumulates W2 = Q1^T Q1 from the panel it just formed.
      double gacc[BS];
#pragma unroll
      for (int s = 0; s < BS; ++s) gacc[s] = 0.0;
      // pass 2 of a least-squares problem: c = Q^T b, lane = row, per column j
      const bool with_c = pass == 2 && pb.b != nullptr;
      double cacc[BNMAX / 8];
#pragma unroll
      for (int q = 0; q < BNMAX / 8; ++q) cacc[q] = 0.0;
      double pf[PF];
      panel_load(X, ldx, m, n, 0, pf);
      for (int64_t r0 = 0; r0 < m; r0 += BPANEL) {
        panel_store(pf, n, sm.P);
        __syncthreads();
        // The next panel's loads go out now. In pass 2, X is Q itself: the
        // next panel's rows are read before this iteration writes (only) the
        // current panel's rows.
        if (r0 + BPANEL < m) panel_load(X, ldx, m, n, r0 + BPANEL, pf);
        // each warp owns columns j = warp, warp+8, ...; lane owns row r0+lane
        double qv[BNMAX / 8];
#pragma unroll
        for (int q = 0; q < BNMAX / 8; ++q) {
          const int j = warp + 8 * q;
          double a = 0.0;
          if (j < n) {
            for (int k = 0; k <= j; ++k) a = fma(sm.P[lane * BLD + k], sm.T[k * BLD + j], a);
          }
          qv[q] = a;
        }
        __syncthreads();  // everyone has read the panel
        const double bv = (with_c && r0 + lane < m) ? pb.b[r0 + lane] : 0.0;
#pragma unroll
        for (int q = 0; q < BNMAX / 8; ++q) {
          const int j = warp + 8 * q;
          if (j < n) {
            sm.P[lane * BLD + j] = qv[q];
            if (r0 + lane < m) pb.Q[r0 + lane + (int64_t)j * pb.ldq] = qv[q];
            if (with_c) cacc[q] = fma(qv[q], bv, cacc[q]);
          }
        }
        __syncthreads();
        if (pass == 1) gram_panel(nslots, sm.P, oi, oj, wact, gacc);
        __syncthreads();
      }
      if (with_c) {
        // c_j = sum over lanes (fixed xor tree), kept in sm.P[j]
#pragma unroll
        for (int q = 0; q < BNMAX / 8; ++q) {
          double v = cacc[q];
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
          const int j = warp + 8 * q;
          if (lane == 0 && j < n) sm.P[j] = v;
        }
        __syncthreads();
      }
      if (pass == 1) {
        // W2 into S for the next CholInv (lower triangle)
#pragma unroll
        for (int s = 0; s < BS; ++s)
          if (s < nslots && t + s * BT < P) sm.S[oi[s] * BLD + oj[s]] = gacc[s];
        __syncthreads();
      }
    }
    // R = R2 R1 with R2 = L2^T: R(i, j) = sum_{i<=k<=j} L2(k, i) R1(k, j),
    // also kept in T (Y2 is no longer needed) for the solve
    for (int e = t; e < n * n; e += BT) {
      const int i = e % n, j = e / n;
      double v = 0.0;
      if (i <= j)
        for (int k = i; k <= j; ++k) v = fma(sm.S[i * BLD + k], sm.R1[j * BLD + k], v);
      pb.R[i + (int64_t)j * pb.ldr] = v;
      sm.T[j * BLD + i] = v;
    }
    if (pb.b != nullptr) {
      __syncthreads();
      if (warp == 0) {
        // back substitution R x = c; lane l holds rows l and l + 32
        double c0 = lane < n ? sm.P[lane] : 0.0, c1 = lane + 32 < n ? sm.P[lane + 32] : 0.0;
        for (int j = n - 1; j >= 0; --j) {
          const double cj = __shfl_sync(0xffffffffu, j < 32 ? c0 : c1, j & 31);
          const double xj = cj / sm.T[j * BLD + j];
          if (lane == (j & 31)) {
            if (j < 32) c0 = xj;
            else c1 = xj;
          }
          if (lane < j) c0 = fma(-sm.T[j * BLD + lane], xj, c0);
          if (lane + 32 < j) c1 = fma(-sm.T[j * BLD + lane + 32], xj, c1);
        }
        if (lane < n) pb.x[lane] = c0;
        if (lane + 32 < n) pb.x[lane + 32] = c1;
      }
    }
    if (t == 0) {
      status[job].failed_pass = fail_pass;
      status[job].failed_pivot = fail_pivot;
    }
    __syncthreads();
  }
}

}  // namespace

size_t batched_small_smem() { return sizeof(SmallSmem); }

cudaError_t cqr2_small_batched(const BatchProblem* probs, int count, int* next, BatchStatus* status, cudaStream_t s) {
  const size_t sm = sizeof(SmallSmem);
  cudaError_t e = cudaFuncSetAttribute(k_cqr2_small_batched, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 148, per = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_cqr2_small_batched, BT, sm);
  const int grid = std::max(1, std::min(count, sms * std::max(1, per)));
  if ((e = cudaMemsetAsync(next, 0, sizeof(int), s)) != cudaSuccess) return e;
  k_cqr2_small_batched<<<grid, BT, sm, s>>>(probs, count, next, status);
  count_launch();
  return cudaGetLastError();
}

}  // namespace cqr2
