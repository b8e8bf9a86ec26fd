// Split-precision (Ozaki-scheme) emulation of the two FP64 contractions of
// CholeskyQR2 -- the Gram W = X^T X and the Q-forming Q = X R^-1 -- on the
// BF16 tensor cores (tcgen05), with CholInv and R2 R1 left in native FP64.
// This is not part of the paper; it serves the same Algorithm CQR2.
//
// Error-free split. With a shared exponent e along the contraction (per
// column of X, for both products; for the Q-form X's column exponents are
// folded into the rows of R^-1, which then has one exponent per column)
// every entry is rounded once to a fixed-point integer
//     x' = round(x * 2^(7 + 8(S-1) - e)),  |x'| <= 2^(7 + 8(S-1)),
// and cut into S balanced base-256 digits, x = 2^e sum_s d_s 2^(-7-8s),
// |d_0| <= 128, d_s in [-128, 127]. Every digit is exact in BF16. This is
// done with integer operations on the FP64 bit pattern (GB300's FP64 pipe is
// far too slow even for conversions).
//
// Products. Slice pairs (s, t) with s + t <= S - 1 are kept (triangular
// truncation, S(S+1)/2 products). Pairs with the same g = s + t share a
// scale, so each group g accumulates into its own FP32 accumulator in TMEM.
// A chunk of 128 contraction indices keeps every group sum an integer below
// 2^24, so the FP32 accumulation is exact. After each chunk the epilogue
// warps move the group sums into two int64 fixed-point accumulators per
// output (T = X 2^24 + Y, X: groups 0-3, Y: groups 4-6), which stays exact
// as well. The only roundings are the one of x' and the final conversion to
// FP64 with integer operations: correctly rounded for the Gram, within one
// ulp for the Q-form (a shorter sequence; far below its truncation error).
//
// Kernel: persistent, one CTA per SM. BF16 operands in 128-byte swizzled
// shared memory, loaded by TMA from the column slice planes, stored K-block
// tiled as [slice][m / 64][column][m % 64] so that every box is contiguous
// (the Q-form's X as an MN-major operand, everything else K-major). Warp 0
// produces (TMA), warp 1 issues tcgen05.mma (M = 128, one MMA per A slice and
// K = 16 step covering all its products), the other warps drain the group
// accumulators. Gram: 128 x 64 tiles, one accumulator buffer; Q-form:
// 128 x 32 tiles, two. All waits are bounded; a timeout sets the status word
// and the CTA unwinds.
#include <cuda.h>

#include <algorithm>
#include <climits>

#include "kernels.h"
#include "oz_fixed.cuh"

namespace cqr2 {
namespace {

constexpr int OZ_BK = 64;          // contraction per K-block (128-byte rows)
constexpr int OZ_QFORM_NA_MAX = 10;  // A ring slots of the Q-form (the Gram keeps 8)
constexpr int OZ_BM = 128;         // tile rows
constexpr int EXP_NONFINITE = OZ_EXP_NONFINITE;
constexpr long long WAIT_LIMIT = 1ll << 24;

// ------------------------------------------------------------ digits

__device__ __forceinline__ int exp_from_bits(unsigned long long absbits) {
  // smallest e with |x| < 2^e for |x| <= max, from the FP64 bit pattern of max
  const int ex = (int)((absbits >> 52) & 0x7FF);
  if (ex == 0x7FF) return EXP_NONFINITE;
  if (absbits == 0) return 0;
  if (ex == 0) return -1021;  // subnormal maximum
  return ex - 1022;
}

// FP32 bits of a small integer |d| <= 2^8: placing d in the low mantissa
// bits of 1.5 * 2^23 and subtracting 1.5 * 2^23 gives d exactly in FP32 (one
// integer add, one FP32 add); with at most 8 significant bits its low 16 bits
// are zero, so the top half is the exact BF16 value.
__device__ __forceinline__ unsigned small_int_f32bits(int d) {
  return __float_as_uint(__int_as_float(0x4B400000 + d) - 12582912.0f);
}

// The S balanced base-256 digits of x (shared exponent e), most significant
// first, as FP32 bit patterns whose top halves are the BF16 digits.
template <int S>
__device__ __forceinline__ void digits_f32bits(double x, int e, unsigned (&out)[S]) {
  int d[S];
  oz_balanced_digits<S>(oz_to_fixed(x, e, S), d);
#pragma unroll
  for (int s = 0; s < S; ++s) out[s] = small_int_f32bits(d[s]);
}

// Writes the S digits of x (with shared exponent e) as BF16 to out[s * stride].
template <int S>
__device__ __forceinline__ void write_digits(double x, int e, unsigned short* out, size_t stride) {
  unsigned d[S];
  digits_f32bits<S>(x, e, d);
#pragma unroll
  for (int s = 0; s < S; ++s) out[(size_t)s * stride] = (unsigned short)(d[s] >> 16);
}

// Digits of four consecutive entries, written as one 8-byte store per slice
// (the BF16 halves of two FP32 patterns joined by one byte permute).
template <int S>
__device__ __forceinline__ void write_digits4(const double (&x)[4], const int (&e)[4], unsigned short* out,
                                              size_t stride) {
  unsigned d[4][S];
#pragma unroll
  for (int q = 0; q < 4; ++q) digits_f32bits<S>(x[q], e[q], d[q]);
#pragma unroll
  for (int s = 0; s < S; ++s) {
    uint2 w;
    w.x = __byte_perm(d[0][s], d[1][s], 0x7632);
    w.y = __byte_perm(d[2][s], d[3][s], 0x7632);
    *reinterpret_cast<uint2*>(out + (size_t)s * stride) = w;
  }
}

// ------------------------------------------------------------ slicing kernels

// colmax[j] = max_i |X(i, j)| as FP64 bits (atomicMax on the bit pattern).
__global__ void __launch_bounds__(256) k_colmax(const double* __restrict__ X, int64_t ld, int64_t m, int n,
                                                int64_t rows_per, unsigned long long* __restrict__ colmax) {
  const int j = blockIdx.y;
  const int64_t r0 = (int64_t)blockIdx.x * rows_per;
  const int64_t r1 = min(m, r0 + rows_per);
  const double* col = X + (int64_t)j * ld;
  unsigned long long mx = 0;
  for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(col[r]) & 0x7FFFFFFFFFFFFFFFull;
    mx = b > mx ? b : mx;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long v = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = v > mx ? v : mx;
  }
  __shared__ unsigned long long red[8];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mx = red[w] > mx ? red[w] : mx;
    atomicMax(colmax + j, mx);
  }
}

__global__ void k_exps_from_max(const unsigned long long* __restrict__ mx, int n, int* __restrict__ e) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) e[j] = exp_from_bits(mx[j]);
}

// Column slices for the Gram: planes[s][j][k], k < mp (zero for k >= m).
template <int S>
__global__ void __launch_bounds__(256) k_slice_cols(const double* __restrict__ X, int64_t ld, int64_t m, int n,
                                                    int64_t mp, const int* __restrict__ cexp,
                                                    unsigned short* __restrict__ planes, const int* __restrict__ gate) {
  if (gate && *gate != S) return;  // routed to the other slice count
  // four consecutive rows per thread: 32 contiguous bytes read, one 8-byte
  // store per slice (mp is a multiple of 64)
  const int j = blockIdx.y;
  const int e = cexp[j];
  const int ee[4] = {e, e, e, e};
  const size_t stride = (size_t)n * mp;
  const double* col = X + (int64_t)j * ld;
  for (int64_t k = 4 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x); k < mp;
       k += 4 * (int64_t)gridDim.x * blockDim.x) {
    double x[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) x[q] = k + q < m ? col[k + q] : 0.0;
    // K-block tiled: [slice][k / 64][column][k % 64], so that a TMA box of
    // columns x 64 rows is one contiguous run of memory
    write_digits4<S>(x, ee, planes + (size_t)(k >> 6) * ((size_t)n * 64) + (size_t)j * 64 + (k & 63), stride);
  }
}

// Right operand of the Q-form, R^-1 in slices planes[s][j][k] (k < np). The
// left operand is X in its column slices, x(i,k) = 2^c_k xt(i,k) with the
// Gram's column exponents c_k; the scale 2^c_k moves into row k of R^-1
// (exact), r'(k,j) = 2^c_k r(k,j), so that the contraction over k has one
// exponent per column j of R^-1: f_j = max_k (c_k + e(r(k,j))) over the
// nonzero entries, and r'(k,j) is cut with exponent f_j (digits of r(k,j) with
// exponent f_j - c_k). cexp == nullptr means c_k = 0. With from_upper the
// input is R^-1 itself (upper triangular, R^-1(k, j) at Y[k + j * ldy])
// instead of Y = (R^-1)^T.
template <int S>
__global__ void __launch_bounds__(256) k_slice_rinv(const double* __restrict__ Y, int64_t ldy, int n, int np,
                                                    bool from_upper, const int* __restrict__ cexp,
                                                    unsigned short* __restrict__ planes, int* __restrict__ fexp,
                                                    const int* __restrict__ gate) {
  if (gate && *gate != S) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j = blockIdx.x * 8 + warp;
  if (j >= n) return;
  const int64_t sj = from_upper ? (int64_t)j * ldy : (int64_t)j;  // offset of (j, 0) in Y-coordinates
  const int64_t sk = from_upper ? 1 : ldy;                        // stride along k
  int f = INT_MIN;
  for (int k = lane; k <= j; k += 32) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(Y[sj + k * sk]) & 0x7FFFFFFFFFFFFFFFull;
    if (b == 0) continue;
    const int ck = cexp ? cexp[k] : 0;
    const int e = exp_from_bits(b);
    const int ef = (e >= EXP_NONFINITE || ck >= EXP_NONFINITE) ? EXP_NONFINITE : e + ck;
    f = ef > f ? ef : f;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const int v = __shfl_xor_sync(0xffffffffu, f, o);
    f = v > f ? v : f;
  }
  if (f == INT_MIN) f = 0;  // an all-zero column
  if (lane == 0) fexp[j] = f;
  const size_t stride = (size_t)n * np;
  for (int k = lane; k < np; k += 32) {
    const double x = k <= j ? Y[sj + k * sk] : 0.0;
    const int ck = cexp && k < n ? cexp[k] : 0;
    write_digits<S>(x, f >= EXP_NONFINITE ? EXP_NONFINITE : f - ck, planes + (size_t)j * np + k, stride);
  }
}

// ------------------------------------------------------------ tcgen05 helpers

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t cnt) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(cnt));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
// Bounded wait on a phase parity. Gives up (false) after WAIT_LIMIT polls, or
// as soon as another CTA has recorded a timeout in the status word.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t phase, const DevStatus* st) {
  const uint32_t addr = smem_u32(b);
  for (long long i = 0; i < WAIT_LIMIT; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(addr), "r"(phase)
        : "memory");
    if (ok) return true;
    if ((i & 4095) == 4095 && *(volatile const int*)&st->status == 5) return false;
  }
  return false;
}

// Bounded wait that ignores the status word: after a timeout, the unwinding
// CTA still waits (up to the limit) for its own copies and MMAs in flight.
__device__ __forceinline__ bool mbar_wait_drain(uint64_t* b, uint32_t phase) {
  const uint32_t addr = smem_u32(b);
  for (long long i = 0; i < (1ll << 22); ++i) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(addr), "r"(phase)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// Records a timeout (status 5) in the status word; the first reporter wins.
__device__ __forceinline__ void report_timeout(DevStatus* st) {
  if (atomicCAS(&st->lock, 0, 1) == 0) {
    st->pass = -1;
    st->pivot = -1;
    st->value = 0.0;
    __threadfence();
    st->status = 5;
  }
}
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1, int c2,
                                            int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5, %6}], [%2];" ::
          "r"(smem_u32(dst)),
      "l"(map), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
      : "memory");
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(
          smem_u32(dst)),
      "l"(map), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}
// MN-major operand (the Q-form's X tile, [k][m] rows of 64 m-values): 128-byte
// swizzle, 64-element atoms along M 8192 bytes apart (the two TMA boxes), 8-row
// groups along K 1024 bytes apart; 16 k further is 2048 bytes.
__device__ __forceinline__ uint64_t sdesc_mn(const void* p) {
  const uint64_t a = (smem_u32(p) & 0x3FFFF) >> 4;
  return a | ((uint64_t)(8192 >> 4) << 16) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) | (2ull << 61);
}
// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sdesc(const void* p) {
  const uint64_t a = (smem_u32(p) & 0x3FFFF) >> 4;
  return a | (1ull << 16) | (64ull << 32) | (1ull << 46) | (2ull << 61);
}
__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          tmem_d),
      "l"(da), "l"(db), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// ------------------------------------------------------------ GEMM kernel

enum { OZ_GRAM = 0, OZ_QFORM = 1 };

// Tile shapes. The Gram uses 128 x 64 tiles (more operand reuse; the S group
// accumulators take 64 S <= 448 TMEM columns, one buffer). The Q-form uses
// 128 x 32 tiles with two accumulator buffers (2 x 32 S <= 448 columns) and
// 16 epilogue warps, since its epilogue (S conversions to integer and one to
// FP64 per output) is as long as its MMAs. The epilogue warps may also be
// split into two groups that take alternate tiles (NGRP = 2); measured on
// 2^20 x 128 that was slower (1.88 ms against 1.37 ms per Q-form), so both
// shapes run one group.
constexpr int OZ_GRAM_BN = 64, OZ_GRAM_EPI = 8, OZ_GRAM_GRP = 1;
constexpr int OZ_QFORM_BN = 32, OZ_QFORM_EPI = 16, OZ_QFORM_GRP = 1;

template <int S, int BN, int EPI, int NGRP>
struct OzCfg {
  static constexpr int NBUF = 2 * S * BN <= 512 ? 2 : 1;         // accumulator buffers in TMEM
  static constexpr int THREADS = 64 + 32 * EPI;                   // producer, MMA, epilogue warps
  static constexpr int A_BYTES = OZ_BM * OZ_BK * 2;               // one A slice tile
  static constexpr int B_BYTES = BN * OZ_BK * 2;                  // one B slice tile
  // A ring slots: what shared memory leaves beside the B double buffer, the
  // barriers and (Q-form) the column-max keys, at most 8 (Gram) or 10
  static constexpr int RESERVED = BN == 32 ? 6200 : 2048, NA_CAP = BN == 32 ? OZ_QFORM_NA_MAX : 8;
  static constexpr int NA = (227 * 1024 - RESERVED - 2 * S * B_BYTES) / A_BYTES < NA_CAP
                                ? (227 * 1024 - RESERVED - 2 * S * B_BYTES) / A_BYTES
                                : NA_CAP;
  static constexpr int CPT = BN * 4 * NGRP / EPI;                 // columns per epilogue thread
  static constexpr int TMAX = 256 / BN;                           // products per MMA (N <= 256)
  static constexpr int NBAR = 2 * NA + 4 + 2 * NBUF * S + 1;  // + the drain barrier
  static constexpr size_t SMEM = 1024 + (size_t)NA * A_BYTES + (size_t)2 * S * B_BYTES + 8 * NBAR + 16;
  static_assert(NBUF * S * BN <= 512, "accumulators must fit in TMEM");
  static_assert(CPT == 8 || CPT == 16 || CPT == 32, "epilogue load width");
  static_assert(NA >= S, "a K-block of A slices must fit the ring");
  static_assert((EPI / NGRP) % 4 == 0 && (NGRP == 1 || NBUF == 2), "epilogue groups");
};

struct OzParams {
  int64_t m;
  int n;
  int64_t rows_per_split;  // Gram: rows per CTA range (multiple of 128)
  int ntile_j;             // column tiles, ceil(n / BN)
  int ntiles;              // Gram: tiles touching the upper triangle
  int64_t nitems;          // work items (tiles x row ranges, or output tiles)
  const int* eA;           // Gram: column exponents; Q-form: unused (null)
  const int* eB;           // Gram: column exponents; Q-form: column exponents of the scaled R^-1
  double* out;             // Gram: partial[split][n][n]; Q-form: Q
  int64_t ldo;
  DevStatus* st;
  // Q-form, n <= OZ_CMAX_N: if set, the column maxima of |Q| (as the FP64
  // bit pattern of a value with the maximum's exponent, k_colmax's meaning)
  // are atomically folded in, so the next pass needs no column-max sweep
  unsigned long long* cmax;
  // if set, the launch does nothing unless *gate equals its slice count (a
  // plan routed between 6 and 7 slices launches both and one returns)
  const int* gate;
};
constexpr int OZ_CMAX_N = OZAKI_FUSED_COLMAX_MAX_N;

// Order-preserving 32-bit key of |x| for the column exponent: the high word
// of its bit pattern (sign cleared), and back to a bit pattern with that
// high word. exp_from_bits of the result equals that of the column's maximum
// except for a column whose maximum lies below 2^-1042 (a high word of zero),
// which reads as all zero instead of subnormal.
__device__ __forceinline__ uint32_t oz_exp_key(double x) { return (uint32_t)__double2hiint(x) & 0x7FFFFFFFu; }
__device__ __forceinline__ unsigned long long oz_key_bits(uint32_t k) { return (unsigned long long)k << 32; }

// One work item: an output tile and its contraction range.
struct OzItem {
  int64_t i0, j0, kbase;
  int nk;     // K-blocks of 64
  int split;  // Gram: row range
};

// K-blocks of a Q-form tile with first column j0: R^-1 is upper triangular,
// so only k < j0 + BN contributes.
template <int BN>
__device__ __forceinline__ int oz_qform_nk(int64_t j0, int n) {
  return min((int)((j0 + BN + OZ_BK - 1) / OZ_BK), (n + OZ_BK - 1) / OZ_BK);
}

template <int MODE, int BN>
__device__ __forceinline__ OzItem oz_item(const OzParams& p, int64_t it) {
  OzItem w;
  constexpr int R = OZ_BM / BN;  // column tiles per 128-row block
  if (MODE == OZ_GRAM) {
    // the tiles of one row range are neighbours: their slices are shared in L2
    int t = (int)(it % p.ntiles), I = 0;
    w.split = (int)(it / p.ntiles);
    while (t >= p.ntile_j - R * I) {
      t -= p.ntile_j - R * I;
      ++I;
    }
    w.i0 = (int64_t)OZ_BM * I;
    w.j0 = (int64_t)BN * (R * I + t);
    w.kbase = (int64_t)w.split * p.rows_per_split;
    const int64_t kend = min(p.m, w.kbase + p.rows_per_split);
    w.nk = kend > w.kbase ? (int)((kend - w.kbase + OZ_BK - 1) / OZ_BK) : 0;
  } else {
    // the column tiles of one row tile are neighbours: they share A slices in L2
    w.j0 = (int64_t)BN * (it % p.ntile_j);
    w.i0 = (int64_t)OZ_BM * (it / p.ntile_j);
    w.kbase = 0;
    w.split = 0;
    w.nk = oz_qform_nk<BN>(w.j0, p.n);
  }
  return w;
}

// First work item of CTA b of G (CTA G gives the end) when each CTA takes a
// contiguous range of items (the Q-form; the Gram deals its equal-cost items
// round-robin instead). A Q-form item costs its K-blocks plus a fixed epilogue (model:
// nk + 1); the ranges split the total cost evenly, so that no CTA is left with
// only the widest tiles.
template <int MODE, int BN>
__device__ __forceinline__ int64_t oz_range_begin(const OzParams& p, int64_t b, int64_t G) {
  if (MODE == OZ_GRAM) return b * p.nitems / G;
  const int J = p.ntile_j;
  int64_t P = 0;  // cost of one row tile
  for (int j = 0; j < J; ++j) P += oz_qform_nk<BN>((int64_t)BN * j, p.n) + 1;
  const int64_t rows = p.nitems / J;
  const int64_t target = b * (rows * P) / G;  // cost before the range
  const int64_t rt = target / P;
  int64_t rem = target - rt * P;
  int j = 0;
  while (j < J && rem > 0) {
    rem -= oz_qform_nk<BN>((int64_t)BN * j, p.n) + 1;
    ++j;
  }
  return rt * J + j;
}

// acc += x * w in one integer multiply-add (32 x 32 -> 64 bits).
__device__ __forceinline__ void mad_wide(long long& acc, int x, int w) {
  asm("mad.wide.s32 %0, %1, %2, %0;" : "+l"(acc) : "r"(x), "r"(w));
}

// Adds the group sums of one chunk (exact integers in FP32) into the two
// fixed-point accumulators, T = X 2^24 + Y: groups 0-3 into X with weights
// 2^24, 2^16, 2^8, 1 and groups 4-6 into Y with weights 2^16, 2^8, 1.
template <int G, int N>
__device__ __forceinline__ void oz_accumulate(const uint32_t* v, long long* X, long long* Y) {
  constexpr int W = G <= 3 ? 1 << (8 * (3 - G)) : 1 << (8 * (6 - G));
#pragma unroll
  for (int cc = 0; cc < N; ++cc) {
    const int x = __float2int_rn(__uint_as_float(v[cc]));
    if (G <= 3) mad_wide(X[cc], x, W);
    else mad_wide(Y[cc], x, W);
  }
}

template <int N>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, uint32_t* v);
template <>
__device__ __forceinline__ void tmem_ld<8>(uint32_t taddr, uint32_t* v) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
template <>
__device__ __forceinline__ void tmem_ld<16>(uint32_t taddr, uint32_t* v) {
  uint32_t(&w)[16] = *reinterpret_cast<uint32_t(*)[16]>(v);
  tmem_ld16(taddr, w);
}

// TMEM load of 8 columns without the wait (the caller waits once for several).
__device__ __forceinline__ void tmem_ld8_nw(uint32_t taddr, uint32_t* v) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
               : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Drains group G of one chunk for this thread's CPT columns (16 at a time).
template <int G, int CPT>
__device__ __forceinline__ void oz_drain_group(uint32_t ta, long long* X, long long* Y) {
  constexpr int W = CPT >= 32 ? 16 : 8;  // columns per TMEM load (register budget)
#pragma unroll
  for (int h = 0; h < CPT / W; ++h) {
    uint32_t v[W];
    tmem_ld<W>(ta + W * h, v);
    oz_accumulate<G, W>(v, X + W * h, Y + W * h);
  }
}

// Item number of a CTA's it-th item (see it_begin below).
template <int MODE>
__device__ __forceinline__ int64_t oz_item_id(int64_t it) {
  return MODE == OZ_GRAM ? (int64_t)blockIdx.x + it * gridDim.x : it;
}

// Walks a CTA's items. The Q-form's items are consecutive, so the row tile
// and column tile advance by a counter instead of a 64-bit division per item
// (which the single MMA-issuing thread would pay between items).
template <int MODE, int BN>
struct OzCursor {
  int64_t rt = 0;  // Q-form: row tile
  int jt = 0;      // Q-form: column tile
  __device__ __forceinline__ void init(const OzParams& p, int64_t it0) {
    if (MODE == OZ_QFORM) {
      rt = it0 / p.ntile_j;
      jt = (int)(it0 - rt * p.ntile_j);
    }
  }
  __device__ __forceinline__ void next(const OzParams& p) {
    if (MODE == OZ_QFORM && ++jt == p.ntile_j) {
      jt = 0;
      ++rt;
    }
  }
  __device__ __forceinline__ OzItem item(const OzParams& p, int64_t it) const {
    if (MODE == OZ_GRAM) return oz_item<MODE, BN>(p, oz_item_id<MODE>(it));
    OzItem w;
    w.j0 = (int64_t)BN * jt;
    w.i0 = (int64_t)OZ_BM * rt;
    w.kbase = 0;
    w.split = 0;
    w.nk = oz_qform_nk<BN>(w.j0, p.n);
    return w;
  }
};

// Persistent: CTA b takes its items in order. The producer, the
// MMA issuer and the epilogue walk the same item sequence with running
// counters (K-blocks, A slices, chunks), so the mbarrier phases continue
// across items. Group g of chunk c lives in accumulator buffer c % NBUF; the
// epilogue drains a group as soon as its last product is done and the MMAs
// overwrite it only after that drain. Warp w of the epilogue reads TMEM lanes
// 32 (w % 4) .. +31 (its rows) and one column slice of each group.
template <int S, int MODE, int BN, int EPI, int NGRP>
__global__ void __launch_bounds__(OzCfg<S, BN, EPI, NGRP>::THREADS, 1)
    k_ozaki_gemm(const __grid_constant__ CUtensorMap tA, const __grid_constant__ CUtensorMap tB, OzParams p) {
  using C = OzCfg<S, BN, EPI, NGRP>;
  if (p.gate && *p.gate != S) return;  // uniform for the whole grid, before any barrier or TMEM
  constexpr int NA = C::NA, NBUF = C::NBUF, CPT = C::CPT;
  constexpr int A_BYTES = C::A_BYTES, B_BYTES = C::B_BYTES;
  constexpr uint32_t ACC_COLS = S * BN;  // one accumulator buffer
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = smem;                  // NA slots
  uint8_t* sB = sA + NA * A_BYTES;     // 2 buffers x S planes
  uint64_t* bar = (uint64_t*)(sB + 2 * S * B_BYTES);
  uint64_t* afull = bar;
  uint64_t* aempty = afull + NA;
  uint64_t* bfull = aempty + NA;
  uint64_t* bempty = bfull + 2;
  uint64_t* accfull = bempty + 2;       // [NBUF][S]
  uint64_t* accempty = accfull + NBUF * S;
  uint64_t* drainbar = accempty + NBUF * S;  // MMA completion on the timeout path
  uint32_t* tmem_slot = (uint32_t*)(drainbar + 1);
  uint32_t* s_key = tmem_slot + 4;  // Q-form with p.cmax: column max keys [n]
  const bool fuse_cmax = MODE == OZ_QFORM && p.cmax != nullptr;
  if (fuse_cmax)
    for (int c = threadIdx.x; c < p.n; c += blockDim.x) s_key[c] = 0u;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int i = 0; i < NA; ++i) {
      mbar_init(&afull[i], 1);
      mbar_init(&aempty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&bfull[i], 1);
      mbar_init(&bempty[i], 1);
    }
    for (int i = 0; i < NBUF * S; ++i) {
      mbar_init(&accfull[i], 1);
      mbar_init(&accempty[i], EPI / NGRP);  // one group drains a chunk
    }
    mbar_init(drainbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tmem_slot;
  // Gram items are dealt round-robin (the CTA's k-th item is blockIdx.x + k
  // gridDim.x): the CTAs running side by side then hold the tiles of the same
  // row ranges and read each slice K-block from DRAM once between them, the
  // others finding it in L2. Q-form items go in cost-balanced contiguous
  // ranges (oz_range_begin).
  const int64_t it_begin = MODE == OZ_GRAM ? 0 : oz_range_begin<MODE, BN>(p, blockIdx.x, gridDim.x);
  const int64_t it_end = MODE == OZ_GRAM
                             ? (p.nitems > (int64_t)blockIdx.x ? (p.nitems - blockIdx.x + gridDim.x - 1) / gridDim.x : 0)
                             : oz_range_begin<MODE, BN>(p, blockIdx.x + 1, gridDim.x);

  // Ring positions run on across items: A slot and its phase parity, B buffer
  // and its parity. The single issuing threads keep their loops short (no
  // divisions, slices and products unrolled): an MMA of N < 192 costs about
  // as long to issue as to run.
  if (warp == 0) {
    if (lane == 0) {
      bool ok = true;
      int slot = 0, buf = 0;
      uint32_t aph = 0, bph = 0;
      bool awrapped = false, bwrapped = false;  // ring slots used once already
      int alast[NA], blast[2];                   // parity of each slot's last fill (-1: none)
      for (int i = 0; i < NA; ++i) alast[i] = -1;
      blast[0] = blast[1] = -1;
      OzCursor<MODE, BN> cur;
      cur.init(p, it_begin);
      for (int64_t it = it_begin; it < it_end && ok; ++it, cur.next(p)) {
        const OzItem w = cur.item(p, it);
        for (int kb = 0; kb < w.nk; ++kb) {
          const int k0 = (int)(w.kbase + (int64_t)kb * OZ_BK);
          if (bwrapped && !(ok = mbar_wait(&bempty[buf], bph ^ 1u, p.st))) break;
          mbar_expect_tx(&bfull[buf], S * B_BYTES);
          blast[buf] = (int)bph;
#pragma unroll
          for (int t = 0; t < S; ++t) {
            if (MODE == OZ_GRAM)  // column slices, K-block tiled: (k % 64, column, k / 64, slice)
              tma_load_4d(sB + (buf * S + t) * B_BYTES, &tB, &bfull[buf], 0, (int)w.j0, k0 >> 6, t);
            else  // R^-1 slices [slice][column][k]
              tma_load_3d(sB + (buf * S + t) * B_BYTES, &tB, &bfull[buf], k0, (int)w.j0, t);
          }
#pragma unroll
          for (int s = 0; s < S; ++s) {
            if (awrapped && !(ok = mbar_wait(&aempty[slot], aph ^ 1u, p.st))) break;
            mbar_expect_tx(&afull[slot], A_BYTES);
            alast[slot] = (int)aph;
            if (MODE == OZ_GRAM) {
              tma_load_4d(sA + slot * A_BYTES, &tA, &afull[slot], 0, (int)w.i0, k0 >> 6, s);
            } else {  // X from its column slices: two boxes of 64 rows (m) x 64 columns (k)
              const int kb = (int)(w.i0 >> 6);
              tma_load_4d(sA + slot * A_BYTES, &tA, &afull[slot], 0, k0, kb, s);
              tma_load_4d(sA + slot * A_BYTES + A_BYTES / 2, &tA, &afull[slot], 0, k0, kb + 1, s);
            }
            if (++slot == NA) {
              slot = 0;
              aph ^= 1u;
              awrapped = true;
            }
          }
          if (!ok) break;
          if ((buf ^= 1) == 0) {
            bph ^= 1u;
            bwrapped = true;
          }
        }
      }
      if (!ok) {
        report_timeout(p.st);
        // wait for the copies still in flight: the last issued fill of every slot
        for (int i = 0; i < NA; ++i)
          if (alast[i] >= 0) mbar_wait_drain(&afull[i], (uint32_t)alast[i]);
        for (int i = 0; i < 2; ++i)
          if (blast[i] >= 0) mbar_wait_drain(&bfull[i], (uint32_t)blast[i]);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // kind::f16, BF16 A and B, FP32 accumulate, M = 128; B K-major; A K-major
      // (Gram) or MN-major (Q-form, bit 15)
      const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | (MODE == OZ_QFORM ? 1u << 15 : 0u) |
                             ((uint32_t)(OZ_BM >> 4) << 24);
      bool ok = true;
      int slot = 0, buf = 0;
      uint32_t aph = 0, bph = 0;
      int64_t gc = 0;            // chunks issued
      int64_t used0 = 0, used1 = 0;  // two epilogue groups: chunks issued into buffer 0, 1
      OzCursor<MODE, BN> cur;
      cur.init(p, it_begin);
      for (int64_t it = it_begin; it < it_end && ok; ++it, cur.next(p)) {
        const OzItem w = cur.item(p, it);
        const int par_it = (int)((it - it_begin) & 1);
        for (int kb = 0; kb < w.nk; ++kb) {
          const bool first = (kb & 1) == 0;  // the chunk's first K-block overwrites its groups
          const bool last = (kb & 1) == 1 || kb == w.nk - 1;
          // Accumulator buffer of this chunk. One epilogue group: chunks
          // alternate between the buffers. Two groups: group g drains the
          // items of parity g from buffer g only, so that each waits on its
          // buffer's phases strictly in turn (a waiter two phases ahead
          // would see the earlier phase's parity as complete).
          const int ab = NGRP == 2 ? par_it : (NBUF == 2 ? (int)(gc & 1) : 0);
          const int64_t use = NGRP == 2 ? (par_it ? used1 : used0) : (NBUF == 2 ? gc >> 1 : gc);  // earlier chunks in it
          const bool wait_acc = first && use >= 1;
          const uint32_t acc = tmem + (uint32_t)ab * ACC_COLS;
          if (!(ok = mbar_wait(&bfull[buf], bph, p.st))) break;
          const uint64_t db0 = sdesc(sB + buf * S * B_BYTES);
#pragma unroll
          for (int s = 0; s < S; ++s) {
            if (!(ok = mbar_wait(&afull[slot], aph, p.st))) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint64_t da = MODE == OZ_GRAM ? sdesc(sA + slot * A_BYTES) : sdesc_mn(sA + slot * A_BYTES);
            constexpr uint64_t DA_K16 = MODE == OZ_GRAM ? 2 : 2048 >> 4;  // descriptor step per 16 k
            // Products (s, t), t = t0 .. t0+nt-1, in one MMA of N = BN nt: the
            // B slices lie back to back in shared memory (one 1024-byte pitch
            // per 8 rows throughout) and group g = s + t is the BN-column
            // accumulator at column BN g, so each product lands in its group.
            // The S - s products of slice s go in as few MMAs as N <= 256
            // allows, split evenly: an MMA below N = 192 costs a fixed ~75
            // clocks, so 3 + 3 beats 4 + 2 and 3 + 2 beats 4 + 1.
            constexpr int NMMA_MAX = (S + C::TMAX - 1) / C::TMAX;
#pragma unroll
            for (int q = 0, t0 = 0; q < NMMA_MAX && t0 < S - s; ++q) {
              const int nm = (S - s + C::TMAX - 1) / C::TMAX;  // MMAs for this slice
              const int nt = (S - s - t0 + (nm - q) - 1) / (nm - q);
              if (s == 0 && wait_acc) {  // first write of groups t0 .. t0+nt-1 in this buffer
#pragma unroll
                for (int g = t0; g < t0 + nt; ++g) {
                  // the epilogue releases each half (groups 0-3, 4..S-1) on its last group's barrier
                  const bool rep = g == 3 || g == S - 1 || g == t0 + nt - 1;
                  const int gb = g <= 3 ? 3 : S - 1;
                  if (rep && !(ok = mbar_wait(&accempty[ab * S + gb], (uint32_t)((use - 1) & 1), p.st))) break;
                }
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;");
              }
              const uint32_t idesc_n = idesc | ((uint32_t)((BN * nt) >> 3) << 17);
              const uint64_t db = db0 + (uint64_t)((t0 * B_BYTES) >> 4);
              const uint32_t d = acc + (uint32_t)((s + t0) * BN);
              mma_bf16(d, da, db, idesc_n, (s == 0 && first) ? 0u : 1u);
#pragma unroll
              for (int k = 1; k < OZ_BK / 16; ++k) mma_bf16(d, da + DA_K16 * k, db + 2 * k, idesc_n, 1u);
              t0 += nt;
            }
            if (!ok) break;
            mma_commit(&aempty[slot]);
            // every product of group s is issued; the Q-form's epilogue waits on groups 3 and S-1 only
            if (last && (MODE == OZ_GRAM || CPT != 8 || s == 3 || s == S - 1)) mma_commit(&accfull[ab * S + s]);
            if (++slot == NA) {
              slot = 0;
              aph ^= 1u;
            }
          }
          if (!ok) break;
          mma_commit(&bempty[buf]);
          if ((buf ^= 1) == 0) bph ^= 1u;
          if (last) {
            ++gc;
            if (NGRP == 2) (par_it ? used1 : used0) += 1;
          }
        }
      }
      if (!ok) {
        report_timeout(p.st);
        mma_commit(drainbar);  // arrives once every MMA issued so far has completed
        mbar_wait_drain(drainbar, 0);
      }
    }
  } else {
    const int ew = warp - 2;                            // epilogue warp
    const int grp = NGRP == 2 ? ew / (EPI / NGRP) : 0;  // its group: items of its parity
    const int q4 = warp & 3;                            // TMEM lane quarter (rows)
    const int cs = (ew % (EPI / NGRP)) >> 2;            // column slice of each accumulator
    bool ok = true;
    int64_t gc = 0;  // chunks drained (by this group)
    OzCursor<MODE, BN> cur;
    cur.init(p, it_begin);
    for (int64_t it = it_begin; it < it_end && ok; ++it, cur.next(p)) {
      if (NGRP == 2 && (int)((it - it_begin) & 1) != grp) continue;
      const OzItem w = cur.item(p, it);
      const int nchunks = (w.nk + 1) >> 1;
      long long X[CPT], Y[CPT];
#pragma unroll
      for (int c = 0; c < CPT; ++c) X[c] = Y[c] = 0;
      const int64_t row = w.i0 + q4 * 32 + lane;
      const int64_t nrow = MODE == OZ_GRAM ? p.n : p.m;
      const int ea = 0;  // Q-form: X's column exponents live in R^-1's slices
      // Q-form: the output columns' exponents, loaded now so that the loads
      // overlap the drains (the Gram converts once per many chunks and keeps
      // its registers for the accumulators)
      constexpr int NEB = MODE == OZ_QFORM ? CPT : 1;
      int eb[NEB];
#pragma unroll
      for (int cc = 0; cc < NEB; ++cc) {
        const int64_t col = w.j0 + cs * CPT + cc;
        eb[cc] = (MODE == OZ_QFORM && col < p.n) ? p.eB[col] : 0;
      }
      for (int c = 0; c < nchunks && ok; ++c, ++gc) {
        const int ab = NGRP == 2 ? grp : (int)(gc % NBUF);
        const uint32_t par = (uint32_t)((NGRP == 2 ? gc : gc / NBUF) & 1);
        const uint32_t ta = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)ab * ACC_COLS + (uint32_t)(cs * CPT);
#define OZ_DRAIN(G)                                                        \
  if (G < S && ok) {                                                       \
    ok = mbar_wait(&accfull[ab * S + G], par, p.st);                       \
    if (ok) {                                                              \
      asm volatile("tcgen05.fence::after_thread_sync;");                   \
      oz_drain_group<G, CPT>(ta + G * BN, X, Y);                           \
      asm volatile("tcgen05.fence::before_thread_sync;");                  \
      __syncwarp();                                                        \
      if (lane == 0 && (G == 3 || G == S - 1)) mbar_arrive(&accempty[ab * S + G]); \
    }                                                                      \
  }
        if (MODE == OZ_QFORM && CPT == 8) {
          // two waits per chunk: groups 0-3 are complete once slice 3's
          // commit has arrived (a commit tracks every earlier MMA), the rest
          // once the last slice's has; all loads of a half share one wait,
          // and each half is released on its last group's barrier (fewer
          // barrier operations per tile: the Q-form is bound by its tile
          // pipeline's hand-offs)
#define OZ_HALF(G0, G1)                                                      \
  if (ok) {                                                                  \
    ok = mbar_wait(&accfull[ab * S + (G1)], par, p.st);                      \
    if (ok) {                                                                \
      asm volatile("tcgen05.fence::after_thread_sync;");                     \
      uint32_t v[4][8];                                                      \
      _Pragma("unroll") for (int g = G0; g <= G1; ++g) tmem_ld8_nw(ta + g * BN, v[g - G0]); \
      tmem_wait_ld();                                                        \
      asm volatile("tcgen05.fence::before_thread_sync;");                    \
      __syncwarp();                                                          \
      if (lane == 0)                                                         \
        mbar_arrive(&accempty[ab * S + (G1)]);                               \
      if (G0 <= 0 && 0 <= G1) oz_accumulate<0, 8>(v[0 - G0], X, Y);         \
      if (G0 <= 1 && 1 <= G1) oz_accumulate<1, 8>(v[1 - G0], X, Y);         \
      if (G0 <= 2 && 2 <= G1) oz_accumulate<2, 8>(v[2 - G0], X, Y);         \
      if (G0 <= 3 && 3 <= G1) oz_accumulate<3, 8>(v[3 - G0], X, Y);         \
      if (G0 <= 4 && 4 <= G1) oz_accumulate<4, 8>(v[4 - G0 < 4 ? 4 - G0 : 0], X, Y); \
      if (G0 <= 5 && 5 <= G1) oz_accumulate<5, 8>(v[5 - G0 < 4 ? 5 - G0 : 0], X, Y); \
      if (G0 <= 6 && 6 <= G1) oz_accumulate<6, 8>(v[6 - G0 < 4 ? 6 - G0 : 0], X, Y); \
    }                                                                        \
  }
          OZ_HALF(0, 3)
          OZ_HALF(4, S - 1)
#undef OZ_HALF
        } else {
          OZ_DRAIN(0)
          OZ_DRAIN(1)
          OZ_DRAIN(2)
          OZ_DRAIN(3)
          OZ_DRAIN(4)
          OZ_DRAIN(5)
          OZ_DRAIN(6)
        }
#undef OZ_DRAIN
      }
      if (!ok) break;
      uint32_t ck[NEB];  // Q-form: column max keys of this thread's row
#pragma unroll
      for (int cc = 0; cc < NEB; ++cc) ck[cc] = 0u;
      if (row < nrow) {
        const int ea2 = MODE == OZ_GRAM ? p.eA[row] : ea;
        double* out = MODE == OZ_GRAM ? p.out + (int64_t)w.split * p.n * p.n : p.out;
        const int64_t ld = MODE == OZ_GRAM ? p.n : p.ldo;
#pragma unroll
        for (int cc = 0; cc < CPT; ++cc) {
          const int64_t col = w.j0 + cs * CPT + cc;
          if (col < p.n) {
            const int e2 = MODE == OZ_QFORM ? eb[cc < NEB ? cc : 0] : p.eB[col];
            // Gram: exact rounding; Q-form: within one ulp (far below its
            // truncation error), with a shorter integer sequence
            const double v = (ea2 >= EXP_NONFINITE || e2 >= EXP_NONFINITE)
                                 ? __longlong_as_double(0x7FF8000000000000ll)
                             : MODE == OZ_GRAM ? oz_xy_to_double(X[cc], Y[cc], ea2 + e2 - 14 - 48)
                                               : oz_xy_to_double_fast(X[cc], Y[cc], ea2 + e2 - 14 - 48);
            out[row + col * ld] = v;
            if (MODE == OZ_QFORM && fuse_cmax) ck[cc < NEB ? cc : 0] = oz_exp_key(v);
          }
        }
      }
      if (fuse_cmax) {
        // the warp's 32 rows reduced per column, then one shared atomic
        const unsigned mask = __activemask();
#pragma unroll
        for (int cc = 0; cc < NEB; ++cc) {
          const uint32_t mk = __reduce_max_sync(mask, ck[cc]);
          const int64_t col = w.j0 + cs * CPT + cc;
          if (lane == __ffs(mask) - 1 && col < p.n && mk != 0u) atomicMax(&s_key[col], mk);
        }
      }
    }
    if (!ok) report_timeout(p.st);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (fuse_cmax)
    for (int c = threadIdx.x; c < p.n; c += blockDim.x)
      if (s_key[c] != 0u) atomicMax(p.cmax + c, oz_key_bits(s_key[c]));
  if (warp == 0) {
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
  }
}

// Self-test of the timeout path: one thread waits, with the GEMM's bounded
// wait and a short limit, on an mbarrier that nothing arrives at; it then
// reports the timeout and drains exactly as the GEMM's roles do. No memory is
// touched but the status word.
__global__ void k_selftest_wait(long long polls, DevStatus* st) {
  __shared__ uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  const uint32_t addr = smem_u32(&bar);
  bool ok = false;
  for (long long i = 0; i < polls && !ok; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(addr), "r"(0u)
        : "memory");
    ok = done != 0;
  }
  if (!ok) report_timeout(st);
}

// Sum the split partials of the computed Gram tiles and mirror.
__global__ void k_oz_gram_reduce(const double* __restrict__ partial, int nsplit, int n, double* __restrict__ W,
                                 int64_t ldw, const int* __restrict__ gate, int S) {
  if (gate && *gate != S) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i >= n || i > j) return;
  double s = 0.0;
  for (int b = 0; b < nsplit; ++b) s += partial[(int64_t)b * n * n + i + (int64_t)j * n];
  W[i + (int64_t)j * ldw] = s;
  W[j + (int64_t)i * ldw] = s;
}

// Slice-count routing of a 6-slice plan. A column's split keeps 7 + 8(S-1)
// bits relative to its scale 2^e (the power of two above its largest entry),
// so its normwise error grows with the crest ratio sqrt(m) 2^e / ||x_j||, the
// scale over the column's root-mean-square (about 5 to 10 for Gaussian-like
// columns). Where that ratio exceeds 2^OZ_ROUTE_LOG2_CREST for any column,
// the gate is set to 7 and the rest of the factorization runs with 7 slices;
// otherwise to 6. ||x_j||^2 is the diagonal of W = X^T X; with W null the
// columns are taken to have unit norm (the second pass's X, Q1, has columns
// of norm 1 up to the first pass's error). keep: an earlier 7 stays.
constexpr double OZ_ROUTE_LOG2_CREST = 4.0;
__global__ void k_oz_route(const int* __restrict__ cexp, const double* __restrict__ W, int64_t ldw, int n, int64_t m,
                           int* __restrict__ gate, bool keep) {
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  const double lm = log2((double)m);
  int mine = 0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const int e = cexp[j];
    const double w = W ? W[j + (int64_t)j * ldw] : 1.0;
    if (e >= EXP_NONFINITE || !(w > 0.0) || !(w < INFINITY)) continue;  // breakdown is reported elsewhere
    if ((double)e + 0.5 * (lm - log2(w)) > OZ_ROUTE_LOG2_CREST) mine = 1;
  }
  if (mine) any = 1;
  __syncthreads();
  if (threadIdx.x == 0) *gate = (any || (keep && *gate == 7)) ? 7 : 6;
}

// ------------------------------------------------------------ host side

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

template <int S, int MODE, int BN, int EPI, int NGRP>
cudaError_t launch_oz(const CUtensorMap& a, const CUtensorMap& b, const OzParams& p, dim3 grid, cudaStream_t s) {
  using Cfg = OzCfg<S, BN, EPI, NGRP>;
  // the Q-form also holds the column max keys (after the TMEM slot)
  constexpr size_t SMEM = Cfg::SMEM + (MODE == OZ_QFORM ? 4 * OZ_CMAX_N + 16 : 0);
  static_assert(SMEM <= 227 * 1024, "shared memory per CTA");
  auto kern = k_ozaki_gemm<S, MODE, BN, EPI, NGRP>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
  if (e != cudaSuccess) return e;
  kern<<<grid, Cfg::THREADS, SMEM, s>>>(a, b, p);
  count_launch();
  return cudaGetLastError();
}

}  // namespace

int64_t sm_count_oz() {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;  // one CTA per SM (shared memory and the 512 TMEM columns)
}

// ------------------------------------------------------------ public (internal) API

cudaError_t ozaki_selftest_wait(long long polls, DevStatus* st, cudaStream_t s) {
  k_selftest_wait<<<1, 32, 0, s>>>(polls, st);
  count_launch();
  return cudaGetLastError();
}

bool ozaki_supported(int n, int S) { return n >= 1 && n <= OZAKI_MAX_N && S >= 6 && S <= 7; }

namespace {
constexpr int64_t OZ_MAX_CHUNKS_PER_SPLIT = (1 << 20) / 128;  // fixed-point headroom

// About two waves of one CTA per SM over all tiles.
int64_t oz_split_target(int ntiles) {
  return std::max<int64_t>(1, ceil_div((int64_t)2 * sm_count_oz(), ntiles));
}
}  // namespace

OzGeom ozaki_geometry(int64_t m, int n) {
  OzGeom g;
  g.mp = ceil_div(m, OZ_BK) * OZ_BK;
  g.np = (int)(ceil_div(n, OZ_BK) * OZ_BK);
  g.ntile_j = (int)ceil_div(n, OZ_GRAM_BN);
  g.ntiles = 0;
  constexpr int R = OZ_BM / OZ_GRAM_BN;  // column tiles per 128-row block
  for (int I = 0; R * I < g.ntile_j; ++I) g.ntiles += g.ntile_j - R * I;
  // ranges of at most 2^20 rows (8192 chunks) keep the int64 accumulators exact
  const int64_t chunks = ceil_div(m, 128);
  const int64_t want = std::max(std::min(oz_split_target(g.ntiles), chunks), ceil_div(chunks, OZ_MAX_CHUNKS_PER_SPLIT));
  g.rows_per_split = ceil_div(chunks, want) * 128;
  g.nsplit = (int)ceil_div(m, g.rows_per_split);  // <= want
  return g;
}

int64_t ozaki_split_capacity(int64_t m, int n) {
  const OzGeom g = ozaki_geometry(m, n);
  return std::max<int64_t>(oz_split_target(g.ntiles), ceil_div(ceil_div(m, 128), OZ_MAX_CHUNKS_PER_SPLIT));
}

size_t ozaki_plane_elems(int64_t m, int n, int S) {
  const OzGeom g = ozaki_geometry(m, n);
  return (size_t)S * n * g.mp;
}

cudaError_t ozaki_make_maps(OzMaps& maps, int64_t m, int n, int S, void* planes, void* rinv_planes) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  const OzGeom g = ozaki_geometry(m, n);
  auto make = [&](CUtensorMap* map, void* base, uint64_t inner, uint64_t rows, uint32_t box_rows) -> bool {
    cuuint64_t dims[3] = {inner, rows, (cuuint64_t)S};
    cuuint64_t strides[2] = {inner * 2, inner * rows * 2};
    cuuint32_t box[3] = {(cuuint32_t)OZ_BK, box_rows, 1};
    cuuint32_t es[3] = {1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
  };
  // column slices, K-block tiled: dims (k % 64, column, k / 64, slice)
  auto make_tiled = [&](CUtensorMap* map, uint32_t box_cols) -> bool {
    cuuint64_t dims[4] = {(cuuint64_t)OZ_BK, (cuuint64_t)n, (cuuint64_t)(g.mp / OZ_BK), (cuuint64_t)S};
    cuuint64_t strides[3] = {(cuuint64_t)OZ_BK * 2, (cuuint64_t)n * OZ_BK * 2, (cuuint64_t)n * g.mp * 2};
    cuuint32_t box[4] = {(cuuint32_t)OZ_BK, box_cols, 1, 1};
    cuuint32_t es[4] = {1, 1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, planes, dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
  };
  static_assert(sizeof(CUtensorMap) <= sizeof(OzMaps::col_a), "tensor map storage");
  bool ok = make_tiled((CUtensorMap*)maps.col_a, OZ_BM) && make_tiled((CUtensorMap*)maps.col_b, OZ_GRAM_BN) &&
            make_tiled((CUtensorMap*)maps.col_a_mn, OZ_BK) &&
            make((CUtensorMap*)maps.rinv_b, rinv_planes, (uint64_t)g.np, (uint64_t)n, OZ_QFORM_BN);
  return ok ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t ozaki_exps(const unsigned long long* colmax, int n, int* cexp, cudaStream_t s) {
  k_exps_from_max<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(colmax, n, cexp);
  count_launch();
  return cudaGetLastError();
}

cudaError_t ozaki_colmax(const double* X, int64_t ld, int64_t m, int n, unsigned long long* colmax, int* cexp,
                         cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(colmax, 0, (size_t)n * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  const int64_t rows_per = 8192;
  dim3 grid((unsigned)ceil_div(m, rows_per), (unsigned)n);
  k_colmax<<<grid, 256, 0, s>>>(X, ld, m, n, rows_per, colmax);
  count_launch();
  k_exps_from_max<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(colmax, n, cexp);
  count_launch();
  return cudaGetLastError();
}

cudaError_t ozaki_slice_cols(const double* X, int64_t ld, int64_t m, int n, int S, const int* cexp,
                             unsigned short* planes, cudaStream_t s, const int* gate) {
  const OzGeom g = ozaki_geometry(m, n);
  dim3 grid((unsigned)std::min<int64_t>(ceil_div(g.mp, 4 * 256), 1024), (unsigned)n);
  if (S == 7) k_slice_cols<7><<<grid, 256, 0, s>>>(X, ld, m, n, g.mp, cexp, planes, gate);
  else k_slice_cols<6><<<grid, 256, 0, s>>>(X, ld, m, n, g.mp, cexp, planes, gate);
  count_launch();
  return cudaGetLastError();
}


cudaError_t ozaki_slice_rinv(const double* Y, int64_t ldy, int n, int S, bool from_upper, const int* cexp,
                             unsigned short* planes, int* fexp, cudaStream_t s, const int* gate) {
  const int np = (int)(ceil_div(n, OZ_BK) * OZ_BK);
  const unsigned grid = (unsigned)ceil_div(n, 8);
  if (S == 7) k_slice_rinv<7><<<grid, 256, 0, s>>>(Y, ldy, n, np, from_upper, cexp, planes, fexp, gate);
  else k_slice_rinv<6><<<grid, 256, 0, s>>>(Y, ldy, n, np, from_upper, cexp, planes, fexp, gate);
  count_launch();
  return cudaGetLastError();
}

cudaError_t ozaki_gram(const OzMaps& maps, int64_t m, int n, int S, const int* cexp, double* partial,
                       int64_t max_splits, double* W, int64_t ldw, DevStatus* st, cudaStream_t s, const int* gate) {
  const OzGeom g = ozaki_geometry(m, n);
  if (g.nsplit > max_splits) return cudaErrorInvalidValue;
  OzParams p{};
  p.m = m;
  p.n = n;
  p.rows_per_split = g.rows_per_split;
  p.ntile_j = g.ntile_j;
  p.eA = cexp;
  p.eB = cexp;
  p.out = partial;
  p.ldo = n;
  p.st = st;
  p.ntiles = g.ntiles;
  p.nitems = (int64_t)g.ntiles * g.nsplit;
  p.gate = gate;
  dim3 grid((unsigned)std::min<int64_t>(p.nitems, sm_count_oz()));
  const CUtensorMap& a = *(const CUtensorMap*)maps.col_a;
  const CUtensorMap& b = *(const CUtensorMap*)maps.col_b;
  cudaError_t e = S == 7 ? launch_oz<7, OZ_GRAM, OZ_GRAM_BN, OZ_GRAM_EPI, OZ_GRAM_GRP>(a, b, p, grid, s)
                         : launch_oz<6, OZ_GRAM, OZ_GRAM_BN, OZ_GRAM_EPI, OZ_GRAM_GRP>(a, b, p, grid, s);
  if (e != cudaSuccess) return e;
  dim3 rg((unsigned)ceil_div(n, 128), (unsigned)n);
  k_oz_gram_reduce<<<rg, 128, 0, s>>>(partial, g.nsplit, n, W, ldw, gate, S);
  count_launch();
  return cudaGetLastError();
}

cudaError_t ozaki_qform(const OzMaps& maps, int64_t m, int n, int S, const int* fexp, double* Q, int64_t ldq,
                        DevStatus* st, cudaStream_t s, unsigned long long* colmax, const int* gate) {
  const OzGeom g = ozaki_geometry(m, n);
  OzParams p{};
  p.cmax = n <= OZ_CMAX_N ? colmax : nullptr;
  p.m = m;
  p.n = n;
  p.eA = nullptr;  // X enters through its column slices, whose exponents are folded into R^-1
  p.eB = fexp;
  p.out = Q;
  p.ldo = ldq;
  p.st = st;
  p.ntile_j = (int)ceil_div(n, OZ_QFORM_BN);
  p.ntiles = 1;
  p.nitems = (int64_t)p.ntile_j * ceil_div(m, OZ_BM);
  p.gate = gate;
  dim3 grid((unsigned)std::min<int64_t>(p.nitems, sm_count_oz()));
  const CUtensorMap& a = *(const CUtensorMap*)maps.col_a_mn;
  const CUtensorMap& b = *(const CUtensorMap*)maps.rinv_b;
  return S == 7 ? launch_oz<7, OZ_QFORM, OZ_QFORM_BN, OZ_QFORM_EPI, OZ_QFORM_GRP>(a, b, p, grid, s)
                : launch_oz<6, OZ_QFORM, OZ_QFORM_BN, OZ_QFORM_EPI, OZ_QFORM_GRP>(a, b, p, grid, s);
}

cudaError_t ozaki_route(const int* cexp, const double* W, int64_t ldw, int n, int64_t m, int* gate, bool keep,
                        cudaStream_t s) {
  k_oz_route<<<1, 256, 0, s>>>(cexp, W, ldw, n, m, gate, keep);
  count_launch();
  return cudaGetLastError();
}

}  // namespace cqr2
