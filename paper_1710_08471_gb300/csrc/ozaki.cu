// Split-precision (Ozaki-scheme) emulation of the two FP64 contractions of
// CholeskyQR2 -- the Gram W = X^T X and the Q-forming Q = X R^-1 -- on the
// BF16 tensor cores (tcgen05), with CholInv and R2 R1 left in native FP64.
// This is not part of the paper; it serves the same Algorithm CQR2.
//
// Error-free split. With a shared exponent e along the contraction (per
// column of X for the Gram, per row of X and per column of R^-1 for the
// Q-form) every entry is rounded once to a fixed-point integer
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
// output (groups 0-2 and 3-6), which stays exact as well. The only rounding
// is the one of x' and the final conversion to FP64, done with integer
// operations.
//
// Kernel: 128 x 64 output tile per CTA, BF16 operands K-major in 128-byte
// swizzled shared memory, loaded by TMA (3-D maps over [slice][row][k]).
// Warp 0 produces (TMA), warp 1 issues tcgen05.mma (M=128, N=64, K=16) into
// the 7 group accumulators (448 TMEM columns), warps 2-9 drain groups. All
// waits are bounded; a timeout sets the status word and the CTA unwinds.
#include <cuda.h>

#include <algorithm>

#include "kernels.h"

namespace cqr2 {
namespace {

constexpr int OZ_BK = 64;          // contraction per K-block (128-byte rows)
constexpr int OZ_BM = 128;         // tile rows
constexpr int OZ_BN = 64;          // tile columns
constexpr int OZ_NA = 4;           // A-plane ring slots
constexpr int OZ_THREADS = 320;    // producer + MMA + 8 epilogue warps
constexpr int OZ_EPI_WARPS = 8;
constexpr int EXP_NONFINITE = 1 << 20;  // exponent sentinel: a non-finite entry was seen
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

__device__ __forceinline__ long long to_fixed(double x, int e, int S) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  int ex = (int)((b >> 52) & 0x7FF);
  unsigned long long mant = b & ((1ull << 52) - 1);
  if (ex == 0) {
    if (mant == 0) return 0;
    ex = 1;
  } else {
    mant |= 1ull << 52;
  }
  if (e >= EXP_NONFINITE || ex == 0x7FF) return 0;
  const int sh = ex - 1075 + 7 + 8 * (S - 1) - e;  // < 8S - 53 because |x| < 2^e
  long long v;
  if (sh >= 0) {
    v = (long long)(mant << sh);
  } else if (sh > -63) {
    v = (long long)((mant + (1ull << (-sh - 1))) >> (-sh));
  } else {
    v = 0;
  }
  return (b >> 63) ? -v : v;
}

__device__ __forceinline__ unsigned short small_int_to_bf16(int d) {
  if (d == 0) return 0;
  const unsigned s = d < 0 ? 0x8000u : 0u;
  const unsigned a = (unsigned)(d < 0 ? -d : d);
  const int msb = 31 - __clz(a);
  const unsigned frac = (a << (7 - msb)) & 0x7Fu;
  return (unsigned short)(s | ((unsigned)(127 + msb) << 7) | frac);
}

// Writes the S digits of x (with shared exponent e) as BF16 to out[s * stride].
template <int S>
__device__ __forceinline__ void write_digits(double x, int e, unsigned short* out, size_t stride) {
  long long v = to_fixed(x, e, S);
  int d[S];
#pragma unroll
  for (int s = S - 1; s >= 1; --s) {
    const int lo = (int)(signed char)(v & 0xFF);
    d[s] = lo;
    v = (v - lo) >> 8;
  }
  d[0] = (int)v;
#pragma unroll
  for (int s = 0; s < S; ++s) out[(size_t)s * stride] = small_int_to_bf16(d[s]);
}

// value = (hi * 2^32 + lo) * 2^E, rounded to nearest, with integer operations.
__device__ __forceinline__ double fixed_to_double(long long hi, long long lo, int E) {
  unsigned long long l = (unsigned long long)lo + ((unsigned long long)hi << 32);
  const unsigned long long c = l < (unsigned long long)lo ? 1ull : 0ull;
  unsigned long long h = (unsigned long long)((lo >> 63) + (hi >> 32)) + c;
  const bool neg = (long long)h < 0;
  if (neg) {
    l = ~l + 1ull;
    h = ~h + (l == 0 ? 1ull : 0ull);
  }
  if (h == 0 && l == 0) return 0.0;
  const int lz = h ? __clzll((long long)h) : 64 + __clzll((long long)l);
  unsigned long long th, tl;
  if (lz >= 64) {
    th = l << (lz - 64);
    tl = 0;
  } else if (lz > 0) {
    th = (h << lz) | (l >> (64 - lz));
    tl = l << lz;
  } else {
    th = h;
    tl = l;
  }
  int msb = 127 - lz;
  unsigned long long m = th >> 11;
  const bool round = (th >> 10) & 1ull;
  const bool sticky = ((th & 0x3FFull) != 0) || (tl != 0);
  if (round && (sticky || (m & 1ull))) {
    m += 1;
    if (m >> 53) {
      m >>= 1;
      msb += 1;
    }
  }
  const int biased = msb + E + 1023;
  if (biased <= 0 || biased >= 2047) {
    // outside the normal range: rare, use FP64 arithmetic
    const double mag = ldexp((double)m, msb - 52 + E);
    return neg ? -mag : mag;
  }
  const unsigned long long bits =
      (neg ? (1ull << 63) : 0ull) | ((unsigned long long)biased << 52) | (m & ((1ull << 52) - 1));
  return __longlong_as_double((long long)bits);
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
                                                    unsigned short* __restrict__ planes) {
  const int j = blockIdx.y;
  const int e = cexp[j];
  const size_t stride = (size_t)n * mp;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < mp; k += (int64_t)gridDim.x * blockDim.x) {
    const double x = k < m ? X[k + (int64_t)j * ld] : 0.0;
    write_digits<S>(x, e, planes + (size_t)j * mp + k, stride);
  }
}

// Row slices for the Q-form's left operand: planes[s][r][k], k < np, with one
// exponent per row. A CTA stages 16 rows x n in shared memory.
constexpr int SR_ROWS = 16;
template <int S>
__global__ void __launch_bounds__(256) k_slice_rows(const double* __restrict__ X, int64_t ld, int64_t m, int n, int np,
                                                    unsigned short* __restrict__ planes, int* __restrict__ rexp) {
  extern __shared__ double tile[];  // [n][SR_ROWS]
  __shared__ int sexp[SR_ROWS];
  const int64_t r0 = (int64_t)blockIdx.x * SR_ROWS;
  for (int e = threadIdx.x; e < n * SR_ROWS; e += blockDim.x) {
    const int r = e % SR_ROWS, k = e / SR_ROWS;
    tile[e] = (r0 + r < m) ? X[r0 + r + (int64_t)k * ld] : 0.0;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int r = warp; r < SR_ROWS; r += 8) {
    unsigned long long mx = 0;
    for (int k = lane; k < n; k += 32) {
      const unsigned long long b = (unsigned long long)__double_as_longlong(tile[k * SR_ROWS + r]) & 0x7FFFFFFFFFFFFFFFull;
      mx = b > mx ? b : mx;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long v = __shfl_xor_sync(0xffffffffu, mx, o);
      mx = v > mx ? v : mx;
    }
    if (lane == 0) {
      sexp[r] = exp_from_bits(mx);
      if (r0 + r < m) rexp[r0 + r] = sexp[r];
    }
  }
  __syncthreads();
  const size_t stride = (size_t)m * np;
  for (int e = threadIdx.x; e < SR_ROWS * np; e += blockDim.x) {
    const int r = e / np, k = e % np;
    if (r0 + r >= m) continue;
    const double x = k < n ? tile[k * SR_ROWS + r] : 0.0;
    write_digits<S>(x, sexp[r], planes + (size_t)(r0 + r) * np + k, stride);
  }
}

// Slices of R^-1 = Y^T for the Q-form's right operand: planes[s][j][k] holds
// R^-1(k, j) = Y(j, k) for k <= j, one exponent per column j of R^-1.
// With from_upper the input is R^-1 itself (upper triangular, R^-1(k, j) at
// Y[k + j * ldy]) instead of Y = (R^-1)^T.
template <int S>
__global__ void __launch_bounds__(256) k_slice_rinv(const double* __restrict__ Y, int64_t ldy, int n, int np,
                                                    bool from_upper, unsigned short* __restrict__ planes,
                                                    int* __restrict__ fexp) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j = blockIdx.x * 8 + warp;
  if (j >= n) return;
  const int64_t sj = from_upper ? (int64_t)j * ldy : (int64_t)j;  // offset of (j, 0) in Y-coordinates
  const int64_t sk = from_upper ? 1 : ldy;                        // stride along k
  unsigned long long mx = 0;
  for (int k = lane; k <= j; k += 32) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(Y[sj + k * sk]) & 0x7FFFFFFFFFFFFFFFull;
    mx = b > mx ? b : mx;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long v = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = v > mx ? v : mx;
  }
  const int e = exp_from_bits(mx);
  if (lane == 0) fexp[j] = e;
  const size_t stride = (size_t)n * np;
  for (int k = lane; k < np; k += 32) {
    const double x = k <= j ? Y[sj + k * sk] : 0.0;
    write_digits<S>(x, e, planes + (size_t)j * np + k, stride);
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
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(
          smem_u32(dst)),
      "l"(map), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
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
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
      "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
        "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
        "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// ------------------------------------------------------------ GEMM kernel

enum { OZ_GRAM = 0, OZ_QFORM = 1 };

struct OzParams {
  int64_t m;
  int n;
  int64_t rows_per_split;  // Gram: rows per CTA range (multiple of 128)
  int ntile_j;             // number of 64-column tiles, ceil(n / 64)
  const int* eA;           // Gram: column exponents; Q-form: row exponents of X
  const int* eB;           // Gram: column exponents; Q-form: column exponents of R^-1
  double* out;             // Gram: partial[split][n][n]; Q-form: Q
  int64_t ldo;
  DevStatus* st;
};

template <int S, int MODE>
__global__ void __launch_bounds__(OZ_THREADS, 1) k_ozaki_gemm(const __grid_constant__ CUtensorMap tA,
                                                               const __grid_constant__ CUtensorMap tB, OzParams p) {
  constexpr int A_BYTES = OZ_BM * OZ_BK * 2;
  constexpr int B_BYTES = OZ_BN * OZ_BK * 2;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = smem;                              // OZ_NA slots
  uint8_t* sB = sA + OZ_NA * A_BYTES;              // 2 buffers x S planes
  uint64_t* bar = (uint64_t*)(sB + 2 * S * B_BYTES);
  uint64_t* afull = bar;
  uint64_t* aempty = afull + OZ_NA;
  uint64_t* bfull = aempty + OZ_NA;
  uint64_t* bempty = bfull + 2;
  uint64_t* accfull = bempty + 2;
  uint64_t* accempty = accfull + S;
  uint32_t* tmem_slot = (uint32_t*)(accempty + S);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  // Tile and contraction range.
  int64_t i0, j0, kbase;
  int nk;
  int split = 0;
  if (MODE == OZ_GRAM) {
    int t = blockIdx.x, I = 0;
    while (t >= p.ntile_j - 2 * I) {
      t -= p.ntile_j - 2 * I;
      ++I;
    }
    i0 = (int64_t)OZ_BM * I;
    j0 = (int64_t)OZ_BN * (2 * I + t);
    split = blockIdx.y;
    kbase = (int64_t)split * p.rows_per_split;
    const int64_t kend = min(p.m, kbase + p.rows_per_split);
    nk = kend > kbase ? (int)((kend - kbase + OZ_BK - 1) / OZ_BK) : 0;
  } else {
    // 1-D grid: the column tiles of one row tile are neighbours, so the A
    // slices they share are read once from memory and then from L2.
    const int64_t lin = (int64_t)blockIdx.x;
    j0 = (int64_t)OZ_BN * (lin % p.ntile_j);
    i0 = (int64_t)OZ_BM * (lin / p.ntile_j);
    kbase = 0;
    nk = (int)((j0 + OZ_BN + OZ_BK - 1) / OZ_BK);  // R^-1 upper triangular: k < j0 + 64
    const int nkmax = (p.n + OZ_BK - 1) / OZ_BK;
    nk = min(nk, nkmax);
  }

  if (threadIdx.x == 0) {
    for (int i = 0; i < OZ_NA; ++i) {
      mbar_init(&afull[i], 1);
      mbar_init(&aempty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&bfull[i], 1);
      mbar_init(&bempty[i], 1);
    }
    for (int g = 0; g < S; ++g) {
      mbar_init(&accfull[g], 1);
      mbar_init(&accempty[g], OZ_EPI_WARPS);
    }
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

  if (warp == 0) {
    if (lane == 0) {
      bool ok = true;
      for (int kb = 0; kb < nk && ok; ++kb) {
        const int buf = kb & 1;
        const int k0 = (int)(kbase + (int64_t)kb * OZ_BK);
        if (kb >= 2) ok = mbar_wait(&bempty[buf], ((kb >> 1) - 1) & 1, p.st);
        if (!ok) break;
        mbar_expect_tx(&bfull[buf], S * B_BYTES);
        for (int t = 0; t < S; ++t) tma_load_3d(sB + (buf * S + t) * B_BYTES, &tB, &bfull[buf], k0, (int)j0, t);
        for (int s = 0; s < S; ++s) {
          const int q = kb * S + s, slot = q % OZ_NA;
          if (q >= OZ_NA) ok = mbar_wait(&aempty[slot], ((q / OZ_NA) - 1) & 1, p.st);
          if (!ok) break;
          mbar_expect_tx(&afull[slot], A_BYTES);
          tma_load_3d(sA + slot * A_BYTES, &tA, &afull[slot], k0, (int)i0, s);
        }
      }
      if (!ok) report_timeout(p.st);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(OZ_BN >> 3) << 17) |
                             ((uint32_t)(OZ_BM >> 4) << 24);
      bool ok = true;
      for (int kb = 0; kb < nk && ok; ++kb) {
        const int buf = kb & 1;
        const bool first = (kb & 1) == 0;
        const bool last = (kb & 1) == 1 || kb == nk - 1;
        const int c = kb >> 1;
        ok = mbar_wait(&bfull[buf], (kb >> 1) & 1, p.st);
        if (!ok) break;
        for (int s = 0; s < S && ok; ++s) {
          const int q = kb * S + s, slot = q % OZ_NA;
          ok = mbar_wait(&afull[slot], (q / OZ_NA) & 1, p.st);
          if (!ok) break;
          asm volatile("tcgen05.fence::after_thread_sync;");
          const uint64_t da = sdesc(sA + slot * A_BYTES);
          // Products (s, t) for t = t0 .. t0+nt-1 in one MMA of N = 64 nt: the
          // B slices lie back to back in shared memory (one 1024-byte group
          // pitch throughout) and the groups g = s + t are adjacent 64-column
          // accumulators in TMEM, so the wide MMA lands every product in its
          // own group.
          for (int t0 = 0; t0 + s < S && ok; t0 += 4) {
            const int nt = min(4, S - s - t0);
            if (first && s == 0 && c >= 1) {
              for (int g = t0; g < t0 + nt && ok; ++g) ok = mbar_wait(&accempty[g], (c - 1) & 1, p.st);
              if (!ok) break;
              asm volatile("tcgen05.fence::after_thread_sync;");
            }
            const uint32_t idesc_n = (idesc & ~(0x3Fu << 17)) | ((uint32_t)((OZ_BN * nt) >> 3) << 17);
            const uint64_t db = sdesc(sB + (buf * S + t0) * B_BYTES);
#pragma unroll
            for (int k = 0; k < OZ_BK / 16; ++k)
              mma_bf16(tmem + (uint32_t)((s + t0) * OZ_BN), da + 2 * k, db + 2 * k, idesc_n,
                       (first && s == 0 && k == 0) ? 0u : 1u);
          }
          mma_commit(&aempty[slot]);
          if (last) mma_commit(&accfull[s]);  // every product of group s is issued
        }
        mma_commit(&bempty[buf]);
      }
      if (!ok) report_timeout(p.st);
    }
  } else {
    // Epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31, columns half*32 .. +31.
    const int q4 = warp & 3;
    const int half = (warp - 2) >> 2;
    long long hi[32], lo[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) hi[c] = lo[c] = 0;
    const int nchunks = (nk + 1) >> 1;
    bool ok = true;
    for (int c = 0; c < nchunks && ok; ++c) {
#pragma unroll 1
      for (int g = 0; g < S; ++g) {
        ok = mbar_wait(&accfull[g], c & 1, p.st);
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;");
        uint32_t v[32];
        tmem_ld32(tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(g * OZ_BN + half * 32), v);
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncwarp();
        if (lane == 0) mbar_arrive(&accempty[g]);
        if (g <= 2) {
          const int sh = 8 * (2 - g);
#pragma unroll
          for (int cc = 0; cc < 32; ++cc)
            hi[cc] += (long long)((unsigned long long)(long long)__float2int_rn(__uint_as_float(v[cc])) << sh);
        } else {
          const int sh = 8 * (6 - g);
#pragma unroll
          for (int cc = 0; cc < 32; ++cc)
            lo[cc] += (long long)((unsigned long long)(long long)__float2int_rn(__uint_as_float(v[cc])) << sh);
        }
      }
    }
    if (!ok) report_timeout(p.st);
    const int64_t row = i0 + q4 * 32 + lane;
    if (MODE == OZ_GRAM) {
      if (row < p.n) {
        const int ea = p.eA[row];
        double* out = p.out + (int64_t)split * p.n * p.n;
#pragma unroll
        for (int cc = 0; cc < 32; ++cc) {
          const int64_t col = j0 + half * 32 + cc;
          if (col < p.n) {
            const int eb = p.eB[col];
            double v = (ea >= EXP_NONFINITE || eb >= EXP_NONFINITE) ? __longlong_as_double(0x7FF8000000000000ll)
                                                                    : fixed_to_double(hi[cc], lo[cc], ea + eb - 14 - 48);
            out[row + col * p.n] = v;
          }
        }
      }
    } else {
      if (row < p.m) {
        const int ea = p.eA[row];
#pragma unroll
        for (int cc = 0; cc < 32; ++cc) {
          const int64_t col = j0 + half * 32 + cc;
          if (col < p.n) {
            const int eb = p.eB[col];
            double v = (ea >= EXP_NONFINITE || eb >= EXP_NONFINITE) ? __longlong_as_double(0x7FF8000000000000ll)
                                                                    : fixed_to_double(hi[cc], lo[cc], ea + eb - 14 - 48);
            p.out[row + col * p.ldo] = v;
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) {
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
  }
}

// Sum the split partials of the computed Gram tiles and mirror.
__global__ void k_oz_gram_reduce(const double* __restrict__ partial, int nsplit, int n, double* __restrict__ W,
                                 int64_t ldw) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i >= n || i > j) return;
  double s = 0.0;
  for (int b = 0; b < nsplit; ++b) s += partial[(int64_t)b * n * n + i + (int64_t)j * n];
  W[i + (int64_t)j * ldw] = s;
  W[j + (int64_t)i * ldw] = s;
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

template <int S>
size_t oz_smem() {
  return 1024 + (size_t)OZ_NA * OZ_BM * OZ_BK * 2 + (size_t)2 * S * OZ_BN * OZ_BK * 2 + 8 * (2 * OZ_NA + 4 + 2 * S) +
         16;
}

template <int S, int MODE>
cudaError_t launch_oz(const CUtensorMap& a, const CUtensorMap& b, const OzParams& p, dim3 grid, cudaStream_t s) {
  const size_t sm = oz_smem<S>();
  auto kern = k_ozaki_gemm<S, MODE>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  kern<<<grid, OZ_THREADS, sm, s>>>(a, b, p);
  count_launch();
  return cudaGetLastError();
}

}  // namespace

// ------------------------------------------------------------ public (internal) API

bool ozaki_supported(int n, int S) { return n >= 1 && n <= OZAKI_MAX_N && S >= 6 && S <= 7; }

OzGeom ozaki_geometry(int64_t m, int n) {
  OzGeom g;
  g.mp = ceil_div(m, OZ_BK) * OZ_BK;
  g.np = (int)(ceil_div(n, OZ_BK) * OZ_BK);
  g.ntile_j = (int)ceil_div(n, OZ_BN);
  g.ntiles = 0;
  for (int I = 0; 2 * I < g.ntile_j; ++I) g.ntiles += g.ntile_j - 2 * I;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // one CTA per SM at a time; about two waves, ranges of at most 2^20 rows (fixed-point headroom)
  int64_t want = std::max<int64_t>(1, ceil_div((int64_t)2 * sms, g.ntiles));
  const int64_t chunks = ceil_div(m, 128);
  want = std::min<int64_t>(want, chunks);
  g.rows_per_split = ceil_div(chunks, want) * 128;
  while (g.rows_per_split > (1 << 20)) {
    ++want;
    g.rows_per_split = ceil_div(chunks, want) * 128;
  }
  g.nsplit = (int)ceil_div(m, g.rows_per_split);
  return g;
}

size_t ozaki_plane_elems(int64_t m, int n, int S) {
  const OzGeom g = ozaki_geometry(m, n);
  return (size_t)S * std::max<size_t>((size_t)n * g.mp, (size_t)m * g.np);
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
  static_assert(sizeof(CUtensorMap) <= sizeof(OzMaps::col_a), "tensor map storage");
  bool ok = make((CUtensorMap*)maps.col_a, planes, (uint64_t)g.mp, (uint64_t)n, OZ_BM) &&
            make((CUtensorMap*)maps.col_b, planes, (uint64_t)g.mp, (uint64_t)n, OZ_BN) &&
            make((CUtensorMap*)maps.row_a, planes, (uint64_t)g.np, (uint64_t)m, OZ_BM) &&
            make((CUtensorMap*)maps.rinv_b, rinv_planes, (uint64_t)g.np, (uint64_t)n, OZ_BN);
  return ok ? cudaSuccess : cudaErrorInvalidValue;
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
                             unsigned short* planes, cudaStream_t s) {
  const OzGeom g = ozaki_geometry(m, n);
  dim3 grid((unsigned)std::min<int64_t>(ceil_div(g.mp, 256), 1024), (unsigned)n);
  if (S == 7) k_slice_cols<7><<<grid, 256, 0, s>>>(X, ld, m, n, g.mp, cexp, planes);
  else k_slice_cols<6><<<grid, 256, 0, s>>>(X, ld, m, n, g.mp, cexp, planes);
  count_launch();
  return cudaGetLastError();
}

cudaError_t ozaki_slice_rows(const double* X, int64_t ld, int64_t m, int n, int S, unsigned short* planes, int* rexp,
                             cudaStream_t s) {
  const OzGeom g = ozaki_geometry(m, n);
  const size_t sm = (size_t)n * SR_ROWS * sizeof(double);
  cudaError_t e;
  if (S == 7) {
    e = cudaFuncSetAttribute(k_slice_rows<7>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_slice_rows<7><<<(unsigned)ceil_div(m, SR_ROWS), 256, sm, s>>>(X, ld, m, n, g.np, planes, rexp);
  } else {
    e = cudaFuncSetAttribute(k_slice_rows<6>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_slice_rows<6><<<(unsigned)ceil_div(m, SR_ROWS), 256, sm, s>>>(X, ld, m, n, g.np, planes, rexp);
  }
  count_launch();
  return cudaGetLastError();
}

cudaError_t ozaki_slice_rinv(const double* Y, int64_t ldy, int n, int S, bool from_upper, unsigned short* planes,
                             int* fexp, cudaStream_t s) {
  const int np = (int)(ceil_div(n, OZ_BK) * OZ_BK);
  const unsigned grid = (unsigned)ceil_div(n, 8);
  if (S == 7) k_slice_rinv<7><<<grid, 256, 0, s>>>(Y, ldy, n, np, from_upper, planes, fexp);
  else k_slice_rinv<6><<<grid, 256, 0, s>>>(Y, ldy, n, np, from_upper, planes, fexp);
  count_launch();
  return cudaGetLastError();
}

cudaError_t ozaki_gram(const OzMaps& maps, int64_t m, int n, int S, const int* cexp, double* partial, double* W,
                       int64_t ldw, DevStatus* st, cudaStream_t s) {
  const OzGeom g = ozaki_geometry(m, n);
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
  dim3 grid((unsigned)g.ntiles, (unsigned)g.nsplit);
  const CUtensorMap& a = *(const CUtensorMap*)maps.col_a;
  const CUtensorMap& b = *(const CUtensorMap*)maps.col_b;
  cudaError_t e = S == 7 ? launch_oz<7, OZ_GRAM>(a, b, p, grid, s) : launch_oz<6, OZ_GRAM>(a, b, p, grid, s);
  if (e != cudaSuccess) return e;
  dim3 rg((unsigned)ceil_div(n, 128), (unsigned)n);
  k_oz_gram_reduce<<<rg, 128, 0, s>>>(partial, g.nsplit, n, W, ldw);
  count_launch();
  return cudaGetLastError();
}

cudaError_t ozaki_qform(const OzMaps& maps, int64_t m, int n, int S, const int* rexp, const int* fexp, double* Q,
                        int64_t ldq, DevStatus* st, cudaStream_t s) {
  const OzGeom g = ozaki_geometry(m, n);
  OzParams p{};
  p.m = m;
  p.n = n;
  p.eA = rexp;
  p.eB = fexp;
  p.out = Q;
  p.ldo = ldq;
  p.st = st;
  p.ntile_j = g.ntile_j;
  dim3 grid((unsigned)(g.ntile_j * ceil_div(m, OZ_BM)));
  const CUtensorMap& a = *(const CUtensorMap*)maps.row_a;
  const CUtensorMap& b = *(const CUtensorMap*)maps.rinv_b;
  return S == 7 ? launch_oz<7, OZ_QFORM>(a, b, p, grid, s) : launch_oz<6, OZ_QFORM>(a, b, p, grid, s);
}

}  // namespace cqr2
