// Split-m Gram (Syrk, Section II-A; Algorithm CQR step 1): W = A^T A.
//
// The n x n upper triangle is cut into T x T tiles (diagonal and strictly
// upper). Each CTA owns one tile and one contiguous range of rows of A and
// accumulates that range's partial tile in registers; a second kernel sums the
// ranges' partials in a fixed order (deterministic), which is the one-GPU
// counterpart of the 1D algorithm's local Syrk + Allreduce (Algorithm 1D-CQR).
//
// GB300 FP64 runs at about 2 FMA per clock per SM and a warp instruction pays
// for all 32 lanes whether or not they are active, so the diagonal tiles use a
// flattened list of the T(T+1)/2 upper pairs (no lane computes a pair below
// the diagonal) and off-diagonal tiles give each lane one column j and a
// strided set of rows i (the row operand is a shared-memory broadcast).
// Row panels of KC rows are staged through double-buffered shared memory with
// cp.async; the layout [row][column] (padded) makes lanes that differ in the
// column index hit distinct banks.
#include <algorithm>
#include <mutex>

#include "../../include/cqr2.h"
#include "kernels.h"

namespace cqr2 {
namespace {

constexpr int KC = 32;  // rows per staged chunk

// Scratch of the allocation-free Gram entry point (cqr2_syrk_noalloc): the
// split-m partial tiles live in this fixed device array instead of a plan's
// workspace. It belongs to this file's module: a device holds it from the
// first time the module is loaded there (the first Gram kernel or
// cqr2_syrk_noalloc call on that device, under CUDA's default lazy loading)
// until the process exits.
constexpr size_t NOALLOC_DOUBLES = CQR2_NOALLOC_SCRATCH_BYTES / sizeof(double);
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_DOUBLES];

template <int T>
__host__ __device__ constexpr int lds() {
  return T + 1;
}

template <int T, int NT, bool DIAG>
__global__ void __launch_bounds__(NT) k_gram_tile(const double* __restrict__ A, int64_t lda, int64_t m, int n,
                                                  int64_t rows_per_split, int ntile, int ntiles_total,
                                                  double* __restrict__ partial) {
  constexpr int LDS = lds<T>();
  constexpr int NBLK = DIAG ? 1 : 2;
  constexpr int P = DIAG ? T * (T + 1) / 2 : T * T;
  constexpr int S = (P + NT - 1) / NT;
  constexpr int STEP = NT / T;  // off-diagonal: row stride between a lane's slots
  constexpr int E = KC * T / NT;  // elements per thread per block per chunk
  static_assert((KC * T) % NT == 0, "chunk must split evenly");
  static_assert(DIAG || (NT % T == 0), "off-diagonal mapping needs NT multiple of T");
  extern __shared__ double smem[];

  const int t = threadIdx.x;
  int I, J, tile_index;
  if (DIAG) {
    I = J = blockIdx.y;
    tile_index = I;
  } else {
    int rem = blockIdx.y;
    I = 0;
    while (rem >= ntile - 1 - I) {
      rem -= ntile - 1 - I;
      ++I;
    }
    J = I + 1 + rem;
    tile_index = ntile + blockIdx.y;
  }
  const int cI = I * T, cJ = J * T;
  const int64_t r_begin = (int64_t)blockIdx.x * rows_per_split;
  const int64_t r_end = min(m, r_begin + rows_per_split);

  // Slot -> (i, j) inside the tile.
  int oi[DIAG ? S : 1], oj[DIAG ? S : 1];
  bool last_ok = true;
  if (DIAG) {
    int i = 0, start = 0;  // start = first flattened index of row i
#pragma unroll
    for (int s = 0; s < S; ++s) {
      int p = t + s * NT;
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
  const int jcol = t % T;       // off-diagonal lane column
  const int irow0 = t / T;      // off-diagonal first row

  double acc[S];
#pragma unroll
  for (int s = 0; s < S; ++s) acc[s] = 0.0;

  auto load_chunk = [&](int buf, int64_t r0) {
#pragma unroll
    for (int blk = 0; blk < NBLK; ++blk) {
      const int cbase = blk ? cJ : cI;
      double* dst = smem + (size_t)((buf * NBLK + blk) * KC) * LDS;
#pragma unroll
      for (int q = 0; q < E; ++q) {
        const int e = t + q * NT;
        const int kk = e % KC, c = e / KC;
        const int64_t row = r0 + kk;
        const int col = cbase + c;
        const bool ok = (row < r_end) && (col < n);
        const double* src = ok ? (A + row + (int64_t)col * lda) : A;
        cp_async8(dst + kk * LDS + c, src, ok ? 8 : 0);
      }
    }
  };

  const int64_t nchunks = r_end > r_begin ? (r_end - r_begin + KC - 1) / KC : 0;
  if (nchunks > 0) load_chunk(0, r_begin);
  cp_async_commit();
  for (int64_t ch = 0; ch < nchunks; ++ch) {
    const int buf = (int)(ch & 1);
    if (ch + 1 < nchunks) load_chunk(buf ^ 1, r_begin + (ch + 1) * KC);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    const double* As = smem + (size_t)(buf * NBLK * KC) * LDS;
    if (DIAG) {
#pragma unroll 4
      for (int kk = 0; kk < KC; ++kk) {
        const double* row = As + kk * LDS;
#pragma unroll
        for (int s = 0; s < S; ++s) acc[s] = fma(row[oi[s]], row[oj[s]], acc[s]);
      }
    } else {
      const double* Bs = As + KC * LDS;
#pragma unroll 4
      for (int kk = 0; kk < KC; ++kk) {
        const double bj = Bs[kk * LDS + jcol];
        const double* arow = As + kk * LDS + irow0;
#pragma unroll
        for (int s = 0; s < S; ++s) acc[s] = fma(arow[s * STEP], bj, acc[s]);
      }
    }
    __syncthreads();
  }

  double* out = partial + ((int64_t)blockIdx.x * ntiles_total + tile_index) * (int64_t)(T * T);
  if (DIAG) {
#pragma unroll
    for (int s = 0; s < S; ++s) {
      if (s < S - 1 || last_ok) out[oi[s] + oj[s] * T] = acc[s];
    }
  } else {
#pragma unroll
    for (int s = 0; s < S; ++s) out[(irow0 + s * STEP) + jcol * T] = acc[s];
  }
}

// W = the sum of the row ranges' partial tiles, mirrored. The ranges are cut
// into RC contiguous chunks: warp c of a block sums chunk c for 32 elements
// of one column, in range order, and thread c = 0 adds the chunk sums in
// chunk order -- the same fixed order on every call (deterministic), with RC
// warps sharing each element's long sum (the FP64 pipe charges every warp
// instruction in full, so one thread per element and hundreds of ranges left
// most of the GPU idle).
constexpr int GRAM_RC = 8;
__global__ void __launch_bounds__(32 * GRAM_RC) k_gram_reduce(const double* __restrict__ partial, int64_t nsplit,
                                                              int T, int ntile, int ntiles_total, int n,
                                                              double* __restrict__ W, int64_t ldw) {
  __shared__ double part[GRAM_RC][32];
  const int lane = threadIdx.x & 31, c = threadIdx.x >> 5;
  const int i = blockIdx.x * 32 + lane;
  const int j = blockIdx.y;
  const bool live = i < n && i <= j;
  double s = 0.0;
  if (live) {
    const int I = i / T, Jt = j / T;
    const int tile = I == Jt ? I : ntile + I * ntile - I * (I + 1) / 2 + (Jt - I - 1);
    const int64_t loc = (i - I * T) + (int64_t)(j - Jt * T) * T;
    const int64_t stride = (int64_t)ntiles_total * T * T;
    const double* p = partial + (int64_t)tile * T * T + loc;
    const int64_t b0 = nsplit * c / GRAM_RC, b1 = nsplit * (c + 1) / GRAM_RC;
    for (int64_t b = b0; b < b1; ++b) s += p[b * stride];
  }
  part[c][lane] = s;
  __syncthreads();
  if (c == 0 && live) {
    double t = part[0][lane];
#pragma unroll
    for (int k = 1; k < GRAM_RC; ++k) t += part[k][lane];
    W[i + (int64_t)j * ldw] = t;
    W[j + (int64_t)i * ldw] = t;
  }
}

template <int T, int NT, bool DIAG>
size_t gram_smem() {
  return (size_t)2 * (DIAG ? 1 : 2) * KC * lds<T>() * sizeof(double);
}

template <int T, int NT, bool DIAG>
cudaError_t launch_tile(const double* A, int64_t lda, int64_t m, int n, const GramGeom& g, double* partial,
                        int ntiles_y, cudaStream_t s) {
  if (ntiles_y == 0) return cudaSuccess;
  const size_t sm = gram_smem<T, NT, DIAG>();
  auto kern = k_gram_tile<T, NT, DIAG>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)g.nsplit, (unsigned)ntiles_y);
  kern<<<grid, NT, sm, s>>>(A, lda, m, n, g.rows_per_split, g.ntile, g.ntiles_total, partial);
  count_launch();
  return cudaGetLastError();
}

}  // namespace

GramGeom gram_geometry(int64_t m, int n, int64_t max_splits, int ctas_per_sm) {
  GramGeom g;
  g.T = n <= 32 ? 32 : (n <= 64 ? 64 : 128);
  g.ntile = (int)ceil_div(n, g.T);
  g.ntiles_total = g.ntile + g.ntile * (g.ntile - 1) / 2;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // About ctas_per_sm CTAs per SM in total, but never a range shorter than one chunk.
  int64_t want = std::max<int64_t>(1, ceil_div((int64_t)std::max(1, ctas_per_sm) * sms, g.ntiles_total));
  want = std::min<int64_t>(want, std::max<int64_t>(1, ceil_div(m, KC)));
  if (max_splits > 0) want = std::min<int64_t>(want, max_splits);
  g.rows_per_split = ceil_div(ceil_div(m, want), KC) * KC;
  g.nsplit = std::max<int64_t>(1, ceil_div(m, g.rows_per_split));
  return g;
}

cudaError_t gram_partials(const double* A, int64_t lda, int64_t m, int n, const GramGeom& g, double* partial,
                          cudaStream_t s) {
  const int noff = g.ntiles_total - g.ntile;
  cudaError_t e;
  switch (g.T) {
    case 32:
      e = launch_tile<32, 128, true>(A, lda, m, n, g, partial, g.ntile, s);
      if (e == cudaSuccess) e = launch_tile<32, 128, false>(A, lda, m, n, g, partial, noff, s);
      return e;
    case 64:
      e = launch_tile<64, 256, true>(A, lda, m, n, g, partial, g.ntile, s);
      if (e == cudaSuccess) e = launch_tile<64, 256, false>(A, lda, m, n, g, partial, noff, s);
      return e;
    default:
      e = launch_tile<128, 256, true>(A, lda, m, n, g, partial, g.ntile, s);
      if (e == cudaSuccess) e = launch_tile<128, 256, false>(A, lda, m, n, g, partial, noff, s);
      return e;
  }
}

cudaError_t gram_reduce(const double* partial, const GramGeom& g, int n, double* W, int64_t ldw, cudaStream_t s) {
  dim3 block(32 * GRAM_RC);
  dim3 grid((unsigned)ceil_div(n, 32), (unsigned)n);
  k_gram_reduce<<<grid, block, 0, s>>>(partial, g.nsplit, g.T, g.ntile, g.ntiles_total, n, W, ldw);
  count_launch();
  return cudaGetLastError();
}

}  // namespace cqr2

namespace {

// Device address of g_noalloc_scratch, looked up once per CUDA context (with
// that context current) on the first call there, and cached. Host code must
// not use the symbol itself: on the host it names a stand-in, not device
// memory. The cache is keyed by the context's process-unique id
// (cuCtxGetId), so a context made current by the driver API, or the new
// primary context after a cudaDeviceReset, gets its own lookup instead of a
// stale address; where the driver lacks cuCtxGetId the key is the device
// ordinal (primary contexts only, no cudaDeviceReset in between).
typedef int (*CtxGetCurrentFn)(void**);
typedef int (*CtxGetIdFn)(void*, unsigned long long*);
constexpr int MAX_CONTEXTS = 64;
std::mutex g_scratch_mu;
struct ScratchEntry {
  unsigned long long key;
  double* addr;
};
ScratchEntry g_scratch[MAX_CONTEXTS];
int g_scratch_used = 0;

template <typename F>
F driver_fn(const char* name) {
  void* p = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPoint(name, &p, cudaEnableDefault, &q) != cudaSuccess || q != cudaDriverEntryPointSuccess)
    return nullptr;
  return reinterpret_cast<F>(p);
}

// Key of the current context: its unique id with the top bit set, or the
// device ordinal when the driver cannot tell contexts apart (or no context is
// current yet; the entry point's pointer checks have made the runtime's
// context current by then).
cudaError_t context_key(unsigned long long* key) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  static CtxGetCurrentFn get_cur = driver_fn<CtxGetCurrentFn>("cuCtxGetCurrent");
  static CtxGetIdFn get_id = driver_fn<CtxGetIdFn>("cuCtxGetId");
  void* ctx = nullptr;
  unsigned long long id = 0;
  if (get_cur && get_id && get_cur(&ctx) == 0 && ctx && get_id(ctx, &id) == 0) {
    *key = id | (1ull << 63);
    return cudaSuccess;
  }
  *key = (unsigned long long)dev;
  return cudaSuccess;
}

cudaError_t noalloc_scratch(double** out) {
  unsigned long long key = 0;
  cudaError_t e = context_key(&key);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  for (int i = 0; i < g_scratch_used; ++i)
    if (g_scratch[i].key == key) {
      *out = g_scratch[i].addr;
      return cudaSuccess;
    }
  if (g_scratch_used == MAX_CONTEXTS) return cudaErrorInvalidDevice;
  void* p = nullptr;
  e = cudaGetSymbolAddress(&p, cqr2::g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  g_scratch[g_scratch_used++] = {key, static_cast<double*>(p)};
  *out = static_cast<double*>(p);
  return cudaSuccess;
}

// A pointer the kernels may dereference on the current device: device or
// managed memory of this device. Host and unregistered pointers, and memory
// of another device, are rejected (cudaPointerGetAttributes allocates
// nothing).
bool on_current_device(const void* ptr) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();  // clear the error the failed query recorded
    return false;
  }
  return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

}  // namespace

extern "C" cqr2_status_t cqr2_syrk_noalloc(const double* dA, int64_t m, int64_t n, int64_t lda, double* dW,
                                           int64_t ldw, void* stream) {
  using namespace cqr2;
  if (!dA || !dW || n < 1 || m < n || lda < m || ldw < n) return CQR2_ERR_INVALID_ARG;
  if (n > CQR2_NOALLOC_MAX_N) return CQR2_ERR_UNSUPPORTED;
  if (!on_current_device(dA) || !on_current_device(dW)) return CQR2_ERR_INVALID_ARG;
  const GramGeom g0 = gram_geometry(m, (int)n, 0);
  const int64_t per_split = (int64_t)g0.ntiles_total * g0.T * g0.T;
  const int64_t max_splits = (int64_t)NOALLOC_DOUBLES / per_split;
  if (max_splits < 1) return CQR2_ERR_UNSUPPORTED;
  const GramGeom g = gram_geometry(m, (int)n, max_splits);
  if (g.partial_doubles() > NOALLOC_DOUBLES) return CQR2_ERR_UNSUPPORTED;
  double* scratch = nullptr;
  if (noalloc_scratch(&scratch) != cudaSuccess) return CQR2_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // Every partial entry the reduction reads is written by gram_partials in
  // this same call, so nothing left over from an earlier call is used and no
  // clearing is needed.
  if (gram_partials(dA, lda, m, (int)n, g, scratch, s) != cudaSuccess) return CQR2_ERR_CUDA;
  if (gram_reduce(scratch, g, (int)n, dW, ldw, s) != cudaSuccess) return CQR2_ERR_CUDA;
  return CQR2_OK;
}
