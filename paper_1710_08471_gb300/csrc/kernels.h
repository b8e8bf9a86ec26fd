// Host-side launchers of the CholeskyQR2 kernels (internal, not the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "common.cuh"

struct cqr2_plan_st;

namespace cqr2 {

// Process-wide count of kernel launches issued by this library.
void count_launch();
void count_launches(int64_t k);  // a graph replay: the kernels it runs
int64_t launch_count();

// ---------------------------------------------------------------- Gram
// Split-m Syrk W = A^T A (Section II-A; the tall dimension is cut into row
// ranges whose partial Grams are summed in a fixed order, the single-GPU form
// of the 1D algorithm's Allreduce, Algorithm 1D-CQR).
struct GramGeom {
  int T = 0;              // output tile width (32, 64 or 128)
  int ntile = 0;          // tiles per side
  int ntiles_total = 0;   // ntile diagonal + ntile(ntile-1)/2 off-diagonal
  int64_t nsplit = 0;     // row ranges
  int64_t rows_per_split = 0;
  size_t partial_doubles() const { return (size_t)nsplit * ntiles_total * T * T; }
};
// ctas_per_sm: target number of Gram CTAs per SM (an autotuned knob).
GramGeom gram_geometry(int64_t m, int n, int64_t max_splits, int ctas_per_sm = 4);
cudaError_t gram_partials(const double* A, int64_t lda, int64_t m, int n, const GramGeom& g,
                          double* partial, cudaStream_t s);
cudaError_t gram_reduce(const double* partial, const GramGeom& g, int n, double* W, int64_t ldw,
                        cudaStream_t s);

// ---------------------------------------------------------------- Q-form
// Q = A Rinv for upper-triangular Rinv (Algorithm CQR step 3).
// Small-n path (n <= 256): one row per lane, warps own column groups.
int qform_group_width(int n);  // columns per group (RP_GROUPS groups), 0 if n > 256
constexpr int RP_GROUPS = 16;  // column groups of the packed R^-1 (the Q-form's NGROUP; checked at run time)
size_t rpack_doubles(int n);
// Rp[g][k][c] = Rinv(k, g*w + c) for k <= g*w + c, else 0; Rinv = Y^T.
cudaError_t pack_rinv_from_lower(const double* Y, int64_t ldy, int n, double* Rp, cudaStream_t s);
// Same from an upper-triangular Rinv (strictly lower part ignored).
cudaError_t pack_rinv_from_upper(const double* Rinv, int64_t ld, int n, double* Rp, cudaStream_t s);
// Q may alias A (each CTA reads its whole row panel before writing it).
cudaError_t qform_small(const double* A, int64_t lda, int64_t m, int n, const double* Rp, double* Q,
                        int64_t ldq, cudaStream_t s);
// Fused: Q = A Rinv and the partial Grams of Q (same layout as gram_partials
// with geometry g, which must have T >= n, i.e. one diagonal tile).
bool qform_gram_fusable(int n);
cudaError_t qform_gram_small(const double* A, int64_t lda, int64_t m, int n, const double* Rp, double* Q,
                             int64_t ldq, const GramGeom& g, double* partial, cudaStream_t s);

// ---------------------------------------------------------------- GEMM
// C = alpha op(A) op(B) + beta C, FP64, column-major. Structure flags let
// tiles skip blocks that are zero by triangularity.
enum : unsigned {
  GEMM_TA = 1u << 0,        // op(A) = A^T
  GEMM_TB = 1u << 1,        // op(B) = B^T
  GEMM_A_LOWER = 1u << 2,   // op(A)(i,k) = 0 for k > i
  GEMM_A_UPPER = 1u << 3,   // op(A)(i,k) = 0 for k < i
  GEMM_B_LOWER = 1u << 4,   // op(B)(k,j) = 0 for k < j
  GEMM_B_UPPER = 1u << 5,   // op(B)(k,j) = 0 for k > j
  GEMM_C_LOWER = 1u << 6,   // only C(i,j), i >= j, is computed and written
  GEMM_C_UPPER = 1u << 7,   // only C(i,j), i <= j, is computed; i > j written as 0
  GEMM_BETA0 = 1u << 8,     // C is not read (beta = 0)
};
// With scratch ws (ws_doubles doubles), a product too small to fill the GPU
// splits k over up to 8 CTAs per tile and sums the partials in a fixed order
// (deterministic; ws must not alias A, B or C).
cudaError_t gemm_f64(int64_t M, int64_t N, int64_t K, double alpha, const double* A, int64_t lda,
                     const double* B, int64_t ldb, double beta, double* C, int64_t ldc, unsigned flags,
                     cudaStream_t s, double* ws = nullptr, size_t ws_doubles = 0);

// R = op(A) B for upper-triangular n x n factors, n <= TRMM_SMALL_MAX, one
// launch; op(A) = A^T (A lower) when a_trans. C below the diagonal is zeroed.
constexpr int TRMM_SMALL_MAX = 128;
cudaError_t trmm_upper_small(int n, const double* A, int64_t lda, bool a_trans, const double* B, int64_t ldb,
                             double* C, int64_t ldc, cudaStream_t s);

// ---------------------------------------------------------------- CholInv
// [L, Y] = CholInv(W) (Algorithm 1): recursive halving with FP64 GEMMs and a
// one-CTA base case of size <= 64. `work` and `U` are n x n scratch (ld n).
constexpr int CHOLINV_BASE = 64;
// ws (wsn doubles, may be null) is split-k scratch for the recursion's small
// products; cholinv_splitk_doubles() is enough for any n.
// With Rt, also R = L^T (ld ldrt, zeros below the diagonal); with Rp, also
// the Q-form's packed R^-1 (pack_rinv_from_lower). At n = 64 one kernel writes
// everything; otherwise the transpose and the packing are launches of their own.
cudaError_t cholinv(int n, const double* W, int64_t ldw, double* L, int64_t ldl, double* Y, int64_t ldy,
                    double* work, double* U, DevStatus* st, int pass, cudaStream_t s, double* ws = nullptr,
                    size_t wsn = 0, double* Rt = nullptr, int64_t ldrt = 0, double* Rp = nullptr);
size_t cholinv_splitk_doubles();
// Inverse depth (the paper's triangular inverted blocks): the top `depth`
// halvings form L21 = W21 L11^-T by block forward substitution and leave Y21
// zero, so Y holds the inverses of L's diagonal blocks only. T is scratch of
// n x right_solve_temp_cols(n) doubles (ld ldt >= n).
cudaError_t cholinv_depth(int n, const double* W, int64_t ldw, double* L, int64_t ldl, double* Y, int64_t ldy,
                          double* work, double* U, double* T, int64_t ldt, DevStatus* st, int pass, int depth,
                          cudaStream_t s, double* ws = nullptr, size_t wsn = 0);
// X = B L^-T (M x N) for lower-triangular L whose diagonal-block inverses of a
// depth-`depth` halving are in Y: X1 = B1 L11^-T, X2 = (B2 - X1 L21^T) L22^-T.
// X may equal B. T is scratch of M x right_solve_temp_cols(N) (ld ldt >= M).
cudaError_t right_solve(int64_t M, int N, const double* B, int64_t ldb, double* X, int64_t ldx, const double* L,
                        int64_t ldl, const double* Y, int64_t ldy, int depth, double* T, int64_t ldt,
                        cudaStream_t s);
int right_solve_temp_cols(int n);
// Shifted CholeskyQR: W += s I, s = 11 (m n + n (n+1)) 2^-53 trace(W).
cudaError_t add_shift(double* W, int64_t ldw, int n, int64_t m, cudaStream_t s);
// R = L^T (upper) with zeros below the diagonal.
cudaError_t transpose_lower(const double* L, int64_t ldl, int n, double* R, int64_t ldr, cudaStream_t s);
// R = upper part of X with zeros below the diagonal.
cudaError_t copy_upper(const double* X, int64_t ldx, int n, double* R, int64_t ldr, cudaStream_t s);

// ---------------------------------------------------------------- Ozaki
// Split-precision Gram and Q-form on BF16 tensor cores (see ozaki.cu).
constexpr int OZAKI_MAX_N = 16384;
struct OzGeom {
  int64_t mp = 0;            // m rounded up to 64
  int np = 0;                // n rounded up to 64
  int ntile_j = 0;           // Gram: 64-column tiles
  int ntiles = 0;            // Gram tiles (128 x 64) touching the upper triangle
  int64_t rows_per_split = 0;
  int nsplit = 0;
};
// Four TMA descriptors (CUtensorMap is 128 bytes, 64-byte aligned).
struct OzMaps {
  alignas(64) unsigned char col_a[128];
  alignas(64) unsigned char col_b[128];
  alignas(64) unsigned char col_a_mn[128];  // the column slices as the Q-form's MN-major left operand
  alignas(64) unsigned char rinv_b[128];
};
bool ozaki_supported(int n, int S);
OzGeom ozaki_geometry(int64_t m, int n);
// Upper bound on ozaki_geometry(m', n).nsplit for every m' <= m.
int64_t ozaki_split_capacity(int64_t m, int n);
size_t ozaki_plane_elems(int64_t m, int n, int S);
cudaError_t ozaki_make_maps(OzMaps& maps, int64_t m, int n, int S, void* planes, void* rinv_planes);
cudaError_t ozaki_colmax(const double* X, int64_t ld, int64_t m, int n, unsigned long long* colmax, int* cexp,
                         cudaStream_t s);
// A non-null gate makes a launch do nothing unless *gate == S (device-side
// routing of a 6-slice plan between 6 and 7 slices; see ozaki_route).
cudaError_t ozaki_slice_cols(const double* X, int64_t ld, int64_t m, int n, int S, const int* cexp,
                             unsigned short* planes, cudaStream_t s, const int* gate = nullptr);
// R^-1 slices with X's column exponents cexp folded into its rows (cexp may be null).
cudaError_t ozaki_slice_rinv(const double* Y, int64_t ldy, int n, int S, bool from_upper, const int* cexp,
                             unsigned short* planes, int* fexp, cudaStream_t s, const int* gate = nullptr);
// partial holds max_splits n x n blocks; a geometry needing more is refused.
cudaError_t ozaki_gram(const OzMaps& maps, int64_t m, int n, int S, const int* cexp, double* partial,
                       int64_t max_splits, double* W, int64_t ldw, DevStatus* st, cudaStream_t s,
                       const int* gate = nullptr);
// One thread waits on an mbarrier nothing arrives at (bounded, `polls`
// polls) and records a timeout in *st, as the split-precision GEMM does.
cudaError_t ozaki_selftest_wait(long long polls, DevStatus* st, cudaStream_t s);
// Q = X R^-1 from X's column slices (the Gram's planes) and R^-1's slices.
// With colmax (zeroed by the caller) and n <= OZAKI_FUSED_COLMAX_MAX_N, the
// column maxima of Q are folded into it as k_colmax would compute them.
cudaError_t ozaki_qform(const OzMaps& maps, int64_t m, int n, int S, const int* fexp, double* Q, int64_t ldq,
                        DevStatus* st, cudaStream_t s, unsigned long long* colmax = nullptr,
                        const int* gate = nullptr);
// Sets *gate to 7 when some column's crest ratio sqrt(m) 2^cexp[j] / sqrt(W_jj)
// exceeds 16 (or, with keep, when *gate is 7 already), else to 6.
cudaError_t ozaki_route(const int* cexp, const double* W, int64_t ldw, int n, int64_t m, int* gate, bool keep,
                        cudaStream_t s);
constexpr int OZAKI_FUSED_COLMAX_MAX_N = 1024;
// Column exponents from column maxima (the second half of ozaki_colmax).
cudaError_t ozaki_exps(const unsigned long long* colmax, int n, int* cexp, cudaStream_t s);

// ---------------------------------------------------------------- batched
// One problem of a grouped launch (same layout as cqr2_problem_t).
struct BatchProblem {
  int64_t m, n;
  const double* A;
  int64_t lda;
  double* Q;
  int64_t ldq;
  double* R;
  int64_t ldr;
  const double* b;  // optional right-hand side (m), with x (n): least squares
  double* x;
};
struct BatchStatus {
  int failed_pass;   // 0 = ok
  int failed_pivot;  // -1 = none
};
constexpr int BATCH_SMALL_MAX_N = 64;
// Enqueue a copy of a plan's device status word (outcome of its last call).
cudaError_t plan_status_copy(struct ::cqr2_plan_st* p, DevStatus* dst, cudaStream_t s);
size_t batched_small_smem();
// Persistent grouped kernel: every problem (n <= 64) factored by one CTA.
cudaError_t cqr2_small_batched(const BatchProblem* probs, int count, int* next, BatchStatus* status,
                               cudaStream_t s);

// ---------------------------------------------------------------- panels
// B(0:rows, 0:cols) += A(0:rows, 0:cols).
cudaError_t add_block(const double* A, int64_t lda, double* B, int64_t ldb, int64_t rows, int64_t cols,
                      cudaStream_t s);
// Copies a panel's first breakdown (status word `inner`) into `outer`, unless
// outer holds one already, with the pivot index shifted by col0.
cudaError_t status_merge(DevStatus* outer, const DevStatus* inner, int64_t col0, cudaStream_t s);

// ---------------------------------------------------------------- lstsq
// c = Q^T b as split-m partials, then x solves R x = c (back substitution).
int64_t gemv_splits(int64_t m, int n);
cudaError_t gemv_t_partials(const double* Q, int64_t ldq, int64_t m, int n, const double* b, int64_t nsplit,
                            double* partial, cudaStream_t s);
cudaError_t lstsq_solve(const double* partial, int64_t nsplit, int n, const double* R, int64_t ldr, double* x,
                        cudaStream_t s);

}  // namespace cqr2
