/*
 * cqr2.h -- C ABI of the GB300 (sm_103a) CholeskyQR2 library.
 *
 * CholeskyQR2 (Hutter & Solomonik, "Communication-avoiding CholeskyQR2 for
 * rectangular matrices", arXiv 1710.08471, Section II-E, Algorithms CQR and
 * CQR2) computes the reduced QR factorization A = QR of an m x n matrix,
 * m >= n: Q is m x n with orthonormal columns, R is n x n upper triangular
 * with a positive diagonal. It runs CholeskyQR twice:
 *
 *   pass 1:  W1 = A^T A            (Syrk, Section II-A)
 *            [L1, Y1] = CholInv(W1) (Algorithm 1, Section II-D), R1 = L1^T
 *            Q1 = A R1^-1 = A Y1^T
 *   pass 2:  the same on Q1, giving Q and R2
 *   finally: R = R2 R1              (Algorithm CQR2, step 3)
 *
 * Conventions shared by every entry point:
 *   - Matrices are FP64 and column-major (LAPACK layout): element (i, j) of a
 *     matrix with leading dimension ld is at ptr[i + j * ld], ld >= rows.
 *   - Pointers named d* are DEVICE pointers on the current CUDA device; the
 *     caller owns them and keeps them alive until the stream work completes.
 *     Host pointers are named h* and may be pageable or pinned.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream). All device work of a plan is enqueued on its stream,
 *     asynchronously, unless an entry point says it synchronizes.
 *   - Every step runs in this library's own CUDA kernels. There is no CPU
 *     fallback: without a usable GPU, plan creation fails with CQR2_ERR_CUDA.
 *   - No C++ exception crosses this boundary. A plan is not thread-safe; use
 *     one plan per host thread (plans are independent).
 *   - Errors: CQR2_ERR_INVALID_ARG for null pointers, m < n, n < 1, or a
 *     leading dimension smaller than the row count; nothing is enqueued then.
 *     CQR2_ERR_CUDA when a CUDA call fails. CQR2_ERR_NOT_SPD when a
 *     Cholesky pivot was not a finite positive number (reported only by calls
 *     that synchronize, see cqr2_info_t).
 */
#ifndef CQR2_H
#define CQR2_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cqr2_plan_st* cqr2_plan_t;

typedef enum {
  CQR2_OK = 0,
  CQR2_ERR_INVALID_ARG = 1,
  CQR2_ERR_NOT_SPD = 2,     /* Cholesky breakdown in pass 1 or 2 */
  CQR2_ERR_CUDA = 3,        /* a CUDA runtime call failed */
  CQR2_ERR_OOM = 4,         /* device workspace allocation failed */
  CQR2_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up */
  CQR2_ERR_UNSUPPORTED = 6  /* valid request this build does not serve */
} cqr2_status_t;

/* Arithmetic of the two O(m n^2) contractions (Gram and Q-forming).
 * CQR2_FP64: native FP64 FMA throughout.
 * CQR2_OZAKI_BF16: the Gram and Q-forming products are emulated on the
 *   BF16 tensor cores from 7 error-free slices of every FP64 entry (about 55
 *   significant bits, Ozaki scheme) with exact accumulation; CholInv and
 *   R = R2 R1 stay native FP64. Not part of the paper. n <= 16384.
 *   Admissible inputs: every entry is cut with its column's shared exponent
 *   (the power of two 2^e above the column's largest entry), so the accuracy
 *   is normwise and degrades with a column's crest ratio c_j =
 *   sqrt(m) 2^e_j / ||a_j||_2 (about 5 to 10 for Gaussian-like columns).
 *   Tested within ten times the FP64 bounds for kappa(A) <= 1e7 and c_j up to
 *   about 150 (rows whose norms span twelve orders of magnitude, a column
 *   entry 1e8 times its column's median, columns scaled by 1e-20 or 1e15);
 *   the residual grows about like c_j 2^-55.
 * CQR2_OZAKI_BF16_S6: the same with 6 slices (about 47 bits): faster, with
 *   errors within 10x of the FP64 bounds for kappa(A) <= 1e4 when every
 *   crest ratio is at most 16. The plan checks the crest ratios on the device
 *   (A's after the first Gram, Q1's before the second) and, where one exceeds
 *   16, runs the rest of the factorization with 7 slices
 *   (cqr2_plan_split_slices reports which);
 *   at larger kappa the 6-slice residual grows (about 1e-12 at kappa 1e6,
 *   m = 2^23). */
typedef enum { CQR2_FP64 = 0, CQR2_OZAKI_BF16 = 1, CQR2_OZAKI_BF16_S6 = 2 } cqr2_precision_t;

/* Plan flags. */
#define CQR2_FUSED 0x1u /* fuse pass-1 Q-forming with the pass-2 Gram: Q1 is
                           produced and its Gram accumulated in one sweep, so
                           Q1 makes one fewer trip through memory (FP64,
                           n <= 128; ignored otherwise) */
#define CQR2_SHIFTED 0x4u /* shifted CholeskyQR3: a first CholeskyQR pass on
                             A^T A + s I with s = 11 (m n + n (n+1)) 2^-53
                             ||A||_F^2, then CholeskyQR2 of its Q; R is the
                             product of the three R factors. The third-pass,
                             shifted variant the paper cites for unconditional
                             stability (Section I) and names as future work
                             (Section V): accurate to kappa(A) near 1e12, where
                             plain CholeskyQR2 breaks down. Breakdown passes
                             are reported as 1 (shifted), 2 and 3. */
#define CQR2_INPLACE 0x8u /* allow dQ == dA (with ldq == lda): Q overwrites A.
                             Every path reads each part of A before Q lands on
                             it: FP64 n <= 256 stages each row panel on chip
                             before writing it, wider FP64 forms Q1 in the
                             plan's workspace, and the split-precision Q-form
                             reads only A's slices. Without this flag dQ == dA
                             is CQR2_ERR_INVALID_ARG. Q and A must never
                             overlap partially. */
#define CQR2_GRAPH 0x2u /* capture the launch sequence of a factorization in
                           a CUDA graph and replay it while the call's
                           pointers, leading dimensions and m repeat; needs a
                           non-NULL stream; per-stage profiling bypasses it */

/* Device-side outcome of a factorization. */
typedef struct {
  int32_t status;       /* CQR2_OK, CQR2_ERR_NOT_SPD, or CQR2_ERR_TIMEOUT when a
                           bounded device-side wait of a tensor-core kernel gave up */
  int32_t failed_pass;  /* 0 = none, 1 or 2 = CholeskyQR pass that broke down */
  int64_t failed_pivot; /* 0-based index of the first bad pivot, -1 = none */
  double pivot_value;   /* value of that pivot (may be NaN) */
} cqr2_info_t;

/* Create a plan for m x n factorizations (m >= n >= 1) with the given
 * precision (cqr2_precision_t) and flags (CQR2_FUSED or 0). Allocates the
 * device workspace: the split-m partial Gram matrices, W, L, Y and scratch
 * n x n matrices, and a status word. `stream` may be changed later with
 * cqr2_plan_set_stream. On failure *plan is set to NULL. */
cqr2_status_t cqr2_plan_create(cqr2_plan_t* plan, int64_t m, int64_t n, int32_t precision,
                               uint32_t flags, void* stream);

/* Bytes of device workspace the plan owns. */
size_t cqr2_workspace_bytes(cqr2_plan_t plan);

/* Change the stream subsequent calls enqueue on. */
cqr2_status_t cqr2_plan_set_stream(cqr2_plan_t plan, void* stream);

/* Release the plan and its workspace. Synchronizes the plan's stream first.
 * NULL is ignored. */
void cqr2_plan_destroy(cqr2_plan_t plan);

/* CholeskyQR2 (Algorithm CQR2): A = Q R.
 * dA: m x n input, not modified. dQ: m x n output (may not alias dA).
 * dR: n x n output, upper triangular with its strictly lower part set to 0.
 * Q1 is staged in dQ, so the call needs no m x n workspace.
 * info: if non-NULL, the call synchronizes the stream and fills *info, and
 * returns CQR2_ERR_NOT_SPD on breakdown; if NULL the call is fully
 * asynchronous and the outcome can be read later with cqr2_plan_info. */
cqr2_status_t cqr2_factor(cqr2_plan_t plan, const double* dA, int64_t lda, double* dQ, int64_t ldq,
                          double* dR, int64_t ldr, cqr2_info_t* info);

/* Least squares min_x ||A x - b||_2 through CholeskyQR2 (the paper names
 * least squares as the use, Section I; the solve itself is this library's
 * reading): factor A = QR, c = Q^T b, then x solves R x = c by back
 * substitution. db: m-vector, dx: n-vector (device). dQ (m x n, ldq)
 * receives Q; it may be NULL, and then Q goes to an m x n buffer the plan
 * allocates on the first such call and keeps (CQR2_ERR_OOM if that fails).
 * dR may be NULL, else receives R. info as in cqr2_factor. */
cqr2_status_t cqr2_lstsq(cqr2_plan_t plan, const double* dA, int64_t lda, const double* db, double* dx,
                         double* dQ, int64_t ldq, double* dR, int64_t ldr, cqr2_info_t* info);

/* cqr2_factor / cqr2_lstsq for an m x n matrix with n <= m <= the plan's m
 * (the plan's m is the largest row count it serves; its workspace is sized
 * for it). Lets one plan per n serve matrices of uneven height. The launch
 * geometry (row ranges, and tensor-map descriptors of a split-precision
 * plan) is recomputed on the host when m changes between calls. */
cqr2_status_t cqr2_factor_rows(cqr2_plan_t plan, int64_t m, const double* dA, int64_t lda, double* dQ,
                               int64_t ldq, double* dR, int64_t ldr, cqr2_info_t* info);
cqr2_status_t cqr2_lstsq_rows(cqr2_plan_t plan, int64_t m, const double* dA, int64_t lda, const double* db,
                              double* dx, double* dQ, int64_t ldq, double* dR, int64_t ldr, cqr2_info_t* info);

/* Tuning knobs of a plan (set by the autotuner, cqr2_autotune, or by hand):
 * the number of Gram CTAs per SM (1..8, default 4), and whether to fuse the
 * pass-1 Q-form with the pass-2 Gram (honoured only where CQR2_FUSED is). */
cqr2_status_t cqr2_plan_set_gram_ctas(cqr2_plan_t plan, int32_t ctas_per_sm);
cqr2_status_t cqr2_plan_set_fused(cqr2_plan_t plan, int32_t fused);

/* Inverse depth (the paper's alternative of triangular inverted blocks,
 * Section III-A "3D-CQR2", and its InverseDepth parameter, Section IV): with
 * depth d > 0 the top d halvings of CholInv (Algorithm 1) do not form the
 * off-diagonal inverse block Y21; L21 = A21 L11^-T and Q = A R^-1 are then
 * computed by block forward substitution through the inverses of L's diagonal
 * blocks (X1 = B1 L11^-T, X2 = (B2 - X1 L21^T) L22^-T). d = 0 (the default)
 * forms the whole inverse. The result is the same factorization up to
 * rounding, with less work in CholInv.
 * Applies to native-FP64 plans with n > 256 (the general path); d > 0 on
 * another plan returns CQR2_ERR_UNSUPPORTED, d outside 0..16
 * CQR2_ERR_INVALID_ARG. The first d > 0 allocates an m x (about n/2) scratch
 * buffer (CQR2_ERR_OOM if that fails). Not for use while the plan's stream
 * has a call in flight. */
cqr2_status_t cqr2_plan_set_inverse_depth(cqr2_plan_t plan, int32_t depth);

/* CholeskyQR2 on column panels of width b (the paper's conclusion, Section
 * V, names a CholeskyQR2 that operates on subpanels, to cut the extra
 * computation on near-square matrices, as future work; this is the library's
 * reading of it). With 1 <= b < n, cqr2_factor (and the _rows, _host and
 * least-squares forms) factors A panel by panel, left to right: panel k's
 * columns are copied to their place in Q, projected twice against the
 * panels before it (C = Q_<k^T V, V -= Q_<k C; the second projection
 * reorthogonalises), and factored in place by CholeskyQR2, which gives its
 * columns of Q and R's diagonal block; R's block above it is the sum of the
 * two projections' coefficients. CholInv then works on b x b Gram matrices
 * only, where plain CholeskyQR2 factors and inverts two n x n ones and forms
 * R2 R1. The same factorization up to rounding; accurate while each
 * projected panel satisfies CholeskyQR2's own condition (its condition
 * number well below 1e8). A breakdown reports the pass of the panel's
 * CholeskyQR2 and the pivot as a column index of A.
 * b = 0 or b >= n turns it off (plain CholeskyQR2). Native-FP64 plans
 * without CQR2_SHIFTED only (else CQR2_ERR_UNSUPPORTED); b < 0 is
 * CQR2_ERR_INVALID_ARG. Allocates the panels' own plans (m x b, and the
 * narrower last panel) and n x b doubles (CQR2_ERR_OOM on failure);
 * synchronizes the plan's stream; not for use while the plan has a call in
 * flight. */
cqr2_status_t cqr2_plan_set_panel_width(cqr2_plan_t plan, int64_t b);

/* Self-test of the bounded-wait timeout path (no counterpart in the paper):
 * runs one thread that waits, with the library's bounded mbarrier wait, on a
 * barrier that nothing arrives at, for at most `polls` polls (1..2^24), and
 * reports through a device status word exactly as the split-precision GEMM
 * does when one of its waits runs out. Returns CQR2_ERR_TIMEOUT when the wait
 * ran out (the expected outcome), CQR2_OK if it did not,
 * CQR2_ERR_INVALID_ARG for polls outside the range, CQR2_ERR_CUDA or
 * CQR2_ERR_OOM on a CUDA failure. Synchronises `stream` (may be NULL). The
 * CUDA context stays usable afterwards. */
cqr2_status_t cqr2_selftest_wait_timeout(int64_t polls, void* stream);

/* Synchronize the plan's stream and report the outcome of the last
 * factorization enqueued on the plan. */
cqr2_status_t cqr2_plan_info(cqr2_plan_t plan, cqr2_info_t* info);

/* Slices per entry the plan's last factorization used: 0 for CQR2_FP64, 7
 * for CQR2_OZAKI_BF16, and 6 or 7 for CQR2_OZAKI_BF16_S6 (7 when a column's
 * crest ratio routed it, see cqr2_precision_t; 0 before its first
 * factorization). Not part of the paper. Synchronizes the plan's stream;
 * CQR2_ERR_INVALID_ARG for null arguments, CQR2_ERR_CUDA if the read fails. */
cqr2_status_t cqr2_plan_split_slices(cqr2_plan_t plan, int32_t* slices);

/* ---- Step-level entry points (each one step of Algorithm CQR on the
 * plan's m x n shape, on the plan's stream, asynchronous). ---- */

/* Syrk (Section II-A, Algorithm CQR step 1): W = A^T A, n x n, both
 * triangles written (symmetric). dA m x n. */
cqr2_status_t cqr2_syrk(cqr2_plan_t plan, const double* dA, int64_t lda, double* dW, int64_t ldw);

/* CholInv (Algorithm 1): W = L L^T with L lower triangular, Y = L^-1.
 * dW n x n symmetric (only its lower triangle and diagonal are read); dL and
 * dY n x n outputs, strictly upper parts set to 0. info as in cqr2_factor
 * (failed_pass is reported as 1). */
cqr2_status_t cqr2_cholinv(cqr2_plan_t plan, const double* dW, int64_t ldw, double* dL, int64_t ldl,
                           double* dY, int64_t ldy, cqr2_info_t* info);

/* Q-forming multiply (Algorithm CQR step 3): Q = A Rinv with Rinv n x n
 * upper triangular (its strictly lower part is ignored). dA m x n, dQ m x n
 * (may not alias dA). */
cqr2_status_t cqr2_qform(cqr2_plan_t plan, const double* dA, int64_t lda, const double* dRinv,
                         int64_t ldri, double* dQ, int64_t ldq);

/* R = R2 R1 for n x n upper-triangular R2, R1 (Algorithm CQR2 step 3);
 * strictly lower part of R set to 0. dR may not alias the inputs. */
cqr2_status_t cqr2_trmm_upper(cqr2_plan_t plan, const double* dR2, int64_t ld2, const double* dR1,
                              int64_t ld1, double* dR, int64_t ldr);

/* ---- Many independent factorizations ---- */

/* One problem of a batch: A (m x n, lda) is factored into Q (m x n, ldq) and
 * R (n x n, ldr), all device pointers, m >= n >= 1, Q not aliasing A.
 * b and x are both NULL (a factorization) or both set (least squares: x, n
 * entries, minimizes ||A x - b|| for b, m entries, by R x = Q^T b, as
 * cqr2_lstsq does). */
typedef struct {
  int64_t m, n;
  const double* A;
  int64_t lda;
  double* Q;
  int64_t ldq;
  double* R;
  int64_t ldr;
  const double* b;
  double* x;
} cqr2_problem_t;

typedef struct cqr2_batch_st* cqr2_batch_t;

/* Routing and concurrency of a batch.
 * small_work_limit: problems with n <= 64 and m n^2 <= this are factored by
 *   the persistent grouped kernel (one launch for all of them, one CTA per
 *   problem at a time, FP64 whatever the batch precision).
 * streams: the other problems run on per-(n, stream) plans spread over this
 *   many streams (1..16) forked from and joined to the batch stream.
 * fused: use CQR2_FUSED for those plans.
 * graph: when a call repeats the previous call's problem list exactly (same
 *   descriptors, same order), capture its whole launch sequence -- the
 *   grouped launch and every planned problem's kernels on the forked
 *   streams -- into a CUDA graph, and replay that graph while the list keeps
 *   repeating. Needs a non-NULL batch stream; 0 = off. */
typedef struct {
  int64_t small_work_limit;
  int32_t streams;
  int32_t fused;
  int32_t graph;
} cqr2_batch_config_t;

/* Create a batch context for up to max_count problems per call, with the
 * precision used by the planned problems (cqr2_precision_t). cfg may be NULL
 * for the defaults (the tuned small-problem limit, 4 streams, fused, no
 * graph). Plans
 * are created lazily per (n, stream) and grow to the largest m seen. */
cqr2_status_t cqr2_batch_create(cqr2_batch_t* batch, int32_t max_count, int32_t precision,
                                const cqr2_batch_config_t* cfg, void* stream);

/* Factor (or solve, where b is given) `count` problems (host array of
 * descriptors). All work is enqueued on the batch's stream (and streams
 * joined back into it). With infos (a host array of count entries) the call
 * synchronizes and reports every problem's outcome, returning
 * CQR2_ERR_NOT_SPD if any broke down; with NULL it is asynchronous and
 * cqr2_batch_info reports the outcomes later. A call first waits until the
 * batch's previous call has finished on the device (its descriptors and
 * status words are reused). A problem's result depends only on the problem
 * and the batch's configuration, not on the rest of the batch: the route
 * (grouped kernel or plan) is chosen from m and n alone. */
cqr2_status_t cqr2_batch_factor(cqr2_batch_t batch, const cqr2_problem_t* problems, int32_t count,
                                cqr2_info_t* infos);

/* Outcomes of the batch's last cqr2_batch_factor call (count must equal that
 * call's count): waits for the batch's stream, then fills infos as the
 * synchronous form does and returns the same status. */
cqr2_status_t cqr2_batch_info(cqr2_batch_t batch, int32_t count, cqr2_info_t* infos);

void cqr2_batch_destroy(cqr2_batch_t batch);

/* ---- Autotuner ---- */

typedef struct {
  int32_t gram_ctas;   /* best Gram CTAs per SM */
  int32_t fused;       /* best fusion choice */
  double ms;           /* its time per factorization */
  int32_t candidates;  /* configurations timed */
} cqr2_tune_result_t;

/* Time the candidate configurations (Gram CTAs per SM 1, 2, 4, 8; fused or
 * not where fusion applies) of an m x n factorization at `precision` on the
 * current device, with temporary device buffers, and record the fastest in a
 * process-wide table keyed by (n, floor(log2 m), precision). Batches use the
 * table for the plans they create. Synchronizes; allocates. */
cqr2_status_t cqr2_autotune(int64_t m, int64_t n, int32_t precision, cqr2_tune_result_t* out);

/* Tune the batch routing limit for batches of `count` problems of width n
 * (1 <= n <= 64): times the same batch through the grouped kernel and
 * through plans on 4 streams for m = max(n, 64), doubling while the grouped
 * launch is at least as fast (up to about 4 GB of scratch, so the result is a
 * lower bound when the grouped launch still wins there), and sets the limit
 * on m n^2 used by batches created later (cfg NULL) to the largest m n^2
 * where it was; 0 if it never was. *limit_out receives it. Synchronizes;
 * allocates. */
cqr2_status_t cqr2_autotune_batch(int64_t n, int32_t count, int64_t* limit_out);

/* Set the batch routing limit on m n^2 used by batches created later. */
cqr2_status_t cqr2_tune_set_small_limit(int64_t limit);

/* Write the tuning table as text into buf (NUL-terminated, truncated to
 * size); returns the size needed including the NUL. */
int64_t cqr2_tune_table(char* buf, int64_t size);

/* ---- Allocation-free Gram ---- */

/* Fixed device scratch of cqr2_syrk_noalloc (32 MiB per GPU) and the largest
 * n it serves. */
#define CQR2_NOALLOC_SCRATCH_BYTES (32u << 20)
#define CQR2_NOALLOC_MAX_N 2816

/* W = A^T A, the same Gram as cqr2_syrk, for callers that cannot allocate
 * device memory. The paper has no counterpart: it exists because some
 * callers must not call cudaMalloc, for example a host program that hands all
 * device memory to its own pool allocator up front, or code running where a
 * device allocation could fail under memory pressure or stall other work in
 * the middle of a job. This entry point needs no plan and calls no
 * cudaMalloc, cudaFree or allocating library routine: its split-m partial
 * Gram tiles live in one file-scope device array of
 * CQR2_NOALLOC_SCRATCH_BYTES. A device takes that array when the library's
 * Gram module is first loaded on it (the first Gram kernel of any entry point,
 * or the first cqr2_syrk_noalloc call, there) and holds it until the process
 * exits.
 *   dA: m x n (lda >= m) device input; dW: n x n (ldw >= n) device output,
 *   both triangles written. Both must be device (or managed) memory of the
 *   current device. stream: cudaStream_t as void* (NULL = default).
 *   Errors: CQR2_ERR_INVALID_ARG for null pointers, n < 1, m < n, a bad
 *   leading dimension, or a pointer that is host memory or belongs to another
 *   device; CQR2_ERR_UNSUPPORTED for n > CQR2_NOALLOC_MAX_N (the partial
 *   tiles of one row range would not fit the scratch); CQR2_ERR_CUDA if a
 *   CUDA call fails. Larger m only means fewer row ranges.
 * The first call in a CUDA context looks up the scratch array's device
 * address there (cudaGetSymbolAddress, with that context current) and caches
 * it under the context's unique id, so a new context (another device, a
 * driver-API context, or the primary context again after cudaDeviceReset)
 * gets its own lookup; make that first call before any stream capture. All
 * calls on a device share the one array and it keeps the last call's
 * contents; every entry a call reads is written earlier in the same call, so
 * nothing needs clearing, but calls whose work overlaps on the GPU (other
 * streams, other host threads) race on the array: serialize them. */
cqr2_status_t cqr2_syrk_noalloc(const double* dA, int64_t m, int64_t n, int64_t lda, double* dW, int64_t ldw,
                                void* stream);

/* ---- Host-buffer entry point ---- */

/* CholeskyQR2 of a matrix in HOST memory: copies hA (m x n, lda) to the
 * device, factors it exactly as cqr2_factor, and copies Q (m x n, ldq) and R
 * (n x n, ldr) back. Pinned host buffers give full copy bandwidth; pageable
 * ones work too. The first call allocates device staging for A, Q and R
 * (2 m n + n^2 doubles) that the plan keeps until it is destroyed. Always
 * synchronizes; returns CQR2_ERR_NOT_SPD on breakdown (info may be NULL). */
cqr2_status_t cqr2_factor_host(cqr2_plan_t plan, const double* hA, int64_t lda, double* hQ, int64_t ldq,
                               double* hR, int64_t ldr, cqr2_info_t* info);

/* ---- Measurement ---- */

/* Stages of a factorization timed by the per-plan profiler. With
 * CQR2_FUSED, CQR2_STAGE_QFORM1 also accumulates pass 2's partial Grams and
 * CQR2_STAGE_GRAM2 only sums them. With a split-precision plan, the slicing
 * of the operands into BF16 digits is timed as CQR2_STAGE_SPLIT and the
 * GRAM/QFORM stages hold the tensor-core contractions alone. */
typedef enum {
  CQR2_STAGE_GRAM1 = 0,
  CQR2_STAGE_CHOLINV1 = 1,
  CQR2_STAGE_QFORM1 = 2,
  CQR2_STAGE_GRAM2 = 3,
  CQR2_STAGE_CHOLINV2 = 4,
  CQR2_STAGE_QFORM2 = 5,
  CQR2_STAGE_TRMM = 6,
  CQR2_STAGE_LSTSQ = 7,
  CQR2_STAGE_H2D = 8,
  CQR2_STAGE_D2H = 9,
  CQR2_STAGE_SPLIT = 10,
  CQR2_NUM_STAGES = 11
} cqr2_stage_t;

/* Turn per-stage timing on (1) or off (0) and clear what was recorded. While
 * on, every stage of every call records a CUDA event before and after it on
 * the plan's stream (at most 8192 stage records are kept). Synchronizes. */
cqr2_status_t cqr2_plan_set_profiling(cqr2_plan_t plan, int32_t enable);

/* Synchronize the stream and write, for stages 0..nstages-1, the total
 * milliseconds recorded since profiling was enabled into ms[] and the
 * number of timed instances into count[] (count may be NULL). */
cqr2_status_t cqr2_plan_stage_times(cqr2_plan_t plan, double* ms, int64_t* count, int32_t nstages);

/* Static name of a stage ("gram1", "qform2", ...). */
const char* cqr2_stage_name(int32_t stage);

/* Number of CUDA kernels this library has launched in this process (a CUDA
 * graph replay adds the kernels the graph runs). */
int64_t cqr2_launch_count(void);

/* Human-readable name of a status code (static string). */
const char* cqr2_status_string(cqr2_status_t status);

/* Library version string, e.g. "cqr2 0.1 sm_103a". */
const char* cqr2_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CQR2_H */
