// C ABI of the CholeskyQR2 library: plans, workspace, and the sequencing of
// the kernels of Algorithm CQR2 on the caller's stream.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/cqr2.h"
#include "kernels.h"

using namespace cqr2;

namespace cqr2 {
static std::atomic<int64_t> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launches(int64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
int64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }
}  // namespace cqr2

struct cqr2_plan_st {
  int64_t m = 0, n = 0;  // m is the largest row count the plan serves
  int64_t cm = 0;        // row count of the call in progress (geometry below is for cm)
  int gram_cps = 4;      // Gram CTAs per SM (autotuned knob, 1..GRAM_CPS_MAX)
  int64_t gram_cap = 0;  // row ranges the Gram partials have room for (any cm <= m)
  int inv_depth = 0;         // CholInv levels without Y21 (0: whole inverse)
  // CholeskyQR2 on column panels of width panel_b (0: off): plans for the
  // panels' own CholeskyQR2 (width panel_b, and the narrower last panel) and
  // n x panel_b doubles for the second projection's coefficients
  int64_t panel_b = 0;
  cqr2_plan_st* pan_full = nullptr;
  cqr2_plan_st* pan_tail = nullptr;
  double* pan_C = nullptr;
  double* Tsolve = nullptr;  // block-substitution scratch, ldt x right_solve_temp_cols(n)
  double* skws = nullptr;    // split-k scratch of CholInv's small products
  int64_t ldt = 0;
  int64_t oz_cap = 0;    // same for the split-precision Gram partials
  int precision = CQR2_FP64;
  unsigned flags = 0;
  int device = 0;
  cudaStream_t stream = nullptr;
  GramGeom g;
  bool small = false;  // n <= 256: panel Q-form kernel, Q1 staged in the output Q
  bool fused = false;  // CQR2_FUSED requested and n small enough to fuse
  int64_t gemv_nsplit = 0;
  // device workspace (one allocation)
  char* ws = nullptr;
  size_t ws_bytes = 0;
  double* partial = nullptr;
  double* W = nullptr;
  double* Wk = nullptr;
  double* L = nullptr;
  double* Y = nullptr;
  double* U = nullptr;
  double* R1 = nullptr;
  double* Rf = nullptr;  // final R when the caller passes no R
  double* R0 = nullptr;  // R of the shifted pass (CQR2_SHIFTED)
  double* Rt = nullptr;  // R of the CholeskyQR2 that follows it
  double* Rp = nullptr;
  double* Q1 = nullptr;  // m x n, only when !small
  double* lspart = nullptr;
  DevStatus* st = nullptr;
  DevStatus* h_st = nullptr;  // pinned host copy
  // device staging for cqr2_factor_host (allocated on its first call)
  double* hA_dev = nullptr;
  double* lsQ = nullptr;  // Q of least-squares calls given no dQ (m x n, on demand)
  double* hQ_dev = nullptr;
  double* hR_dev = nullptr;
  // cqr2_factor_host overlaps its copies with the factorization: A arrives
  // in row blocks on a copy stream while the pass-1 Gram consumes them, and
  // Q leaves block by block as the last Q-form writes it.
  cudaStream_t copy_stream = nullptr;
  double* hx_partial = nullptr;  // Gram partials of the row blocks (HX_BLOCKS x hx_cap ranges)
  int64_t hx_cap = 0;
  std::vector<cudaEvent_t> hx_ev;  // [0, HX_BLOCKS): A block in; [HX_BLOCKS, 2 HX_BLOCKS): Q block out; 2 more
  struct {
    bool on = false;         // a host-buffer call is in progress
    bool a_pending = false;  // A's blocks are still in flight (no kernel has waited for them)
    bool q_sent = false;     // Q has been copied out block by block
    double* hQ = nullptr;
    int64_t ldq = 0;
  } hx;
  // split-precision (Ozaki) path
  int oz_S = 0;     // slices per entry, 0 = native FP64
  int oz_Scap = 0;  // slices the planes have room for (7 for a 6-slice plan, which may route to 7)
  int* oz_gate = nullptr;  // device: slice count the current factorization uses (6-slice plans)
  unsigned short* oz_planes = nullptr;
  unsigned short* oz_rinv = nullptr;
  unsigned long long* oz_colmax = nullptr;
  int* oz_cexp = nullptr;
  int* oz_fexp = nullptr;
  double* oz_partial = nullptr;
  OzMaps oz_maps;
  // CUDA graph of the last factorization (CQR2_GRAPH), keyed by its arguments
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  struct {
    const void* A;
    void* Q;
    void* R;
    int64_t lda, ldq, ldr, m;
  } gkey{};
  int64_t g_kernels = 0;  // kernels in the captured graph
  // per-stage CUDA-event timing
  bool profiling = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_marks;
};

namespace {

constexpr int GRAM_CPS_MAX = 8;

#define TRY(call)                             \
  do {                                        \
    cudaError_t e_ = (call);                  \
    if (e_ != cudaSuccess) return CQR2_ERR_CUDA; \
  } while (0)

// R = op(A) B of two upper-triangular factors (R = R2 R1 of Algorithm CQR2,
// R = R' R0 of the shifted variant); op(A) = A^T when A holds a lower
// Cholesky factor.
cudaError_t r_product(cqr2_plan_st* p, int n, const double* A, int64_t lda, bool a_trans, const double* B,
                      int64_t ldb, double* C, int64_t ldc, cudaStream_t s) {
  if (n <= TRMM_SMALL_MAX) return trmm_upper_small(n, A, lda, a_trans, B, ldb, C, ldc, s);
  return gemm_f64(n, n, n, 1.0, A, lda, B, ldb, 0.0, C, ldc,
                  (a_trans ? GEMM_TA : 0u) | GEMM_A_UPPER | GEMM_B_UPPER | GEMM_C_UPPER | GEMM_BETA0, s, p->skws,
                  cholinv_splitk_doubles());
}

// Copy a column-major rows x cols block: one linear copy when both sides are
// packed (ld == rows), which runs at full link bandwidth, else a pitched copy.
cudaError_t copy_cols(double* dst, int64_t ldd, const double* src, int64_t lds, int64_t rows, int64_t cols,
                      cudaMemcpyKind kind, cudaStream_t s) {
  const size_t colb = (size_t)rows * sizeof(double);
  if (ldd == rows && lds == rows) return cudaMemcpyAsync(dst, src, colb * (size_t)cols, kind, s);
  return cudaMemcpy2DAsync(dst, (size_t)ldd * sizeof(double), src, (size_t)lds * sizeof(double), colb, (size_t)cols,
                           kind, s);
}

cqr2_status_t check_device(const cqr2_plan_st* p) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return CQR2_ERR_CUDA;
  return dev == p->device ? CQR2_OK : CQR2_ERR_INVALID_ARG;
}

constexpr size_t MAX_MARKS = 8192;

cudaEvent_t take_event(cqr2_plan_st* p) {
  if (p->ev_used == p->ev_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    p->ev_pool.push_back(e);
  }
  return p->ev_pool[p->ev_used++];
}

// Records CUDA events around one stage when profiling, on the plan's stream
// or on another one (the host-copy stream).
struct Stage {
  cqr2_plan_st* p;
  int id;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  Stage(cqr2_plan_st* p_, int id_, cudaStream_t s_ = nullptr) : p(p_), id(id_), s(s_ ? s_ : p_->stream) {
    if (p->profiling && p->ev_marks.size() < MAX_MARKS) {
      a = take_event(p);
      if (a) cudaEventRecord(a, s);
    }
  }
  ~Stage() {
    if (!a) return;
    cudaEvent_t b = take_event(p);
    if (!b) return;
    cudaEventRecord(b, s);
    p->ev_marks.push_back({id, {a, b}});
  }
};

// ---- host-buffer calls: row blocks of the copies
constexpr int HX_BLOCKS = 8;
inline int64_t hx_row(int64_t m, int r) { return r == HX_BLOCKS ? m : ((m * r / HX_BLOCKS) & ~(int64_t)63); }

// A kernel about to read A (the host-staged input) as a whole waits for all
// of its blocks first; the blocked pass-1 Gram waits block by block instead.
cudaError_t hx_wait_input(cqr2_plan_st* p, cudaStream_t s) {
  if (!p->hx.on || !p->hx.a_pending) return cudaSuccess;
  p->hx.a_pending = false;
  return cudaStreamWaitEvent(s, p->hx_ev[HX_BLOCKS - 1], 0);
}

// [L, Y] = CholInv(W) of the plan's pass, with the plan's inverse depth.
// [L, Y] = CholInv(W) into the plan's L and Y, and, when given, R = L^T into Rt
// (ld n) and the Q-form's packed R^-1 into Rp.
cudaError_t plan_cholinv(cqr2_plan_st* p, int pass, cudaStream_t s, double* Rt = nullptr, double* Rp = nullptr) {
  const int n = (int)p->n;
  if (p->inv_depth > 0) {
    cudaError_t e = cholinv_depth(n, p->W, n, p->L, n, p->Y, n, p->Wk, p->U, p->Tsolve, p->ldt, p->st, pass,
                                  p->inv_depth, s, p->skws, cholinv_splitk_doubles());
    if (e == cudaSuccess && Rt != nullptr) e = transpose_lower(p->L, n, n, Rt, n, s);
    if (e == cudaSuccess && Rp != nullptr) e = pack_rinv_from_lower(p->Y, n, n, Rp, s);
    return e;
  }
  return cholinv(n, p->W, n, p->L, n, p->Y, n, p->Wk, p->U, p->st, pass, s, p->skws, cholinv_splitk_doubles(), Rt,
                 n, Rp);
}

// X = B R^-1 = B L^-T (general path, rows x n): one triangular multiply by
// the whole inverse, or block forward substitution at inverse depth d > 0.
cudaError_t plan_apply_rinv(cqr2_plan_st* p, int64_t rows, const double* B, int64_t ldb, double* X, int64_t ldx,
                            cudaStream_t s) {
  const int n = (int)p->n;
  if (p->inv_depth > 0)
    return right_solve(rows, n, B, ldb, X, ldx, p->L, n, p->Y, n, p->inv_depth, p->Tsolve, p->ldt, s);
  return gemm_f64(rows, n, n, 1.0, B, ldb, p->Y, n, 0.0, X, ldx, GEMM_TB | GEMM_B_UPPER | GEMM_BETA0, s);
}

cqr2_status_t read_info(cqr2_plan_st* p, cqr2_info_t* info) {
  TRY(cudaMemcpyAsync(p->h_st, p->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, p->stream));
  TRY(cudaStreamSynchronize(p->stream));
  const int st = p->h_st->status;
  info->status = st == 0 ? CQR2_OK : (st == 5 ? CQR2_ERR_TIMEOUT : CQR2_ERR_NOT_SPD);
  info->failed_pass = st == 2 ? p->h_st->pass : 0;
  info->failed_pivot = st == 2 ? p->h_st->pivot : -1;
  info->pivot_value = st == 2 ? p->h_st->value : 0.0;
  return (cqr2_status_t)info->status;
}

}  // namespace

cudaError_t cqr2::plan_status_copy(cqr2_plan_st* p, DevStatus* dst, cudaStream_t s) {
  return cudaMemcpyAsync(dst, p->st, sizeof(DevStatus), cudaMemcpyDeviceToDevice, s);
}

namespace {

// Prepares the plan's launch geometry for an m-row call (m <= plan m).
cqr2_status_t set_rows(cqr2_plan_st* p, int64_t m) {
  if (m < p->n || m > p->m) return CQR2_ERR_INVALID_ARG;
  if (m == p->cm) return CQR2_OK;
  p->g = gram_geometry(m, (int)p->n, p->gram_cap, p->gram_cps);
  p->gemv_nsplit = gemv_splits(m, (int)p->n);
  if (p->oz_S && ozaki_make_maps(p->oz_maps, m, (int)p->n, p->oz_Scap, p->oz_planes, p->oz_rinv) != cudaSuccess) {
    p->cm = 0;
    return CQR2_ERR_CUDA;
  }
  p->cm = m;
  return CQR2_OK;
}

// Split-precision CholeskyQR2: the Gram and Q-forming contractions on the
// BF16 tensor cores (Ozaki slices), CholInv and R2 R1 in native FP64.
// A 6-slice plan routes on the device by the columns' crest ratios (scale
// over root-mean-square, ozaki_route). Pass 1 runs its Gram with 6 slices
// (that Gram only sets how well conditioned Q1 is), then checks A's columns
// with the norms from W's diagonal; where a ratio is above 16 it re-slices A
// with 7 slices for its Q-form. Pass 2 checks Q1's columns (unit norm) before
// slicing, keeping an earlier 7, so its Gram -- which sets Q's orthogonality
// -- and its Q-form use the chosen count. Both variants of each routed step
// are launched and the one the gate does not select returns at once, so the
// host never waits for the decision.
cqr2_status_t factor_impl_ozaki(cqr2_plan_st* p, const double* dA, int64_t lda, double* dQ, int64_t ldq, double* dR,
                                int64_t ldr, int pass_base = 0) {
  const int n = (int)p->n, S = p->oz_S;
  const int64_t m = p->cm;
  cudaStream_t s = p->stream;
  const bool route = S == 6;
  const int* gate = route ? p->oz_gate : nullptr;
  if (!pass_base) TRY(cudaMemsetAsync(p->st, 0, sizeof(DevStatus), s));
  TRY(hx_wait_input(p, s));
  // Up to OZAKI_FUSED_COLMAX_MAX_N columns the pass-1 Q-form also folds Q1's
  // column maxima into oz_colmax, so pass 2 skips the column-max sweep.
  const bool fused_cmax = n <= OZAKI_FUSED_COLMAX_MAX_N;
  // launch a gated step for both slice counts (6-slice plans) or once
  auto each = [&](auto&& step) -> cudaError_t {
    if (!route) return step(S, (const int*)nullptr);
    cudaError_t e = step(6, gate);
    return e == cudaSuccess ? step(7, gate) : e;
  };
  for (int pass = 1; pass <= 2; ++pass) {
    const double* X = pass == 1 ? dA : dQ;
    const int64_t ldx = pass == 1 ? lda : ldq;
    {
      Stage st(p, CQR2_STAGE_SPLIT);
      if (pass == 2 && fused_cmax) {
        TRY(ozaki_exps(p->oz_colmax, n, p->oz_cexp, s));
      } else {
        TRY(ozaki_colmax(X, ldx, m, n, p->oz_colmax, p->oz_cexp, s));
      }
      if (pass == 1 || !route) {
        TRY(ozaki_slice_cols(X, ldx, m, n, S, p->oz_cexp, p->oz_planes, s));
      } else {
        TRY(ozaki_route(p->oz_cexp, nullptr, n, n, m, p->oz_gate, true, s));
        TRY(each([&](int Sx, const int* g) {
          return ozaki_slice_cols(X, ldx, m, n, Sx, p->oz_cexp, p->oz_planes, s, g);
        }));
      }
    }
    {
      Stage st(p, pass == 1 ? CQR2_STAGE_GRAM1 : CQR2_STAGE_GRAM2);
      if (pass == 1 || !route) {
        TRY(ozaki_gram(p->oz_maps, m, n, S, p->oz_cexp, p->oz_partial, p->oz_cap, p->W, n, p->st, s));
      } else {
        TRY(each([&](int Sx, const int* g) {
          return ozaki_gram(p->oz_maps, m, n, Sx, p->oz_cexp, p->oz_partial, p->oz_cap, p->W, n, p->st, s, g);
        }));
      }
    }
    if (route && pass == 1) {
      Stage st(p, CQR2_STAGE_SPLIT);
      TRY(ozaki_route(p->oz_cexp, p->W, n, n, m, p->oz_gate, false, s));
      // routed to 7: A again in 7 slices for this pass's Q-form
      TRY(ozaki_slice_cols(X, ldx, m, n, 7, p->oz_cexp, p->oz_planes, s, gate));
    }
    {
      Stage st(p, pass == 1 ? CQR2_STAGE_CHOLINV1 : CQR2_STAGE_CHOLINV2);
      TRY(plan_cholinv(p, pass_base + pass, s, pass == 1 ? p->R1 : nullptr));  // R1 = L1^T
    }
    {
      Stage st(p, CQR2_STAGE_SPLIT);
      TRY(each([&](int Sx, const int* g) {
        return ozaki_slice_rinv(p->Y, n, n, Sx, false, p->oz_cexp, p->oz_rinv, p->oz_fexp, s, g);
      }));
    }
    {
      // The Q-form reads only the slices of X, so pass 2 may overwrite Q1 in place.
      Stage st(p, pass == 1 ? CQR2_STAGE_QFORM1 : CQR2_STAGE_QFORM2);
      const bool cm = pass == 1 && fused_cmax;
      if (cm) TRY(cudaMemsetAsync(p->oz_colmax, 0, (size_t)n * sizeof(unsigned long long), s));
      TRY(each([&](int Sx, const int* g) {
        return ozaki_qform(p->oz_maps, m, n, Sx, p->oz_fexp, dQ, ldq, p->st, s, cm ? p->oz_colmax : nullptr, g);
      }));
    }
  }
  {
    Stage st(p, CQR2_STAGE_TRMM);
    TRY(r_product(p, n, p->L, n, true, p->R1, n, dR, ldr, s));
  }
  return CQR2_OK;
}

cqr2_status_t factor_impl(cqr2_plan_st* p, const double* dA, int64_t lda, double* dQ, int64_t ldq, double* dR,
                          int64_t ldr, int pass_base = 0) {
  if (p->oz_S) return factor_impl_ozaki(p, dA, lda, dQ, ldq, dR, ldr, pass_base);
  const int n = (int)p->n;
  cudaStream_t s = p->stream;
  if (!pass_base) TRY(cudaMemsetAsync(p->st, 0, sizeof(DevStatus), s));
  // ---- pass 1: W1 = A^T A, [L1, Y1] = CholInv(W1)
  {
    Stage st(p, CQR2_STAGE_GRAM1);
    if (p->hx.on && p->hx.a_pending && pass_base == 0) {
      // A is arriving in row blocks: each block's row ranges go to their own
      // partials as soon as the block has landed; one fixed-order sum follows.
      const int64_t per_split = (int64_t)p->g.ntiles_total * p->g.T * p->g.T;
      int64_t used = 0;
      for (int b = 0; b < HX_BLOCKS; ++b) {
        const int64_t r0 = hx_row(p->cm, b), r1 = hx_row(p->cm, b + 1);
        TRY(cudaStreamWaitEvent(s, p->hx_ev[b], 0));
        if (r1 <= r0) continue;
        const GramGeom gr = gram_geometry(r1 - r0, n, p->hx_cap, p->gram_cps);
        TRY(gram_partials(dA + r0, lda, r1 - r0, n, gr, p->hx_partial + used * per_split, s));
        used += gr.nsplit;
      }
      p->hx.a_pending = false;
      GramGeom gall = p->g;
      gall.nsplit = used;
      TRY(gram_reduce(p->hx_partial, gall, n, p->W, n, s));
    } else {
      TRY(hx_wait_input(p, s));
      TRY(gram_partials(dA, lda, p->cm, n, p->g, p->partial, s));
      TRY(gram_reduce(p->partial, p->g, n, p->W, n, s));
    }
  }
  {
    Stage st(p, CQR2_STAGE_CHOLINV1);
    // R1 = L1^T, and on the small path R1^-1 packed for the Q-form
    TRY(plan_cholinv(p, pass_base + 1, s, p->R1, p->small ? p->Rp : nullptr));
  }
  // ---- Q1 = A R1^-1 (staged in dQ on the small path), then pass 2 on Q1
  const double* X2 = dQ;
  int64_t ldx2 = ldq;
  if (p->small) {
    Stage st(p, CQR2_STAGE_QFORM1);
    if (p->fused) {
      // Q1 and the partial Grams of Q1 in one sweep over A
      TRY(qform_gram_small(dA, lda, p->cm, n, p->Rp, dQ, ldq, p->g, p->partial, s));
    } else {
      TRY(qform_small(dA, lda, p->cm, n, p->Rp, dQ, ldq, s));
    }
  } else {
    Stage st(p, CQR2_STAGE_QFORM1);
    TRY(plan_apply_rinv(p, p->cm, dA, lda, p->Q1, p->m, s));
    X2 = p->Q1;
    ldx2 = p->m;
  }
  {
    Stage st(p, CQR2_STAGE_GRAM2);
    if (!p->fused) TRY(gram_partials(X2, ldx2, p->cm, n, p->g, p->partial, s));
    TRY(gram_reduce(p->partial, p->g, n, p->W, n, s));
  }
  {
    Stage st(p, CQR2_STAGE_CHOLINV2);
    TRY(plan_cholinv(p, pass_base + 2, s, nullptr, p->small ? p->Rp : nullptr));
  }
  {
    Stage st(p, CQR2_STAGE_QFORM2);
    // Host-buffer call: the last Q-form runs by row blocks, each copied out on
    // the copy stream while the next block is formed.
    const int nb = p->hx.on ? HX_BLOCKS : 1;
    for (int b = 0; b < nb; ++b) {
      const int64_t r0 = nb == 1 ? 0 : hx_row(p->cm, b), r1 = nb == 1 ? p->cm : hx_row(p->cm, b + 1);
      if (r1 > r0) {
        if (p->small) {
          TRY(qform_small(dQ + r0, ldq, r1 - r0, n, p->Rp, dQ + r0, ldq, s));  // in place, panel by panel
        } else {
          TRY(plan_apply_rinv(p, r1 - r0, X2 + r0, ldx2, dQ + r0, ldq, s));
        }
      }
      if (p->hx.on) {
        cudaEvent_t ev = p->hx_ev[HX_BLOCKS + b];
        TRY(cudaEventRecord(ev, s));
        TRY(cudaStreamWaitEvent(p->copy_stream, ev, 0));
        if (r1 > r0) {
          Stage sd(p, CQR2_STAGE_D2H, p->copy_stream);
          TRY(cudaMemcpy2DAsync(p->hx.hQ + r0, (size_t)p->hx.ldq * sizeof(double), dQ + r0, (size_t)ldq * sizeof(double),
                                (size_t)(r1 - r0) * sizeof(double), (size_t)n, cudaMemcpyDeviceToHost, p->copy_stream));
        }
      }
    }
    if (p->hx.on) p->hx.q_sent = true;
  }
  // ---- R = R2 R1 with R2 = L2^T
  {
    Stage st(p, CQR2_STAGE_TRMM);
    TRY(r_product(p, n, p->L, n, true, p->R1, n, dR, ldr, s));
  }
  return CQR2_OK;
}

// CholeskyQR2, or with CQR2_SHIFTED shifted CholeskyQR3: a shifted first
// pass (W = A^T A + s I, [L0, Y0] = CholInv(W), Q0 = A Y0^T staged in Q),
// CholeskyQR2 of Q0 in place (its passes report as 2 and 3), R = R' R0.
cqr2_status_t factor_any(cqr2_plan_st* p, const double* dA, int64_t lda, double* dQ, int64_t ldq, double* dR,
                         int64_t ldr);

// CholeskyQR2 on column panels (Section V names a CholeskyQR2 that works on
// subpanels, to cut the extra computation near-square matrices cost, as
// future work; this is the library's reading of it). Left to right, each
// panel of b columns is copied into its place in Q, projected twice against
// the panels before it (block Gram-Schmidt with one reorthogonalisation:
// C = Q_<k^T V, V -= Q_<k C, twice, R's block above the diagonal gets the sum
// of both C), and factored by CholeskyQR2 in place, which gives its Q columns
// and R's diagonal block. CholInv then only ever sees b x b Gram matrices,
// instead of the whole n x n ones (twice) and R2 R1 of plain CQR2.
cqr2_status_t factor_panels(cqr2_plan_st* p, const double* dA, int64_t lda, double* dQ, int64_t ldq, double* dR,
                            int64_t ldr) {
  const int64_t n = p->n, m = p->cm, b = p->panel_b;
  cudaStream_t s = p->stream;
  TRY(cudaMemsetAsync(p->st, 0, sizeof(DevStatus), s));
  TRY(hx_wait_input(p, s));
  // R's strictly lower part stays zero; its blocks are written panel by panel
  TRY(cudaMemset2DAsync(dR, (size_t)ldr * sizeof(double), 0, (size_t)n * sizeof(double), (size_t)n, s));
  for (int64_t c0 = 0; c0 < n; c0 += b) {
    const int64_t bk = std::min(b, n - c0);
    cqr2_plan_st* in = bk == b ? p->pan_full : p->pan_tail;
    double* Qk = dQ + c0 * ldq;
    if (dQ != dA) TRY(copy_cols(Qk, ldq, dA + c0 * lda, lda, m, bk, cudaMemcpyDeviceToDevice, s));
    if (c0 > 0) {
      double* Rk = dR + c0 * ldr;  // R(0:c0, c0:c0+bk)
      TRY(gemm_f64(c0, bk, m, 1.0, dQ, ldq, Qk, ldq, 0.0, Rk, ldr, GEMM_TA | GEMM_BETA0, s, p->skws,
                   cholinv_splitk_doubles()));
      TRY(gemm_f64(m, bk, c0, -1.0, dQ, ldq, Rk, ldr, 1.0, Qk, ldq, 0, s));
      TRY(gemm_f64(c0, bk, m, 1.0, dQ, ldq, Qk, ldq, 0.0, p->pan_C, c0, GEMM_TA | GEMM_BETA0, s, p->skws,
                   cholinv_splitk_doubles()));
      TRY(gemm_f64(m, bk, c0, -1.0, dQ, ldq, p->pan_C, c0, 1.0, Qk, ldq, 0, s));
      TRY(add_block(p->pan_C, c0, Rk, ldr, c0, bk, s));
    }
    in->stream = s;
    cqr2_status_t r = set_rows(in, m);
    if (r != CQR2_OK) return r;
    if ((r = factor_any(in, Qk, ldq, Qk, ldq, dR + c0 + c0 * ldr, ldr)) != CQR2_OK) return r;
    TRY(status_merge(p->st, in->st, c0, s));
  }
  return CQR2_OK;
}

cqr2_status_t factor_any(cqr2_plan_st* p, const double* dA, int64_t lda, double* dQ, int64_t ldq, double* dR,
                         int64_t ldr) {
  if (p->panel_b) return factor_panels(p, dA, lda, dQ, ldq, dR, ldr);
  if (!(p->flags & CQR2_SHIFTED)) return factor_impl(p, dA, lda, dQ, ldq, dR, ldr, 0);
  const int n = (int)p->n;
  const int64_t m = p->cm;
  cudaStream_t s = p->stream;
  TRY(cudaMemsetAsync(p->st, 0, sizeof(DevStatus), s));
  TRY(hx_wait_input(p, s));
  {
    Stage st(p, CQR2_STAGE_GRAM1);
    if (p->oz_S) {
      TRY(ozaki_colmax(dA, lda, m, n, p->oz_colmax, p->oz_cexp, s));
      TRY(ozaki_slice_cols(dA, lda, m, n, p->oz_S, p->oz_cexp, p->oz_planes, s));
      TRY(ozaki_gram(p->oz_maps, m, n, p->oz_S, p->oz_cexp, p->oz_partial, p->oz_cap, p->W, n, p->st, s));
    } else {
      TRY(gram_partials(dA, lda, m, n, p->g, p->partial, s));
      TRY(gram_reduce(p->partial, p->g, n, p->W, n, s));
    }
    TRY(add_shift(p->W, n, n, m, s));
  }
  {
    Stage st(p, CQR2_STAGE_CHOLINV1);
    TRY(plan_cholinv(p, 1, s, p->R0));  // R0 = L0^T
  }
  {
    Stage st(p, CQR2_STAGE_QFORM1);
    if (p->oz_S) {
      TRY(ozaki_slice_rinv(p->Y, n, n, p->oz_S, false, p->oz_cexp, p->oz_rinv, p->oz_fexp, s));
      TRY(ozaki_qform(p->oz_maps, m, n, p->oz_S, p->oz_fexp, dQ, ldq, p->st, s));
    } else if (p->small) {
      TRY(pack_rinv_from_lower(p->Y, n, n, p->Rp, s));
      TRY(qform_small(dA, lda, m, n, p->Rp, dQ, ldq, s));
    } else if ((const void*)dA == (const void*)dQ) {
      // in place: the tiled multiply may not write over its input, so Q0 is
      // formed in the workspace and copied over A
      TRY(plan_apply_rinv(p, m, dA, lda, p->Q1, p->m, s));
      TRY(cudaMemcpy2DAsync(dQ, (size_t)ldq * sizeof(double), p->Q1, (size_t)p->m * sizeof(double),
                            (size_t)m * sizeof(double), (size_t)n, cudaMemcpyDeviceToDevice, s));
    } else {
      TRY(plan_apply_rinv(p, m, dA, lda, dQ, ldq, s));
    }
  }
  cqr2_status_t r = factor_impl(p, dQ, ldq, dQ, ldq, p->Rt, n, 1);
  if (r != CQR2_OK) return r;
  Stage st(p, CQR2_STAGE_TRMM);
  TRY(r_product(p, n, p->Rt, n, false, p->R0, n, dR, ldr, s));
  return CQR2_OK;
}

bool bad_ld(int64_t ld, int64_t rows) { return ld < std::max<int64_t>(1, rows); }

// Q may be A itself only on a CQR2_INPLACE plan, with the same leading dimension.
bool bad_alias(const cqr2_plan_st* p, const double* dA, int64_t lda, const double* dQ, int64_t ldq) {
  if ((const void*)dA != (const void*)dQ) return false;
  return !(p->flags & CQR2_INPLACE) || lda != ldq;
}

size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

extern "C" {

const char* cqr2_status_string(cqr2_status_t s) {
  switch (s) {
    case CQR2_OK: return "CQR2_OK";
    case CQR2_ERR_INVALID_ARG: return "CQR2_ERR_INVALID_ARG";
    case CQR2_ERR_NOT_SPD: return "CQR2_ERR_NOT_SPD";
    case CQR2_ERR_CUDA: return "CQR2_ERR_CUDA";
    case CQR2_ERR_OOM: return "CQR2_ERR_OOM";
    case CQR2_ERR_TIMEOUT: return "CQR2_ERR_TIMEOUT";
    case CQR2_ERR_UNSUPPORTED: return "CQR2_ERR_UNSUPPORTED";
  }
  return "CQR2_ERR_UNKNOWN";
}

const char* cqr2_version(void) { return "cqr2 0.1 sm_103a"; }

cqr2_status_t cqr2_plan_create(cqr2_plan_t* plan, int64_t m, int64_t n, int32_t precision, uint32_t flags,
                               void* stream) {
  if (!plan) return CQR2_ERR_INVALID_ARG;
  *plan = nullptr;
  if (n < 1 || m < n || n > 65535) return CQR2_ERR_INVALID_ARG;
  if (precision != CQR2_FP64 && precision != CQR2_OZAKI_BF16 && precision != CQR2_OZAKI_BF16_S6)
    return CQR2_ERR_INVALID_ARG;
  if (flags & ~(CQR2_FUSED | CQR2_GRAPH | CQR2_SHIFTED | CQR2_INPLACE)) return CQR2_ERR_INVALID_ARG;
  const int oz_S = precision == CQR2_OZAKI_BF16 ? 7 : (precision == CQR2_OZAKI_BF16_S6 ? 6 : 0);
  if (oz_S && !ozaki_supported((int)n, oz_S)) return CQR2_ERR_UNSUPPORTED;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CQR2_ERR_CUDA;
  auto* p = new (std::nothrow) cqr2_plan_st();
  if (!p) return CQR2_ERR_OOM;
  p->m = m;
  p->n = n;
  p->precision = precision;
  p->flags = flags;
  p->device = dev;
  p->stream = static_cast<cudaStream_t>(stream);
  // Size the Gram partials for every row count the plan serves: a smaller m
  // can round to more (shorter) ranges than m itself, up to the CTA target.
  p->g = gram_geometry(m, (int)n, 0, GRAM_CPS_MAX);
  {
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    p->gram_cap = std::max<int64_t>(p->g.nsplit, ceil_div((int64_t)GRAM_CPS_MAX * sms, p->g.ntiles_total));
    p->g.nsplit = p->gram_cap;
  }
  p->small = qform_group_width((int)n) > 0;
  p->fused = (flags & CQR2_FUSED) && qform_gram_fusable((int)n);
  p->gemv_nsplit = gemv_splits(m, (int)n);
  p->oz_S = oz_S;
  const size_t nn = (size_t)n * n * sizeof(double);
  OzGeom og;
  if (oz_S) {
    og = ozaki_geometry(m, (int)n);
    p->oz_cap = ozaki_split_capacity(m, (int)n);
    p->oz_Scap = oz_S == 6 ? 7 : oz_S;
    p->small = false;  // no m x n FP64 workspace: Q1 is staged in the output Q
    p->fused = false;
  }
  size_t off[24];
  size_t sz = 0;
  int k = 0;
  auto take = [&](size_t bytes) {
    off[k++] = sz;
    sz += align_up(bytes);
  };
  take(p->g.partial_doubles() * sizeof(double));                     // 0 partial
  take(nn);                                                          // 1 W
  take(nn);                                                          // 2 Wk
  take(nn);                                                          // 3 L
  take(nn);                                                          // 4 Y
  take(nn);                                                          // 5 U
  take(nn);                                                          // 6 R1
  take(nn);                                                          // 7 Rf
  take(rpack_doubles((int)n) * sizeof(double));                      // 8 Rp
  take((p->small || oz_S) ? 0 : (size_t)m * n * sizeof(double));    // 9 Q1
  take((size_t)p->gemv_nsplit * n * sizeof(double));                 // 10 lspart
  take(sizeof(DevStatus));                                           // 11 st
  take(nn);                                                          // 12 R0
  take(nn);                                                          // 13 Rt
  if (oz_S) {
    take(ozaki_plane_elems(m, (int)n, p->oz_Scap) * 2);              // 14 slice planes (bf16)
    take((size_t)p->oz_Scap * n * og.np * 2);                        // 15 R^-1 planes
    take((size_t)n * sizeof(unsigned long long));                    // 16 column max
    take((size_t)n * sizeof(int));                                   // 17 column exponents
    take(sizeof(int));                                               // 18 slice-count gate
    take((size_t)n * sizeof(int));                                   // 19 R^-1 exponents
    take((size_t)p->oz_cap * n * n * sizeof(double));                // 20 Gram partials
  }
  const int i_sk = k;
  take(cholinv_splitk_doubles() * sizeof(double));                   // split-k scratch of CholInv
  if (cudaMalloc(&p->ws, sz) != cudaSuccess) {
    cudaGetLastError();
    delete p;
    return CQR2_ERR_OOM;
  }
  if (cudaMallocHost(&p->h_st, sizeof(DevStatus)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(p->ws);
    delete p;
    return CQR2_ERR_OOM;
  }
  p->ws_bytes = sz;
  auto at = [&](int i) { return reinterpret_cast<double*>(p->ws + off[i]); };
  p->partial = at(0);
  p->W = at(1);
  p->Wk = at(2);
  p->L = at(3);
  p->Y = at(4);
  p->U = at(5);
  p->R1 = at(6);
  p->Rf = at(7);
  p->R0 = at(12);
  p->Rt = at(13);
  p->Rp = at(8);
  p->Q1 = p->small ? nullptr : at(9);
  p->lspart = at(10);
  p->st = reinterpret_cast<DevStatus*>(p->ws + off[11]);
  p->skws = at(i_sk);
  if (oz_S) {
    p->oz_planes = reinterpret_cast<unsigned short*>(p->ws + off[14]);
    p->oz_rinv = reinterpret_cast<unsigned short*>(p->ws + off[15]);
    p->oz_colmax = reinterpret_cast<unsigned long long*>(p->ws + off[16]);
    p->oz_cexp = reinterpret_cast<int*>(p->ws + off[17]);
    p->oz_fexp = reinterpret_cast<int*>(p->ws + off[19]);
    p->oz_gate = reinterpret_cast<int*>(p->ws + off[18]);
    p->oz_partial = at(20);
    // zero the planes once so that padding rows/columns read as zero
    if (cudaMemsetAsync(p->oz_planes, 0, ozaki_plane_elems(m, (int)n, p->oz_Scap) * 2, p->stream) != cudaSuccess ||
        cudaMemsetAsync(p->oz_rinv, 0, (size_t)p->oz_Scap * n * og.np * 2, p->stream) != cudaSuccess ||
        cudaMemsetAsync(p->oz_gate, 0, sizeof(int), p->stream) != cudaSuccess ||
        ozaki_make_maps(p->oz_maps, m, (int)n, p->oz_Scap, p->oz_planes, p->oz_rinv) != cudaSuccess) {
      cudaGetLastError();
      cudaFreeHost(p->h_st);
      cudaFree(p->ws);
      delete p;
      return CQR2_ERR_CUDA;
    }
  }
  p->g = gram_geometry(m, (int)n, p->gram_cap, p->gram_cps);
  p->cm = m;  // geometry and tensor maps above are for the full row count
  std::memset(p->h_st, 0, sizeof(DevStatus));
  if (cudaMemsetAsync(p->st, 0, sizeof(DevStatus), p->stream) != cudaSuccess) {
    cudaFreeHost(p->h_st);
    cudaFree(p->ws);
    delete p;
    return CQR2_ERR_CUDA;
  }
  *plan = p;
  return CQR2_OK;
}

size_t cqr2_workspace_bytes(cqr2_plan_t plan) { return plan ? plan->ws_bytes : 0; }

cqr2_status_t cqr2_plan_set_stream(cqr2_plan_t plan, void* stream) {
  if (!plan) return CQR2_ERR_INVALID_ARG;
  plan->stream = static_cast<cudaStream_t>(stream);
  return CQR2_OK;
}

void cqr2_plan_destroy(cqr2_plan_t plan) {
  if (!plan) return;
  cudaStreamSynchronize(plan->stream);
  cqr2_plan_destroy(plan->pan_full);
  cqr2_plan_destroy(plan->pan_tail);
  cudaFree(plan->pan_C);
  for (cudaEvent_t e : plan->ev_pool) cudaEventDestroy(e);
  if (plan->gexec) cudaGraphExecDestroy(plan->gexec);
  if (plan->graph) cudaGraphDestroy(plan->graph);
  if (plan->copy_stream) {
    cudaStreamSynchronize(plan->copy_stream);
    cudaStreamDestroy(plan->copy_stream);
  }
  for (cudaEvent_t e : plan->hx_ev) cudaEventDestroy(e);
  cudaFree(plan->hx_partial);
  cudaFree(plan->Tsolve);
  cudaFree(plan->hA_dev);
  cudaFree(plan->lsQ);
  cudaFree(plan->hQ_dev);
  cudaFree(plan->hR_dev);
  cudaFree(plan->ws);
  cudaFreeHost(plan->h_st);
  delete plan;
}

cqr2_status_t cqr2_plan_info(cqr2_plan_t plan, cqr2_info_t* info) {
  if (!plan || !info) return CQR2_ERR_INVALID_ARG;
  return read_info(plan, info);
}

cqr2_status_t cqr2_plan_set_panel_width(cqr2_plan_t p, int64_t b) {
  if (!p || b < 0) return CQR2_ERR_INVALID_ARG;
  if (b > 0 && b < p->n && (p->oz_S || (p->flags & CQR2_SHIFTED))) return CQR2_ERR_UNSUPPORTED;
  if (check_device(p) != CQR2_OK) return CQR2_ERR_INVALID_ARG;
  if (b >= p->n) b = 0;  // one panel is plain CholeskyQR2
  if (b == p->panel_b) return CQR2_OK;
  if (cudaStreamSynchronize(p->stream) != cudaSuccess) return CQR2_ERR_CUDA;
  cqr2_plan_destroy(p->pan_full);
  cqr2_plan_destroy(p->pan_tail);
  cudaFree(p->pan_C);
  p->pan_full = p->pan_tail = nullptr;
  p->pan_C = nullptr;
  p->panel_b = 0;
  if (b == 0) return CQR2_OK;
  const int64_t tail = p->n % b;
  const uint32_t fl = CQR2_INPLACE | CQR2_FUSED;
  cqr2_status_t r = cqr2_plan_create(&p->pan_full, p->m, b, CQR2_FP64, fl, p->stream);
  if (r == CQR2_OK && tail) r = cqr2_plan_create(&p->pan_tail, p->m, tail, CQR2_FP64, fl, p->stream);
  if (r == CQR2_OK && cudaMalloc(&p->pan_C, (size_t)p->n * b * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    r = CQR2_ERR_OOM;
  }
  if (r != CQR2_OK) {
    cqr2_plan_destroy(p->pan_full);
    cqr2_plan_destroy(p->pan_tail);
    cudaFree(p->pan_C);
    p->pan_full = p->pan_tail = nullptr;
    p->pan_C = nullptr;
    return r;
  }
  if (p->gexec) {  // a captured graph of the unpaneled sequence no longer applies
    cudaGraphExecDestroy(p->gexec);
    cudaGraphDestroy(p->graph);
    p->gexec = nullptr;
    p->graph = nullptr;
  }
  p->panel_b = b;
  return CQR2_OK;
}

cqr2_status_t cqr2_plan_split_slices(cqr2_plan_t plan, int32_t* slices) {
  if (!plan || !slices) return CQR2_ERR_INVALID_ARG;
  if (plan->oz_S != 6) {
    *slices = plan->oz_S;
    return CQR2_OK;
  }
  int g = 0;
  if (cudaMemcpyAsync(&g, plan->oz_gate, sizeof(int), cudaMemcpyDeviceToHost, plan->stream) != cudaSuccess ||
      cudaStreamSynchronize(plan->stream) != cudaSuccess)
    return CQR2_ERR_CUDA;
  *slices = g;
  return CQR2_OK;
}

cqr2_status_t cqr2_factor_rows(cqr2_plan_t p, int64_t m, const double* dA, int64_t lda, double* dQ, int64_t ldq,
                               double* dR, int64_t ldr, cqr2_info_t* info) {
  if (!p || !dA || !dQ || !dR) return CQR2_ERR_INVALID_ARG;
  if (m < p->n || m > p->m) return CQR2_ERR_INVALID_ARG;
  if (bad_ld(lda, m) || bad_ld(ldq, m) || bad_ld(ldr, p->n)) return CQR2_ERR_INVALID_ARG;
  if (bad_alias(p, dA, lda, dQ, ldq)) return CQR2_ERR_INVALID_ARG;
  cqr2_status_t r = check_device(p);
  if (r != CQR2_OK) return r;
  if ((r = set_rows(p, m)) != CQR2_OK) return r;
  if ((p->flags & CQR2_GRAPH) && p->stream && !p->profiling) {
    // Replay the captured launch sequence when the arguments repeat;
    // otherwise capture this call's sequence into a new graph first.
    const bool same = p->gexec && p->gkey.A == dA && p->gkey.Q == dQ && p->gkey.R == dR && p->gkey.lda == lda &&
                      p->gkey.ldq == ldq && p->gkey.ldr == ldr && p->gkey.m == m;
    if (!same) {
      if (p->gexec) cudaGraphExecDestroy(p->gexec);
      if (p->graph) cudaGraphDestroy(p->graph);
      p->gexec = nullptr;
      p->graph = nullptr;
      TRY(cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal));
      const int64_t l0 = launch_count();
      r = factor_any(p, dA, lda, dQ, ldq, dR, ldr);
      p->g_kernels = launch_count() - l0;  // counted once here, and again at every replay
      cudaGraph_t g = nullptr;
      const cudaError_t ce = cudaStreamEndCapture(p->stream, &g);
      if (r != CQR2_OK || ce != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return r != CQR2_OK ? r : CQR2_ERR_CUDA;
      }
      if (cudaGraphInstantiate(&p->gexec, g, 0) != cudaSuccess) {
        cudaGraphDestroy(g);
        p->gexec = nullptr;
        return CQR2_ERR_CUDA;
      }
      p->graph = g;
      p->gkey.A = dA;
      p->gkey.Q = dQ;
      p->gkey.R = dR;
      p->gkey.lda = lda;
      p->gkey.ldq = ldq;
      p->gkey.ldr = ldr;
      p->gkey.m = m;
    }
    if (same) count_launches(p->g_kernels);
    TRY(cudaGraphLaunch(p->gexec, p->stream));
  } else if ((r = factor_any(p, dA, lda, dQ, ldq, dR, ldr)) != CQR2_OK) {
    return r;
  }
  if (info) return read_info(p, info);
  return CQR2_OK;
}

cqr2_status_t cqr2_plan_set_gram_ctas(cqr2_plan_t p, int32_t ctas_per_sm) {
  if (!p || ctas_per_sm < 1 || ctas_per_sm > GRAM_CPS_MAX) return CQR2_ERR_INVALID_ARG;
  p->gram_cps = ctas_per_sm;
  p->cm = 0;  // recompute the geometry on the next call
  if (p->gexec) cudaGraphExecDestroy(p->gexec);
  if (p->graph) cudaGraphDestroy(p->graph);
  p->gexec = nullptr;
  p->graph = nullptr;
  return CQR2_OK;
}

cqr2_status_t cqr2_plan_set_inverse_depth(cqr2_plan_t p, int32_t depth) {
  if (!p || depth < 0 || depth > 16) return CQR2_ERR_INVALID_ARG;
  if (depth > 0 && (p->oz_S || p->small)) return CQR2_ERR_UNSUPPORTED;
  if (depth > 0 && !p->Tsolve) {
    const int64_t ldt = std::max(p->m, p->n);
    if (cudaMalloc(&p->Tsolve, (size_t)ldt * right_solve_temp_cols((int)p->n) * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      p->Tsolve = nullptr;
      return CQR2_ERR_OOM;
    }
    p->ldt = ldt;
  }
  p->inv_depth = depth;
  if (p->gexec) cudaGraphExecDestroy(p->gexec);  // a captured launch sequence no longer applies
  if (p->graph) cudaGraphDestroy(p->graph);
  p->gexec = nullptr;
  p->graph = nullptr;
  return CQR2_OK;
}

cqr2_status_t cqr2_selftest_wait_timeout(int64_t polls, void* stream) {
  if (polls < 1 || polls > (int64_t(1) << 24)) return CQR2_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DevStatus* st = nullptr;
  if (cudaMalloc(&st, sizeof(DevStatus)) != cudaSuccess) {
    cudaGetLastError();
    return CQR2_ERR_OOM;
  }
  DevStatus h{};
  cqr2_status_t r = CQR2_OK;
  if (cudaMemsetAsync(st, 0, sizeof(DevStatus), s) != cudaSuccess || ozaki_selftest_wait(polls, st, s) != cudaSuccess ||
      cudaMemcpyAsync(&h, st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    r = CQR2_ERR_CUDA;
  else if (h.status == 5)
    r = CQR2_ERR_TIMEOUT;
  cudaFree(st);
  return r;
}

cqr2_status_t cqr2_plan_set_fused(cqr2_plan_t p, int32_t fused) {
  if (!p) return CQR2_ERR_INVALID_ARG;
  p->fused = fused && !p->oz_S && qform_gram_fusable((int)p->n) && p->small;
  if (p->gexec) cudaGraphExecDestroy(p->gexec);
  if (p->graph) cudaGraphDestroy(p->graph);
  p->gexec = nullptr;
  p->graph = nullptr;
  return CQR2_OK;
}

cqr2_status_t cqr2_factor(cqr2_plan_t p, const double* dA, int64_t lda, double* dQ, int64_t ldq, double* dR,
                          int64_t ldr, cqr2_info_t* info) {
  if (!p) return CQR2_ERR_INVALID_ARG;
  return cqr2_factor_rows(p, p->m, dA, lda, dQ, ldq, dR, ldr, info);
}

cqr2_status_t cqr2_lstsq(cqr2_plan_t p, const double* dA, int64_t lda, const double* db, double* dx, double* dQ,
                         int64_t ldq, double* dR, int64_t ldr, cqr2_info_t* info) {
  if (!p) return CQR2_ERR_INVALID_ARG;
  return cqr2_lstsq_rows(p, p->m, dA, lda, db, dx, dQ, ldq, dR, ldr, info);
}

cqr2_status_t cqr2_lstsq_rows(cqr2_plan_t p, int64_t m, const double* dA, int64_t lda, const double* db, double* dx,
                              double* dQ, int64_t ldq, double* dR, int64_t ldr, cqr2_info_t* info) {
  if (!p || !dA || !db || !dx) return CQR2_ERR_INVALID_ARG;
  if (m < p->n || m > p->m) return CQR2_ERR_INVALID_ARG;
  if (bad_ld(lda, m) || (dQ && bad_ld(ldq, m))) return CQR2_ERR_INVALID_ARG;
  if (dR && bad_ld(ldr, p->n)) return CQR2_ERR_INVALID_ARG;
  if (dQ && bad_alias(p, dA, lda, dQ, ldq)) return CQR2_ERR_INVALID_ARG;
  cqr2_status_t r = check_device(p);
  if (r != CQR2_OK) return r;
  if (!dQ) {
    // Q into the plan's own m x n buffer, allocated once
    if (!p->lsQ && cudaMalloc(&p->lsQ, (size_t)p->m * p->n * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      p->lsQ = nullptr;
      return CQR2_ERR_OOM;
    }
    dQ = p->lsQ;
    ldq = p->m;
  }
  if ((r = set_rows(p, m)) != CQR2_OK) return r;
  double* R = dR ? dR : p->Rf;
  const int64_t ldR = dR ? ldr : p->n;
  if ((r = factor_any(p, dA, lda, dQ, ldq, R, ldR)) != CQR2_OK) return r;
  {
    Stage st(p, CQR2_STAGE_LSTSQ);
    TRY(gemv_t_partials(dQ, ldq, p->cm, (int)p->n, db, p->gemv_nsplit, p->lspart, p->stream));
    TRY(lstsq_solve(p->lspart, p->gemv_nsplit, (int)p->n, R, ldR, dx, p->stream));
  }
  if (info) return read_info(p, info);
  return CQR2_OK;
}

cqr2_status_t cqr2_syrk(cqr2_plan_t p, const double* dA, int64_t lda, double* dW, int64_t ldw) {
  if (!p || !dA || !dW || bad_ld(lda, p->m) || bad_ld(ldw, p->n)) return CQR2_ERR_INVALID_ARG;
  cqr2_status_t r = check_device(p);
  if (r != CQR2_OK) return r;
  if ((r = set_rows(p, p->m)) != CQR2_OK) return r;
  if (p->oz_S) {
    const int n = (int)p->n;
    TRY(cudaMemsetAsync(p->st, 0, sizeof(DevStatus), p->stream));
    TRY(ozaki_colmax(dA, lda, p->cm, n, p->oz_colmax, p->oz_cexp, p->stream));
    TRY(ozaki_slice_cols(dA, lda, p->cm, n, p->oz_S, p->oz_cexp, p->oz_planes, p->stream));
    TRY(ozaki_gram(p->oz_maps, p->cm, n, p->oz_S, p->oz_cexp, p->oz_partial, p->oz_cap, dW, ldw, p->st, p->stream));
    return CQR2_OK;
  }
  TRY(gram_partials(dA, lda, p->cm, (int)p->n, p->g, p->partial, p->stream));
  TRY(gram_reduce(p->partial, p->g, (int)p->n, dW, ldw, p->stream));
  return CQR2_OK;
}

cqr2_status_t cqr2_cholinv(cqr2_plan_t p, const double* dW, int64_t ldw, double* dL, int64_t ldl, double* dY,
                           int64_t ldy, cqr2_info_t* info) {
  if (!p || !dW || !dL || !dY || bad_ld(ldw, p->n) || bad_ld(ldl, p->n) || bad_ld(ldy, p->n))
    return CQR2_ERR_INVALID_ARG;
  cqr2_status_t r = check_device(p);
  if (r != CQR2_OK) return r;
  TRY(cudaMemsetAsync(p->st, 0, sizeof(DevStatus), p->stream));
  TRY(cholinv((int)p->n, dW, ldw, dL, ldl, dY, ldy, p->Wk, p->U, p->st, 1, p->stream, p->skws,
              cholinv_splitk_doubles()));
  if (info) return read_info(p, info);
  return CQR2_OK;
}

cqr2_status_t cqr2_qform(cqr2_plan_t p, const double* dA, int64_t lda, const double* dRinv, int64_t ldri,
                         double* dQ, int64_t ldq) {
  if (!p || !dA || !dRinv || !dQ || bad_ld(lda, p->m) || bad_ld(ldri, p->n) || bad_ld(ldq, p->m))
    return CQR2_ERR_INVALID_ARG;
  if ((const void*)dA == (const void*)dQ) return CQR2_ERR_INVALID_ARG;
  cqr2_status_t r = check_device(p);
  if (r != CQR2_OK) return r;
  if ((r = set_rows(p, p->m)) != CQR2_OK) return r;
  const int n = (int)p->n;
  if (p->oz_S) {
    TRY(cudaMemsetAsync(p->st, 0, sizeof(DevStatus), p->stream));
    TRY(ozaki_colmax(dA, lda, p->cm, n, p->oz_colmax, p->oz_cexp, p->stream));
    TRY(ozaki_slice_cols(dA, lda, p->cm, n, p->oz_S, p->oz_cexp, p->oz_planes, p->stream));
    TRY(ozaki_slice_rinv(dRinv, ldri, n, p->oz_S, true, p->oz_cexp, p->oz_rinv, p->oz_fexp, p->stream));
    TRY(ozaki_qform(p->oz_maps, p->cm, n, p->oz_S, p->oz_fexp, dQ, ldq, p->st, p->stream));
  } else if (p->small) {
    TRY(pack_rinv_from_upper(dRinv, ldri, n, p->Rp, p->stream));
    TRY(qform_small(dA, lda, p->cm, n, p->Rp, dQ, ldq, p->stream));
  } else {
    TRY(gemm_f64(p->cm, n, n, 1.0, dA, lda, dRinv, ldri, 0.0, dQ, ldq, GEMM_B_UPPER | GEMM_BETA0, p->stream));
  }
  return CQR2_OK;
}

cqr2_status_t cqr2_trmm_upper(cqr2_plan_t p, const double* dR2, int64_t ld2, const double* dR1, int64_t ld1,
                              double* dR, int64_t ldr) {
  if (!p || !dR2 || !dR1 || !dR || bad_ld(ld2, p->n) || bad_ld(ld1, p->n) || bad_ld(ldr, p->n))
    return CQR2_ERR_INVALID_ARG;
  cqr2_status_t r = check_device(p);
  if (r != CQR2_OK) return r;
  const int n = (int)p->n;
  TRY(r_product(p, n, dR2, ld2, false, dR1, ld1, dR, ldr, p->stream));
  return CQR2_OK;
}

const char* cqr2_stage_name(int32_t stage) {
  static const char* names[CQR2_NUM_STAGES] = {"gram1", "cholinv1", "qform1", "gram2", "cholinv2",
                                               "qform2", "trmm",  "lstsq",  "h2d",   "d2h", "split"};
  return (stage >= 0 && stage < CQR2_NUM_STAGES) ? names[stage] : "unknown";
}

int64_t cqr2_launch_count(void) { return launch_count(); }

cqr2_status_t cqr2_plan_set_profiling(cqr2_plan_t p, int32_t enable) {
  if (!p) return CQR2_ERR_INVALID_ARG;
  if (cudaStreamSynchronize(p->stream) != cudaSuccess) return CQR2_ERR_CUDA;
  p->profiling = enable != 0;
  p->ev_marks.clear();
  p->ev_used = 0;
  return CQR2_OK;
}

cqr2_status_t cqr2_plan_stage_times(cqr2_plan_t p, double* ms, int64_t* count, int32_t nstages) {
  if (!p || !ms || nstages < 0) return CQR2_ERR_INVALID_ARG;
  for (int i = 0; i < nstages; ++i) {
    ms[i] = 0.0;
    if (count) count[i] = 0;
  }
  if (cudaStreamSynchronize(p->stream) != cudaSuccess) return CQR2_ERR_CUDA;
  for (auto& mk : p->ev_marks) {
    if (mk.first >= nstages) continue;
    float t = 0.f;
    if (cudaEventElapsedTime(&t, mk.second.first, mk.second.second) != cudaSuccess) return CQR2_ERR_CUDA;
    ms[mk.first] += t;
    if (count) count[mk.first] += 1;
  }
  return CQR2_OK;
}

cqr2_status_t cqr2_factor_host(cqr2_plan_t p, const double* hA, int64_t lda, double* hQ, int64_t ldq, double* hR,
                               int64_t ldr, cqr2_info_t* info) {
  if (!p || !hA || !hQ || !hR) return CQR2_ERR_INVALID_ARG;
  if (bad_ld(lda, p->m) || bad_ld(ldq, p->m) || bad_ld(ldr, p->n)) return CQR2_ERR_INVALID_ARG;
  cqr2_status_t r = check_device(p);
  if (r != CQR2_OK) return r;
  if ((r = set_rows(p, p->m)) != CQR2_OK) return r;
  const size_t mn = (size_t)p->m * p->n * sizeof(double);
  if (!p->hA_dev) {
    // Partials for the row-blocked pass-1 Gram: each block may use as many
    // ranges as the largest CTA target asks for.
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
    p->hx_cap = std::max<int64_t>(1, ceil_div((int64_t)GRAM_CPS_MAX * sms, p->g.ntiles_total));
    const size_t part = (size_t)HX_BLOCKS * p->hx_cap * p->g.ntiles_total * p->g.T * p->g.T * sizeof(double);
    if (cudaMalloc(&p->hA_dev, mn) != cudaSuccess || cudaMalloc(&p->hQ_dev, mn) != cudaSuccess ||
        cudaMalloc(&p->hR_dev, (size_t)p->n * p->n * sizeof(double)) != cudaSuccess ||
        (!p->oz_S && cudaMalloc(&p->hx_partial, part) != cudaSuccess)) {
      cudaGetLastError();
      cudaFree(p->hA_dev);
      cudaFree(p->hQ_dev);
      cudaFree(p->hR_dev);
      cudaFree(p->hx_partial);
      p->hA_dev = p->hQ_dev = p->hR_dev = nullptr;
      p->hx_partial = nullptr;
      return CQR2_ERR_OOM;
    }
  }
  if (!p->copy_stream) {
    if (cudaStreamCreateWithFlags(&p->copy_stream, cudaStreamNonBlocking) != cudaSuccess) return CQR2_ERR_CUDA;
    p->hx_ev.resize(2 * HX_BLOCKS + 1);
    for (cudaEvent_t& e : p->hx_ev)
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return CQR2_ERR_CUDA;
  }
  cudaStream_t cs = p->copy_stream;
  cudaEvent_t ev_ready = p->hx_ev[2 * HX_BLOCKS];
  // The copy stream starts after the plan stream's earlier work (the staging
  // buffers may still be read by a previous call).
  TRY(cudaEventRecord(ev_ready, p->stream));
  TRY(cudaStreamWaitEvent(cs, ev_ready, 0));
  {
    Stage st(p, CQR2_STAGE_H2D, cs);
    for (int b = 0; b < HX_BLOCKS; ++b) {
      const int64_t r0 = hx_row(p->m, b), r1 = hx_row(p->m, b + 1);
      if (r1 > r0)
        TRY(cudaMemcpy2DAsync(p->hA_dev + r0, (size_t)p->m * sizeof(double), hA + r0, (size_t)lda * sizeof(double),
                              (size_t)(r1 - r0) * sizeof(double), (size_t)p->n, cudaMemcpyHostToDevice, cs));
      TRY(cudaEventRecord(p->hx_ev[b], cs));
    }
  }
  p->hx.on = true;
  p->hx.a_pending = true;
  p->hx.q_sent = false;
  p->hx.hQ = hQ;
  p->hx.ldq = ldq;
  r = factor_any(p, p->hA_dev, p->m, p->hQ_dev, p->m, p->hR_dev, p->n);
  const bool q_sent = p->hx.q_sent;
  p->hx.on = false;
  p->hx.a_pending = false;  // every path waits for the input blocks before reading A
  if (r != CQR2_OK) {
    cudaStreamSynchronize(cs);
    return r;
  }
  {
    Stage st(p, CQR2_STAGE_D2H);
    if (!q_sent) TRY(copy_cols(hQ, ldq, p->hQ_dev, p->m, p->m, p->n, cudaMemcpyDeviceToHost, p->stream));
    TRY(copy_cols(hR, ldr, p->hR_dev, p->n, p->n, p->n, cudaMemcpyDeviceToHost, p->stream));
  }
  // the plan stream (and read_info's synchronisation) covers the copy stream
  TRY(cudaEventRecord(ev_ready, cs));
  TRY(cudaStreamWaitEvent(p->stream, ev_ready, 0));
  cqr2_info_t local;
  r = read_info(p, info ? info : &local);
  return r;
}

}  // extern "C"
