// C ABI for many independent factorizations and for the autotuner.
//
// cqr2_batch_factor routes every problem of a batch:
//   * small ones (n <= 64 and m n^2 at most the tuned limit) go to one launch
//     of the persistent grouped kernel, which factors a whole problem per CTA
//     from a device work queue, largest first;
//   * the others run on per-(n, stream) plans spread over several streams
//     that fork from and join back into the batch's stream, so their kernels
//     overlap on the device.
// cqr2_autotune times candidate configurations on the device and keeps the
// fastest per (n, m bucket, precision) in a process-wide table.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/cqr2.h"
#include "kernels.h"

using namespace cqr2;

struct cqr2_batch_st {
  int device = 0;
  int precision = CQR2_FP64;
  cudaStream_t stream = nullptr;
  int32_t max_count = 0;
  cqr2_batch_config_t cfg{};
  BatchProblem* d_probs = nullptr;
  BatchStatus* d_status = nullptr;
  int* d_next = nullptr;
  BatchProblem* h_probs = nullptr;
  BatchStatus* h_status = nullptr;
  DevStatus* d_lstatus = nullptr;  // status words of the planned problems
  DevStatus* h_lstatus = nullptr;
  std::vector<cudaStream_t> side;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> joins;
  struct PlanSlot {
    cqr2_plan_t plan = nullptr;
    int64_t m_max = 0;
  };
  std::map<std::pair<int64_t, int>, PlanSlot> plans;  // (n, side stream) -> plan
  // the last call: its end on the batch stream and where each outcome lives
  cudaEvent_t done = nullptr;
  bool pending = false;
  int32_t last_count = 0;
  std::vector<int> last_small;                 // problem index per grouped job
  std::vector<int> last_used;                  // problem index per planned status word
  // graph replay of a repeating problem list (cfg.graph)
  std::vector<cqr2_problem_t> gkey;            // the previous call's list
  bool gkey_valid = false;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;             // captured for gkey, if any
  std::vector<int> g_small, g_used;            // its outcome locations
  int64_t replays = 0;
  int64_t g_kernels = 0;                       // kernels in the captured graph
};

namespace {

struct TuneEntry {
  int32_t gram_ctas;
  int32_t fused;
  double ms;
};
std::mutex g_tune_mu;
std::map<std::string, TuneEntry> g_tune;  // key "n:mbucket:precision"
int64_t g_small_limit = -1;                 // tuned grouped-kernel limit on m n^2 (-1 = default)

std::string tune_key(int64_t m, int64_t n, int precision) {
  const int mb = (int)std::floor(std::log2((double)std::max<int64_t>(m, 1)));
  char buf[64];
  std::snprintf(buf, sizeof(buf), "%lld:%d:%d", (long long)n, mb, precision);
  return buf;
}

constexpr int64_t DEFAULT_SMALL_LIMIT = (int64_t)32768 * 64 * 64;

bool lookup_tune(int64_t m, int64_t n, int precision, TuneEntry* e) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune.find(tune_key(m, n, precision));
  if (it == g_tune.end()) return false;
  *e = it->second;
  return true;
}

// Enqueue one batch call on b's stream: routing, the grouped launch, the
// planned problems on side streams, and the copies of every outcome to the
// host. Records where each outcome lives in b->last_small / b->last_used.
cqr2_status_t batch_enqueue(cqr2_batch_t b, const cqr2_problem_t* problems, int32_t count) {
  // route by shape alone
  std::vector<int> small, large;
  for (int i = 0; i < count; ++i) {
    const cqr2_problem_t& q = problems[i];
    const bool is_small = q.n <= BATCH_SMALL_MAX_N && (double)q.m * q.n * q.n <= (double)b->cfg.small_work_limit;
    (is_small ? small : large).push_back(i);
  }
  std::sort(small.begin(), small.end(), [&](int a, int c) {
    return (double)problems[a].m * problems[a].n * problems[a].n > (double)problems[c].m * problems[c].n * problems[c].n;
  });
  // grouped launch for the small problems (on the batch stream)
  if (!small.empty()) {
    for (size_t k = 0; k < small.size(); ++k) {
      const cqr2_problem_t& q = problems[small[k]];
      b->h_probs[k] = BatchProblem{q.m, q.n, q.A, q.lda, q.Q, q.ldq, q.R, q.ldr, q.b, q.x};
    }
    if (cudaMemcpyAsync(b->d_probs, b->h_probs, sizeof(BatchProblem) * small.size(), cudaMemcpyHostToDevice,
                        b->stream) != cudaSuccess)
      return CQR2_ERR_CUDA;
    if (cqr2_small_batched(b->d_probs, (int)small.size(), b->d_next, b->d_status, b->stream) != cudaSuccess)
      return CQR2_ERR_CUDA;
  }
  b->last_small = small;
  // the others: plans on side streams forked from the batch stream
  if (!large.empty()) {
    if (cudaEventRecord(b->fork, b->stream) != cudaSuccess) return CQR2_ERR_CUDA;
    const int ns = (int)std::min<size_t>(b->side.size(), large.size());
    for (int s = 0; s < ns; ++s)
      if (cudaStreamWaitEvent(b->side[s], b->fork, 0) != cudaSuccess) return CQR2_ERR_CUDA;
    for (size_t k = 0; k < large.size(); ++k) {
      const cqr2_problem_t& q = problems[large[k]];
      const int s = (int)(k % ns);
      auto& slot = b->plans[{q.n, s}];
      if (!slot.plan || slot.m_max < q.m) {
        if (slot.plan) {
          cudaStreamSynchronize(b->side[s]);
          cqr2_plan_destroy(slot.plan);
          slot.plan = nullptr;
        }
        const int64_t mm = std::max<int64_t>(q.m, slot.m_max);
        int prec = b->precision;
        if (prec != CQR2_FP64 && q.n > OZAKI_MAX_N) prec = CQR2_FP64;
        cqr2_status_t r = cqr2_plan_create(&slot.plan, mm, q.n, prec, b->cfg.fused ? CQR2_FUSED : 0, b->side[s]);
        if (r != CQR2_OK) return r;
        slot.m_max = mm;
        TuneEntry te;
        if (lookup_tune(q.m, q.n, prec, &te)) {
          cqr2_plan_set_gram_ctas(slot.plan, te.gram_ctas);
          cqr2_plan_set_fused(slot.plan, te.fused);
        }
      }
      cqr2_status_t r = q.b ? cqr2_lstsq_rows(slot.plan, q.m, q.A, q.lda, q.b, q.x, q.Q, q.ldq, q.R, q.ldr, nullptr)
                            : cqr2_factor_rows(slot.plan, q.m, q.A, q.lda, q.Q, q.ldq, q.R, q.ldr, nullptr);
      if (r != CQR2_OK) return r;
      if (plan_status_copy(slot.plan, b->d_lstatus + b->last_used.size(), b->side[s]) != cudaSuccess)
        return CQR2_ERR_CUDA;
      b->last_used.push_back(large[k]);
    }
    for (int s = 0; s < ns; ++s) {
      if (cudaEventRecord(b->joins[s], b->side[s]) != cudaSuccess) return CQR2_ERR_CUDA;
      if (cudaStreamWaitEvent(b->stream, b->joins[s], 0) != cudaSuccess) return CQR2_ERR_CUDA;
    }
  }
  // the outcomes travel to the host with the work, so cqr2_batch_info only waits
  if (!small.empty() && cudaMemcpyAsync(b->h_status, b->d_status, sizeof(BatchStatus) * small.size(),
                                        cudaMemcpyDeviceToHost, b->stream) != cudaSuccess)
    return CQR2_ERR_CUDA;
  if (!b->last_used.empty() && cudaMemcpyAsync(b->h_lstatus, b->d_lstatus, sizeof(DevStatus) * b->last_used.size(),
                                               cudaMemcpyDeviceToHost, b->stream) != cudaSuccess)
    return CQR2_ERR_CUDA;
  return CQR2_OK;
}

bool same_problem(const cqr2_problem_t& a, const cqr2_problem_t& c) {
  return a.m == c.m && a.n == c.n && a.A == c.A && a.lda == c.lda && a.Q == c.Q && a.ldq == c.ldq && a.R == c.R &&
         a.ldr == c.ldr && a.b == c.b && a.x == c.x;
}

void drop_graph(cqr2_batch_t b) {
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->gexec = nullptr;
  b->graph = nullptr;
}

// cfg.graph: the first call of a list runs eagerly (plans get created and
// sized outside any capture); when the next call repeats it, that call's
// sequence is captured and launched, and later repeats replay the graph.
cqr2_status_t batch_enqueue_graph(cqr2_batch_t b, const cqr2_problem_t* problems, int32_t count) {
  bool same = b->gkey_valid && (int32_t)b->gkey.size() == count;
  for (int i = 0; same && i < count; ++i) same = same_problem(b->gkey[i], problems[i]);
  if (!same) {
    drop_graph(b);
    b->gkey.assign(problems, problems + count);
    b->gkey_valid = false;
    const cqr2_status_t r = batch_enqueue(b, problems, count);
    b->gkey_valid = r == CQR2_OK;
    return r;
  }
  if (!b->gexec) {
    if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return CQR2_ERR_CUDA;
    const int64_t l0 = launch_count();
    const cqr2_status_t r = batch_enqueue(b, problems, count);
    b->g_kernels = launch_count() - l0;
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(b->stream, &g);
    if (r != CQR2_OK || ce != cudaSuccess || cudaGraphInstantiate(&b->gexec, g, 0) != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      b->gexec = nullptr;
      b->gkey_valid = false;
      cudaGetLastError();
      return r != CQR2_OK ? r : CQR2_ERR_CUDA;
    }
    b->graph = g;
    b->g_small = b->last_small;
    b->g_used = b->last_used;
  } else {
    b->last_small = b->g_small;
    b->last_used = b->g_used;
    ++b->replays;
    count_launches(b->g_kernels);
  }
  return cudaGraphLaunch(b->gexec, b->stream) == cudaSuccess ? CQR2_OK : CQR2_ERR_CUDA;
}

}  // namespace

extern "C" {

cqr2_status_t cqr2_batch_create(cqr2_batch_t* batch, int32_t max_count, int32_t precision,
                                const cqr2_batch_config_t* cfg, void* stream) {
  if (!batch) return CQR2_ERR_INVALID_ARG;
  *batch = nullptr;
  if (max_count < 1) return CQR2_ERR_INVALID_ARG;
  if (precision != CQR2_FP64 && precision != CQR2_OZAKI_BF16 && precision != CQR2_OZAKI_BF16_S6)
    return CQR2_ERR_INVALID_ARG;
  auto* b = new (std::nothrow) cqr2_batch_st();
  if (!b) return CQR2_ERR_OOM;
  if (cudaGetDevice(&b->device) != cudaSuccess) {
    delete b;
    return CQR2_ERR_CUDA;
  }
  b->precision = precision;
  b->stream = static_cast<cudaStream_t>(stream);
  b->max_count = max_count;
  if (cfg) {
    b->cfg = *cfg;
  } else {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    b->cfg.small_work_limit = g_small_limit >= 0 ? g_small_limit : DEFAULT_SMALL_LIMIT;
    b->cfg.streams = 4;
    b->cfg.fused = 1;
  }
  b->cfg.streams = std::max(1, std::min(16, (int)b->cfg.streams));
  bool ok = cudaMalloc(&b->d_probs, sizeof(BatchProblem) * max_count) == cudaSuccess &&
            cudaMalloc(&b->d_status, sizeof(BatchStatus) * max_count) == cudaSuccess &&
            cudaMalloc(&b->d_next, sizeof(int)) == cudaSuccess &&
            cudaMallocHost(&b->h_probs, sizeof(BatchProblem) * max_count) == cudaSuccess &&
            cudaMallocHost(&b->h_status, sizeof(BatchStatus) * max_count) == cudaSuccess &&
            cudaMalloc(&b->d_lstatus, sizeof(DevStatus) * max_count) == cudaSuccess &&
            cudaMallocHost(&b->h_lstatus, sizeof(DevStatus) * max_count) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming) == cudaSuccess;
  for (int i = 0; ok && i < b->cfg.streams; ++i) {
    cudaStream_t s;
    cudaEvent_t e;
    ok = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
    if (ok) {
      b->side.push_back(s);
      b->joins.push_back(e);
    }
  }
  if (!ok) {
    cudaGetLastError();
    cqr2_batch_destroy(b);
    return CQR2_ERR_OOM;
  }
  *batch = b;
  return CQR2_OK;
}

void cqr2_batch_destroy(cqr2_batch_t b) {
  if (!b) return;
  if (b->stream || true) cudaStreamSynchronize(b->stream);
  for (auto& kv : b->plans) cqr2_plan_destroy(kv.second.plan);
  for (cudaStream_t s : b->side) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->joins) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->done) cudaEventDestroy(b->done);
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->graph) cudaGraphDestroy(b->graph);
  cudaFree(b->d_probs);
  cudaFree(b->d_status);
  cudaFree(b->d_next);
  cudaFreeHost(b->h_probs);
  cudaFreeHost(b->h_status);
  cudaFree(b->d_lstatus);
  cudaFreeHost(b->h_lstatus);
  delete b;
}

cqr2_status_t cqr2_batch_factor(cqr2_batch_t b, const cqr2_problem_t* problems, int32_t count, cqr2_info_t* infos) {
  if (!b || (!problems && count > 0) || count < 0 || count > b->max_count) return CQR2_ERR_INVALID_ARG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return CQR2_ERR_CUDA;
  if (dev != b->device) return CQR2_ERR_INVALID_ARG;
  for (int i = 0; i < count; ++i) {
    const cqr2_problem_t& q = problems[i];
    if (q.n < 1 || q.m < q.n || !q.A || !q.Q || !q.R || q.lda < q.m || q.ldq < q.m || q.ldr < q.n ||
        (const void*)q.A == (const void*)q.Q || (q.b == nullptr) != (q.x == nullptr))
      return CQR2_ERR_INVALID_ARG;
  }
  // the previous call's descriptors and status words are about to be reused
  if (b->pending && cudaEventSynchronize(b->done) != cudaSuccess) return CQR2_ERR_CUDA;
  b->pending = false;
  b->last_count = 0;
  b->last_small.clear();
  b->last_used.clear();
  // whatever gets enqueued, the next call waits for it
  const cqr2_status_t r = b->cfg.graph && b->stream ? batch_enqueue_graph(b, problems, count)
                                                    : batch_enqueue(b, problems, count);
  const bool recorded = cudaEventRecord(b->done, b->stream) == cudaSuccess;
  b->pending = recorded;
  if (r != CQR2_OK || !recorded) {
    b->last_small.clear();
    b->last_used.clear();
    return r != CQR2_OK ? r : CQR2_ERR_CUDA;
  }
  b->last_count = count;
  if (!infos) return CQR2_OK;
  return cqr2_batch_info(b, count, infos);
}

cqr2_status_t cqr2_batch_info(cqr2_batch_t b, int32_t count, cqr2_info_t* infos) {
  if (!b || !infos || count != b->last_count) return CQR2_ERR_INVALID_ARG;
  if (b->pending && cudaEventSynchronize(b->done) != cudaSuccess) return CQR2_ERR_CUDA;
  b->pending = false;
  cqr2_status_t worst = CQR2_OK;
  for (size_t k = 0; k < b->last_small.size(); ++k) {
    cqr2_info_t& in = infos[b->last_small[k]];
    const BatchStatus& st = b->h_status[k];
    in.status = st.failed_pass ? CQR2_ERR_NOT_SPD : CQR2_OK;
    in.failed_pass = st.failed_pass;
    in.failed_pivot = st.failed_pass ? st.failed_pivot : -1;
    in.pivot_value = 0.0;
    if (st.failed_pass) worst = CQR2_ERR_NOT_SPD;
  }
  for (size_t k = 0; k < b->last_used.size(); ++k) {
    cqr2_info_t& in = infos[b->last_used[k]];
    const DevStatus& st = b->h_lstatus[k];
    in.status = st.status == 0 ? CQR2_OK : (st.status == 5 ? CQR2_ERR_TIMEOUT : CQR2_ERR_NOT_SPD);
    in.failed_pass = st.status == 2 ? st.pass : 0;
    in.failed_pivot = st.status == 2 ? st.pivot : -1;
    in.pivot_value = st.status == 2 ? st.value : 0.0;
    if (in.status != CQR2_OK) worst = (cqr2_status_t)in.status;
  }
  return worst;
}

cqr2_status_t cqr2_autotune(int64_t m, int64_t n, int32_t precision, cqr2_tune_result_t* out) {
  if (n < 1 || m < n || !out) return CQR2_ERR_INVALID_ARG;
  std::memset(out, 0, sizeof(*out));
  double* A = nullptr;
  double* Q = nullptr;
  double* R = nullptr;
  const size_t mn = (size_t)m * n * sizeof(double);
  if (cudaMalloc(&A, mn) != cudaSuccess || cudaMalloc(&Q, mn) != cudaSuccess ||
      cudaMalloc(&R, (size_t)n * n * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(A);
    cudaFree(Q);
    return CQR2_ERR_OOM;
  }
  cudaStream_t s;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
    cudaFree(A);
    cudaFree(Q);
    cudaFree(R);
    return CQR2_ERR_CUDA;
  }
  // A well-conditioned scratch matrix: the first n rows are the identity
  // (the timings do not depend on the values).
  bool filled = cudaMemsetAsync(A, 0, mn, s) == cudaSuccess;
  for (int64_t j = 0; filled && j < n; ++j) {
    const double one = 1.0;
    filled = cudaMemcpyAsync(A + j + j * m, &one, sizeof(double), cudaMemcpyHostToDevice, s) == cudaSuccess;
  }
  if (!filled) {
    cudaStreamDestroy(s);
    cudaFree(A);
    cudaFree(Q);
    cudaFree(R);
    return CQR2_ERR_CUDA;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cqr2_plan_t plan = nullptr;
  cqr2_status_t r = cqr2_plan_create(&plan, m, n, precision, CQR2_FUSED, s);
  if (r != CQR2_OK) {
    cudaStreamDestroy(s);
    cudaFree(A);
    cudaFree(Q);
    cudaFree(R);
    return r;
  }
  const int cps_list[] = {1, 2, 4, 8};
  const int fused_list[] = {0, 1};
  double best = 1e30;
  TuneEntry bestE{4, 1, 0.0};
  int tried = 0;
  for (int f : fused_list) {
    if (f && (precision != CQR2_FP64 || n > 128)) continue;
    for (int cps : cps_list) {
      cqr2_plan_set_fused(plan, f);
      cqr2_plan_set_gram_ctas(plan, cps);
      cqr2_factor(plan, A, m, Q, m, R, n, nullptr);  // warm
      cudaEventRecord(e0, s);
      const int reps = 3;
      for (int i = 0; i < reps; ++i) cqr2_factor(plan, A, m, Q, m, R, n, nullptr);
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      ms /= reps;
      ++tried;
      if (ms < best) {
        best = ms;
        bestE = TuneEntry{cps, f, ms};
      }
    }
  }
  cqr2_plan_destroy(plan);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(s);
  cudaFree(A);
  cudaFree(Q);
  cudaFree(R);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[tune_key(m, n, precision)] = bestE;
  }
  out->gram_ctas = bestE.gram_ctas;
  out->fused = bestE.fused;
  out->ms = bestE.ms;
  out->candidates = tried;
  return CQR2_OK;
}

cqr2_status_t cqr2_autotune_batch(int64_t n, int32_t count, int64_t* limit_out) {
  if (n < 1 || n > BATCH_SMALL_MAX_N || count < 1 || !limit_out) return CQR2_ERR_INVALID_ARG;
  *limit_out = 0;
  // Largest m measured: keep the scratch (one A shared by all problems, a Q
  // and an R each) near 4 GB.
  int64_t m_cap = std::max<int64_t>(n, ((int64_t)1 << 32) / ((int64_t)count * n * 8 * 2));
  m_cap = std::min<int64_t>(m_cap, (int64_t)1 << 20);
  double *A = nullptr, *Q = nullptr, *R = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cqr2_batch_t grouped = nullptr, planned = nullptr;
  auto cleanup = [&]() {
    if (s) cudaStreamSynchronize(s);
    cqr2_batch_destroy(grouped);
    cqr2_batch_destroy(planned);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    cudaFree(A);
    cudaFree(Q);
    cudaFree(R);
    cudaGetLastError();
  };
  if (cudaMalloc(&A, (size_t)m_cap * n * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&Q, (size_t)count * m_cap * n * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&R, (size_t)count * n * n * sizeof(double)) != cudaSuccess) {
    cleanup();
    return CQR2_ERR_OOM;
  }
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
      cudaMemsetAsync(A, 0, (size_t)m_cap * n * sizeof(double), s) != cudaSuccess) {
    cleanup();
    return CQR2_ERR_CUDA;
  }
  for (int64_t j = 0; j < n; ++j) {  // identity on top: well conditioned for every m
    const double one = 1.0;
    if (cudaMemcpyAsync(A + j + j * m_cap, &one, sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess) {
      cleanup();
      return CQR2_ERR_CUDA;
    }
  }
  // the same problems routed to the grouped kernel, and to plans
  cqr2_batch_config_t cg{(int64_t)1 << 62, 4, 1, 0}, cp{0, 4, 1, 0};
  if (cqr2_batch_create(&grouped, count, CQR2_FP64, &cg, s) != CQR2_OK ||
      cqr2_batch_create(&planned, count, CQR2_FP64, &cp, s) != CQR2_OK) {
    cleanup();
    return CQR2_ERR_OOM;
  }
  std::vector<cqr2_problem_t> probs(count);
  auto time_batch = [&](cqr2_batch_t b, int64_t m, float* ms) -> cqr2_status_t {
    for (int i = 0; i < count; ++i)
      probs[i] = cqr2_problem_t{m, n, A, m_cap, Q + (size_t)i * m_cap * n, m_cap, R + (size_t)i * n * n, n,
                                nullptr, nullptr};
    cqr2_status_t r = cqr2_batch_factor(b, probs.data(), count, nullptr);  // warm (plans, first loads)
    if (r != CQR2_OK) return r;
    if (cudaEventRecord(e0, s) != cudaSuccess) return CQR2_ERR_CUDA;
    const int reps = 3;
    for (int k = 0; k < reps; ++k)
      if ((r = cqr2_batch_factor(b, probs.data(), count, nullptr)) != CQR2_OK) return r;
    if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) return CQR2_ERR_CUDA;
    if (cudaEventElapsedTime(ms, e0, e1) != cudaSuccess) return CQR2_ERR_CUDA;
    *ms /= reps;
    return CQR2_OK;
  };
  // double m from n while the grouped launch is at least as fast
  int64_t limit = 0;
  for (int64_t m = std::max<int64_t>(n, 64); m <= m_cap; m *= 2) {
    float tg = 0.f, tp = 0.f;
    cqr2_status_t r = time_batch(grouped, m, &tg);
    if (r == CQR2_OK) r = time_batch(planned, m, &tp);
    if (r != CQR2_OK) {
      cleanup();
      return r;
    }
    if (tg > tp) break;
    limit = m * n * n;
  }
  cleanup();
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_small_limit = limit;
  }
  *limit_out = limit;
  return CQR2_OK;
}

cqr2_status_t cqr2_tune_set_small_limit(int64_t limit) {
  if (limit < 0) return CQR2_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_small_limit = limit;
  return CQR2_OK;
}

int64_t cqr2_tune_table(char* buf, int64_t size) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  std::string s;
  char line[160];
  for (auto& kv : g_tune) {
    std::snprintf(line, sizeof(line), "%s gram_ctas=%d fused=%d ms=%.4f\n", kv.first.c_str(), kv.second.gram_ctas,
                  kv.second.fused, kv.second.ms);
    s += line;
  }
  std::snprintf(line, sizeof(line), "small_work_limit=%lld\n",
                (long long)(g_small_limit >= 0 ? g_small_limit : DEFAULT_SMALL_LIMIT));
  s += line;
  if (buf && size > 0) {
    const size_t k = std::min<size_t>((size_t)size - 1, s.size());
    std::memcpy(buf, s.data(), k);
    buf[k] = 0;
  }
  return (int64_t)s.size() + 1;
}

}  // extern "C"
