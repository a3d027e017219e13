// Launch schedules, their autotuner, and many independent regressions in one call.
//
// A batch is a set of unrelated problems (own n, d, dtype, Π1 and Π2 draws).
// Each problem runs the same kernel chain as l1_coreset (Figure 2, steps 1-7)
// and optionally the coreset solve and objective (step 8).  The chains are
// spread over a pool of library-owned streams that fork from the caller's
// stream on one event and join back into it, so the whole batch is one unit of
// stream work: it can be captured into a CUDA graph and replayed with a single
// launch.  λ keeps M in shared memory in this form, because the constant bank
// holds one M per device and the chains run concurrently.
#include <stdio.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <numeric>
#include <tuple>
#include <vector>

#include "l1s_common.cuh"

namespace l1s {

// defined in api.cu
int64_t coreset_capacity_of(const l1s_params* p);
bool check_ws(const Plan& pl, const void* ws, size_t ws_bytes);
bool check_a(const void* A, int64_t lda, const float* b, int d);
int coreset_impl(const Plan& pl, const void* A, int64_t lda, l1s_dtype dtype, const float* b,
                 const l1s_params* params, int64_t capacity, int64_t* idx, double* wts, double* coreset,
                 int64_t* count, unsigned char* w, cudaStream_t st);
bool launch_solve(const double* X, const double* w, const int64_t* count, int64_t capacity, int d,
                  int max_iter, double* x_out, double* obj_out, int nblocks, double* partials,
                  void* state, float* scratch, StatusBlock* status, cudaStream_t st, int k,
                  uint32_t* flags_out);
bool launch_objective(const void* A, int64_t lda, l1s_dtype dt, const float* b, int64_t n, int d,
                      const double* x, double* out, int nblocks, double* partials, cudaStream_t st);

// ---------------------------------------------------------------------------
// Schedule table, keyed by (device, d, dtype, log2 s).
// ---------------------------------------------------------------------------
using SchedKey = std::tuple<int, int, int, int>;
static std::mutex g_sched_mu;
static std::map<SchedKey, l1s_schedule> g_sched;

bool schedule_lookup(int d, l1s_dtype dt, int log2s, l1s_schedule* out) {
  *out = l1s_schedule{};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  std::lock_guard<std::mutex> lock(g_sched_mu);
  auto it = g_sched.find(SchedKey{dev, d, static_cast<int>(dt), log2s});
  if (it == g_sched.end()) return false;
  *out = it->second;
  return true;
}

static bool valid_schedule(const l1s_schedule& s) {
  return s.fct_variant >= 0 && s.fct_variant <= 7 && s.fct_ctas_per_sm >= 0 && s.fct_ctas_per_sm <= 64 &&
         s.lam_ctas_per_sm >= 0 && s.lam_ctas_per_sm <= 32 && s.smp_chunks_per_sm >= 0 &&
         s.smp_chunks_per_sm <= 16;
}

// ---------------------------------------------------------------------------
// Stream pool (per device): kPool non-blocking streams, one fork event and one
// join event per stream.  Enqueueing a batch holds the pool's mutex.
// ---------------------------------------------------------------------------
constexpr int kPool = 16;
struct StreamPool {
  bool ready = false;
  cudaStream_t st[kPool];
  cudaEvent_t fork;
  cudaEvent_t join[kPool];
  std::mutex mu;
};
static StreamPool g_pools[64];
static std::mutex g_pools_mu;

static StreamPool* stream_pool() {
  int dev = 0;
  if (!cuda_ok(cudaGetDevice(&dev), "cudaGetDevice") || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lock(g_pools_mu);
  StreamPool& P = g_pools[dev];
  if (!P.ready) {
    for (int k = 0; k < kPool; ++k) {
      if (!cuda_ok(cudaStreamCreateWithFlags(&P.st[k], cudaStreamNonBlocking), "create pool stream") ||
          !cuda_ok(cudaEventCreateWithFlags(&P.join[k], cudaEventDisableTiming), "create join event"))
        return nullptr;
    }
    if (!cuda_ok(cudaEventCreateWithFlags(&P.fork, cudaEventDisableTiming), "create fork event")) return nullptr;
    P.ready = true;
  }
  return &P;
}

// Per-problem view of a batch: its plan, its workspace slice and its output buffers.
struct Member {
  Plan pl;
  size_t ws_off;
  int64_t cap;            // rows the kept-row buffers hold
  bool internal_rows;     // idx/w live in the workspace
  bool internal_core;     // the coreset lives in the workspace
  double cost;            // estimated device time (ns), for stream assignment
};

static size_t member_plans(const l1s_problem* probs, int32_t count, std::vector<Member>* out) {
  out->assign(static_cast<size_t>(count), Member{});
  size_t off = 256;
  for (int32_t i = 0; i < count; ++i) {
    const l1s_problem& pr = probs[i];
    Member& m = (*out)[i];
    if (!make_plan(&pr.params, pr.n, pr.d, pr.dtype, false, &m.pl)) {
      char msg[512];
      snprintf(msg, sizeof(msg), "%s", l1s_last_error());
      set_error("problem %d: %s", i, msg);
      return 0;
    }
    m.pl.lam_m_in_smem = 1;
    m.ws_off = off;
    off = align_up(off + m.pl.total);
    const double esz = pr.dtype == L1S_BF16 ? 2.0 : 4.0;
    // Two reads of X plus the λ round trip at ~6 bytes/ns, plus ~25 µs of dependent
    // launches and the conditioning's serial FP64 work.
    m.cost = static_cast<double>(pr.n) * (2.0 * (pr.d * esz + 4.0) + 8.0) / 6.0 + 25000.0;
  }
  return off;
}

static bool check_member(const l1s_problem& pr, int i) {
  if (!check_a(pr.A_dev, pr.lda, pr.b_dev, pr.d)) {
    char msg[512];
    snprintf(msg, sizeof(msg), "%s", l1s_last_error());
    return set_error("problem %d: %s", i, msg), false;
  }
  if ((pr.idx_dev == nullptr) != (pr.w_dev == nullptr))
    return set_error("problem %d: idx_dev and w_dev must both be given or both be NULL", i), false;
  if (pr.idx_dev && pr.capacity < 1) return set_error("problem %d: capacity must be >= 1", i), false;
  if (pr.coreset_dev && !pr.idx_dev) return set_error("problem %d: coreset_dev needs idx_dev and w_dev", i), false;
  if (pr.objective_dev && !pr.x_dev) return set_error("problem %d: objective_dev needs x_dev", i), false;
  return true;
}

// Enqueue one member's chain on `st`.
static int enqueue_member(const l1s_problem& pr, const Member& m, unsigned char* base, uint32_t* flags_dev,
                          int index, cudaStream_t st) {
  const Plan& pl = m.pl;
  unsigned char* w = base + m.ws_off;
  const int q = pr.d + 1;
  const int64_t cap_ws = coreset_capacity_of(&pr.params);
  StatusBlock* sb = reinterpret_cast<StatusBlock*>(w + pl.off_status);
  int64_t* idx_ws = reinterpret_cast<int64_t*>(w + pl.off_idx_tmp);
  double* w_ws = reinterpret_cast<double*>(idx_ws + cap_ws);
  double* core_ws = w_ws + cap_ws;
  double* obj_ws = core_ws + cap_ws * q + (q + 1);   // coreset objective of the solve
  int64_t* idx = m.internal_rows ? idx_ws : pr.idx_dev;
  double* wts = m.internal_rows ? w_ws : pr.w_dev;
  double* core = pr.coreset_dev ? pr.coreset_dev : (m.internal_core ? core_ws : nullptr);
  int64_t* cnt = pr.count_dev ? pr.count_dev : &sb->count;
  int rc = coreset_impl(pl, pr.A_dev, pr.lda, pr.dtype, pr.b_dev, &pr.params, m.cap, idx, wts, core, cnt, w, st);
  if (rc != L1S_OK) return rc;
  if (pr.x_dev) {
    const DeviceInfo di = device_info();
    if (!launch_solve(core, wts, cnt, m.cap, pr.d, 100, pr.x_dev, obj_ws, di.sms,
                      reinterpret_cast<double*>(w + pl.off_irls), w + pl.off_x,
                      reinterpret_cast<float*>(w + pl.off_objp), sb, st, 1, nullptr))
      return L1S_ERR_CUDA;
    if (pr.objective_dev &&
        !launch_objective(pr.A_dev, pr.lda, pr.dtype, pr.b_dev, pr.n, pr.d, pr.x_dev, pr.objective_dev,
                          pl.lam_ctas, reinterpret_cast<double*>(w + pl.off_lamsum), st))
      return L1S_ERR_CUDA;
  }
  if (flags_dev && !cuda_ok(cudaMemcpyAsync(flags_dev + index, &sb->flags, sizeof(uint32_t),
                                            cudaMemcpyDeviceToDevice, st),
                            "copy status word"))
    return L1S_ERR_CUDA;
  return L1S_OK;
}

static void settle_member(const l1s_problem& pr, Member* m) {
  const int64_t cap_ws = coreset_capacity_of(&pr.params);
  m->internal_rows = pr.idx_dev == nullptr;
  m->internal_core = pr.coreset_dev == nullptr && pr.x_dev != nullptr;
  // Rows kept in the workspace, and the rows the solve reads, are bounded by its
  // 2·m_s + 64 slots.
  m->cap = m->internal_rows ? cap_ws : pr.capacity;
  if (pr.x_dev) m->cap = std::min(m->cap, cap_ws);
}

}  // namespace l1s

using namespace l1s;

extern "C" {

int l1s_schedule_set(int32_t d, l1s_dtype dtype, int32_t s, const l1s_schedule* sch) {
  const int l2 = log2_exact(s);
  if (d < 1 || d > kMaxD || l2 < 0 || l2 > kMaxLog2S || (dtype != L1S_F32 && dtype != L1S_BF16))
    return set_error("bad d, dtype or s"), L1S_ERR_INVALID_ARG;
  if (sch && !valid_schedule(*sch)) return set_error("schedule field out of range"), L1S_ERR_INVALID_ARG;
  int dev = 0;
  if (!cuda_ok(cudaGetDevice(&dev), "cudaGetDevice")) return L1S_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_sched_mu);
  const SchedKey key{dev, d, static_cast<int>(dtype), l2};
  if (sch)
    g_sched[key] = *sch;
  else
    g_sched.erase(key);
  return L1S_OK;
}

int l1s_schedule_get(int32_t d, l1s_dtype dtype, int32_t s, l1s_schedule* sch) {
  const int l2 = log2_exact(s);
  if (!sch || l2 < 0) return set_error("bad arguments"), L1S_ERR_INVALID_ARG;
  schedule_lookup(d, dtype, l2, sch);
  return L1S_OK;
}

int l1s_batched_workspace_size(const l1s_problem* probs, int32_t count, size_t* bytes) {
  if (!bytes || count < 0 || (count > 0 && !probs)) return set_error("bad arguments"), L1S_ERR_INVALID_ARG;
  std::vector<Member> mem;
  const size_t total = count ? member_plans(probs, count, &mem) : 256;
  if (total == 0) return L1S_ERR_INVALID_ARG;
  *bytes = total;
  return L1S_OK;
}

int l1_regress_batched(const l1s_problem* probs, int32_t count, uint32_t* flags_dev, void* ws, size_t ws_bytes,
                       void* stream) {
  TraceRange trace_("l1_regress_batched");
  if (count < 0 || (count > 0 && !probs)) return set_error("bad arguments"), L1S_ERR_INVALID_ARG;
  if (count == 0) return L1S_OK;
  if (!ws || reinterpret_cast<uintptr_t>(ws) % 256 != 0)
    return set_error("workspace must be non-NULL and 256-byte aligned"), L1S_ERR_WORKSPACE;
  std::vector<Member> mem;
  const size_t total = member_plans(probs, count, &mem);
  if (total == 0) return L1S_ERR_INVALID_ARG;
  if (ws_bytes < total) return set_error("workspace too small: %zu bytes given, %zu needed", ws_bytes, total),
                               L1S_ERR_WORKSPACE;
  for (int32_t i = 0; i < count; ++i) {
    if (!check_member(probs[i], i)) return L1S_ERR_INVALID_ARG;
    settle_member(probs[i], &mem[i]);
  }
  StreamPool* pool = stream_pool();
  if (!pool) return L1S_ERR_CUDA;

  // Longest-processing-time-first: each problem onto the stream with the least work so far.
  const int nst = std::min<int>(kPool, count);
  std::vector<int> order(static_cast<size_t>(count));
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return mem[a].cost > mem[b].cost; });
  std::vector<double> load(static_cast<size_t>(nst), 0.0);
  std::vector<int> lane(static_cast<size_t>(count));
  for (int i : order) {
    const int k = static_cast<int>(std::min_element(load.begin(), load.end()) - load.begin());
    lane[i] = k;
    load[k] += mem[i].cost;
  }

  std::lock_guard<std::mutex> lock(pool->mu);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!cuda_ok(cudaEventRecord(pool->fork, st), "record fork event")) return L1S_ERR_CUDA;
  for (int k = 0; k < nst; ++k)
    if (!cuda_ok(cudaStreamWaitEvent(pool->st[k], pool->fork, 0), "fork")) return L1S_ERR_CUDA;
  int rc = L1S_OK;
  unsigned char* base = static_cast<unsigned char*>(ws);
  for (int i : order) {
    rc = enqueue_member(probs[i], mem[i], base, flags_dev, i, pool->st[lane[i]]);
    if (rc != L1S_OK) break;
  }
  // Join every pool stream back, also after a failed enqueue, so that a capture in
  // progress on `stream` stays well formed.
  for (int k = 0; k < nst; ++k) {
    if (!cuda_ok(cudaEventRecord(pool->join[k], pool->st[k]), "record join event") ||
        !cuda_ok(cudaStreamWaitEvent(st, pool->join[k], 0), "join"))
      rc = L1S_ERR_CUDA;
  }
  return rc;
}

int l1s_autotune(const l1s_problem* prob, int32_t trials, l1s_schedule* best, double* best_ms, void* ws,
                 size_t ws_bytes, void* stream) {
  TraceRange trace_("l1s_autotune");
  if (!prob || !best || trials < 1 || trials > 1000) return set_error("bad arguments"), L1S_ERR_INVALID_ARG;
  if (!check_member(*prob, 0)) return L1S_ERR_INVALID_ARG;
  const l1s_problem& pr = *prob;
  Plan base;
  const l1s_schedule none{};
  if (!make_plan(&pr.params, pr.n, pr.d, pr.dtype, false, &base, &none)) return L1S_ERR_INVALID_ARG;
  if (!check_ws(base, ws, ws_bytes)) return L1S_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned char* w = static_cast<unsigned char*>(ws);
  const int64_t cap = coreset_capacity_of(&pr.params);
  int64_t* idx = reinterpret_cast<int64_t*>(w + base.off_idx_tmp);
  double* wts = reinterpret_cast<double*>(idx + cap);
  StatusBlock* sb = reinterpret_cast<StatusBlock*>(w + base.off_status);

  cudaEvent_t e0, e1;
  if (!cuda_ok(cudaEventCreate(&e0), "event") || !cuda_ok(cudaEventCreate(&e1), "event")) return L1S_ERR_CUDA;
  // Median time of `trials` runs of the coreset chain under schedule c (+inf if it does not plan).
  auto time_of = [&](const l1s_schedule& c) -> double {
    Plan pl;
    if (!make_plan(&pr.params, pr.n, pr.d, pr.dtype, false, &pl, &c)) return INFINITY;
    pl.lam_m_in_smem = 1;
    std::vector<float> t;
    for (int r = 0; r <= trials; ++r) {
      if (!cuda_ok(cudaEventRecord(e0, st), "record") ||
          coreset_impl(pl, pr.A_dev, pr.lda, pr.dtype, pr.b_dev, &pr.params, cap, idx, wts, nullptr, &sb->count,
                       w, st) != L1S_OK ||
          !cuda_ok(cudaEventRecord(e1, st), "record") || !cuda_ok(cudaEventSynchronize(e1), "synchronize"))
        return INFINITY;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (r > 0) t.push_back(ms);   // the first run warms caches and the instruction path
    }
    std::nth_element(t.begin(), t.begin() + t.size() / 2, t.end());
    return t[t.size() / 2];
  };

  // Coordinate descent: the phase-1 kernel and its residency, then the λ grid, then the
  // sampling chunking, each with the others held at the best found so far.
  l1s_schedule cur{};
  double cur_t = time_of(cur);
  auto try_field = [&](int32_t l1s_schedule::*field, std::initializer_list<int32_t> values) {
    for (int32_t v : values) {
      l1s_schedule c = cur;
      c.*field = v;
      const double t = time_of(c);
      if (t < cur_t) {
        cur_t = t;
        cur = c;
      }
    }
  };
  int v3_slices = 0;
  for (int v = 1; v <= 7; ++v) {
    l1s_schedule c = cur;
    c.fct_variant = v;
    Plan probe;
    if (!make_plan(&pr.params, pr.n, pr.d, pr.dtype, false, &probe, &c)) continue;
    const bool plain = !probe.fct_ws && !probe.fct_sorted && !probe.fct_cols;
    if (v == 3 && plain && !probe.fct_staged) v3_slices = probe.fct_slices;
    const bool applies = (v == 4 && probe.fct_sorted) || (v == 1 && probe.fct_ws && !probe.fct_lean) ||
                         (v == 5 && probe.fct_lean) ||
                         (v == 2 && plain && probe.fct_staged) || (v == 3 && plain && !probe.fct_staged) ||
                         (v == 6 && plain && !probe.fct_staged && probe.fct_slices < v3_slices) ||
                         (v == 7 && probe.fct_cols);
    if (!applies) continue;
    for (int per = 1; per <= 4; ++per) {
      c.fct_ctas_per_sm = per;
      const double t = time_of(c);
      if (t < cur_t) {
        cur_t = t;
        cur = c;
      }
    }
  }
  try_field(&l1s_schedule::lam_ctas_per_sm, {2, 4, 8, 16, 32});
  try_field(&l1s_schedule::smp_chunks_per_sm, {1, 2, 4, 8, 16});
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  set_error("");
  if (!std::isfinite(cur_t)) return set_error("no schedule ran"), L1S_ERR_CUDA;
  *best = cur;
  if (best_ms) *best_ms = cur_t;
  return l1s_schedule_set(pr.d, pr.dtype, pr.params.s, &cur);
}

}  // extern "C"
