// jd_server.cu -- the serving loop: many optimal-control requests solved concurrently
// on one GPU (jd_server_* in include/jd.h).
//
// Requests arrive from any host thread (jd_server_submit copies them into a FIFO).  One
// worker thread owns the device work:
//   * admission: a request is admitted when a slot is free and its device footprint
//     (problem buffers + adjoint plan) fits what is left of the HBM budget; requests
//     behind one that does not fit may go first (backfill);
//   * each admitted request gets a slot: its own CUDA stream, pinned scalar and output
//     buffers, and a problem object whose buffers come from the stream-ordered pool
//     allocator (freeing them does not synchronize the device);
//   * every active request is an optimizer state machine (Algorithm 5.4); the worker
//     polls each slot's event and advances the machines whose phase has finished, so
//     the kernels of all active requests overlap on the device while the host takes
//     one request's line-search decision;
//   * small requests (d <= 2, du = 1, the stored plan, at most batch_paths paths) share
//     launches: their machines defer each phase, and the worker launches the deferred
//     phases of up to kBatchMax requests with the same precision and dimension, whatever
//     their phases, as one batched sequence (jd::opt_launch_batch) on one of a few batch
//     streams -- forward and adjoint sweeps over all their paths, one launch per
//     reduction and per optimizer step, instead of a launch sequence per request;
//   * a finished request frees its slot and memory, and the next ones are admitted.
// Each request runs the arithmetic and the host decisions of jd_optimize on its own
// buffers (a batched launch gives every problem the bits of its own launches), so its
// result does not depend on what else is running.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "jd_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t ticket = 0;
  jd_problem_desc desc{};
  std::vector<double> A, C, B, dA, sigma, x0, q, xd;
  jd_opt_params o{};
  double t_submit = 0, t_admit = -1, t_done = -1;
  size_t bytes = 0;
  jd_adjoint_mode plan = JD_ADJ_AUTO;
  bool done = false, released = false;
  jd_opt_result r{};
  int grads = 0;           // gradient evaluations
  std::vector<double> u;   // final control (Nt*du), dropped once handed out
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;
  double *pinned_scal = nullptr;
  double *pinned_u = nullptr;
  size_t pinned_u_cap = 0;
  jd_problem *p = nullptr;
  Request *req = nullptr;
  jd::OptMachine m;
  bool batch = false;   // the request's phases run in batched launches
};

constexpr int kBatchStreams = 4;

}  // namespace

struct jd_server {
  int device = 0;
  size_t budget = 0, used = 0;
  std::vector<Slot> slots;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Request *> pending;
  std::unordered_map<uint64_t, Request *> all;
  uint64_t next_ticket = 1;
  std::atomic<bool> stop{false};
  std::atomic<int64_t> batch_paths{JD_SERVER_BATCH_PATHS};
  std::atomic<int64_t> batch_launches{0}, batch_phases{0};
  cudaStream_t bstream[kBatchStreams] = {};
  int next_bstream = 0;
  std::thread worker;
  Clock::time_point t0;
  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

// Plan and bytes for a request given the free budget: STORED when it fits in a
// quarter of the budget (so that several large requests can run side by side) and in
// what is free, else RECOMPUTE (d <= 8), else nothing yet.  A request whose smallest
// plan exceeds the whole budget can never run.
bool choose_plan(const jd_problem_desc &q, size_t budget, size_t free_b, jd_adjoint_mode *plan, size_t *bytes,
                 bool *never) {
  const size_t st = jd::problem_bytes(q, JD_ADJ_STORED);
  const bool rec_ok = q.d <= 8;
  if (!rec_ok) {
    // d = 32 has the stored plan only; when all paths do not fit a quarter of the
    // budget, the problem stores them block by block inside the bytes reserved here
    const size_t mn = jd::problem_bytes_min(q);
    *never = mn > budget;
    if (*never) return false;
    const size_t cap = std::max(budget / 4, mn);
    const size_t want = std::min(st, cap);
    if (want > free_b) return false;
    *plan = JD_ADJ_STORED;
    *bytes = want;
    return true;
  }
  const size_t rc = jd::problem_bytes(q, JD_ADJ_RECOMPUTE);
  *never = false;
  jd_adjoint_mode want = q.mode;
  if (want == JD_ADJ_AUTO) want = st <= budget / 4 ? JD_ADJ_STORED : JD_ADJ_RECOMPUTE;
  const size_t need = want == JD_ADJ_STORED ? st : rc;
  if (need > budget) {
    if (q.mode == JD_ADJ_AUTO && want == JD_ADJ_STORED && rc <= budget) {
      want = JD_ADJ_RECOMPUTE;
    } else {
      *never = true;
      return false;
    }
  }
  const size_t need2 = want == JD_ADJ_STORED ? st : rc;
  if (need2 > free_b) return false;
  *plan = want;
  *bytes = need2;
  // room for the second buffer set of jd_optimize's paired trials when it keeps the
  // request within a quarter of the budget and what is free (else single trials)
  const size_t pb = jd::pair_bytes(q, want);
  if (pb && need2 + pb <= budget / 4 && need2 + pb <= free_b) *bytes = need2 + pb;
  return true;
}

void finish_request(jd_server *s, Slot &sl, jd_status st) {
  Request *rq = sl.req;
  const size_t n = (size_t)rq->desc.Nt * rq->desc.du;
  {
    std::lock_guard<std::mutex> g(s->mu);
    rq->grads = sl.m.grads;
    if (st == JD_OK) {
      rq->r = sl.m.r;
      rq->u.assign(sl.pinned_u, sl.pinned_u + n);
    } else {
      std::memset(&rq->r, 0, sizeof(rq->r));
      rq->r.status = st;
    }
    rq->t_done = s->now();
    rq->done = true;
  }
  jd::opt_release(sl.m);
  if (sl.p) jd_problem_destroy(sl.p);   // stream-ordered frees: no device-wide sync
  sl.p = nullptr;
  sl.req = nullptr;
  s->used -= rq->bytes;
  s->cv.notify_all();
}

// Admit one request into a free slot; returns false when nothing can be admitted now.
bool admit_one(jd_server *s) {
  Slot *free_slot = nullptr;
  for (auto &sl : s->slots)
    if (!sl.req) {
      free_slot = &sl;
      break;
    }
  if (!free_slot) return false;
  Request *rq = nullptr;
  jd_adjoint_mode plan = JD_ADJ_AUTO;
  size_t bytes = 0;
  std::vector<Request *> rejected;
  {
    std::lock_guard<std::mutex> g(s->mu);
    for (auto it = s->pending.begin(); it != s->pending.end();) {
      bool never = false;
      if (choose_plan((*it)->desc, s->budget, s->budget - s->used, &plan, &bytes, &never)) {
        rq = *it;
        s->pending.erase(it);
        break;
      }
      if (never) {
        rejected.push_back(*it);
        it = s->pending.erase(it);
        continue;
      }
      ++it;
    }
    for (Request *r : rejected) {
      r->r.status = JD_ERR_OOM;
      r->t_admit = r->t_done = s->now();
      r->done = true;
    }
  }
  if (!rejected.empty()) s->cv.notify_all();
  if (!rq) return !rejected.empty();
  Slot &sl = *free_slot;
  sl.m = jd::OptMachine();
  sl.m.ev = sl.ev;
  sl.m.use_graphs = true;   // every phase of a solo request replays a captured graph
  const jd_problem_desc &rd = rq->desc;
  sl.batch = rd.d <= 2 && rd.du == 1 && plan == JD_ADJ_STORED && !rd.use_tensor_cores &&
             rd.M <= s->batch_paths.load();
  rq->t_admit = s->now();
  rq->plan = plan;
  rq->bytes = bytes;
  s->used += bytes;
  sl.req = rq;
  const size_t n = (size_t)rq->desc.Nt * rq->desc.du;
  if (sl.pinned_u_cap < n) {
    if (sl.pinned_u) cudaFreeHost(sl.pinned_u);
    sl.pinned_u = nullptr;
    sl.pinned_u_cap = 0;
    if (cudaMallocHost((void **)&sl.pinned_u, n * 8) != cudaSuccess) {
      finish_request(s, sl, JD_ERR_CUDA);
      return true;
    }
    sl.pinned_u_cap = n;
  }
  jd_problem_desc q = rq->desc;
  q.mode = plan;
  q.mem_budget_bytes = bytes;
  q.cuda_stream = nullptr;
  jd::ProblemOpts opts;
  opts.stream = sl.stream;
  opts.pinned = sl.pinned_scal;
  opts.async_alloc = true;
  opts.no_pre = sl.batch;   // batched sweeps draw in the sweep
  jd_status st = jd::create_problem(q, opts, &sl.p);
  if (st != JD_OK) {
    sl.p = nullptr;
    finish_request(s, sl, st);
    return true;
  }
  if (sl.batch && !jd::opt_batchable(sl.p)) sl.batch = false;
  if (sl.batch) {   // phases deferred to batched launches; no graphs
    sl.m.defer = true;
    sl.m.use_graphs = false;
  }
  // u^0 = 0 projected into the bounds
  const double u0 = std::min(std::max(0.0, q.u_min), q.u_max);
  for (size_t i = 0; i < n; ++i) sl.pinned_u[i] = u0;
  if (cudaMemcpyAsync(sl.p->u_in, sl.pinned_u, n * 8, cudaMemcpyHostToDevice, sl.stream) != cudaSuccess) {
    finish_request(s, sl, JD_ERR_CUDA);
    return true;
  }
  st = jd::opt_begin(sl.m, sl.p, rq->o, sl.pinned_u, JD_MEM_HOST, nullptr);
  if (st != JD_OK) finish_request(s, sl, st);
  return true;
}

// Launch the deferred phases of batched requests: grouped by batch key, up to
// kBatchMax per launch, on the batch streams in turn.
void launch_batches(jd_server *s) {
  std::vector<Slot *> w;
  for (auto &sl : s->slots)
    if (sl.req && sl.batch && jd::opt_batch_key(sl.m) >= 0) w.push_back(&sl);
  std::stable_sort(w.begin(), w.end(),
                   [](const Slot *a, const Slot *b) { return jd::opt_batch_key(a->m) < jd::opt_batch_key(b->m); });
  for (size_t i = 0; i < w.size();) {
    const int key = jd::opt_batch_key(w[i]->m);
    size_t j = i;
    jd::OptMachine *ms[jd::kBatchMax];
    int n = 0;
    while (j < w.size() && n < jd::kBatchMax && jd::opt_batch_key(w[j]->m) == key) ms[n++] = &w[j++]->m;
    cudaStream_t st = s->bstream[s->next_bstream];
    s->next_bstream = (s->next_bstream + 1) % kBatchStreams;
    const jd_status e = jd::opt_launch_batch(ms, n, st);
    if (e != JD_OK) {
      cudaStreamSynchronize(st);   // nothing of the group may still run when its buffers go
      for (size_t k = i; k < j; ++k) finish_request(s, *w[k], e);
    } else {
      s->batch_launches.fetch_add(1);
      s->batch_phases.fetch_add(n);
    }
    i = j;
  }
}

void worker_main(jd_server *s) {
  cudaSetDevice(s->device);
  for (;;) {
    while (admit_one(s)) {
    }
    launch_batches(s);   // the first phases of the requests just admitted
    bool progress = false, active = false;
    for (auto &sl : s->slots) {
      if (!sl.req) continue;
      active = true;
      if (sl.batch && sl.m.want != jd::OptMachine::IDLE) continue;   // not launched yet
      const cudaError_t q = cudaEventQuery(sl.ev);
      if (q == cudaErrorNotReady) continue;
      progress = true;
      if (q != cudaSuccess) {
        finish_request(s, sl, JD_ERR_CUDA);
        continue;
      }
      const jd_status st = jd::opt_advance(sl.m);
      if (st != JD_OK)
        finish_request(s, sl, st);
      else if (sl.m.phase == jd::OptMachine::DONE)
        finish_request(s, sl, JD_OK);
    }
    launch_batches(s);   // the phases decided in this pass
    if (progress) continue;
    std::unique_lock<std::mutex> g(s->mu);
    if (!active) {
      if (s->stop.load() && s->pending.empty()) return;
      if (s->pending.empty())
        s->cv.wait_for(g, std::chrono::milliseconds(50));
      else
        s->cv.wait_for(g, std::chrono::microseconds(200));   // waiting for memory
    } else {
      g.unlock();
      std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
  }
}

void copy_arrays(Request *rq, const jd_problem_desc &q) {
  const size_t d = q.d, dd = d * d;
  rq->A.assign(q.A, q.A + dd);
  if (q.C) rq->C.assign(q.C, q.C + dd);
  rq->B.assign(q.B, q.B + d * q.du);
  if (q.dA) rq->dA.assign(q.dA, q.dA + dd);
  rq->sigma.assign(q.sigma, q.sigma + d);
  rq->x0.assign(q.x0, q.x0 + d);
  rq->q.assign(q.q, q.q + d);
  rq->xd.assign(q.xd, q.xd + (size_t)(q.Nt + 1) * d);
  rq->desc = q;
  rq->desc.A = rq->A.data();
  rq->desc.C = q.C ? rq->C.data() : nullptr;
  rq->desc.B = rq->B.data();
  rq->desc.dA = q.dA ? rq->dA.data() : nullptr;
  rq->desc.sigma = rq->sigma.data();
  rq->desc.x0 = rq->x0.data();
  rq->desc.q = rq->q.data();
  rq->desc.xd = rq->xd.data();
}

}  // namespace

extern "C" {

jd_status jd_server_create(size_t hbm_budget, int max_slots, jd_server **out) {
  if (!out || max_slots < 1 || max_slots > 256) return JD_ERR_INVALID_ARG;
  *out = nullptr;
  jd_server *s = new jd_server();
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    delete s;
    return JD_ERR_CUDA;
  }
  if (!hbm_budget) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      delete s;
      return JD_ERR_CUDA;
    }
    hbm_budget = fr / 10 * 8;
  }
  s->budget = hbm_budget;
  // Keep freed blocks in the stream-ordered pool (no release to the driver between
  // requests), and raise the per-thread stack limit once for every kernel family so
  // that creating a problem never changes a device limit while others run.
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, s->device) == cudaSuccess) {
    uint64_t thr = hbm_budget;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  size_t need = 0;
  for (int prec = 0; prec < 2; ++prec)
    for (int D : {1, 2, 4, 8, 32})
      for (int DU : {1, 4})
        if (const jd::PathOps *ops = jd::path_ops_dims(prec, D, DU)) need = std::max(need, ops->stack_bytes());
  size_t cur = 0;
  if (cudaDeviceGetLimit(&cur, cudaLimitStackSize) == cudaSuccess && cur < need)
    cudaDeviceSetLimit(cudaLimitStackSize, need);
  for (auto &b : s->bstream)
    if (cudaStreamCreateWithFlags(&b, cudaStreamNonBlocking) != cudaSuccess) {
      jd_server_destroy(s);
      return JD_ERR_CUDA;
    }
  s->slots.resize(max_slots);
  for (auto &sl : s->slots) {
    if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaMallocHost((void **)&sl.pinned_scal, jd::kScalars * 8) != cudaSuccess) {
      jd_server_destroy(s);
      return JD_ERR_CUDA;
    }
  }
  s->t0 = Clock::now();
  s->worker = std::thread(worker_main, s);
  *out = s;
  return JD_OK;
}

jd_status jd_server_submit(jd_server *s, const jd_problem_desc *d, const jd_opt_params *o, uint64_t *ticket) {
  if (!s || !d || !o || !ticket) return JD_ERR_INVALID_ARG;
  // the same checks as jd_problem_create, without touching the device
  size_t bytes = 0;
  const jd_status st = jd_problem_footprint(d, d->d > 8 ? JD_ADJ_STORED : JD_ADJ_RECOMPUTE, &bytes);
  if (st != JD_OK) return st;
  if (o->max_iter < 0 || o->max_backtracks < 0 || !(o->armijo_c >= 0.0)) return JD_ERR_INVALID_ARG;
  Request *rq = new Request();
  copy_arrays(rq, *d);
  rq->o = *o;
  {
    std::lock_guard<std::mutex> g(s->mu);
    if (s->stop.load()) {
      delete rq;
      return JD_ERR_INVALID_ARG;
    }
    rq->ticket = s->next_ticket++;
    rq->t_submit = s->now();
    s->pending.push_back(rq);
    s->all[rq->ticket] = rq;
    *ticket = rq->ticket;
  }
  s->cv.notify_all();
  return JD_OK;
}

jd_status jd_server_poll(jd_server *s, uint64_t ticket, double *u_out, jd_opt_result *r) {
  if (!s) return JD_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return JD_ERR_INVALID_ARG;
  Request *rq = it->second;
  if (!rq->done) return JD_ERR_BUSY;
  if (r) *r = rq->r;
  if (u_out) {
    if (rq->released) return JD_ERR_INVALID_ARG;
    if (!rq->u.empty()) std::memcpy(u_out, rq->u.data(), rq->u.size() * 8);
    rq->u.clear();
    rq->u.shrink_to_fit();
    rq->released = true;
  }
  return JD_OK;
}

jd_status jd_server_wait(jd_server *s, uint64_t ticket, double timeout_s) {
  if (!s) return JD_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> g(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return JD_ERR_INVALID_ARG;
  Request *rq = it->second;
  const auto until = Clock::now() + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(
                                        timeout_s > 0 ? timeout_s : 1e9));
  while (!rq->done)
    if (s->cv.wait_until(g, until) == std::cv_status::timeout && !rq->done) return JD_ERR_BUSY;
  return JD_OK;
}

jd_status jd_server_info(jd_server *s, uint64_t ticket, jd_request_info *info) {
  if (!s || !info) return JD_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return JD_ERR_INVALID_ARG;
  const Request *rq = it->second;
  info->submit_s = rq->t_submit;
  info->admit_s = rq->t_admit;
  info->done_s = rq->t_done;
  info->device_bytes = rq->bytes;
  info->plan = rq->plan;
  info->done = rq->done ? 1 : 0;
  info->path_steps = rq->done ? (int64_t)rq->grads * rq->desc.M * rq->desc.Nt : 0;
  info->sweep_steps = rq->done ? (int64_t)(rq->r.sweeps + rq->grads) * rq->desc.M * rq->desc.Nt : 0;
  return JD_OK;
}

jd_status jd_server_set_batching(jd_server *s, int64_t max_paths) {
  if (!s || max_paths < 0) return JD_ERR_INVALID_ARG;
  s->batch_paths.store(max_paths);
  return JD_OK;
}

jd_status jd_server_batch_stats(jd_server *s, int64_t *launches, int64_t *phases) {
  if (!s) return JD_ERR_INVALID_ARG;
  if (launches) *launches = s->batch_launches.load();
  if (phases) *phases = s->batch_phases.load();
  return JD_OK;
}

jd_status jd_server_destroy(jd_server *s) {
  if (!s) return JD_OK;
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->stop.store(true);
    for (Request *r : s->pending) {   // requests never admitted are cancelled
      r->r.status = JD_ERR_INVALID_ARG;
      r->done = true;
    }
    s->pending.clear();
  }
  s->cv.notify_all();
  if (s->worker.joinable()) s->worker.join();   // active requests run to their end
  cudaSetDevice(s->device);
  for (auto &sl : s->slots) {
    if (sl.p) jd_problem_destroy(sl.p);
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    if (sl.stream) cudaStreamDestroy(sl.stream);
    if (sl.ev) cudaEventDestroy(sl.ev);
    if (sl.pinned_scal) cudaFreeHost(sl.pinned_scal);
    if (sl.pinned_u) cudaFreeHost(sl.pinned_u);
  }
  for (auto &b : s->bstream)
    if (b) {
      cudaStreamSynchronize(b);
      cudaStreamDestroy(b);
    }
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, s->device) == cudaSuccess) cudaMemPoolTrimTo(pool, 0);
  for (auto &kv : s->all) delete kv.second;
  delete s;
  return JD_OK;
}

}  // extern "C"
