// Serving form: a request loop with continuous batching on one GPU.
//
// Trajectory requests (a fused circuit, a seed, a trajectory range, a sample
// count) are submitted as they arrive.  A fixed set of workers, each with
// its own CUDA stream, takes requests in arrival order as soon as a worker is
// free and the request's device footprint fits the memory budget
// (8 * 2^n bytes per resident state, the paper's memory rule of Sec. IV.A),
// so requests that arrive while others run are admitted as slots and memory
// free up and their kernels overlap on the device.  Small states run their
// trajectories in one batched persistent launch (batch.cu), larger ones the
// plain trajectory loop (runtime.cu); either way every request's results
// depend only on its own circuit, seed and trajectory ids, so a request gives
// the same result alone and in any mix.
//
// Failure handling is host-side: a request that hits an out-of-memory error
// is deferred and retried, a request whose worker thread died is requeued by
// the watchdog and a replacement worker is started, and queued requests can
// be cancelled.  qt_server_inject drives these paths deterministically (for
// tests); a dry-run mode replaces the GPU work by a timed wait so the
// scheduling logic runs without a GPU.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "kernels.h"
#include "qt_internal.h"

namespace qt {
namespace {

using Clock = std::chrono::steady_clock;

double now_s() {
  return std::chrono::duration<double>(Clock::now().time_since_epoch()).count();
}

enum ReqState : int32_t { kQueued = 0, kRunning = 1, kDone = 2, kFailed = 3, kCancelled = 4 };

struct Req {
  const qt_fused* f = nullptr;
  qt_server_request r{};
  uint32_t n = 0;
  uint64_t bytes = 0;
  int32_t state = kQueued;
  qt_status status = QT_OK;
  std::string err;
  uint32_t attempts = 0;
  int32_t worker = -1;
  bool batched = false;
  double t_submit = 0, t_start = 0, t_done = 0;
  std::vector<uint64_t> samples;
  uint64_t flushes = 0;
};

struct Worker {
  std::thread th;
  cudaStream_t stream = nullptr;
  std::atomic<bool> finished{false};
  std::atomic<bool> crashed{false};
  uint64_t current = 0;          // request being run (0: none)
};

}  // namespace
}  // namespace qt

using namespace qt;

struct qt_server {
  qt_server_config cfg{};
  int device = 0;
  uint32_t sms = 152;        // SMs of the device (sizes the batched form's arena)
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, Req> reqs;
  uint64_t next_id = 1;
  uint64_t inflight = 0, peak_inflight = 0;
  uint32_t requeued = 0, deferred = 0;
  bool stop = false;
  std::vector<std::unique_ptr<Worker>> workers;
  std::thread watchdog;
  // fault injection (host side)
  uint32_t inj_exit = 0, inj_oom = 0;

  void start_worker(size_t w);
  void worker_loop(size_t w);
  void watchdog_loop();
  qt_status execute(Req& q, cudaStream_t st);
};

namespace qt {
namespace {

uint64_t footprint(uint32_t n, bool batched, uint32_t sms) {
  const uint64_t state = 8ull << n;
  // batched form: states <= 2^14 sit in shared memory; larger ones take one
  // global slot per SM (the arena qt_batch_run sizes by the SM count).  Plain
  // loop: one resident state.  Plus scratch.
  uint64_t b = batched ? (n > 14 ? state * sms : 0) : state;
  b += (16ull << 20) + (state >> 8);
  return b;
}

// One trajectory per SM in the batched kernel: worth it for states that fit
// in shared memory, and for larger ones (up to small_n_max) only when the
// request has enough trajectories to occupy the GPU.
bool use_batched(const qt_server_config& c, const qt_fused* f, uint32_t num_traj) {
  if (c.small_n_max == 0 || f->c->n > c.small_n_max || f->c->n > 20) return false;
  if (f->c->n > 14 && num_traj < 64) return false;
  for (const auto& g : f->gates)
    if (g.targets.size() > 4) return false;
  for (const auto& op : f->c->ops)
    if (op.q > 2) return false;
  return true;
}

}  // namespace
}  // namespace qt

qt_status qt_server::execute(Req& q, cudaStream_t st) {
  if (cfg.flags & QT_SERVER_DRY_RUN) {
    // scheduling only: hold the slot for a time that grows with the work
    const double us = 20.0 + 1e-3 * static_cast<double>(q.r.num_traj) * static_cast<double>(1ull << q.n);
    std::this_thread::sleep_for(std::chrono::microseconds(static_cast<int64_t>(std::min(us, 2e5))));
    q.samples.assign(static_cast<size_t>(q.r.num_traj) * q.r.samples_per_traj, 0);
    return QT_OK;
  }
  if (q.batched) {
    std::vector<const qt_fused*> fs(q.r.num_traj, q.f);
    qt_batch* b = nullptr;
    qt_status s = qt_batch_create(q.r.num_traj, fs.data(), &b);
    if (s != QT_OK) return s;
    qt_batch_params p{};
    p.seed = q.r.seed;
    p.first_traj = q.r.first_traj;
    p.samples_per_traj = q.r.samples_per_traj;
    p.stream = st;
    s = qt_batch_run(b, &p);
    if (s == QT_OK) {
      q.samples.assign(static_cast<size_t>(q.r.num_traj) * q.r.samples_per_traj, 0);
      s = qt_batch_samples(b, q.samples.data(), q.samples.size());
      qt_batch_stats_t bs{};
      if (s == QT_OK && qt_batch_stats(b, &bs) == QT_OK) q.flushes = bs.flushes;
    }
    qt_batch_destroy(b);
    return s;
  }
  qt_run_params p{};
  p.seed = q.r.seed;
  p.first_traj = q.r.first_traj;
  p.num_traj = q.r.num_traj;
  p.mode = QT_DELAYED;
  p.precision = QT_FP32;
  p.samples_per_traj = q.r.samples_per_traj;
  p.stream = st;
  qt_run* run = nullptr;
  qt_status s = qt_run_trajectories(q.f, &p, &run);
  if (s != QT_OK) return s;
  q.samples.assign(static_cast<size_t>(q.r.num_traj) * q.r.samples_per_traj, 0);
  s = qt_sample(run, q.r.samples_per_traj, q.samples.data());
  qt_run_stats_t rs{};
  if (s == QT_OK && qt_run_stats(run, &rs) == QT_OK) q.flushes = rs.flushes;
  qt_run_destroy(run);
  return s;
}

void qt_server::worker_loop(size_t w) {
  Worker& me = *workers[w];
  struct Done {
    Worker& w;
    ~Done() { w.finished = true; }
  } done{me};
  cudaSetDevice(device);
  for (;;) {
    uint64_t id = 0;
    Req* q = nullptr;
    {
      std::unique_lock<std::mutex> lk(mu);
      cv_work.wait(lk, [&] {
        if (stop) return true;
        if (queue.empty()) return false;
        const Req& head = reqs[queue.front()];
        return inflight + head.bytes <= cfg.budget_bytes;     // FIFO admission by footprint
      });
      if (stop) return;
      id = queue.front();
      queue.pop_front();
      q = &reqs[id];
      q->state = kRunning;
      q->worker = static_cast<int32_t>(w);
      q->attempts++;
      if (q->attempts == 1) q->t_start = now_s();
      inflight += q->bytes;
      peak_inflight = std::max(peak_inflight, inflight);
      me.current = id;
      if (inj_exit) {                 // injected fault: this worker dies holding the request
        --inj_exit;
        me.crashed = true;
        return;
      }
    }
    qt_status s;
    bool oom = false;
    {
      std::unique_lock<std::mutex> lk(mu);
      if (inj_oom) { --inj_oom; oom = true; }
    }
    if (oom) {
      s = set_error(QT_ERR_OUT_OF_MEMORY, "injected allocation failure");
    } else {
      s = execute(*q, me.stream);
    }
    std::string msg = s == QT_OK ? std::string() : std::string(qt_last_error());
    {
      std::lock_guard<std::mutex> lk(mu);
      inflight -= q->bytes;
      me.current = 0;
      if (s == QT_ERR_OUT_OF_MEMORY && q->attempts < 4 && q->state != kCancelled) {
        q->state = kQueued;                 // deferred, not lost: back to the head of the queue
        queue.push_front(id);
        deferred++;
      } else {
        q->state = s == QT_OK ? kDone : kFailed;
        q->status = s;
        q->err = msg;
        q->t_done = now_s();
      }
    }
    cv_work.notify_all();
    cv_done.notify_all();
  }
}

void qt_server::start_worker(size_t w) {
  workers[w]->finished = false;
  workers[w]->crashed = false;
  workers[w]->th = std::thread([this, w] { worker_loop(w); });
}

void qt_server::watchdog_loop() {
  std::unique_lock<std::mutex> lk(mu);
  while (!stop) {
    cv_done.wait_for(lk, std::chrono::milliseconds(5));
    if (stop) break;
    for (size_t w = 0; w < workers.size(); ++w) {
      Worker& k = *workers[w];
      if (!k.finished || !k.crashed) continue;
      // the worker died holding a request: requeue it by id, start a replacement
      const uint64_t id = k.current;
      if (id) {
        Req& q = reqs[id];
        inflight -= q.bytes;
        if (q.state == kRunning) {
          q.state = kQueued;
          queue.push_front(id);
          requeued++;
        }
        k.current = 0;
      }
      lk.unlock();
      if (k.th.joinable()) k.th.join();
      lk.lock();
      if (!stop) start_worker(w);
      cv_work.notify_all();
    }
  }
}

extern "C" {

qt_status qt_server_create(const qt_server_config* cfg, qt_server** out) {
  clear_error();
  if (!cfg || !out) return set_error(QT_ERR_INVALID_ARG, "qt_server_create: NULL argument");
  *out = nullptr;
  if (cfg->max_slots < 1 || cfg->max_slots > 64)
    return set_error(QT_ERR_INVALID_ARG, "qt_server_create: max_slots %u outside 1..64", cfg->max_slots);
  if (cfg->budget_bytes == 0) return set_error(QT_ERR_INVALID_ARG, "qt_server_create: zero budget");
  std::unique_ptr<qt_server> S(new (std::nothrow) qt_server());
  if (!S) return set_error(QT_ERR_OUT_OF_MEMORY, "qt_server_create: host allocation");
  S->cfg = *cfg;
  if (!(cfg->flags & QT_SERVER_DRY_RUN)) {
    if (cudaGetDevice(&S->device) != cudaSuccess) return set_error(QT_ERR_CUDA, "qt_server_create: no CUDA device");
    S->sms = static_cast<uint32_t>(sm_count());
  }
  S->workers.resize(cfg->max_slots);
  for (uint32_t w = 0; w < cfg->max_slots; ++w) {
    S->workers[w] = std::make_unique<Worker>();
    if (!(cfg->flags & QT_SERVER_DRY_RUN)) {
      if (cudaStreamCreateWithFlags(&S->workers[w]->stream, cudaStreamNonBlocking) != cudaSuccess)
        return set_error(QT_ERR_CUDA, "qt_server_create: cudaStreamCreate");
    }
  }
  for (uint32_t w = 0; w < cfg->max_slots; ++w) S->start_worker(w);
  S->watchdog = std::thread([s = S.get()] { s->watchdog_loop(); });
  *out = S.release();
  return QT_OK;
}

qt_status qt_server_submit(qt_server* s, const qt_fused* f, const qt_server_request* r, uint64_t* id) {
  clear_error();
  if (!s || !f || !r || !id) return set_error(QT_ERR_INVALID_ARG, "qt_server_submit: NULL argument");
  if (r->num_traj == 0) return set_error(QT_ERR_INVALID_ARG, "qt_server_submit: num_traj is 0");
  Req q;
  q.f = f;
  q.r = *r;
  q.n = f->c->n;
  q.batched = use_batched(s->cfg, f, r->num_traj);
  q.bytes = footprint(q.n, q.batched, s->sms);
  if (q.bytes > s->cfg.budget_bytes)
    return set_error(QT_ERR_OUT_OF_MEMORY, "qt_server_submit: footprint %llu bytes exceeds the budget %llu",
                     static_cast<unsigned long long>(q.bytes), static_cast<unsigned long long>(s->cfg.budget_bytes));
  q.t_submit = now_s();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    const uint64_t i = s->next_id++;
    s->reqs.emplace(i, std::move(q));
    s->queue.push_back(i);
    *id = i;
  }
  s->cv_work.notify_all();
  return QT_OK;
}

qt_status qt_server_poll(qt_server* s, uint64_t id, int32_t* state) {
  clear_error();
  if (!s || !state) return set_error(QT_ERR_INVALID_ARG, "qt_server_poll: NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return set_error(QT_ERR_INVALID_ARG, "qt_server_poll: unknown request %llu", (unsigned long long)id);
  *state = it->second.state;
  return QT_OK;
}

qt_status qt_server_wait(qt_server* s, uint64_t id, uint64_t timeout_ns) {
  clear_error();
  if (!s) return set_error(QT_ERR_INVALID_ARG, "qt_server_wait: NULL server");
  std::unique_lock<std::mutex> lk(s->mu);
  auto done = [&] {
    auto it = s->reqs.find(id);
    return it == s->reqs.end() || it->second.state >= kDone;
  };
  if (timeout_ns == 0) s->cv_done.wait(lk, done);
  else if (!s->cv_done.wait_for(lk, std::chrono::nanoseconds(timeout_ns), done))
    return set_error(QT_ERR_TIMEOUT, "qt_server_wait: request %llu not finished", (unsigned long long)id);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return set_error(QT_ERR_INVALID_ARG, "qt_server_wait: unknown request");
  return QT_OK;
}

qt_status qt_server_cancel(qt_server* s, uint64_t id) {
  clear_error();
  if (!s) return set_error(QT_ERR_INVALID_ARG, "qt_server_cancel: NULL server");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return set_error(QT_ERR_INVALID_ARG, "qt_server_cancel: unknown request");
  if (it->second.state != kQueued)
    return set_error(QT_ERR_INVALID_ARG, "qt_server_cancel: request %llu is not queued", (unsigned long long)id);
  s->queue.erase(std::remove(s->queue.begin(), s->queue.end(), id), s->queue.end());
  it->second.state = kCancelled;
  it->second.t_done = now_s();
  s->cv_done.notify_all();
  s->cv_work.notify_all();
  return QT_OK;
}

qt_status qt_server_result(qt_server* s, uint64_t id, uint64_t* samples, size_t cap, qt_server_req_info* info) {
  clear_error();
  if (!s) return set_error(QT_ERR_INVALID_ARG, "qt_server_result: NULL server");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return set_error(QT_ERR_INVALID_ARG, "qt_server_result: unknown request");
  const Req& q = it->second;
  if (info) {
    info->state = q.state;
    info->status = q.status;
    info->attempts = q.attempts;
    info->worker = q.worker;
    info->batched = q.batched ? 1u : 0u;
    info->num_traj = q.r.num_traj;
    info->samples_per_traj = q.r.samples_per_traj;
    info->bytes = q.bytes;
    info->flushes = q.flushes;
    info->queued_s = (q.t_start > 0 ? q.t_start : q.t_done) - q.t_submit;
    info->latency_s = q.t_done > 0 ? q.t_done - q.t_submit : -1.0;
  }
  if (samples) {
    if (q.state != kDone) return set_error(QT_ERR_INVALID_ARG, "qt_server_result: request not done");
    if (cap < q.samples.size()) return set_error(QT_ERR_INVALID_ARG, "qt_server_result: cap %zu < %zu", cap, q.samples.size());
    std::memcpy(samples, q.samples.data(), sizeof(uint64_t) * q.samples.size());
  }
  if (q.state == kFailed) return set_error(q.status, "qt_server_result: request failed: %s", q.err.c_str());
  return QT_OK;
}

qt_status qt_server_release(qt_server* s, uint64_t id) {
  clear_error();
  if (!s) return set_error(QT_ERR_INVALID_ARG, "qt_server_release: NULL server");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return set_error(QT_ERR_INVALID_ARG, "qt_server_release: unknown request");
  if (it->second.state < kDone) return set_error(QT_ERR_INVALID_ARG, "qt_server_release: request still active");
  s->reqs.erase(it);
  return QT_OK;
}

qt_status qt_server_stats(qt_server* s, qt_server_stats_t* out) {
  clear_error();
  if (!s || !out) return set_error(QT_ERR_INVALID_ARG, "qt_server_stats: NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  std::memset(out, 0, sizeof(*out));
  out->budget = s->cfg.budget_bytes;
  out->inflight_bytes = s->inflight;
  out->peak_inflight_bytes = s->peak_inflight;
  out->requeued = s->requeued;
  out->deferred = s->deferred;
  for (const auto& kv : s->reqs) {
    if (kv.second.state == kQueued) out->queued++;
    else if (kv.second.state == kRunning) out->running++;
    else if (kv.second.state == kDone) out->done++;
    else if (kv.second.state == kFailed) out->failed++;
  }
  for (const auto& w : s->workers) out->workers_alive += w->finished ? 0u : 1u;
  return QT_OK;
}

qt_status qt_server_inject(qt_server* s, uint32_t fault, uint32_t count) {
  clear_error();
  if (!s) return set_error(QT_ERR_INVALID_ARG, "qt_server_inject: NULL server");
  std::lock_guard<std::mutex> lk(s->mu);
  if (fault == QT_FAULT_WORKER_EXIT) s->inj_exit += count;
  else if (fault == QT_FAULT_ALLOC) s->inj_oom += count;
  else return set_error(QT_ERR_INVALID_ARG, "qt_server_inject: unknown fault %u", fault);
  return QT_OK;
}

void qt_server_destroy(qt_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  s->cv_done.notify_all();
  if (s->watchdog.joinable()) s->watchdog.join();
  for (auto& w : s->workers)
    if (w->th.joinable()) w->th.join();
  for (auto& w : s->workers)
    if (w->stream) cudaStreamDestroy(w->stream);
  delete s;
}

}  // extern "C"
