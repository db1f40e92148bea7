// Serving form: a request loop with continuous batching on one GPU.
//
// Trajectory requests (a fused circuit, a seed, a trajectory range, a sample
// count) are submitted as they arrive and served by two kinds of executor:
//
//   - the batch lane: requests of small states (n <= 14, or up to
//     small_n_max with >= 64 trajectories) wait in their own queue; whenever
//     the lane is free it takes every queued small request at once and runs
//     all their trajectories -- each with its own circuit, seed and
//     trajectory id -- in one merged launch of the batched persistent kernel
//     (batch.cu), whose CTAs take trajectories from a device work counter.
//     Requests that arrive during a launch join the next one.  The lane's
//     device buffers are kept between launches; the global-memory state
//     slots it needs for states above 2^14 amplitudes are reserved against
//     the budget once, when the server starts;
//   - plain workers: the other requests run the plain trajectory loop
//     (runtime.cu), each worker on its own CUDA stream, admitted in arrival
//     order as soon as a worker is free and the request's device footprint
//     fits the memory budget (8 * 2^n bytes per resident state, the memory
//     rule of Sec. IV.A).  The trajectories of one request share their
//     default-choice prefix (QT_FLAG_SHARE_PREFIX): one state advances along
//     the operators every trajectory applies, and each trajectory copies it
//     at its first non-default channel, so a request holds two states.
//
// Requests that arrive while others run are admitted as the lane and slots
// and memory free up, and their kernels overlap on the device.  Every
// request's results depend only on its own circuit, seed and trajectory ids
// (the batched kernel runs each trajectory in one CTA with a fixed reduction
// order; the plain loop's prefix sharing is decided by the request alone), so
// a request gives the same result alone and in any mix.
//
// Failure handling is host-side: a request that hits an out-of-memory error
// is deferred and retried, a request whose executor thread died is requeued
// by the watchdog (every request of a merged launch, for the lane) and a
// replacement thread is started, and queued requests can be cancelled.
// qt_server_inject drives these paths deterministically (for tests); a
// dry-run mode replaces the GPU work by a timed wait so the scheduling logic
// runs without a GPU.
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

constexpr uint32_t kSmemStateMaxN = 14;       // states the batched kernel holds in shared memory
constexpr uint64_t kLaneMaxTraj = 1u << 15;   // trajectories per merged launch
constexpr uint64_t kScratch = 16ull << 20;    // per-request scratch allowance

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
  std::vector<uint64_t> held;    // requests being run (one, or a merged launch for the lane)
};

}  // namespace
}  // namespace qt

using namespace qt;

struct qt_server {
  qt_server_config cfg{};
  int device = 0;
  uint32_t sms = 152;        // SMs of the device (sizes the lane's state slots)
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<uint64_t> queue;     // plain-loop requests
  std::deque<uint64_t> bqueue;    // requests for the batch lane
  std::unordered_map<uint64_t, Req> reqs;
  uint64_t next_id = 1;
  uint64_t inflight = 0, peak_inflight = 0;
  uint32_t requeued = 0, deferred = 0;
  uint64_t lane_launches = 0, lane_trajectories = 0;
  bool stop = false;
  std::vector<std::unique_ptr<Worker>> workers;   // plain workers, then the lane (if any)
  uint32_t lane_max_n = 0;                        // 0: no lane
  uint64_t lane_bytes = 0;                        // reserved for the lane's state slots
  BatchLane* lane = nullptr;
  std::thread watchdog;
  // fault injection (host side)
  uint32_t inj_exit = 0, inj_oom = 0;

  bool is_lane(size_t w) const { return lane_max_n && w + 1 == workers.size(); }
  void start_worker(size_t w);
  void worker_loop(size_t w);
  void lane_loop(size_t w);
  void watchdog_loop();
  qt_status execute(Req& q, cudaStream_t st);
  qt_status execute_lane(const std::vector<uint64_t>& ids);
  void finish(uint64_t id, qt_status s, const std::string& msg);
};

namespace qt {
namespace {

// Device memory a plain-loop request holds while it runs: its states (two
// with the shared prefix, which needs more than one trajectory) and scratch.
uint64_t footprint(uint32_t n, uint32_t num_traj, bool share) {
  const uint64_t state = 8ull << n;
  return state * (share && num_traj > 1 ? 2 : 1) + kScratch + (state >> 8);
}

// One trajectory per CTA in the batched kernel: worth it for states that fit
// in shared memory, and for larger ones (up to the lane's limit) only when
// the request has enough trajectories to occupy the GPU.
bool use_batched(uint32_t lane_max_n, const qt_fused* f, uint32_t num_traj) {
  if (lane_max_n == 0 || f->c->n > lane_max_n) return false;
  if (f->c->n > kSmemStateMaxN && num_traj < 64) return false;
  for (const auto& g : f->gates)
    if (g.targets.size() > 6) return false;
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
  qt_run_params p{};
  p.seed = q.r.seed;
  p.first_traj = q.r.first_traj;
  p.num_traj = q.r.num_traj;
  p.mode = QT_DELAYED;
  p.precision = QT_FP32;
  p.samples_per_traj = q.r.samples_per_traj;
  p.flags = (cfg.flags & QT_SERVER_NO_SHARED_PREFIX) ? 0u : QT_FLAG_SHARE_PREFIX;
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

// One merged launch over every trajectory of the requests `ids`.
qt_status qt_server::execute_lane(const std::vector<uint64_t>& ids) {
  std::vector<LaneTraj> tr;
  std::vector<Req*> rq;
  {
    std::lock_guard<std::mutex> lk(mu);
    for (uint64_t id : ids) rq.push_back(&reqs[id]);
  }
  uint64_t nsamp = 0;
  for (Req* q : rq)
    for (uint32_t t = 0; t < q->r.num_traj; ++t) {
      tr.push_back(LaneTraj{q->f, q->r.seed, q->r.first_traj + t, q->r.samples_per_traj});
      nsamp += q->r.samples_per_traj;
    }
  std::vector<uint64_t> samples(nsamp, 0);
  std::vector<uint32_t> flushes(tr.size(), 0);
  if (cfg.flags & QT_SERVER_DRY_RUN) {
    double us = 20.0;
    for (Req* q : rq) us += 1e-4 * static_cast<double>(q->r.num_traj) * static_cast<double>(1ull << q->n);
    std::this_thread::sleep_for(std::chrono::microseconds(static_cast<int64_t>(std::min(us, 2e5))));
  } else {
    const qt_status s = lane_run(lane, static_cast<uint32_t>(tr.size()), tr.data(), samples.data(), flushes.data());
    if (s != QT_OK) return s;
  }
  uint64_t so = 0, to = 0;
  for (Req* q : rq) {
    const size_t ns = static_cast<size_t>(q->r.num_traj) * q->r.samples_per_traj;
    q->samples.assign(samples.begin() + so, samples.begin() + so + ns);
    q->flushes = 0;
    for (uint32_t t = 0; t < q->r.num_traj; ++t) q->flushes += flushes[to + t];
    so += ns;
    to += q->r.num_traj;
  }
  {
    std::lock_guard<std::mutex> lk(mu);
    lane_launches++;
    lane_trajectories += tr.size();
  }
  return QT_OK;
}

// Record the outcome of a run (caller holds mu): an allocation failure puts
// the request back at the head of its queue (up to 4 attempts).
void qt_server::finish(uint64_t id, qt_status s, const std::string& msg) {
  Req& q = reqs[id];
  if (s == QT_ERR_OUT_OF_MEMORY && q.attempts < 4 && q.state != kCancelled) {
    q.state = kQueued;                 // deferred, not lost: back to the head of the queue
    (q.batched ? bqueue : queue).push_front(id);
    deferred++;
  } else {
    q.state = s == QT_OK ? kDone : kFailed;
    q.status = s;
    q.err = msg;
    q.t_done = now_s();
  }
}

void qt_server::worker_loop(size_t w) {
  Worker& me = *workers[w];
  struct Done {
    Worker& w;
    ~Done() { w.finished = true; }
  } done{me};
  if (!(cfg.flags & QT_SERVER_DRY_RUN)) cudaSetDevice(device);
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
      me.held.assign(1, id);
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
      me.held.clear();
      finish(id, s, msg);
    }
    cv_work.notify_all();
    cv_done.notify_all();
  }
}

void qt_server::lane_loop(size_t w) {
  Worker& me = *workers[w];
  struct Done {
    Worker& w;
    ~Done() { w.finished = true; }
  } done{me};
  if (!(cfg.flags & QT_SERVER_DRY_RUN)) cudaSetDevice(device);
  for (;;) {
    std::vector<uint64_t> ids;
    {
      std::unique_lock<std::mutex> lk(mu);
      cv_work.wait(lk, [&] { return stop || !bqueue.empty(); });
      if (stop) return;
      // every queued small request, in arrival order, up to the launch's cap
      uint64_t traj = 0;
      while (!bqueue.empty()) {
        Req& q = reqs[bqueue.front()];
        if (!ids.empty() && traj + q.r.num_traj > kLaneMaxTraj) break;
        traj += q.r.num_traj;
        ids.push_back(bqueue.front());
        bqueue.pop_front();
        q.state = kRunning;
        q.worker = static_cast<int32_t>(w);
        q.attempts++;
        if (q.attempts == 1) q.t_start = now_s();
      }
      me.held = ids;
      if (inj_exit) {                 // injected fault: the lane dies holding its launch
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
      s = execute_lane(ids);
    }
    std::string msg = s == QT_OK ? std::string() : std::string(qt_last_error());
    {
      std::lock_guard<std::mutex> lk(mu);
      me.held.clear();
      // deferred requests go back to the head of the queue in their order
      for (auto it = ids.rbegin(); it != ids.rend(); ++it) finish(*it, s, msg);
    }
    cv_work.notify_all();
    cv_done.notify_all();
  }
}

void qt_server::start_worker(size_t w) {
  workers[w]->finished = false;
  workers[w]->crashed = false;
  if (is_lane(w)) workers[w]->th = std::thread([this, w] { lane_loop(w); });
  else workers[w]->th = std::thread([this, w] { worker_loop(w); });
}

void qt_server::watchdog_loop() {
  std::unique_lock<std::mutex> lk(mu);
  while (!stop) {
    cv_done.wait_for(lk, std::chrono::milliseconds(5));
    if (stop) break;
    for (size_t w = 0; w < workers.size(); ++w) {
      Worker& k = *workers[w];
      if (!k.finished || !k.crashed) continue;
      // the thread died holding requests: requeue them by id (in their
      // order, at the head of their queue) and start a replacement
      for (auto it = k.held.rbegin(); it != k.held.rend(); ++it) {
        Req& q = reqs[*it];
        if (!q.batched) inflight -= q.bytes;
        if (q.state == kRunning) {
          q.state = kQueued;
          (q.batched ? bqueue : queue).push_front(*it);
          requeued++;
        }
      }
      k.held.clear();
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
  const bool dry = (cfg->flags & QT_SERVER_DRY_RUN) != 0;
  if (!dry) {
    if (cudaGetDevice(&S->device) != cudaSuccess) return set_error(QT_ERR_CUDA, "qt_server_create: no CUDA device");
    S->sms = static_cast<uint32_t>(sm_count());
  }
  // the batch lane: states up to small_n_max (<= 20); the slots of states
  // above 2^14 amplitudes (one per SM) are reserved against the budget, and
  // the lane keeps to shared-memory states when they would take more than
  // half of it
  if (cfg->small_n_max > 0) {
    S->lane_max_n = std::min<uint32_t>(std::max<uint32_t>(cfg->small_n_max, kSmemStateMaxN), 20);
    if (S->lane_max_n > kSmemStateMaxN) {
      S->lane_bytes = (8ull << S->lane_max_n) * S->sms;
      if (S->lane_bytes > cfg->budget_bytes / 2) {
        S->lane_max_n = kSmemStateMaxN;
        S->lane_bytes = 0;
      }
    }
    S->inflight = S->peak_inflight = S->lane_bytes;
  }
  const uint32_t nw = cfg->max_slots + (S->lane_max_n ? 1 : 0);
  S->workers.resize(nw);
  for (uint32_t w = 0; w < nw; ++w) {
    S->workers[w] = std::make_unique<Worker>();
    if (!dry) {
      if (cudaStreamCreateWithFlags(&S->workers[w]->stream, cudaStreamNonBlocking) != cudaSuccess)
        return set_error(QT_ERR_CUDA, "qt_server_create: cudaStreamCreate");
    }
  }
  if (S->lane_max_n && !dry) {
    const qt_status s = lane_create(S->lane_max_n, S->workers[nw - 1]->stream, &S->lane);
    if (s != QT_OK) return s;
  }
  for (uint32_t w = 0; w < nw; ++w) S->start_worker(w);
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
  q.batched = use_batched(s->lane_max_n, f, r->num_traj) && r->num_traj <= kLaneMaxTraj;
  q.bytes = q.batched ? 0 : footprint(q.n, r->num_traj, !(s->cfg.flags & QT_SERVER_NO_SHARED_PREFIX));
  // (the lane's memory is reserved up front)
  if (q.bytes + s->lane_bytes > s->cfg.budget_bytes)
    return set_error(QT_ERR_OUT_OF_MEMORY, "qt_server_submit: footprint %llu bytes exceeds the budget %llu",
                     static_cast<unsigned long long>(q.bytes), static_cast<unsigned long long>(s->cfg.budget_bytes));
  q.t_submit = now_s();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    const uint64_t i = s->next_id++;
    const bool b = q.batched;
    s->reqs.emplace(i, std::move(q));
    (b ? s->bqueue : s->queue).push_back(i);
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
  std::deque<uint64_t>& qu = it->second.batched ? s->bqueue : s->queue;
  qu.erase(std::remove(qu.begin(), qu.end(), id), qu.end());
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
  out->lane_bytes = s->lane_bytes;
  out->lane_launches = s->lane_launches;
  out->lane_trajectories = s->lane_trajectories;
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
  if (s->lane) lane_destroy(s->lane);
  for (auto& w : s->workers)
    if (w->stream) cudaStreamDestroy(w->stream);
  delete s;
}

}  // extern "C"
