// Request loop with continuous batching (pump_server_*).
//
// Requests are queued in arrival order.  Admission happens whenever a request
// arrives or one finishes: the queue head is admitted while a slot is free and
// its estimated device memory fits next to the requests already admitted (a
// request larger than the whole budget is admitted only when nothing runs).  A
// slot is a worker thread with its own CUDA stream; it builds the request's
// graph, plans on it and frees it, so admitted requests overlap on the device
// (graph build of one next to Explore or certification of another).  Each
// request runs exactly the calls a caller would make alone, on its own graph,
// so its result does not depend on what else runs.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "pump_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Job {
  int64_t ticket = 0;
  int64_t bytes = 0;  // estimated device memory
  Clock::time_point t_submit;
  std::vector<float> states, xi;
  std::vector<int32_t> goal;
  std::vector<pump_aabb> boxes;
  int32_t n = 0, start = 0;
  pump_graph_params gp{};
  pump_plan_params pp{};
};

struct Done {
  bool done = false;
  int status = PUMP_OK;
  pump_plan_result result{};
  std::vector<int32_t> path;
  double latency_ms = 0.0;
};

// Device memory of a request, estimated from its sizes: graph arrays for an out-degree of about
// 60 ln n / ln 4000 (1.5x the calibrated mean), the build's pair bitmaps, the plan arena and
// fixed scratch.  Admission control only: a request whose allocations fail reports OOM.
int64_t estimate_bytes(const pump_request* r) {
  const double n = (double)r->n;
  const double W = (double)r->graph.n_waypoints, w = (double)(r->graph.n_particles / 32);
  const double deg = 60.0 * std::log(std::max(n, 2.0)) / std::log(4000.0);
  const double E = n * deg;
  const double per_edge = 4 + 4 + 4 + 4 + 16 + 12 + 12 * W + 4 * w + 24 + 4 + 16 + 32;
  const double build = 2.0 * n * n / 8.0 + 64.0 * n;
  // per plan: head, parent, edge, creation and expansion stamps, cost, popcount (7 x 4 B), mask
  // words, group slot (4), group record (16) and offset (8), goal lists (2 x 4), row record (8)
  const double arena = (double)r->plan.max_plans * (72.0 + 4.0 * w);
  return (int64_t)(E * per_edge + build + arena) + (16ll << 20);
}

}  // namespace

struct pump_server {
  int device = 0;
  int64_t budget = 0;
  std::mutex mu;
  std::condition_variable cv_work;  // workers: a job was assigned or the server stops
  std::condition_variable cv_done;  // waiters: a job finished
  std::deque<Job*> queue;
  std::vector<Job*> slot_job;
  std::vector<cudaStream_t> streams;
  std::vector<std::thread> workers;
  std::unordered_map<int64_t, Done> results;
  int64_t next_ticket = 1;
  int64_t in_use = 0, peak_bytes = 0;
  int64_t submitted = 0, admitted = 0, completed = 0;
  int running = 0, peak_running = 0;
  bool stop = false;

  // Under mu: admit queue heads while a slot is free and the memory fits.
  void admit() {
    while (!queue.empty()) {
      Job* j = queue.front();
      int free_slot = -1;
      for (size_t k = 0; k < slot_job.size(); ++k)
        if (!slot_job[k]) {
          free_slot = (int)k;
          break;
        }
      if (free_slot < 0) return;
      const bool fits = in_use + j->bytes <= budget || running == 0;
      if (!fits) return;
      queue.pop_front();
      slot_job[free_slot] = j;
      in_use += j->bytes;
      peak_bytes = std::max(peak_bytes, in_use);
      ++running;
      peak_running = std::max(peak_running, running);
      ++admitted;
      cv_work.notify_all();
    }
  }

  void run(Job* j, cudaStream_t s, Done* d) {
    pump_graph* g = nullptr;
    int rc = pump_build_graph(j->states.data(), j->n, j->start, j->goal.data(), (int32_t)j->goal.size(),
                              j->boxes.empty() ? nullptr : j->boxes.data(), (int32_t)j->boxes.size(), j->xi.data(),
                              &j->gp, s, &g);
    std::memset(&d->result, 0, sizeof(d->result));
    d->result.chosen_plan = -1;
    if (!rc) {
      d->path.assign(kPathCap, 0);
      rc = pump_plan(g, &j->pp, d->path.data(), kPathCap, &d->result, s);
      d->path.resize(std::min<int32_t>(d->result.path_len, kPathCap));
    }
    if (g) pump::destroy_on_stream(g, s);
    d->status = rc;
    if (rc && d->result.status == PUMP_OK) d->result.status = rc;
  }

  void worker(int k) {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
      cv_work.wait(lk, [&] { return stop || slot_job[k] != nullptr; });
      if (!slot_job[k]) return;  // stopping and idle
      Job* j = slot_job[k];
      lk.unlock();
      Done d;
      run(j, streams[k], &d);
      const double ms = std::chrono::duration<double, std::milli>(Clock::now() - j->t_submit).count();
      lk.lock();
      d.done = true;
      d.latency_ms = ms;
      results[j->ticket] = std::move(d);
      in_use -= j->bytes;
      --running;
      ++completed;
      slot_job[k] = nullptr;
      delete j;
      if (!stop) admit();
      cv_done.notify_all();
    }
  }

  static constexpr int32_t kPathCap = pump::kMaxPathEdges + 1;
};

extern "C" {

int pump_server_create(int32_t max_slots, int64_t device_bytes, pump_server** out) {
  if (!out || max_slots < 1 || max_slots > 64 || device_bytes <= 0) return PUMP_ERR_INVALID_ARG;
  pump_server* s = new pump_server();
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    delete s;
    return PUMP_ERR_CUDA;
  }
  s->budget = device_bytes;
  s->slot_job.assign(max_slots, nullptr);
  s->streams.assign(max_slots, nullptr);
  for (int k = 0; k < max_slots; ++k)
    if (cudaStreamCreateWithFlags(&s->streams[k], cudaStreamNonBlocking) != cudaSuccess) {
      for (auto st : s->streams)
        if (st) cudaStreamDestroy(st);
      delete s;
      return PUMP_ERR_CUDA;
    }
  for (int k = 0; k < max_slots; ++k) s->workers.emplace_back([s, k] { s->worker(k); });
  *out = s;
  return PUMP_OK;
}

int pump_server_submit(pump_server* s, const pump_request* r, int64_t* ticket) {
  if (!s || !r || !ticket || !r->states || !r->goal_idx || !r->xi) return PUMP_ERR_INVALID_ARG;
  const int N = r->graph.n_particles, W = r->graph.n_waypoints;
  if (r->n < 2 || r->n_goal < 1 || r->n_boxes < 0 || r->n_boxes > pump::kMaxBoxes || (r->n_boxes > 0 && !r->boxes) ||
      N < 32 || N > pump::kMaxParticles || N % 32 || W < 1 || W > pump::kMaxWaypoints || r->plan.max_plans < 1)
    return PUMP_ERR_INVALID_ARG;
  Job* j = new (std::nothrow) Job();
  if (!j) return PUMP_ERR_OOM;
  try {
    j->states.assign(r->states, r->states + 6 * (size_t)r->n);
    j->goal.assign(r->goal_idx, r->goal_idx + r->n_goal);
    j->boxes.assign(r->boxes, r->boxes + r->n_boxes);
    j->xi.assign(r->xi, r->xi + (size_t)N * (W + 1) * 3 * 2);
  } catch (...) {
    delete j;
    return PUMP_ERR_OOM;
  }
  j->n = r->n;
  j->start = r->start_idx;
  j->gp = r->graph;
  // requests overlap on the device: their masks keep their own launch, and the build lays out no
  // edge order for the fused form
  j->gp.flags |= PUMP_GRAPH_SEPARATE_MASKS;
  j->pp = r->plan;
  j->bytes = estimate_bytes(r);
  j->t_submit = Clock::now();
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) {
    delete j;
    return PUMP_ERR_INVALID_ARG;
  }
  j->ticket = s->next_ticket++;
  *ticket = j->ticket;
  s->results[j->ticket] = Done();
  s->queue.push_back(j);
  ++s->submitted;
  s->admit();
  return PUMP_OK;
}

int pump_server_wait(pump_server* s, int64_t ticket, double timeout_s, pump_plan_result* out, int32_t* path,
                     int32_t path_cap, double* latency_ms) {
  if (!s || !out || path_cap < 0 || (path_cap > 0 && !path) || !(timeout_s >= 0.0)) return PUMP_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->results.find(ticket);
  if (it == s->results.end()) return PUMP_ERR_INVALID_ARG;
  const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(
                                           std::min(timeout_s, 1e6)));
  while (!it->second.done) {
    if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && !it->second.done) return PUMP_ERR_TIMEOUT;
    it = s->results.find(ticket);
    if (it == s->results.end()) return PUMP_ERR_INVALID_ARG;
  }
  Done d = std::move(it->second);
  s->results.erase(it);
  lk.unlock();
  *out = d.result;
  const int32_t np = std::min<int32_t>((int32_t)d.path.size(), path_cap);
  if (np > 0) std::memcpy(path, d.path.data(), sizeof(int32_t) * np);
  if (latency_ms) *latency_ms = d.latency_ms;
  return d.status;
}

int pump_server_stats(pump_server* s, int64_t* c) {
  if (!s || !c) return PUMP_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  c[0] = s->submitted;
  c[1] = s->admitted;
  c[2] = s->completed;
  c[3] = (int64_t)s->queue.size();
  c[4] = s->running;
  c[5] = s->peak_running;
  c[6] = s->in_use;
  c[7] = s->peak_bytes;
  return PUMP_OK;
}

void pump_server_destroy(pump_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    for (Job* j : s->queue) {
      s->results.erase(j->ticket);
      delete j;
    }
    s->queue.clear();
    s->cv_work.notify_all();
  }
  for (auto& t : s->workers) t.join();
  for (auto st : s->streams)
    if (st) cudaStreamDestroy(st);
  delete s;
}

}  // extern "C"
