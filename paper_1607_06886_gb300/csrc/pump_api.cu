// C entry points of libpump (include/pump.h): argument checks, staging of
// host arrays, device memory through the installed allocator, and the order
// of the device stages.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "pump_internal.cuh"

namespace pump {

int run_goal_finalize(pump_graph* g, const ExploreArgs& A, cudaStream_t s);
int launch_node_flags(pump_graph* g, const int32_t* goal_dev, cudaStream_t s);
int launch_transpose_xi(pump_graph* g, const float* xi_dev, cudaStream_t s);
int launch_linf(pump_graph* g, float* out_dev, cudaStream_t s);

namespace {
void* (*g_alloc)(size_t, void*, void*) = nullptr;
void (*g_free)(void*, void*, void*) = nullptr;
void* g_ctx = nullptr;
}  // namespace

static std::atomic<unsigned long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

// The stream-ordered pool of each device the library allocates on keeps what it has (release
// threshold raised once per device): by default it hands memory back at every synchronisation and
// the next query pays to map it again.
static void keep_pool_memory() {
  static std::atomic<unsigned long long> done{0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return;
  }
  const unsigned long long bit = 1ull << dev;
  if (done.load(std::memory_order_relaxed) & bit) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t thr = ~0ull;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  cudaGetLastError();
  done.fetch_or(bit, std::memory_order_relaxed);
}

void* dev_alloc(size_t bytes, cudaStream_t s) {
  if (bytes == 0) bytes = 16;
  if (g_alloc) return g_alloc(bytes, (void*)s, g_ctx);
  keep_pool_memory();
  void* p = nullptr;
  if (cudaMallocAsync(&p, bytes, s) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void dev_free(void* p, cudaStream_t s) {
  if (!p) return;
  if (g_alloc) {
    if (g_free) g_free(p, (void*)s, g_ctx);
    return;
  }
  cudaFreeAsync(p, s);
}

void* graph_alloc(pump_graph* g, size_t bytes, cudaStream_t s) {
  void* p = dev_alloc(bytes, s);
  if (p) g->bufs.push_back(DevBuf{p, bytes});
  return p;
}

// Replace a tracked buffer by a larger one (old contents are not kept).
void* graph_realloc(pump_graph* g, void* old, size_t bytes, cudaStream_t s) {
  if (old) {
    for (size_t k = 0; k < g->bufs.size(); ++k)
      if (g->bufs[k].ptr == old) {
        dev_free(old, s);
        g->bufs.erase(g->bufs.begin() + k);
        break;
      }
  }
  return graph_alloc(g, bytes, s);
}

int num_sms() {
  static int cached[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (!cached[dev]) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    cached[dev] = v > 0 ? v : 1;
  }
  return cached[dev];
}

int ensure_explore_bufs(pump_graph* g, int64_t cap, int32_t kmax, cudaStream_t s) {
  ExploreBufs& X = g->ex;
  const int w = g->n_words;
  if (cap > X.cap || w != X.w_alloc) {
    X.head = (int32_t*)graph_realloc(g, X.head, sizeof(int32_t) * cap, s);
    X.parent = (int32_t*)graph_realloc(g, X.parent, sizeof(int32_t) * cap, s);
    X.pedge = (int32_t*)graph_realloc(g, X.pedge, sizeof(int32_t) * cap, s);
    X.tcre = (int32_t*)graph_realloc(g, X.tcre, sizeof(int32_t) * cap, s);
    X.eexp = (int32_t*)graph_realloc(g, X.eexp, sizeof(int32_t) * cap, s);
    X.cost = (float*)graph_realloc(g, X.cost, sizeof(float) * cap, s);
    X.popc = (int32_t*)graph_realloc(g, X.popc, sizeof(int32_t) * cap, s);
    X.mask = (uint32_t*)graph_realloc(g, X.mask, sizeof(uint32_t) * cap * w, s);
    X.group = (int32_t*)graph_realloc(g, X.group, sizeof(int32_t) * cap, s);
    X.ginfo = (int4*)graph_realloc(g, X.ginfo, sizeof(int4) * cap, s);
    X.goff = (int64_t*)graph_realloc(g, X.goff, sizeof(int64_t) * (cap + 1), s);
    X.goal_all = (int32_t*)graph_realloc(g, X.goal_all, sizeof(int32_t) * cap, s);
    X.goal_sorted = (int32_t*)graph_realloc(g, X.goal_sorted, sizeof(int32_t) * cap, s);
    X.prow = (int2*)graph_realloc(g, X.prow, sizeof(int2) * cap, s);
    if (!X.head || !X.parent || !X.pedge || !X.tcre || !X.eexp || !X.cost || !X.popc || !X.mask || !X.group ||
        !X.ginfo || !X.goff || !X.goal_all || !X.goal_sorted || !X.prow) {
      X.cap = 0;
      return PUMP_ERR_OOM;
    }
    X.cap = cap;
    X.w_alloc = w;
  }
  if (kmax > X.kmax_alloc) {
    X.mbest = (uint32_t*)graph_realloc(g, X.mbest, sizeof(uint32_t) * (size_t)g->n * kmax, s);
    if (!X.mbest) {
      X.kmax_alloc = 0;
      return PUMP_ERR_OOM;
    }
    X.kmax_alloc = kmax;
  }
  if (!X.ctl) {
    X.ctl = (ExploreCtl*)graph_alloc(g, sizeof(ExploreCtl), s);
    X.bcnt = (int32_t*)graph_alloc(g, sizeof(int32_t) * 4096, s);
    X.bdeg = (int64_t*)graph_alloc(g, sizeof(int64_t) * 4096, s);
    if (!X.ctl || !X.bcnt || !X.bdeg) return PUMP_ERR_OOM;
  }
  return PUMP_OK;
}

// K = #{k >= 0 : k < a} for a = (eta*alpha)*N (K_max) or (alpha/eta)*N (K_min), in double.
static int32_t popc_bound(double a, int N) {
  if (!(a > 0.0)) return 0;
  double k = std::ceil(a);
  return (int32_t)std::min<double>(k, (double)N + 1.0);
}

void fill_explore_stats(pump_graph* g, const ExploreCtl& h, pump_plan_result* st) {
  g->explored = true;
  // a fused launch that refused its launch shape counted no row: zero the counts before the next
  if (g->last_fused && h.status == PUMP_ERR_CUDA) g->rowcnt_dirty = true;
  g->last_plans = h.n_plans;
  g->last_goal = h.status ? 0 : h.n_goal;
  st->n_candidates = h.n_candidates;
  st->n_kept = h.n_kept;
  st->n_plans = h.n_plans;
  st->n_iterations = h.iter;
  st->n_groups = h.n_groups;
  st->n_goal = g->last_goal;
}

// Explore's arguments for graph g and plan parameters p (buffers allocated as needed).
int prepare_explore_args(pump_graph* g, const pump_plan_params* p, float radius, ExploreArgs* out, cudaStream_t s) {
  const double alpha = (double)p->alpha, eta = (double)p->eta;
  const int32_t kmax = popc_bound((eta * alpha) * (double)g->N, g->N);
  const int32_t kmin = popc_bound((alpha / eta) * (double)g->N, g->N);
  int rc = ensure_explore_bufs(g, p->max_plans, std::max(kmax, 1), s);
  if (rc) return rc;
  ExploreBufs& X = g->ex;
  ExploreArgs A;
  A.row_ptr = g->row_ptr;
  A.col = g->col;
  A.ecost = g->ecost;
  A.emask = g->emask;
  A.is_goal = g->is_goal;
  A.n = g->n;
  A.w = g->n_words;
  A.kmin = kmin;
  A.lr = (double)p->lambda * (double)radius;
  A.max_iter = p->max_iterations;
  A.early_stop = (p->flags & PUMP_NO_EARLY_STOP) ? 0 : 1;
  A.head = X.head;
  A.parent = X.parent;
  A.pedge = X.pedge;
  A.tcre = X.tcre;
  A.eexp = X.eexp;
  A.cost = X.cost;
  A.popc = X.popc;
  A.mask = X.mask;
  A.cap = p->max_plans;
  A.mbest = X.mbest;
  A.group = X.group;
  A.ginfo = X.ginfo;
  A.goff = X.goff;
  A.bcnt = X.bcnt;
  A.bdeg = X.bdeg;
  A.goal_all = X.goal_all;
  A.prow = X.prow;
  A.ctl = X.ctl;
  A.spin_limit = 20000000ll;
  A.kstride = std::max(kmax, 1);
  A.kmax = kmax;
  rc = ensure_edge_targets(g, s);
  if (rc) return rc;
  A.etgt = g->etgt;
  *out = A;
  return PUMP_OK;
}

// Enqueue Explore; with `collect` read its control block back and fill `st`.
int run_explore(pump_graph* g, const pump_plan_params* p, float radius, pump_plan_result* st, cudaStream_t s,
                bool collect, bool masks_pending) {
  ExploreArgs A;
  int rc = prepare_explore_args(g, p, radius, &A, s);
  if (rc) return rc;
  ExploreBufs& X = g->ex;
  rc = run_explore_kernels(g, A, explore_mode(p->flags), s, masks_pending);
  if (rc) return rc;
  if (!g->last_fused) {  // the fused launch orders P_goal itself
    rc = run_goal_finalize(g, A, s);
    if (rc) return rc;
  }
  g->explored = false;
  if (!collect) return PUMP_OK;
  ExploreCtl h;
  PUMP_CUDA_TRY(cudaMemcpyAsync(&h, X.ctl, sizeof(h), cudaMemcpyDeviceToHost, s));
  PUMP_CUDA_TRY(cudaStreamSynchronize(s));
  fill_explore_stats(g, h, st);
  return h.status ? h.status : PUMP_OK;
}

static bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Copy `bytes` from host or device memory into device buffer dst.
static int stage(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  if (bytes == 0) return PUMP_OK;
  cudaMemcpyKind k = is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  PUMP_CUDA_TRY(cudaMemcpyAsync(dst, src, bytes, k, s));
  return PUMP_OK;
}

// Host copy of an input array (for validation).
template <typename T>
static int host_copy(std::vector<T>& out, const T* src, size_t count, cudaStream_t s) {
  out.resize(count);
  if (count == 0) return PUMP_OK;
  if (is_device_ptr(src)) {
    PUMP_CUDA_TRY(cudaMemcpyAsync(out.data(), src, sizeof(T) * count, cudaMemcpyDeviceToHost, s));
    PUMP_CUDA_TRY(cudaStreamSynchronize(s));
  } else {
    std::memcpy(out.data(), src, sizeof(T) * count);
  }
  return PUMP_OK;
}

static void destroy(pump_graph* g) {
  if (!g) return;
  cudaStream_t s = 0;
  cudaDeviceSynchronize();
  row_order_end(g, s);  // an edge order still being laid out (a build that failed): its scratch
  for (auto& b : g->bufs) dev_free(b.ptr, s);
  for (auto& e : g->ev)
    if (e) cudaEventDestroy(e);
  cudaDeviceSynchronize();
  delete g;
}

// Frees a graph whose work was all issued on stream s: waits for s only, so other streams keep
// running (the server's workers).
void destroy_on_stream(pump_graph* g, cudaStream_t s) {
  if (!g) return;
  row_order_end(g, s);  // s waits for a side stream still laying out the edge order
  cudaStreamSynchronize(s);
  for (auto& b : g->bufs) dev_free(b.ptr, s);
  for (auto& e : g->ev)
    if (e) cudaEventDestroy(e);
  cudaStreamSynchronize(s);
  delete g;
}

int check_plan_params(const pump_plan_params* p) {
  if (!p) return PUMP_ERR_INVALID_ARG;
  if (!(p->alpha >= 0.f) || !(p->alpha <= 1.f) || !(p->eta > 0.f) || !std::isfinite(p->eta)) return PUMP_ERR_INVALID_ARG;
  if (!(p->lambda > 0.f) || !(p->lambda <= 1.f)) return PUMP_ERR_INVALID_ARG;
  if (p->max_plans < 1 || p->max_plans > (1ll << 31) - 2 || p->max_iterations < 1) return PUMP_ERR_INVALID_ARG;
  if (p->n_mc < 0 || p->mc_substeps < 1 || p->mc_substeps > 64) return PUMP_ERR_INVALID_ARG;
  return PUMP_OK;
}

// Pinned host copy of Explore's control block, one per host thread (a graph is used by one
// thread at a time), allocated once: pinned allocations cost far more than a query's readback.
static ExploreCtl* thread_ctl_host() {
  struct Buf {
    ExploreCtl* p = nullptr;
    ~Buf() {
      if (p) cudaFreeHost(p);
    }
  };
  thread_local Buf b;
  if (!b.p && cudaHostAlloc((void**)&b.p, sizeof(ExploreCtl), cudaHostAllocDefault) != cudaSuccess) b.p = nullptr;
  return b.p;
}

int make_events(pump_graph* g) {
  for (auto& e : g->ev)
    if (!e) PUMP_CUDA_TRY(cudaEventCreate(&e));
  g->ctl_host = thread_ctl_host();
  if (!g->ctl_host) return PUMP_ERR_CUDA;
  return PUMP_OK;
}

}  // namespace pump

using namespace pump;

extern "C" {

int pump_set_allocator(void* (*alloc)(size_t, void*, void*), void (*free_)(void*, void*, void*), void* ctx) {
  g_alloc = alloc;
  g_free = alloc ? free_ : nullptr;
  g_ctx = alloc ? ctx : nullptr;
  return PUMP_OK;
}

const char* pump_status_str(int st) {
  switch (st) {
    case PUMP_OK: return "ok";
    case PUMP_ERR_INVALID_ARG: return "invalid argument";
    case PUMP_ERR_OOM: return "out of device memory";
    case PUMP_ERR_CUDA: return "CUDA error";
    case PUMP_ERR_CAPACITY: return "plan arena capacity exceeded";
    case PUMP_ERR_TIMEOUT: return "iteration cap reached or device wait timed out";
    case PUMP_ERR_INFEASIBLE: return "no plan certified under the CP target";
    default: return "unknown status";
  }
}

int pump_build_graph(const float* states, int32_t n, int32_t start_idx, const int32_t* goal_idx, int32_t n_goal,
                     const pump_aabb* boxes, int32_t n_boxes, const float* xi, const pump_graph_params* prm,
                     void* stream, pump_graph** out) {
  if (!out || !states || !goal_idx || !xi || !prm) return PUMP_ERR_INVALID_ARG;
  if (n < 2 || start_idx < 0 || start_idx >= n || n_goal < 1 || n_boxes < 0 || n_boxes > kMaxBoxes) return PUMP_ERR_INVALID_ARG;
  if (n_boxes > 0 && !boxes) return PUMP_ERR_INVALID_ARG;
  const int N = prm->n_particles, W = prm->n_waypoints;
  if (N < 32 || N > kMaxParticles || N % 32 != 0 || W < 1 || W > kMaxWaypoints) return PUMP_ERR_INVALID_ARG;
  if (!(prm->radius > 0.f) || !std::isfinite(prm->radius) || !(prm->sigma >= 0.f) || !std::isfinite(prm->sigma))
    return PUMP_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<int32_t> gh;
  int rc = host_copy(gh, goal_idx, (size_t)n_goal, s);
  if (rc) return rc;
  for (int32_t v : gh)
    if (v < 0 || v >= n) return PUMP_ERR_INVALID_ARG;
  pump_graph* g = new (std::nothrow) pump_graph();
  if (!g) return PUMP_ERR_OOM;
  cudaGetDevice(&g->device);
  g->n = n;
  g->N = N;
  g->W = W;
  g->n_words = N / 32;
  g->n_boxes = n_boxes;
  g->n_goal = n_goal;
  g->start = start_idx;
  g->radius = prm->radius;
  g->sigma = prm->sigma;
  g->has_geometry = true;
  g->hsmc = (prm->flags & PUMP_GRAPH_HSMC) != 0;
  g->fuse_masks = (prm->flags & PUMP_GRAPH_SEPARATE_MASKS) == 0;
  g->states = (float*)graph_alloc(g, sizeof(float) * 6 * (size_t)n, s);
  g->boxes = (float*)graph_alloc(g, sizeof(float) * 6 * (size_t)std::max(n_boxes, 1), s);
  g->valid = (uint8_t*)graph_alloc(g, (size_t)n, s);
  g->is_goal = (uint8_t*)graph_alloc(g, (size_t)n, s);
  g->xi_t = (float2*)graph_alloc(g, sizeof(float2) * (size_t)(W + 1) * 3 * N, s);
  g->xi_p = (float4*)graph_alloc(g, sizeof(float4) * (size_t)(W + 1) * 3 * ((N / 32 + 1) / 2) * 32, s);
  g->wctr = (unsigned long long*)graph_alloc(g, 2 * sizeof(unsigned long long), s);
  g->linf_dev = (float*)graph_alloc(g, sizeof(float) * 4, s);
  int32_t* goal_dev = (int32_t*)dev_alloc(sizeof(int32_t) * (size_t)n_goal, s);
  float* xi_raw = (float*)dev_alloc(sizeof(float) * (size_t)N * (W + 1) * 6, s);
  rc = PUMP_OK;
  if (!g->states || !g->boxes || !g->valid || !g->is_goal || !g->xi_t || !g->xi_p || !g->wctr || !g->linf_dev ||
      !goal_dev || !xi_raw)
    rc = PUMP_ERR_OOM;
  if (!rc) rc = stage(g->states, states, sizeof(float) * 6 * (size_t)n, s);
  if (!rc && n_boxes) rc = stage(g->boxes, boxes, sizeof(float) * 6 * (size_t)n_boxes, s);
  if (!rc) rc = stage(goal_dev, gh.data(), sizeof(int32_t) * (size_t)n_goal, s);
  if (!rc) rc = stage(xi_raw, xi, sizeof(float) * (size_t)N * (W + 1) * 6, s);
  if (!rc) rc = launch_node_flags(g, goal_dev, s);
  if (!rc) rc = launch_transpose_xi(g, xi_raw, s);
  if (!rc) rc = launch_linf(g, g->linf_dev, s);
  // the start's validity is read back with the build's last copy (a start inside a box still
  // fails the call, after the build)
  bool start_valid = false;
  if (!rc) rc = build_graph_device(g, start_idx, &start_valid, s);
  if (!rc && !start_valid) rc = PUMP_ERR_INVALID_ARG;
  dev_free(goal_dev, s);
  dev_free(xi_raw, s);
  if (rc) {
    destroy(g);
    return rc;
  }
  *out = g;
  return PUMP_OK;
}

// Former name of pump_build_graph, kept for existing callers.
int pump_graph_build(const float* states, int32_t n, int32_t start_idx, const int32_t* goal_idx, int32_t n_goal,
                     const pump_aabb* boxes, int32_t n_boxes, const float* xi, const pump_graph_params* prm,
                     void* stream, pump_graph** out) {
  return pump_build_graph(states, n, start_idx, goal_idx, n_goal, boxes, n_boxes, xi, prm, stream, out);
}

int pump_graph_from_csr(int32_t n, const int32_t* row_ptr, const int32_t* col, const float* ecost,
                        const uint32_t* emask, int32_t n_particles, int32_t start_idx, const int32_t* goal_idx,
                        int32_t n_goal, void* stream, pump_graph** out) {
  if (!out || !row_ptr || !goal_idx || n < 1 || start_idx < 0 || start_idx >= n || n_goal < 1) return PUMP_ERR_INVALID_ARG;
  if (n_particles < 32 || n_particles > kMaxParticles || n_particles % 32) return PUMP_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int w = n_particles / 32;
  std::vector<int32_t> rp, cl, gh;
  std::vector<float> ec;
  int rc = host_copy(rp, row_ptr, (size_t)n + 1, s);
  if (rc) return rc;
  if (rp[0] != 0) return PUMP_ERR_INVALID_ARG;
  for (int v = 0; v < n; ++v)
    if (rp[v + 1] < rp[v]) return PUMP_ERR_INVALID_ARG;
  const int32_t E = rp[n];
  if (E > 0 && (!col || !ecost || !emask)) return PUMP_ERR_INVALID_ARG;
  if ((rc = host_copy(cl, col, (size_t)E, s))) return rc;
  if ((rc = host_copy(ec, ecost, (size_t)E, s))) return rc;
  if ((rc = host_copy(gh, goal_idx, (size_t)n_goal, s))) return rc;
  for (int v = 0; v < n; ++v)
    for (int e = rp[v]; e < rp[v + 1]; ++e) {
      if (cl[e] < 0 || cl[e] >= n || cl[e] == v) return PUMP_ERR_INVALID_ARG;
      if (e > rp[v] && cl[e] <= cl[e - 1]) return PUMP_ERR_INVALID_ARG;
      if (!(ec[e] >= 0.f) || !std::isfinite(ec[e])) return PUMP_ERR_INVALID_ARG;
      if (ec[e] == 0.f) ec[e] = 0.f;  // -0 -> +0: costs are ordered through their bits
    }
  for (int32_t v : gh)
    if (v < 0 || v >= n) return PUMP_ERR_INVALID_ARG;
  pump_graph* g = new (std::nothrow) pump_graph();
  if (!g) return PUMP_ERR_OOM;
  cudaGetDevice(&g->device);
  g->n = n;
  g->E = E;
  g->N = n_particles;
  g->W = 0;
  g->n_words = w;
  g->n_goal = n_goal;
  g->start = start_idx;
  g->n_valid = n;
  g->has_geometry = false;
  const size_t Es = E > 0 ? (size_t)E : 1;
  g->row_ptr = (int32_t*)graph_alloc(g, sizeof(int32_t) * ((size_t)n + 1), s);
  g->col = (int32_t*)graph_alloc(g, sizeof(int32_t) * Es, s);
  g->ecost = (float*)graph_alloc(g, sizeof(float) * Es, s);
  g->emask = (uint32_t*)graph_alloc(g, sizeof(uint32_t) * Es * w, s);
  g->valid = (uint8_t*)graph_alloc(g, (size_t)n, s);
  g->is_goal = (uint8_t*)graph_alloc(g, (size_t)n, s);
  if (!g->row_ptr || !g->col || !g->ecost || !g->emask || !g->valid || !g->is_goal) {
    destroy(g);
    return PUMP_ERR_OOM;
  }
  std::vector<uint8_t> isg((size_t)n, 0), val((size_t)n, 1);
  for (int32_t v : gh) isg[v] = 1;
  rc = stage(g->row_ptr, rp.data(), sizeof(int32_t) * ((size_t)n + 1), s);
  if (!rc && E) rc = stage(g->col, cl.data(), sizeof(int32_t) * (size_t)E, s);
  if (!rc && E) rc = stage(g->ecost, ec.data(), sizeof(float) * (size_t)E, s);
  if (!rc && E) rc = stage(g->emask, emask, sizeof(uint32_t) * (size_t)E * w, s);
  if (!rc) rc = stage(g->is_goal, isg.data(), (size_t)n, s);
  if (!rc) rc = stage(g->valid, val.data(), (size_t)n, s);
  if (!rc && cudaStreamSynchronize(s) != cudaSuccess) rc = PUMP_ERR_CUDA;
  if (rc) {
    destroy(g);
    return rc;
  }
  g->masks_ready = true;
  *out = g;
  return PUMP_OK;
}

int pump_edge_masks(pump_graph* g, void* stream) {
  if (!g || !g->has_geometry) return PUMP_ERR_INVALID_ARG;
  return compute_edge_masks(g, (cudaStream_t)stream);
}

int pump_edge_masks_list(pump_graph* g, const int32_t* edges, int64_t n, uint32_t* out_masks, uint32_t* bad_ids,
                         void* stream) {
  if (!g || !g->has_geometry || g->hsmc || n < 0 || (n > 0 && (!edges || !out_masks))) return PUMP_ERR_INVALID_ARG;
  if (g->E > INT32_MAX) return PUMP_ERR_INVALID_ARG;
  return compute_edge_masks_list(g, edges, (long long)n, out_masks, bad_ids, (cudaStream_t)stream);
}

int pump_explore(pump_graph* g, const pump_plan_params* p, float radius, pump_plan_result* stats, void* stream) {
  if (!g || !stats || check_plan_params(p)) return PUMP_ERR_INVALID_ARG;
  if (!g->masks_ready) return PUMP_ERR_INVALID_ARG;
  const float r = g->has_geometry ? g->radius : radius;
  if (!(r > 0.f) || !std::isfinite(r)) return PUMP_ERR_INVALID_ARG;
  std::memset(stats, 0, sizeof(*stats));
  stats->chosen_plan = -1;
  int rc = run_explore(g, p, r, stats, (cudaStream_t)stream, true);
  stats->status = rc;
  return rc;
}

int pump_plan(pump_graph* g, const pump_plan_params* p, int32_t* path, int32_t path_cap, pump_plan_result* out,
              void* stream) {
  if (!g || !out || check_plan_params(p) || !g->has_geometry) return PUMP_ERR_INVALID_ARG;
  if (path_cap < 0 || (path_cap > 0 && !path)) return PUMP_ERR_INVALID_ARG;
  const bool no_wait = (p->flags & PUMP_NO_WAIT) != 0;
  if (no_wait && !(p->flags & PUMP_EXPLORE_ONLY)) return PUMP_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = make_events(g);
  if (rc) return rc;
  pump_plan_result r;
  std::memset(&r, 0, sizeof(r));
  r.chosen_plan = -1;
  PUMP_CUDA_TRY(cudaEventRecord(g->ev[0], s));
  // box masks run inside the Explore launch where it applies (then ms_masks covers only what
  // precedes it); the graph's first such run also lays out its edge order
  const bool fuse = g->fuse_masks && !g->hsmc && explore_mode(p->flags) == 0 && fused_masks_env();
  if (!fuse) {
    rc = compute_edge_masks(g, s);
    if (rc) return rc;
  }
  PUMP_CUDA_TRY(cudaEventRecord(g->ev[1], s));
  const bool explore_only = (p->flags & PUMP_EXPLORE_ONLY) != 0;
  rc = run_explore(g, p, g->radius, &r, s, false, fuse);
  PUMP_CUDA_TRY(cudaEventRecord(g->ev[2], s));
  if (rc) return rc;
  if (!explore_only) {
    ExploreCtl h;
    rc = run_select(g, p, path, path_cap, &r, &h, s);
    fill_explore_stats(g, h, &r);
    if (rc) return rc;
    PUMP_CUDA_TRY(cudaEventRecord(g->ev[3], s));
    PUMP_CUDA_TRY(cudaEventSynchronize(g->ev[3]));
  } else if (no_wait) {
    // enqueued only: the counters are read by pump_plan_collect
    r.status = PUMP_OK;
    r.fused = fuse && g->last_fused ? 1 : 0;
    *out = r;
    return PUMP_OK;
  } else {
    // one wait for the control block and the events (a pinned copy does not block the host)
    PUMP_CUDA_TRY(cudaMemcpyAsync(g->ctl_host, g->ex.ctl, sizeof(ExploreCtl), cudaMemcpyDeviceToHost, s));
    PUMP_CUDA_TRY(cudaEventRecord(g->ev[3], s));
    PUMP_CUDA_TRY(cudaEventSynchronize(g->ev[3]));
    const ExploreCtl h = *g->ctl_host;
    fill_explore_stats(g, h, &r);
    if (h.status) return h.status;
    r.status = PUMP_OK;
  }
  cudaEventElapsedTime(&r.ms_masks, g->ev[0], g->ev[1]);
  cudaEventElapsedTime(&r.ms_explore, g->ev[1], g->ev[2]);
  cudaEventElapsedTime(&r.ms_select, g->ev[2], g->ev[3]);
  r.fused = fuse && g->last_fused ? 1 : 0;
  *out = r;
  return r.status == PUMP_ERR_INFEASIBLE ? PUMP_ERR_INFEASIBLE : PUMP_OK;
}

int pump_plan_collect(pump_graph* g, pump_plan_result* out, void* stream) {
  if (!g || !out || !g->ex.ctl) return PUMP_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = make_events(g);
  if (rc) return rc;
  PUMP_CUDA_TRY(cudaMemcpyAsync(g->ctl_host, g->ex.ctl, sizeof(ExploreCtl), cudaMemcpyDeviceToHost, s));
  PUMP_CUDA_TRY(cudaStreamSynchronize(s));
  const ExploreCtl h = *g->ctl_host;
  pump_plan_result r;
  std::memset(&r, 0, sizeof(r));
  r.chosen_plan = -1;
  fill_explore_stats(g, h, &r);
  r.status = h.status;
  r.fused = g->last_fused ? 1 : 0;
  *out = r;
  return h.status;
}

int pump_certify(pump_graph* g, const int32_t* path, int32_t path_len, int32_t n_mc, int32_t substeps, uint64_t seed,
                 int64_t* n_collide, double* cp, void* stream) {
  if (!g || !g->has_geometry || !path || path_len < 1 || path_len > kMaxPathEdges + 1 || n_mc < 0 || substeps < 1 ||
      substeps > 64 || !n_collide || !cp)
    return PUMP_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<int32_t> ph;
  int rc = host_copy(ph, path, (size_t)path_len, s);
  if (rc) return rc;
  for (int32_t v : ph)
    if (v < 0 || v >= g->n) return PUMP_ERR_INVALID_ARG;
  int32_t* pd = (int32_t*)dev_alloc(sizeof(int32_t) * (size_t)path_len, s);
  if (!pd) return PUMP_ERR_OOM;
  rc = stage(pd, ph.data(), sizeof(int32_t) * (size_t)path_len, s);
  int64_t c = 0;
  if (!rc) rc = run_certify_path(g, pd, path_len, n_mc, substeps, seed, &c, s);
  dev_free(pd, s);
  if (rc) return rc;
  *n_collide = c;
  *cp = n_mc > 0 ? (double)c / (double)n_mc : 0.0;
  return PUMP_OK;
}

int pump_export(pump_graph* g, int32_t what, void* host_buf, size_t cap, size_t* needed) {
  if (!g || !needed) return PUMP_ERR_INVALID_ARG;
  const size_t E = (size_t)g->E, n = (size_t)g->n, P = (size_t)g->last_plans, w = (size_t)g->n_words;
  const void* src = nullptr;
  size_t bytes = 0;
  int64_t counts[8] = {g->n, g->E, g->last_plans, g->last_goal, g->N, g->W, g->n_words, g->n_valid};
  const bool geo = g->has_geometry;
  const bool ex = g->explored;
  switch (what) {
    case PUMP_EXPORT_COUNTS: bytes = sizeof(counts); break;
    case PUMP_EXPORT_NODE_VALID: src = g->valid; bytes = n; break;
    case PUMP_EXPORT_ROW_PTR: src = g->row_ptr; bytes = 4 * (n + 1); break;
    case PUMP_EXPORT_COL: src = g->col; bytes = 4 * E; break;
    case PUMP_EXPORT_ECOST: src = g->ecost; bytes = 4 * E; break;
    case PUMP_EXPORT_TAU: if (!geo) return PUMP_ERR_INVALID_ARG; src = g->tau; bytes = 4 * E; break;
    case PUMP_EXPORT_H: if (!geo) return PUMP_ERR_INVALID_ARG; src = g->h; bytes = 4 * E; break;
    case PUMP_EXPORT_PHI: if (!geo) return PUMP_ERR_INVALID_ARG; src = g->phi; bytes = 16 * E; break;
    case PUMP_EXPORT_L: if (!geo) return PUMP_ERR_INVALID_ARG; src = g->L; bytes = 12 * E; break;
    case PUMP_EXPORT_NOMINAL: if (!geo) return PUMP_ERR_INVALID_ARG; src = g->nom; bytes = 12 * (size_t)g->W * E; break;
    case PUMP_EXPORT_LINF: if (!geo) return PUMP_ERR_INVALID_ARG; bytes = 12; break;
    case PUMP_EXPORT_MASKS: src = g->emask; bytes = 4 * w * E; break;
    case PUMP_EXPORT_PLAN_HEAD: if (!ex) return PUMP_ERR_INVALID_ARG; src = g->ex.head; bytes = 4 * P; break;
    case PUMP_EXPORT_PLAN_PARENT: if (!ex) return PUMP_ERR_INVALID_ARG; src = g->ex.parent; bytes = 4 * P; break;
    case PUMP_EXPORT_PLAN_COST: if (!ex) return PUMP_ERR_INVALID_ARG; src = g->ex.cost; bytes = 4 * P; break;
    case PUMP_EXPORT_PLAN_MASK: if (!ex) return PUMP_ERR_INVALID_ARG; src = g->ex.mask; bytes = 4 * w * P; break;
    case PUMP_EXPORT_PLAN_POPC: if (!ex) return PUMP_ERR_INVALID_ARG; src = g->ex.popc; bytes = 4 * P; break;
    case PUMP_EXPORT_PLAN_CREATED: if (!ex) return PUMP_ERR_INVALID_ARG; src = g->ex.tcre; bytes = 4 * P; break;
    case PUMP_EXPORT_PLAN_EXPANDED: if (!ex) return PUMP_ERR_INVALID_ARG; src = g->ex.eexp; bytes = 4 * P; break;
    case PUMP_EXPORT_GOAL_PLANS: if (!ex) return PUMP_ERR_INVALID_ARG; src = g->ex.goal_sorted; bytes = 4 * (size_t)g->last_goal; break;
    case PUMP_EXPORT_EDGE_BOX: if (!geo) return PUMP_ERR_INVALID_ARG; src = g->ibox; bytes = 24 * E; break;
    case PUMP_EXPORT_NOMINAL_VEL: if (!geo) return PUMP_ERR_INVALID_ARG; src = g->nvel; bytes = 12 * (size_t)g->W * E; break;
    case PUMP_EXPORT_EDGE_ORDER: if (!g->eorder) return PUMP_ERR_INVALID_ARG; src = g->eorder; bytes = 8 * E; break;
    default: return PUMP_ERR_INVALID_ARG;
  }
  *needed = bytes;
  if (cap < bytes || (bytes && !host_buf)) return PUMP_ERR_INVALID_ARG;
  if (what == PUMP_EXPORT_COUNTS) {
    std::memcpy(host_buf, counts, sizeof(counts));
    return PUMP_OK;
  }
  if (what == PUMP_EXPORT_LINF) {
    std::memcpy(host_buf, g->linf, 12);
    return PUMP_OK;
  }
  if (cudaDeviceSynchronize() != cudaSuccess) return PUMP_ERR_CUDA;
  if (bytes && cudaMemcpy(host_buf, src, bytes, cudaMemcpyDeviceToHost) != cudaSuccess) return PUMP_ERR_CUDA;
  return PUMP_OK;
}

void pump_graph_destroy(pump_graph* g) { destroy(g); }

uint64_t pump_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

}  // extern "C"
