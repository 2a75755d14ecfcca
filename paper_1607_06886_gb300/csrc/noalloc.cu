// Explore for callers that cannot allocate device memory.
//
// Some callers of a motion planner cannot call cudaMalloc while they plan: a
// robot's real-time control loop that reserves all of its device memory at
// start-up (an allocation mid-loop can block for an unbounded time or fail
// when memory is fragmented), an embedded runtime whose memory budget is
// fixed up front, or a process whose device allocator belongs to a host
// framework that must not be re-entered from inside this library.  For them
// pump_explore_noalloc runs the same Explore kernels as pump_explore, but the
// kernels' scratch (per-node dominance table, group list and offsets, block
// counters, control block, goal list) lives in one file-scope device array of
// fixed size instead of freshly allocated buffers.  The caller supplies the
// graph and the plan arena on the device.
//
// The array is a module global: every GPU that loads the library holds
// kStaticScratchBytes of it until the process exits, and every call on a
// device shares it.  Its contents persist from the previous call; everything
// the kernels read is written by the call's own initialisation first.  Two
// calls whose work overlaps on the GPU (different streams, or another thread)
// race on the array.  A call waits for its own work before it returns, also
// when it fails after its first launch, so serialised calls never overlap.
#include <cuda_runtime.h>

#include <mutex>

#include "pump_internal.cuh"

namespace pump {
int run_goal_finalize(pump_graph* g, const ExploreArgs& A, cudaStream_t s);
}  // namespace pump

namespace {

constexpr size_t kStaticScratchBytes = size_t(32) << 20;  // 32 MiB
constexpr int kMaxDevices = 64;
constexpr int kBlockSlots = 4096;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_scratch_mu;
unsigned char* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device, looked up once per device.
int scratch_address(unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PUMP_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return PUMP_ERR_CUDA;
    g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_ptr[dev];
  return PUMP_OK;
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Device memory of device `dev` (the scratch array used is that device's copy), or managed memory.
bool on_device(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

int32_t popc_bound(double a, int N) {
  if (!(a > 0.0)) return 0;
  double k = ceil(a);
  return (int32_t)(k < (double)N + 1.0 ? k : (double)N + 1.0);
}

// Bytes of the scratch array one call needs; `capacity` is the arena size the kernels use
// (min of the caller's buffers and max_plans).
int scratch_bytes(int32_t n, int32_t n_particles, const pump_plan_params* p, int64_t capacity, size_t* bytes) {
  if (!p || !bytes || n < 1 || n_particles < 32 || capacity < 1) return PUMP_ERR_INVALID_ARG;
  const int32_t kmax = popc_bound(((double)p->eta * (double)p->alpha) * (double)n_particles, n_particles);
  const int32_t kstride = kmax > 1 ? kmax : 1;
  *bytes = align256(sizeof(pump::ExploreCtl)) + align256(sizeof(int32_t) * kBlockSlots) +
           align256(sizeof(int64_t) * kBlockSlots) + align256(sizeof(uint32_t) * (size_t)n * kstride) +
           3 * align256(sizeof(int32_t) * (size_t)capacity) + align256(sizeof(int4) * (size_t)capacity) +
           align256(sizeof(int64_t) * ((size_t)capacity + 1));
  return PUMP_OK;
}

}  // namespace

extern "C" int pump_explore_noalloc(int32_t n, const int32_t* row_ptr, const int32_t* col, const float* ecost,
                                    const uint32_t* emask, int32_t n_particles, int32_t start_idx,
                                    const uint8_t* is_goal, float radius, const pump_plan_params* p,
                                    int64_t capacity, int32_t* plan_head, int32_t* plan_parent, float* plan_cost,
                                    uint32_t* plan_mask, int32_t* plan_popc, int32_t* plan_created,
                                    int32_t* plan_expanded, int32_t* goal_plans, pump_plan_result* stats,
                                    void* stream) {
  using namespace pump;
  if (!p || !stats || n < 1 || start_idx < 0 || start_idx >= n || capacity < 1 || capacity > (1ll << 31) - 2)
    return PUMP_ERR_INVALID_ARG;
  if (n_particles < 32 || n_particles > kMaxParticles || n_particles % 32) return PUMP_ERR_INVALID_ARG;
  if (!(radius > 0.f) || !(p->lambda > 0.f) || !(p->lambda <= 1.f) || !(p->alpha >= 0.f) || !(p->eta > 0.f) ||
      p->max_iterations < 1 || p->max_plans < 1)
    return PUMP_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PUMP_ERR_CUDA;
  const void* dev_ptrs[] = {row_ptr, col, ecost, emask, is_goal, plan_head, plan_parent, plan_cost,
                            plan_mask, plan_popc, plan_created, plan_expanded, goal_plans};
  for (const void* q : dev_ptrs)
    if (!q || !on_device(q, dev)) return PUMP_ERR_INVALID_ARG;
  const int64_t cap = capacity < p->max_plans ? capacity : p->max_plans;  // arena the kernels use
  size_t need = 0;
  int rc = scratch_bytes(n, n_particles, p, cap, &need);
  if (rc) return rc;
  if (need > kStaticScratchBytes) return PUMP_ERR_INVALID_ARG;
  unsigned char* base = nullptr;
  rc = scratch_address(&base);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;

  const double alpha = (double)p->alpha, eta = (double)p->eta;
  const int32_t kmax = popc_bound((eta * alpha) * (double)n_particles, n_particles);
  const int32_t kmin = popc_bound((alpha / eta) * (double)n_particles, n_particles);
  const int32_t kstride = kmax > 1 ? kmax : 1;

  unsigned char* at = base;
  auto carve = [&](size_t bytes) {
    unsigned char* r = at;
    at += align256(bytes);
    return r;
  };
  ExploreArgs A;
  A.ctl = reinterpret_cast<ExploreCtl*>(carve(sizeof(ExploreCtl)));
  A.bcnt = reinterpret_cast<int32_t*>(carve(sizeof(int32_t) * kBlockSlots));
  A.bdeg = reinterpret_cast<int64_t*>(carve(sizeof(int64_t) * kBlockSlots));
  A.mbest = reinterpret_cast<uint32_t*>(carve(sizeof(uint32_t) * (size_t)n * kstride));
  A.group = reinterpret_cast<int32_t*>(carve(sizeof(int32_t) * (size_t)cap));
  A.ginfo = reinterpret_cast<int4*>(carve(sizeof(int4) * (size_t)cap));
  A.pedge = reinterpret_cast<int32_t*>(carve(sizeof(int32_t) * (size_t)cap));
  A.goal_all = reinterpret_cast<int32_t*>(carve(sizeof(int32_t) * (size_t)cap));
  A.etgt = nullptr;  // edge targets are read from the graph arrays
  A.goff = reinterpret_cast<int64_t*>(carve(sizeof(int64_t) * ((size_t)cap + 1)));
  A.row_ptr = row_ptr;
  A.col = col;
  A.ecost = ecost;
  A.emask = emask;
  A.is_goal = is_goal;
  A.n = n;
  A.w = n_particles / 32;
  A.kmax = kmax;
  A.kstride = kstride;
  A.kmin = kmin;
  A.lr = (double)p->lambda * (double)radius;
  A.max_iter = p->max_iterations;
  A.early_stop = (p->flags & PUMP_NO_EARLY_STOP) ? 0 : 1;
  A.head = plan_head;
  A.parent = plan_parent;
  A.tcre = plan_created;
  A.eexp = plan_expanded;
  A.cost = plan_cost;
  A.popc = plan_popc;
  A.mask = plan_mask;
  A.cap = cap;
  A.spin_limit = 20000000ll;

  // a stack graph record carries the node count, start and goal output; it owns no memory
  pump_graph shell;
  shell.n = n;
  shell.start = start_idx;
  shell.ex.goal_sorted = goal_plans;
  rc = run_explore_kernels(&shell, A, explore_mode(p->flags), s);
  if (!rc) rc = run_goal_finalize(&shell, A, s);
  if (rc) {
    // kernels enqueued before the failure may still use the shared array: the next call must
    // not start before they end
    cudaStreamSynchronize(s);
    cudaGetLastError();
    return rc;
  }
  ExploreCtl h;
  if (cudaMemcpyAsync(&h, A.ctl, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess) {
    cudaStreamSynchronize(s);
    cudaGetLastError();
    return PUMP_ERR_CUDA;
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) return PUMP_ERR_CUDA;
  pump_plan_result r{};
  r.status = h.status;
  r.chosen_plan = -1;
  r.n_candidates = h.n_candidates;
  r.n_kept = h.n_kept;
  r.n_plans = h.n_plans;
  r.n_iterations = h.iter;
  r.n_groups = h.n_groups;
  r.n_goal = h.status ? 0 : h.n_goal;
  *stats = r;
  return h.status;
}
