// Many independent queries at once (pump_plan_batch).
//
// Each query is the single-query method on its own graph: its edge masks, its
// Explore run, its PlanSelection.  What the batch changes is only how the work
// is launched: the Explore runs of all queries go to one persistent launch of
// several thread-block clusters, each cluster taking the next query from a
// device counter (explore_cluster.cu), and the small per-query steps before and
// after it (starting state, P_goal, reading back the control blocks) are one
// launch each for the whole batch.  Query results therefore equal the
// single-query results bit for bit.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "pump_internal.cuh"

namespace pump {

int plan_cluster_form(int32_t n, int32_t kstride, int want_nr, bool want_global, int* nr_out, bool* dsm_out,
                      size_t* smem_out);
int cluster_capacity(int nr, bool dsm, size_t smem, int* out);
int run_explore_cluster_batch(const ExploreArgs* As_dev, const int32_t* starts_dev, int32_t nq, int nr, bool dsm,
                              size_t smem, int n_clusters, int32_t* next_dev, cudaStream_t s);
int run_goal_finalize(pump_graph* g, const ExploreArgs& A, cudaStream_t s);

namespace {

// Query q (block q): mbest cleared to +inf when it lives in global memory, then the starting state.
__global__ void k_init_batch(const ExploreArgs* __restrict__ As, const int32_t* __restrict__ starts, int32_t nq,
                             int fill_mbest) {
  const ExploreArgs& A = As[blockIdx.x];
  if (fill_mbest) {
    const int64_t m = (int64_t)A.n * A.kstride;
    for (int64_t k = threadIdx.x; k < m; k += blockDim.x) A.mbest[k] = 0x7f800000u;
  }
  __syncthreads();
  if (threadIdx.x == 0) explore_init_thread(A, starts[blockIdx.x]);
}

// Query q (block q): P_goal in PlanSelection order (the group array is free scratch after Explore).
__global__ void k_finalize_batch(const ExploreArgs* __restrict__ As, int32_t* const* __restrict__ sorted) {
  const ExploreArgs& A = As[blockIdx.x];
  goal_finalize_block(A, A.group, sorted[blockIdx.x]);
}

// Control blocks of all queries into one array (a single copy to the host).
__global__ void k_gather_ctl(const ExploreArgs* __restrict__ As, int32_t nq, ExploreCtl* __restrict__ out) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < nq) out[q] = *As[q].ctl;
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace
}  // namespace pump

extern "C" int pump_plan_batch(pump_graph* const* graphs, int32_t nq, const pump_plan_params* params,
                               const pump_batch_config* config, pump_plan_result* results, void* stream) {
  using namespace pump;
  if (!graphs || !params || !results || nq < 1 || nq > (1 << 20)) return PUMP_ERR_INVALID_ARG;
  pump_batch_config cfg = {0, 0, 0, 0, 0, 0};
  if (config) cfg = *config;
  if ((cfg.cluster_size != 0 && cfg.cluster_size != 4 && cfg.cluster_size != 8 && cfg.cluster_size != 16) ||
      (cfg.mbest_global != 0 && cfg.mbest_global != 1) || cfg.max_clusters < 0 || cfg.mask_pairs < 0 ||
      cfg.mask_pairs > 2 || cfg.mask_chunk < 0 || cfg.mask_chunk > 64 || cfg.mask_span < 0 ||
      cfg.mask_span > 65536 || cfg.mask_span % 32)
    return PUMP_ERR_INVALID_ARG;
  std::vector<pump_graph*> gs(graphs, graphs + nq);
  for (int q = 0; q < nq; ++q)
    if (!gs[q] || !gs[q]->has_geometry || check_plan_params(params + q)) return PUMP_ERR_INVALID_ARG;
  {
    std::vector<pump_graph*> sorted(gs);
    std::sort(sorted.begin(), sorted.end());
    if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end()) return PUMP_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  for (auto& e : ev)
    if (cudaEventCreate(&e) != cudaSuccess) {
      for (auto& f : ev)
        if (f) cudaEventDestroy(f);
      return PUMP_ERR_CUDA;
    }
  auto finish = [&](int rc) {
    for (auto& e : ev) cudaEventDestroy(e);
    return rc;
  };
  if (cudaEventRecord(ev[0], s) != cudaSuccess) return finish(PUMP_ERR_CUDA);
  // edge masks of every query in one launch
  {
    const int rc = compute_edge_masks_batch(gs.data(), nq, s, cfg.mask_pairs, cfg.mask_chunk, cfg.mask_span);
    if (rc) return finish(rc);
  }
  if (cudaEventRecord(ev[1], s) != cudaSuccess) return finish(PUMP_ERR_CUDA);
  // Explore for every query
  std::vector<ExploreArgs> hA(nq);
  std::vector<int32_t> hstart(nq);
  std::vector<int32_t*> hsorted(nq);
  int32_t n_max = 1, k_max = 1;
  for (int q = 0; q < nq; ++q) {
    const int rc = prepare_explore_args(gs[q], params + q, gs[q]->radius, &hA[q], s);
    if (rc) return finish(rc);
    hstart[q] = gs[q]->start;
    hsorted[q] = gs[q]->ex.goal_sorted;
    n_max = std::max(n_max, hA[q].n);
    k_max = std::max(k_max, hA[q].kstride);
  }
  int nr = 0;
  bool dsm = false;
  size_t smem = 0;
  int rc = plan_cluster_form(n_max, k_max, cfg.cluster_size, cfg.mbest_global != 0, &nr, &dsm, &smem);
  if (rc) return finish(rc);
  std::vector<ExploreCtl> hctl(nq);
  if (nr > 0) {
    const size_t b_args = align256(sizeof(ExploreArgs) * (size_t)nq), b_starts = align256(sizeof(int32_t) * nq),
                 b_sorted = align256(sizeof(int32_t*) * nq), b_ctl = align256(sizeof(ExploreCtl) * (size_t)nq);
    unsigned char* buf = (unsigned char*)dev_alloc(b_args + b_starts + b_sorted + b_ctl + 256, s);
    if (!buf) return finish(PUMP_ERR_OOM);
    ExploreArgs* As_dev = reinterpret_cast<ExploreArgs*>(buf);
    int32_t* starts_dev = reinterpret_cast<int32_t*>(buf + b_args);
    int32_t** sorted_dev = reinterpret_cast<int32_t**>(buf + b_args + b_starts);
    ExploreCtl* ctl_dev = reinterpret_cast<ExploreCtl*>(buf + b_args + b_starts + b_sorted);
    int32_t* next_dev = reinterpret_cast<int32_t*>(buf + b_args + b_starts + b_sorted + b_ctl);
    int cap = 0;
    rc = cluster_capacity(nr, dsm, smem, &cap);
    int n_clusters = std::min(nq, std::max(cap, 1));
    if (cfg.max_clusters > 0) n_clusters = std::min(n_clusters, cfg.max_clusters);
    if (!rc && cudaMemcpyAsync(As_dev, hA.data(), sizeof(ExploreArgs) * nq, cudaMemcpyHostToDevice, s) != cudaSuccess)
      rc = PUMP_ERR_CUDA;
    if (!rc && cudaMemcpyAsync(starts_dev, hstart.data(), sizeof(int32_t) * nq, cudaMemcpyHostToDevice, s) != cudaSuccess)
      rc = PUMP_ERR_CUDA;
    if (!rc && cudaMemcpyAsync(sorted_dev, hsorted.data(), sizeof(int32_t*) * nq, cudaMemcpyHostToDevice, s) != cudaSuccess)
      rc = PUMP_ERR_CUDA;
    if (!rc) {
      k_init_batch<<<nq, 256, 0, s>>>(As_dev, starts_dev, nq, dsm ? 0 : 1);
      note_launch();
      rc = run_explore_cluster_batch(As_dev, starts_dev, nq, nr, dsm, smem, n_clusters, next_dev, s);
    }
    if (!rc) {
      k_finalize_batch<<<nq, 1024, 0, s>>>(As_dev, sorted_dev);
      note_launch();
      k_gather_ctl<<<(nq + 127) / 128, 128, 0, s>>>(As_dev, nq, ctl_dev);
      note_launch();
      if (cudaGetLastError() != cudaSuccess ||
          cudaMemcpyAsync(hctl.data(), ctl_dev, sizeof(ExploreCtl) * nq, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        rc = PUMP_ERR_CUDA;
    }
    dev_free(buf, s);
    if (!rc && cudaStreamSynchronize(s) != cudaSuccess) rc = PUMP_ERR_CUDA;
    if (rc) return finish(rc);
  } else {
    // no cluster form on this device: the grid kernel, one query after another
    for (int q = 0; q < nq && !rc; ++q) {
      rc = run_explore_kernels(gs[q], hA[q], 1, s);
      if (!rc) rc = run_goal_finalize(gs[q], hA[q], s);
      if (!rc && cudaMemcpyAsync(&hctl[q], hA[q].ctl, sizeof(ExploreCtl), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        rc = PUMP_ERR_CUDA;
    }
    if (!rc && cudaStreamSynchronize(s) != cudaSuccess) rc = PUMP_ERR_CUDA;
    if (rc) return finish(rc);
  }
  if (cudaEventRecord(ev[2], s) != cudaSuccess) return finish(PUMP_ERR_CUDA);
  // PlanSelection, query by query
  int first = PUMP_OK;
  std::vector<int32_t> path(kMaxPathEdges + 1);
  for (int q = 0; q < nq; ++q) {
    pump_graph* g = gs[q];
    pump_plan_result r;
    std::memset(&r, 0, sizeof(r));
    r.chosen_plan = -1;
    fill_explore_stats(g, hctl[q], &r);
    if (hctl[q].status) {
      r.status = hctl[q].status;
    } else if (params[q].flags & PUMP_EXPLORE_ONLY) {
      r.status = PUMP_OK;
    } else {
      ExploreCtl h;
      rc = run_select(g, params + q, path.data(), (int32_t)path.size(), &r, &h, s);
      fill_explore_stats(g, h, &r);
      if (rc) r.status = rc;
    }
    results[q] = r;
    if (first == PUMP_OK && r.status != PUMP_OK) first = r.status;
  }
  if (cudaEventRecord(ev[3], s) != cudaSuccess || cudaEventSynchronize(ev[3]) != cudaSuccess)
    return finish(PUMP_ERR_CUDA);
  float t[3] = {0.f, 0.f, 0.f};
  cudaEventElapsedTime(&t[0], ev[0], ev[1]);
  cudaEventElapsedTime(&t[1], ev[1], ev[2]);
  cudaEventElapsedTime(&t[2], ev[2], ev[3]);
  for (int q = 0; q < nq; ++q) {
    results[q].ms_masks = t[0];
    results[q].ms_explore = t[1];
    results[q].ms_select = t[2];
  }
  return finish(first);
}
