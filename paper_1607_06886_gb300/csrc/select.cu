// P_goal, PlanSelection (Algorithm 5) and MC(p) certification on the device.
//
// P_goal.  Explore records every arena plan whose head is a goal node.  Such a
// plan p was removed by RemoveDominated iff some plan s at the same node with
// s.cost < p.cost and s.popc <= p.popc entered P before p stopped being open,
// i.e. with creating group t_s <= e_p (e_p the group that expanded p, or
// never).  Removed chains end at plans in the arena, so arena plans suffice.
//
// Order.  P_goal is sorted by ascending popc, then descending cost, then
// ascending id; the bisection runs on 1-based indices as in Algorithm 5.  A
// single-thread state machine advances it and stops when it needs a Monte
// Carlo count it has not got; the host then certifies that plan and resumes.
// Small P_goal sets are certified in one batch up front.
//
// MC(p).  Four lanes per rollout (axes x, y, z and one idle lane).  Rollout m,
// step s, axis j draws (xi0, xi1) from Philox4x64-10 with counter (m, s, j, 0)
// and key (seed, 0): the top 24 bits of words 0 and 1 give u1, u2 in (0,1),
// and Box-Muller gives sqrt(-2 ln u1) (cos 2 pi u2, sin 2 pi u2) in float.  The
// deviation starts at Linf xi (step 0) and is carried over the plan's
// connections; each waypoint interval takes `substeps` steps of
// hs = (tau / W) / substeps with Phi(hs), L(hs) and the nominal position at
// t = ((k-1) substeps + s) hs.  A rollout collides iff a step position lies in
// a closed box.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "pump_internal.cuh"

namespace pump {
namespace {

struct SelState {
  int32_t l, u, m, phase, last_m, need, done, status, chosen, n_probes, pad0, pad1;
  long long last_c, chosen_c;
};

__device__ __forceinline__ bool key_less(const ExploreArgs& A, int32_t a, int32_t b) {
  const int32_t pa = A.popc[a], pb = A.popc[b];
  if (pa != pb) return pa < pb;
  const float ca = A.cost[a], cb = A.cost[b];
  if (ca != cb) return ca > cb;
  return a < b;
}

__global__ void k_goal_finalize(ExploreArgs A, int32_t* removed, int32_t* sorted) {
  ExploreCtl* ctl = A.ctl;
  const int G = ctl->n_goal_all;
  for (int k = threadIdx.x; k < G; k += blockDim.x) {
    const int32_t p = A.goal_all[k];
    const int32_t ep = A.eexp[p] >= 0 ? A.eexp[p] : INT_MAX;
    const int32_t x = A.head[p];
    int rem = 0;
    for (int j = 0; j < G && !rem; ++j) {
      const int32_t q = A.goal_all[j];
      if (q == p || A.head[q] != x) continue;
      if (A.tcre[q] <= ep && A.cost[q] < A.cost[p] && A.popc[q] <= A.popc[p]) rem = 1;
    }
    removed[k] = rem;
  }
  __syncthreads();
  __shared__ int count;
  if (threadIdx.x == 0) count = 0;
  __syncthreads();
  for (int k = threadIdx.x; k < G; k += blockDim.x) {
    if (removed[k]) continue;
    const int32_t p = A.goal_all[k];
    int rank = 0;
    for (int j = 0; j < G; ++j)
      if (!removed[j] && key_less(A, A.goal_all[j], p)) ++rank;
    sorted[rank] = p;
    atomicAdd(&count, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) ctl->n_goal = count;
}

// Path of each plan: node ids from x_init and the edge ids between them.
__global__ void k_mc_paths(const int32_t* __restrict__ plans, int n_cert, const int32_t* __restrict__ parent,
                           const int32_t* __restrict__ pedge, const int32_t* __restrict__ head, int32_t* plen,
                           int32_t* pedges, int32_t* pnodes, int32_t* err) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_cert) return;
  int len = 0;
  for (int32_t q = plans[k]; parent[q] >= 0; q = parent[q]) {
    if (++len > kMaxPathEdges) { atomicExch(err, 1); plen[k] = 0; return; }
  }
  plen[k] = len;
  int j = len;
  int32_t q = plans[k];
  pnodes[(size_t)k * (kMaxPathEdges + 1) + j] = head[q];
  while (parent[q] >= 0) {
    --j;
    pedges[(size_t)k * kMaxPathEdges + j] = pedge[q];
    q = parent[q];
    pnodes[(size_t)k * (kMaxPathEdges + 1) + j] = head[q];
  }
}

// Edge ids along a node path given by the caller (binary search in the rows).
__global__ void k_path_edges(const int32_t* __restrict__ nodes, int len, const int32_t* __restrict__ row_ptr,
                             const int32_t* __restrict__ col, int32_t* pedges, int32_t* pnodes, int32_t* plen,
                             int32_t* err) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j == 0) plen[0] = len - 1;
  if (j < len) pnodes[j] = nodes[j];
  if (j >= len - 1) return;
  int v = nodes[j], u = nodes[j + 1];
  int lo = row_ptr[v], hi = row_ptr[v + 1];
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (col[mid] < u) lo = mid + 1; else hi = mid;
  }
  if (lo < row_ptr[v + 1] && col[lo] == u) pedges[j] = lo;
  else atomicExch(err, 1);
}

// Per path edge: Phi(hs) (4), L(hs) (3), pad, then W*S*3 nominal positions.
__global__ void k_mc_prep(int n_cert, const int32_t* __restrict__ plen, const int64_t* __restrict__ toff,
                          const int32_t* __restrict__ pedges, const int32_t* __restrict__ pnodes,
                          const float* __restrict__ states, const float* __restrict__ tau, int W, int S, float sigma,
                          float* table) {
  const int k = blockIdx.y;
  if (k >= n_cert) return;
  const int L = plen[k];
  const int stride = 8 + W * S * 3;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < L; j += gridDim.x * blockDim.x) {
    const int e = pedges[(size_t)k * kMaxPathEdges + j];
    const int v = pnodes[(size_t)k * (kMaxPathEdges + 1) + j], u = pnodes[(size_t)k * (kMaxPathEdges + 1) + j + 1];
    float* T = table + toff[k] + (size_t)j * stride;
    const float t32 = tau[e];
    const float h = __fdiv_rn(t32, (float)W);
    const float hs = __fdiv_rn(h, (float)S);
    double Phi[4], Lm[3], Linf[3];
    model_dev((double)sigma, (double)hs, Phi, Lm, Linf);
    for (int q = 0; q < 4; ++q) T[q] = __double2float_rn(Phi[q]);
    for (int q = 0; q < 3; ++q) T[4 + q] = __double2float_rn(Lm[q]);
    T[7] = 0.f;
    double xv[6], xu[6];
    for (int q = 0; q < 6; ++q) {
      xv[q] = (double)states[6 * v + q];
      xu[q] = (double)states[6 * u + q];
    }
    const double td = (double)t32;
    for (int kk = 1; kk <= W; ++kk)
      for (int s = 1; s <= S; ++s) {
        const double t = (double)((kk - 1) * S + s) * (double)hs;
        for (int a = 0; a < 3; ++a)
          T[8 + (((kk - 1) * S + (s - 1)) * 3) + a] = __double2float_rn(nominal_dev(xv, xu, td, a, t));
      }
  }
}

__device__ __forceinline__ void mc_normals(uint64_t seed, uint64_t m, uint64_t s, uint64_t j, float* z0, float* z1) {
  uint64_t o[4];
  philox4x64(m, s, j, 0ull, seed, 0ull, o);
  const float u1 = ((float)(o[0] >> 40) + 0.5f) * 5.9604644775390625e-08f;
  const float u2 = ((float)(o[1] >> 40) + 0.5f) * 5.9604644775390625e-08f;
  const float r = sqrtf(-2.0f * logf(u1));
  float sn, cs;
  sincospif(2.0f * u2, &sn, &cs);
  *z0 = r * cs;
  *z1 = r * sn;
}

constexpr int kMcThreads = 256;
constexpr int kRollPerBlock = kMcThreads / 4;

__global__ void __launch_bounds__(kMcThreads) k_mc_rollout(int n_cert, int bpp, const int32_t* __restrict__ plen,
                                                            const int64_t* __restrict__ toff,
                                                            const float* __restrict__ table, int W, int S,
                                                            const float* __restrict__ linf_g,
                                                            const float* __restrict__ boxes_g, int nb, int n_mc,
                                                            uint64_t seed, unsigned long long* counts) {
  extern __shared__ float boxes[];
  for (int q = threadIdx.x; q < 6 * nb; q += blockDim.x) boxes[q] = boxes_g[q];
  __syncthreads();
  const int k = blockIdx.x / bpp;
  const int m = (blockIdx.x % bpp) * kRollPerBlock + (threadIdx.x >> 2);
  const int j = threadIdx.x & 3;
  const int lane = threadIdx.x & 31;
  const int qbase = lane & ~3;
  const bool active = m < n_mc;
  const int L = plen[k];
  const int stride = 8 + W * S * 3;
  const float* T0 = table + toff[k];
  float d0 = 0.f, d1 = 0.f;
  if (j < 3) {
    float x0, x1;
    mc_normals(seed, (uint64_t)m, 0ull, (uint64_t)j, &x0, &x1);
    d0 = __fmul_rn(linf_g[0], x0);
    d1 = fmaf(linf_g[1], x0, __fmul_rn(linf_g[2], x1));
  }
  bool hit = false;
  uint64_t step = 0;
  bool finished = false;
  for (int e = 0; e < L && !finished; ++e) {
    const float* T = T0 + (size_t)e * stride;
    const float P0 = T[0], P1 = T[1], P2 = T[2], P3 = T[3], L0 = T[4], L1 = T[5], L2 = T[6];
    for (int q = 0; q < W * S && !finished; ++q) {
      ++step;
      float pos = 0.f;
      if (j < 3) {
        float x0, x1;
        mc_normals(seed, (uint64_t)m, step, (uint64_t)j, &x0, &x1);
        const float n0 = __fmul_rn(L0, x0);
        const float n1 = fmaf(L1, x0, __fmul_rn(L2, x1));
        const float e0 = fmaf(P0, d0, fmaf(P1, d1, n0));
        const float e1 = fmaf(P2, d0, fmaf(P3, d1, n1));
        d0 = e0;
        d1 = e1;
        pos = __fadd_rn(T[8 + q * 3 + j], d0);
      }
      const float px = __shfl_sync(0xffffffffu, pos, qbase + 0);
      const float py = __shfl_sync(0xffffffffu, pos, qbase + 1);
      const float pz = __shfl_sync(0xffffffffu, pos, qbase + 2);
      if (!hit)
        for (int o = 0; o < nb; ++o)
          if (in_box_dev(px, py, pz, boxes + 6 * o)) { hit = true; break; }
      finished = __all_sync(0xffffffffu, hit || !active);
    }
  }
  const unsigned bal = __ballot_sync(0xffffffffu, active && hit && j == 0);
  if (lane == 0 && bal) atomicAdd(counts + k, (unsigned long long)__popc(bal));
}

__global__ void k_counts_store(int n_cert, const unsigned long long* __restrict__ counts, const int32_t* __restrict__ idx,
                               long long* by_index) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n_cert) by_index[idx[k]] = (long long)counts[k];
}

__global__ void k_bisect_run(SelState* st, const int32_t* __restrict__ sorted, int G, const long long* by_index,
                             int n_mc, double alpha) {
  SelState s = *st;
  s.need = -1;
  for (int guard = 0; guard < 256 && !s.done; ++guard) {
    if (s.phase == 0) {
      s.l = 1;
      s.u = G;
      s.m = (s.l + s.u + 1) / 2;
      s.last_m = -1;
      s.n_probes = 0;
      s.phase = (s.l != s.u) ? 1 : 2;
    } else if (s.phase == 1) {
      const long long c = by_index[s.m - 1];
      if (c < 0) { s.need = s.m - 1; break; }
      s.last_m = s.m;
      s.last_c = c;
      s.n_probes++;
      if ((double)c / (double)n_mc > alpha) s.u = s.m - 1; else s.l = s.m;
      s.m = (s.l + s.u + 1) / 2;
      if (s.l == s.u) s.phase = 2;
    } else {
      long long c;
      if (s.last_m == s.m) {
        c = s.last_c;
      } else {
        c = by_index[s.m - 1];
        if (c < 0) { s.need = s.m - 1; break; }
        s.n_probes++;
      }
      s.chosen = sorted[s.m - 1];
      s.chosen_c = c;
      s.status = ((double)c / (double)n_mc > alpha) ? (int)PUMP_ERR_INFEASIBLE : (int)PUMP_OK;
      s.done = 1;
    }
  }
  *st = s;
}

__global__ void k_backtrack(const int32_t* __restrict__ parent, const int32_t* __restrict__ head, int32_t plan,
                            int32_t* out, int32_t cap, int32_t* len_out) {
  int len = 0;
  for (int32_t q = plan; q >= 0; q = parent[q]) ++len;
  *len_out = len;
  int k = len;
  for (int32_t q = plan; q >= 0; q = parent[q]) {
    --k;
    if (k < cap) out[k] = head[q];
  }
}

__global__ void k_gather(int n, const int32_t* __restrict__ idx, const int32_t* __restrict__ src, int32_t* dst) {
  int k = threadIdx.x;
  if (k < n) dst[k] = src[idx[k]];
}

int ensure_sel(pump_graph* g, int G, cudaStream_t s) {
  ExploreBufs& X = g->ex;
  if (!X.sel_state) {
    X.sel_state = graph_alloc(g, sizeof(SelState), s);
    X.sel_toff = (int64_t*)graph_alloc(g, sizeof(int64_t) * 32, s);
    X.sel_err = (int32_t*)graph_alloc(g, sizeof(int32_t) * 2, s);
    X.sel_idx = (int32_t*)graph_alloc(g, sizeof(int32_t) * 32, s);
    if (!X.sel_state || !X.sel_toff || !X.sel_err || !X.sel_idx) return PUMP_ERR_OOM;
  }
  if (G > X.sel_cap) {
    X.sel_by_index = (long long*)graph_realloc(g, X.sel_by_index, sizeof(long long) * G, s);
    if (!X.sel_by_index) {
      X.sel_cap = 0;
      return PUMP_ERR_OOM;
    }
    X.sel_cap = G;
  }
  return PUMP_OK;
}

int ensure_mc(pump_graph* g, int n_cert, cudaStream_t s) {
  ExploreBufs& X = g->ex;
  if (n_cert <= X.mc_cap && X.mc_count) return PUMP_OK;
  int cap = std::max(n_cert, 32);
  X.mc_count = (int64_t*)graph_realloc(g, X.mc_count, sizeof(int64_t) * cap, s);
  X.mc_plan = (int32_t*)graph_realloc(g, X.mc_plan, sizeof(int32_t) * cap, s);
  X.mc_plen = (int32_t*)graph_realloc(g, X.mc_plen, sizeof(int32_t) * (cap + 1), s);
  X.mc_pedges = (int32_t*)graph_realloc(g, X.mc_pedges, sizeof(int32_t) * (size_t)cap * kMaxPathEdges, s);
  X.path_buf = (int32_t*)graph_realloc(g, X.path_buf, sizeof(int32_t) * (size_t)cap * (kMaxPathEdges + 1), s);
  if (!X.mc_count || !X.mc_plan || !X.mc_plen || !X.mc_pedges || !X.path_buf) {
    X.mc_cap = 0;
    return PUMP_ERR_OOM;
  }
  X.mc_cap = cap;
  return PUMP_OK;
}

// Certify plans whose paths are in mc_plen / mc_pedges / path_buf (rows 0..n_cert-1).
int mc_run(pump_graph* g, int n_cert, int n_mc, int S, uint64_t seed, int64_t* toff_dev, int32_t* err_dev,
           cudaStream_t s) {
  ExploreBufs& X = g->ex;
  std::vector<int32_t> plen(n_cert);
  int32_t err = 0;
  PUMP_CUDA_TRY(cudaMemcpyAsync(plen.data(), X.mc_plen, sizeof(int32_t) * n_cert, cudaMemcpyDeviceToHost, s));
  PUMP_CUDA_TRY(cudaMemcpyAsync(&err, err_dev, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  PUMP_CUDA_TRY(cudaStreamSynchronize(s));
  if (err) return PUMP_ERR_INVALID_ARG;
  const int stride = 8 + g->W * S * 3;
  std::vector<int64_t> toff(n_cert);
  int64_t tot = 0;
  int maxL = 0;
  for (int k = 0; k < n_cert; ++k) {
    toff[k] = tot;
    tot += (int64_t)plen[k] * stride;
    maxL = std::max(maxL, plen[k]);
  }
  if (tot > X.mc_table_floats) {
    int64_t want = std::max<int64_t>(tot, 1 << 16);
    X.mc_table = (float*)graph_realloc(g, X.mc_table, sizeof(float) * want, s);
    if (!X.mc_table) return PUMP_ERR_OOM;
    X.mc_table_floats = want;
  }
  PUMP_CUDA_TRY(cudaMemcpyAsync(toff_dev, toff.data(), sizeof(int64_t) * n_cert, cudaMemcpyHostToDevice, s));
  if (maxL > 0) {
    dim3 grid((maxL + 63) / 64, n_cert);
    k_mc_prep<<<grid, 64, 0, s>>>(n_cert, X.mc_plen, toff_dev, X.mc_pedges, X.path_buf, g->states, g->tau, g->W, S,
                                  g->sigma, X.mc_table);
    note_launch();
  }
  PUMP_CUDA_TRY(cudaMemsetAsync(X.mc_count, 0, sizeof(int64_t) * n_cert, s));
  const int bpp = (n_mc + kRollPerBlock - 1) / kRollPerBlock;
  if (n_mc > 0 && bpp > 0) {
    k_mc_rollout<<<n_cert * bpp, kMcThreads, sizeof(float) * 6 * std::max(g->n_boxes, 1), s>>>(
        n_cert, bpp, X.mc_plen, toff_dev, X.mc_table, g->W, S, g->linf_dev, g->boxes, g->n_boxes, n_mc, seed,
        reinterpret_cast<unsigned long long*>(X.mc_count));
    note_launch();
  }
  PUMP_CUDA_TRY(cudaGetLastError());
  return PUMP_OK;
}

}  // namespace

int run_select(pump_graph* g, const pump_plan_params* p, int32_t* path, int32_t path_cap, pump_plan_result* out,
               cudaStream_t s) {
  ExploreBufs& X = g->ex;
  const int G = g->last_goal;
  out->chosen_plan = -1;
  out->path_len = 0;
  out->path_truncated = 0;
  out->n_certified = 0;
  if (G == 0) {
    out->status = PUMP_ERR_INFEASIBLE;
    return PUMP_OK;
  }
  const int S = p->mc_substeps;
  int rc = ensure_mc(g, std::min(G, 32), s);
  if (rc) return rc;
  rc = ensure_sel(g, G, s);
  if (rc) return rc;
  long long* by_index = X.sel_by_index;
  SelState* st = (SelState*)X.sel_state;
  int64_t* toff_dev = X.sel_toff;
  int32_t* err_dev = X.sel_err;
  int32_t* idx_buf = X.sel_idx;
  PUMP_CUDA_TRY(cudaMemsetAsync(by_index, 0xff, sizeof(long long) * G, s));
  PUMP_CUDA_TRY(cudaMemsetAsync(st, 0, sizeof(SelState), s));
  PUMP_CUDA_TRY(cudaMemsetAsync(err_dev, 0, sizeof(int32_t) * 2, s));
  int32_t* sorted = X.goal_sorted;
  // batch 0: all of a small P_goal
  std::vector<int32_t> want;
  if (G <= 32)
    for (int k = 0; k < G; ++k) want.push_back(k);
  SelState hs;
  for (int round = 0; round < 256; ++round) {
    if (!want.empty()) {
      const int nc = (int)want.size();
      PUMP_CUDA_TRY(cudaMemcpyAsync(idx_buf, want.data(), sizeof(int32_t) * nc, cudaMemcpyHostToDevice, s));
      k_gather<<<1, 32, 0, s>>>(nc, idx_buf, sorted, X.mc_plan);
      note_launch();
      k_mc_paths<<<(nc + 63) / 64, 64, 0, s>>>(X.mc_plan, nc, X.parent, X.pedge, X.head, X.mc_plen, X.mc_pedges,
                                               X.path_buf, err_dev);
      note_launch();
      rc = mc_run(g, nc, p->n_mc, S, p->mc_seed, toff_dev, err_dev, s);
      if (rc) return rc;
      k_counts_store<<<1, 32, 0, s>>>(nc, reinterpret_cast<unsigned long long*>(X.mc_count), idx_buf, by_index);
      note_launch();
      out->n_certified += nc;
      want.clear();
    }
    k_bisect_run<<<1, 1, 0, s>>>(st, sorted, G, by_index, p->n_mc, (double)p->alpha);
    note_launch();
    PUMP_CUDA_TRY(cudaMemcpyAsync(&hs, st, sizeof(hs), cudaMemcpyDeviceToHost, s));
    PUMP_CUDA_TRY(cudaStreamSynchronize(s));
    if (hs.done) break;
    if (hs.need < 0) return PUMP_ERR_CUDA;
    want.push_back(hs.need);
  }
  if (!hs.done) return PUMP_ERR_TIMEOUT;
  out->chosen_plan = hs.chosen;
  out->mc_collisions = hs.chosen_c;
  out->cp_mc = p->n_mc > 0 ? (double)hs.chosen_c / (double)p->n_mc : 0.0;
  out->status = hs.status;
  // chosen plan's values and path
  float c = 0.f;
  int32_t pc = 0;
  PUMP_CUDA_TRY(cudaMemcpyAsync(&c, X.cost + hs.chosen, sizeof(float), cudaMemcpyDeviceToHost, s));
  PUMP_CUDA_TRY(cudaMemcpyAsync(&pc, X.popc + hs.chosen, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  int32_t* len_dev = err_dev;
  k_backtrack<<<1, 1, 0, s>>>(X.parent, X.head, hs.chosen, X.path_buf, kMaxPathEdges + 1, len_dev);
  note_launch();
  int32_t len = 0;
  PUMP_CUDA_TRY(cudaMemcpyAsync(&len, len_dev, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  PUMP_CUDA_TRY(cudaStreamSynchronize(s));
  out->cost = c;
  out->popc = pc;
  out->cp_hat = (float)pc / (float)g->N;
  const int ncopy = std::min(std::min(len, path_cap), kMaxPathEdges + 1);
  if (path && ncopy > 0)
    PUMP_CUDA_TRY(cudaMemcpyAsync(path, X.path_buf, sizeof(int32_t) * ncopy, cudaMemcpyDeviceToHost, s));
  PUMP_CUDA_TRY(cudaStreamSynchronize(s));
  out->path_len = std::min(len, path_cap);
  out->path_truncated = len > path_cap ? 1 : 0;
  return PUMP_OK;
}

int run_goal_finalize(pump_graph* g, const ExploreArgs& A, cudaStream_t s) {
  // the group array is free after Explore and serves as scratch
  k_goal_finalize<<<1, 1024, 0, s>>>(A, A.group, g->ex.goal_sorted);
  note_launch();
  PUMP_CUDA_TRY(cudaGetLastError());
  return PUMP_OK;
}

int run_certify_path(pump_graph* g, const int32_t* path_dev, int32_t path_len, int32_t n_mc, int32_t substeps,
                     uint64_t seed, int64_t* n_collide, cudaStream_t s) {
  int rc = ensure_mc(g, 1, s);
  if (rc) return rc;
  rc = ensure_sel(g, 1, s);
  if (rc) return rc;
  ExploreBufs& X = g->ex;
  int64_t* toff_dev = X.sel_toff;
  int32_t* err_dev = X.sel_err;
  PUMP_CUDA_TRY(cudaMemsetAsync(err_dev, 0, sizeof(int32_t) * 2, s));
  k_path_edges<<<(path_len + 63) / 64, 64, 0, s>>>(path_dev, path_len, g->row_ptr, g->col, X.mc_pedges, X.path_buf,
                                                   X.mc_plen, err_dev);
  note_launch();
  rc = mc_run(g, 1, n_mc, substeps, seed, toff_dev, err_dev, s);
  if (rc) return rc;
  long long c = 0;
  PUMP_CUDA_TRY(cudaMemcpyAsync(&c, X.mc_count, sizeof(long long), cudaMemcpyDeviceToHost, s));
  PUMP_CUDA_TRY(cudaStreamSynchronize(s));
  *n_collide = c;
  return PUMP_OK;
}

}  // namespace pump
