// Explore (Algorithm 4) on the device.
//
// State.  Plans live in an append-only arena (SoA: head, parent, incoming
// edge, cost, popc, mask words, creating group index t, expanding group index
// e).  Per node x and popcount k < K_max, mbest[x][k] holds the least cost of
// any plan ever inserted at x with that popcount (float bits, atomicMin).
//
// Dominance.  A plan p at x is dominated iff some plan d at x has
// d.cost < p.cost and d.popc <= p.popc.  A plan that RemoveDominated removed
// was itself dominated by a plan then in P(x) with strictly lower cost; that
// chain ends at a plan still in P(x) (costs strictly fall, and closed plans
// are never removed), and dominance composes along it.  So "dominated by a
// plan in P(x)" equals "dominated by a plan ever inserted at x", which is
// min_{k <= p.popc} mbest[x][k] < p.cost.  Survivors of an iteration are the
// candidates this test keeps after all of the iteration's candidates are in
// mbest; older open plans it marks are never expanded (they were removed
// while open).  Removal of plans that were already expanded only matters for
// P_goal and is settled at the end from the t / e stamps (select.cu).
//
// Groups.  The bucket of a plan is the least i with cost <= float(i lambda r);
// a plan created by group t joins group max(bucket, t + 1) (it cannot join a
// group already closed).  The next group is the least bucket among open,
// undominated plans; empty group indices in between expand nothing and are
// skipped, which leaves every plan, id and stamp unchanged.
//
// Schedule.  One iteration is five phases separated by grid barriers:
//   P1 expand: candidates of the group (plans by id, then out-edges), CP cutoff,
//      atomicMin into mbest; stamp e = i on group plans.
//   P2 count survivors per block (candidate ranges are contiguous per block).
//   P3 write survivors at arena offsets from the block counts (stable order);
//      minimum bucket over new and older open undominated plans.
//   P4 count plans of the next group per block, with their out-degree sums;
//      raise the stop flag on a goal plan with popc < K_min.
//   P5 write the group (ascending id) and its candidate offsets.
// The persistent kernel runs all iterations in one cooperative launch; the
// stepwise driver launches each phase separately.  Every barrier wait is
// bounded: on expiry the kernel records PUMP_ERR_TIMEOUT and returns.
#include <cuda_runtime.h>

#include <cstdlib>

#include "pump_internal.cuh"

namespace pump {
namespace {

constexpr int kT = 256;
constexpr int kWarpsT = kT / 32;

__device__ __forceinline__ int32_t ld32(const int32_t* p) { return __ldcg(p); }
__device__ __forceinline__ int64_t ld64(const int64_t* p) { return __ldcg(reinterpret_cast<const long long*>(p)); }
__device__ __forceinline__ float ldf(const float* p) { return __ldcg(p); }
__device__ __forceinline__ uint32_t ldu(const uint32_t* p) { return __ldcg(p); }

__device__ __forceinline__ void chunk(int64_t total, int b, int nb, int64_t* lo, int64_t* hi) {
  int64_t per = (total + nb - 1) / nb;
  *lo = min(total, (int64_t)b * per);
  *hi = min(total, *lo + per);
}

// Block-wide exclusive scan (blockDim == kT); returns prefix, writes total.
template <typename T>
__device__ T block_scan(T v, T* total) {
  __shared__ T ws[kWarpsT];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[warp] = x;
  __syncthreads();
  if (warp == 0) {
    T s = lane < kWarpsT ? ws[lane] : T(0);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < kWarpsT) ws[lane] = s;
  }
  __syncthreads();
  T pre = (warp > 0 ? ws[warp - 1] : T(0)) + x - v;
  *total = ws[kWarpsT - 1];
  __syncthreads();
  return pre;
}

template <typename T>
__device__ T block_sum(T v) {
  T tot;
  block_scan<T>(v, &tot);
  return tot;
}

__device__ int32_t block_min(int32_t v) {
  __shared__ int32_t wm[kWarpsT];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
  if (lane == 0) wm[warp] = v;
  __syncthreads();
  int32_t r = wm[0];
  for (int k = 1; k < kWarpsT; ++k) r = min(r, wm[k]);
  __syncthreads();
  return r;
}

// Sum over blocks b' < b of cnt[b'] (and over all blocks), read by the whole block.
template <typename T>
__device__ void block_prefix_of(const T* cnt, int b, int nb, T* before, T* all) {
  T s_before = 0, s_all = 0;
  for (int k = threadIdx.x; k < nb; k += blockDim.x) {
    T c = (sizeof(T) == 8) ? (T)ld64(reinterpret_cast<const int64_t*>(cnt + k))
                           : (T)ld32(reinterpret_cast<const int32_t*>(cnt + k));
    s_all += c;
    if (k < b) s_before += c;
  }
  *before = block_sum<T>(s_before);
  *all = block_sum<T>(s_all);
}

__device__ __forceinline__ bool dominated(const ExploreArgs& A, int x, int pc, float c) {
  const uint32_t* mb = A.mbest + (size_t)x * A.kstride;
  for (int k = 0; k <= pc; ++k)
    if (__uint_as_float(ldu(mb + k)) < c) return true;
  return false;
}

__device__ __forceinline__ int32_t eff_bucket(const ExploreArgs& A, float c, int32_t t) {
  return max(bucket_of(c, A.lr), t + 1);
}

struct Cand {
  int32_t x, parent, edge, pc;
  float cost;
};

// Candidate c of the current group (g plans, offsets goff).
__device__ __forceinline__ Cand cand_at(const ExploreArgs& A, int64_t c, int32_t g) {
  int lo = 0, hi = g;
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (ld64(A.goff + mid) <= c) lo = mid; else hi = mid;
  }
  Cand q;
  const int32_t p = ld32(A.group + lo);
  const int32_t v = ld32(A.head + p);
  const int32_t e = A.row_ptr[v] + (int32_t)(c - ld64(A.goff + lo));
  q.x = A.col[e];
  q.parent = p;
  q.edge = e;
  q.cost = __fadd_rn(ldf(A.cost + p), A.ecost[e]);
  int pc = 0;
  const uint32_t* pm = A.mask + (size_t)p * A.w;
  const uint32_t* em = A.emask + (size_t)e * A.w;
  for (int j = 0; j < A.w; ++j) pc += __popc(ldu(pm + j) | em[j]);
  q.pc = pc;
  return q;
}

// ---------------------------------------------------------------- phases
__device__ void phase_expand(const ExploreArgs& A, int b, int nb) {
  ExploreCtl* ctl = A.ctl;
  const int64_t C = ld64(&ctl->group_cands);
  const int32_t g = ld32(&ctl->group_size);
  const int32_t i = ld32(&ctl->iter);
  if (b == 0 && threadIdx.x == 0) {
    ctl->n_plans = ld64(&ctl->n_plans) + ld32(&ctl->survivors);
    ctl->survivors = 0;
    ctl->n_candidates = ld64(&ctl->n_candidates) + C;
    ctl->n_groups = ld32(&ctl->n_groups) + 1;
  }
  for (int64_t s = (int64_t)b * kT + threadIdx.x; s < g; s += (int64_t)nb * kT) A.eexp[ld32(A.group + s)] = i;
  int64_t c0, c1;
  chunk(C, b, nb, &c0, &c1);
  int64_t kept = 0;
  for (int64_t c = c0 + threadIdx.x; c < c1; c += kT) {
    Cand q = cand_at(A, c, g);
    if (q.pc < A.kmax) {
      atomicMin(A.mbest + (size_t)q.x * A.kstride + q.pc, __float_as_uint(q.cost));
      ++kept;
    }
  }
  kept = block_sum<int64_t>(kept);
  if (threadIdx.x == 0 && kept) atomicAdd(reinterpret_cast<unsigned long long*>(&ctl->n_kept), (unsigned long long)kept);
}

__device__ void phase_count(const ExploreArgs& A, int b, int nb) {
  const int64_t C = ld64(&A.ctl->group_cands);
  const int32_t g = ld32(&A.ctl->group_size);
  int64_t c0, c1;
  chunk(C, b, nb, &c0, &c1);
  int32_t cnt = 0;
  for (int64_t c = c0 + threadIdx.x; c < c1; c += kT) {
    Cand q = cand_at(A, c, g);
    if (q.pc < A.kmax && !dominated(A, q.x, q.pc, q.cost)) ++cnt;
  }
  cnt = block_sum<int32_t>(cnt);
  if (threadIdx.x == 0) A.bcnt[b] = cnt;
}

__device__ void phase_write(const ExploreArgs& A, int b, int nb) {
  ExploreCtl* ctl = A.ctl;
  const int64_t C = ld64(&ctl->group_cands);
  const int32_t g = ld32(&ctl->group_size);
  const int32_t i = ld32(&ctl->iter);
  const int32_t parity = ld32(&ctl->it_count) & 1;
  const int64_t base = ld64(&ctl->n_plans);
  int32_t before, total;
  block_prefix_of<int32_t>(A.bcnt, b, nb, &before, &total);
  if (base + total > A.cap) {
    if (b == 0 && threadIdx.x == 0) atomicExch(&ctl->status, (int)PUMP_ERR_CAPACITY);
    return;
  }
  int64_t c0, c1;
  chunk(C, b, nb, &c0, &c1);
  int32_t bmin = kNoBucket;
  int64_t run = base + before;
  for (int64_t t0 = c0; t0 < c1; t0 += kT) {
    const int64_t c = t0 + threadIdx.x;
    bool keep = false;
    Cand q;
    if (c < c1) {
      q = cand_at(A, c, g);
      keep = q.pc < A.kmax && !dominated(A, q.x, q.pc, q.cost);
    }
    int32_t tile_total;
    const int32_t rank = block_scan<int32_t>(keep ? 1 : 0, &tile_total);
    if (keep) {
      const int64_t id = run + rank;
      A.head[id] = q.x;
      A.parent[id] = q.parent;
      A.pedge[id] = q.edge;
      A.cost[id] = q.cost;
      A.popc[id] = q.pc;
      A.tcre[id] = i;
      A.eexp[id] = -1;
      const uint32_t* pm = A.mask + (size_t)q.parent * A.w;
      const uint32_t* em = A.emask + (size_t)q.edge * A.w;
      uint32_t* om = A.mask + (size_t)id * A.w;
      for (int j = 0; j < A.w; ++j) om[j] = ldu(pm + j) | em[j];
      bmin = min(bmin, eff_bucket(A, q.cost, i));
      if (A.is_goal[q.x]) {
        int slot = atomicAdd(&ctl->n_goal_all, 1);
        A.goal_all[slot] = (int32_t)id;
      }
    }
    run += tile_total;
  }
  // older open plans
  for (int64_t p = (int64_t)b * kT + threadIdx.x; p < base; p += (int64_t)nb * kT) {
    if (ld32(A.eexp + p) != -1) continue;
    const float c = ldf(A.cost + p);
    const int32_t pc = ld32(A.popc + p);
    if (dominated(A, ld32(A.head + p), pc, c)) continue;
    bmin = min(bmin, eff_bucket(A, c, ld32(A.tcre + p)));
  }
  bmin = block_min(bmin);
  if (threadIdx.x == 0 && bmin != kNoBucket) atomicMin(&ctl->next_bucket[parity], bmin);
  if (b == 0 && threadIdx.x == 0) ctl->survivors = total;
}

__device__ __forceinline__ bool selected(const ExploreArgs& A, int64_t p, int32_t nbk, int32_t* deg, bool* goal_stop) {
  if (ld32(A.eexp + p) != -1) return false;
  const float c = ldf(A.cost + p);
  const int32_t pc = ld32(A.popc + p);
  const int32_t x = ld32(A.head + p);
  if (eff_bucket(A, c, ld32(A.tcre + p)) != nbk) return false;
  if (dominated(A, x, pc, c)) return false;
  *deg = A.row_ptr[x + 1] - A.row_ptr[x];
  *goal_stop = A.is_goal[x] && pc < A.kmin;
  return true;
}

__device__ void phase_select_count(const ExploreArgs& A, int b, int nb) {
  ExploreCtl* ctl = A.ctl;
  const int32_t parity = ld32(&ctl->it_count) & 1;
  const int32_t nbk = ld32(&ctl->next_bucket[parity]);
  const int64_t n_all = ld64(&ctl->n_plans) + ld32(&ctl->survivors);
  int32_t cnt = 0;
  int64_t dsum = 0;
  int32_t stop = 0;
  if (nbk != kNoBucket) {
    int64_t a0, a1;
    chunk(n_all, b, nb, &a0, &a1);
    for (int64_t p = a0 + threadIdx.x; p < a1; p += kT) {
      int32_t d;
      bool gs;
      if (selected(A, p, nbk, &d, &gs)) {
        ++cnt;
        dsum += d;
        stop |= gs ? 1 : 0;
      }
    }
  }
  cnt = block_sum<int32_t>(cnt);
  dsum = block_sum<int64_t>(dsum);
  stop = block_sum<int32_t>(stop);
  if (threadIdx.x == 0) {
    A.bcnt[b] = cnt;
    A.bdeg[b] = dsum;
    if (stop) atomicOr(&ctl->stop_next, 1);
  }
}

__device__ void phase_select_write(const ExploreArgs& A, int b, int nb) {
  ExploreCtl* ctl = A.ctl;
  const int32_t parity = ld32(&ctl->it_count) & 1;
  const int32_t nbk = ld32(&ctl->next_bucket[parity]);
  const int64_t n_all = ld64(&ctl->n_plans) + ld32(&ctl->survivors);
  int32_t before, total;
  int64_t dbefore, dtotal;
  block_prefix_of<int32_t>(A.bcnt, b, nb, &before, &total);
  block_prefix_of<int64_t>(A.bdeg, b, nb, &dbefore, &dtotal);
  if (nbk != kNoBucket) {
    int64_t a0, a1;
    chunk(n_all, b, nb, &a0, &a1);
    int32_t run = before;
    int64_t drun = dbefore;
    for (int64_t t0 = a0; t0 < a1; t0 += kT) {
      const int64_t p = t0 + threadIdx.x;
      int32_t d = 0;
      bool gs = false;
      const bool sel = p < a1 && selected(A, p, nbk, &d, &gs);
      int32_t tt;
      int64_t dt;
      const int32_t r = block_scan<int32_t>(sel ? 1 : 0, &tt);
      const int64_t dr = block_scan<int64_t>(sel ? (int64_t)d : 0, &dt);
      if (sel) {
        A.group[run + r] = (int32_t)p;
        A.goff[run + r] = drun + dr;
      }
      run += tt;
      drun += dt;
    }
  }
  if (b == 0 && threadIdx.x == 0) {
    const int32_t it = ld32(&ctl->iter);
    ctl->group_size = total;
    ctl->group_cands = dtotal;
    A.goff[total] = dtotal;
    ctl->iter = nbk != kNoBucket ? nbk : it + 1;
    ctl->stop = A.early_stop ? ld32(&ctl->stop_next) : 0;
    ctl->stop_next = 0;
    ctl->next_bucket[parity ^ 1] = kNoBucket;
    ctl->it_count = ld32(&ctl->it_count) + 1;
  }
}

// Bounded grid barrier (all blocks co-resident: cooperative launch).
__device__ bool grid_sync(ExploreCtl* ctl, int nb, long long limit) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile uint32_t* genp = &ctl->bar_gen;
    const uint32_t gen = *genp;
    __threadfence();
    const uint32_t arrived = atomicAdd(&ctl->bar_count, 1u);
    ok = 1;
    if (arrived == (uint32_t)nb - 1) {
      atomicExch(&ctl->bar_count, 0u);
      __threadfence();
      atomicAdd(&ctl->bar_gen, 1u);
    } else {
      long long spins = 0;
      while (*genp == gen) {
        if (++spins > limit) {
          atomicExch(&ctl->status, (int)PUMP_ERR_TIMEOUT);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

__global__ void __launch_bounds__(kT) k_explore_persistent(ExploreArgs A) {
  const int b = blockIdx.x, nb = gridDim.x;
  ExploreCtl* ctl = A.ctl;
  for (;;) {
    const int32_t g = ld32(&ctl->group_size);
    const int32_t st = ld32(&ctl->status);
    const int32_t stop = ld32(&ctl->stop);
    const int32_t it = ld32(&ctl->iter);
    if (st || stop || g == 0) break;
    if (it >= A.max_iter) {
      if (b == 0 && threadIdx.x == 0) atomicExch(&ctl->status, (int)PUMP_ERR_TIMEOUT);
      break;
    }
    phase_expand(A, b, nb);
    if (!grid_sync(ctl, nb, A.spin_limit)) return;
    phase_count(A, b, nb);
    if (!grid_sync(ctl, nb, A.spin_limit)) return;
    phase_write(A, b, nb);
    if (!grid_sync(ctl, nb, A.spin_limit)) return;
    if (ld32(&ctl->status)) break;
    phase_select_count(A, b, nb);
    if (!grid_sync(ctl, nb, A.spin_limit)) return;
    phase_select_write(A, b, nb);
    if (!grid_sync(ctl, nb, A.spin_limit)) return;
  }
}

__global__ void __launch_bounds__(kT) k_phase(ExploreArgs A, int which) {
  switch (which) {
    case 1: phase_expand(A, blockIdx.x, gridDim.x); break;
    case 2: phase_count(A, blockIdx.x, gridDim.x); break;
    case 3: phase_write(A, blockIdx.x, gridDim.x); break;
    case 4: phase_select_count(A, blockIdx.x, gridDim.x); break;
    case 5: phase_select_write(A, blockIdx.x, gridDim.x); break;
  }
}

__global__ void k_fill_u32(uint32_t* p, int64_t n, uint32_t v) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) p[k] = v;
}

__global__ void k_explore_init(ExploreArgs A, int32_t start) {
  ExploreCtl* c = A.ctl;
  A.head[0] = start;
  A.parent[0] = -1;
  A.pedge[0] = -1;
  A.cost[0] = 0.f;
  A.popc[0] = 0;
  A.tcre[0] = -1;
  A.eexp[0] = -1;
  for (int j = 0; j < A.w; ++j) A.mask[j] = 0u;
  A.mbest[(size_t)start * A.kstride] = 0u;  // float 0
  A.group[0] = 0;
  const int64_t d0 = A.row_ptr[start + 1] - A.row_ptr[start];
  A.goff[0] = 0;
  A.goff[1] = d0;
  c->n_plans = 1;
  c->n_candidates = 0;
  c->n_kept = 0;
  c->group_cands = d0;
  c->group_size = 1;
  c->iter = 0;
  c->it_count = 0;
  c->next_bucket[0] = kNoBucket;
  c->next_bucket[1] = kNoBucket;
  c->stop = (A.early_stop && A.is_goal[start] && 0 < A.kmin) ? 1 : 0;
  c->stop_next = 0;
  c->status = 0;
  c->n_groups = 0;
  c->survivors = 0;
  c->n_goal_all = 0;
  c->n_goal = 0;
  c->bar_count = 0;
  c->bar_gen = 0;
  if (A.is_goal[start]) {
    A.goal_all[0] = 0;
    c->n_goal_all = 1;
  }
}

__global__ void k_explore_commit(ExploreCtl* c) {
  c->n_plans += c->survivors;
  c->survivors = 0;
}

}  // namespace

// Blocks of the persistent Explore kernel (PUMP_EXPLORE_BLOCKS overrides; default one per SM).
int explore_blocks() {
  static int v = -1;
  if (v < 0) {
    const char* e = getenv("PUMP_EXPLORE_BLOCKS");
    v = e ? atoi(e) : 0;
  }
  return v;
}

int run_explore_kernels(pump_graph* g, const ExploreArgs& A, bool stepwise, cudaStream_t s) {
  const int64_t mb = (int64_t)g->n * A.kstride;
  k_fill_u32<<<256, 256, 0, s>>>(A.mbest, mb, 0x7f800000u);
  note_launch();
  k_explore_init<<<1, 1, 0, s>>>(A, g->start);
  note_launch();
  PUMP_CUDA_TRY(cudaGetLastError());
  int dev = 0;
  PUMP_CUDA_TRY(cudaGetDevice(&dev));
  int coop = 0;
  PUMP_CUDA_TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  const int sms = num_sms();
  if (!stepwise && coop) {
    int per_sm = 0;
    PUMP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_explore_persistent, kT, 0));
    const int max_nb = sms * (per_sm < 1 ? 1 : per_sm);
    int nb = explore_blocks();
    if (nb <= 0) nb = sms;
    if (nb > max_nb) nb = max_nb;
    ExploreArgs a = A;
    void* args[] = {&a};
    PUMP_CUDA_TRY(cudaLaunchCooperativeKernel((void*)k_explore_persistent, dim3(nb), dim3(kT), args, 0, s));
    note_launch();
    k_explore_commit<<<1, 1, 0, s>>>(A.ctl);
    note_launch();
    PUMP_CUDA_TRY(cudaGetLastError());
    return PUMP_OK;
  }
  // stepwise: phases as separate launches, host reads the control block
  const int nb = sms;
  ExploreCtl h;
  for (;;) {
    PUMP_CUDA_TRY(cudaMemcpyAsync(&h, A.ctl, sizeof(h), cudaMemcpyDeviceToHost, s));
    PUMP_CUDA_TRY(cudaStreamSynchronize(s));
    if (h.status || h.stop || h.group_size == 0) break;
    if (h.iter >= A.max_iter) {
      int st = PUMP_ERR_TIMEOUT;
      PUMP_CUDA_TRY(cudaMemcpyAsync(&A.ctl->status, &st, sizeof(int), cudaMemcpyHostToDevice, s));
      break;
    }
    for (int ph = 1; ph <= 5; ++ph) {
      k_phase<<<nb, kT, 0, s>>>(A, ph);
      note_launch();
      if (ph == 3) {
        // a full arena stops the run before the group is formed
        PUMP_CUDA_TRY(cudaMemcpyAsync(&h, A.ctl, sizeof(h), cudaMemcpyDeviceToHost, s));
        PUMP_CUDA_TRY(cudaStreamSynchronize(s));
        if (h.status) break;
      }
    }
    PUMP_CUDA_TRY(cudaGetLastError());
    if (h.status) break;
  }
  k_explore_commit<<<1, 1, 0, s>>>(A.ctl);
  note_launch();
  PUMP_CUDA_TRY(cudaGetLastError());
  return PUMP_OK;
}

}  // namespace pump
