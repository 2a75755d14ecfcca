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
// Schedule.  One iteration is four phases separated by grid barriers:
//   P1 expand: candidates of the group (plans by id, then out-edges; a warp per
//      group plan, lanes over its edges), CP cutoff, atomicMin into mbest;
//      stamp e = i on group plans.
//   P2 survivors per block (candidate ranges are contiguous per block) and the
//      least group index over open undominated plans, new and older.
//   P3 survivors written at arena ids from the block counts (stable order);
//      next-group members counted per block, older plans and survivors apart,
//      with out-degree sums; stop flag on a goal plan with popc < K_min.
//   P4 the group written in ascending id with its candidate offsets.
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

// Sums of K int64 values over the block in one pass (one shared-memory round).
template <int K>
__device__ void block_sums(int64_t (&v)[K]) {
  __shared__ int64_t wsum[K][kWarpsT];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < K; ++q) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
    if (lane == 0) wsum[q][warp] = v[q];
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < K; ++q) {
    int64_t t = 0;
#pragma unroll
    for (int w = 0; w < kWarpsT; ++w) t += wsum[q][w];
    v[q] = t;
  }
  __syncthreads();
}

// Packed (count, degree sum): count in bits 40.., sum in bits 0..39.
constexpr int kPackShift = 40;
__device__ __forceinline__ int64_t pack_cd(int64_t c, int64_t d) { return (c << kPackShift) | d; }
__device__ __forceinline__ int32_t pack_c(int64_t x) { return (int32_t)(x >> kPackShift); }
__device__ __forceinline__ int64_t pack_d(int64_t x) { return x & ((int64_t(1) << kPackShift) - 1); }

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
  const int4 gi = __ldcg(A.ginfo + lo);
  const int32_t p = gi.x;
  const int32_t e = gi.z + (int32_t)(c - ld64(A.goff + lo));
  q.x = A.col[e];
  q.parent = p;
  q.edge = e;
  q.cost = __fadd_rn(__int_as_float(gi.w), A.ecost[e]);
  int pc = 0;
  const uint32_t* pm = A.mask + (size_t)p * A.w;
  const uint32_t* em = A.emask + (size_t)e * A.w;
  for (int j = 0; j < A.w; ++j) pc += __popc(ldu(pm + j) | em[j]);
  q.pc = pc;
  return q;
}

// ---------------------------------------------------------------- phases
//
// Shared memory of the persistent kernel: a block keeps the candidates of its chunk (and
// bucket flags of its chunk of older plans) from P1 to P4, so each is computed once.  The
// stepwise driver (separate launches) and chunks that do not fit recompute instead; both
// paths produce the same values.
constexpr int kCandCap = 1536;
constexpr int kOldCap = 2048;
constexpr int kMaxBlocks = 1024;

struct ExploreSmem {
  int32_t cx[kCandCap];     // candidate target node
  int32_t cpar[kCandCap];   // parent plan
  int32_t cedge[kCandCap];  // edge; after P3 the survivor's id
  float ccost[kCandCap];
  int32_t ceff[kCandCap];   // group of a kept candidate (-1 = not kept), from P2
  int16_t cpc[kCandCap];
  int32_t oeff[kOldCap];    // group of an open undominated older plan (-1 otherwise), from P2
  int32_t slot0;
};

__device__ __forceinline__ int32_t deg_of(const ExploreArgs& A, int32_t x) { return A.row_ptr[x + 1] - A.row_ptr[x]; }

// Largest slot s < g with goff[s] <= c.
__device__ __forceinline__ int32_t slot_of(const ExploreArgs& A, int64_t c, int32_t g) {
  int lo = 0, hi = g;
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (ld64(A.goff + mid) <= c) lo = mid; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ int32_t old_eff(const ExploreArgs& A, int64_t p) {
  if (ld32(A.eexp + p) != -1) return -1;
  const float c = ldf(A.cost + p);
  if (dominated(A, ld32(A.head + p), ld32(A.popc + p), c)) return -1;
  return eff_bucket(A, c, ld32(A.tcre + p));
}

// P1: candidates of the group, CP cutoff, dominance table; group plans stamped expanded.
template <bool kC>
__device__ void phase_expand(const ExploreArgs& A, int b, int nb, ExploreSmem* sm, int k) {
  ExploreCtl* ctl = A.ctl;
  const IterState* cur = &ctl->st[k & 1];
  const int64_t C = ld64(&cur->group_cands);
  const int32_t g = ld32(&cur->group_size);
  const int32_t i = ld32(&cur->iter);
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
  if (kC && c1 - c0 <= kCandCap) {
    if (c0 < c1) {
      if (threadIdx.x == 0) sm->slot0 = slot_of(A, c0, g);
      __syncthreads();
      const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
      for (int32_t s = sm->slot0 + warp; s < g; s += kWarpsT) {
        const int64_t lo_s = ld64(A.goff + s);
        if (lo_s >= c1) break;
        const int64_t hi_s = ld64(A.goff + s + 1);
        const int64_t lo = max(lo_s, c0), hi = min(hi_s, c1);
        if (lo >= hi) continue;
        const int4 gi = __ldcg(A.ginfo + s);
        const int32_t p = gi.x;
        const int32_t rp = gi.z;
        const float pcost = __int_as_float(gi.w);
        const uint32_t* pm = A.mask + (size_t)p * A.w;
        for (int64_t c = lo + lane; c < hi; c += 32) {
          const int32_t e = rp + (int32_t)(c - lo_s);
          const int32_t x = A.col[e];
          const float cost = __fadd_rn(pcost, A.ecost[e]);
          const uint32_t* em = A.emask + (size_t)e * A.w;
          int pc = 0;
          for (int j = 0; j < A.w; ++j) pc += __popc(ldu(pm + j) | em[j]);
          const int jl = (int)(c - c0);
          sm->cx[jl] = x;
          sm->cpar[jl] = p;
          sm->cedge[jl] = e;
          sm->ccost[jl] = cost;
          sm->cpc[jl] = (int16_t)pc;
          if (pc < A.kmax) {
            atomicMin(A.mbest + (size_t)x * A.kstride + pc, __float_as_uint(cost));
            ++kept;
          }
        }
      }
    }
  } else {
    for (int64_t c = c0 + threadIdx.x; c < c1; c += kT) {
      Cand q = cand_at(A, c, g);
      if (q.pc < A.kmax) {
        atomicMin(A.mbest + (size_t)q.x * A.kstride + q.pc, __float_as_uint(q.cost));
        ++kept;
      }
    }
  }
  kept = block_sum<int64_t>(kept);
  if (threadIdx.x == 0 && kept) atomicAdd(reinterpret_cast<unsigned long long*>(&ctl->n_kept), (unsigned long long)kept);
}

// Candidate jl of the block's chunk (from shared memory or recomputed).
template <bool kC>
__device__ __forceinline__ Cand local_cand(const ExploreArgs& A, const ExploreSmem* sm, bool fits, int64_t c0, int jl,
                                           int32_t g) {
  if (kC && fits) {
    Cand q;
    q.x = sm->cx[jl];
    q.parent = sm->cpar[jl];
    q.edge = sm->cedge[jl];
    q.cost = sm->ccost[jl];
    q.pc = sm->cpc[jl];
    return q;
  }
  return cand_at(A, c0 + jl, g);
}

// P2: survivors per block (kept and undominated after all of the group's candidates), and the
// least group index among open undominated plans, new and older.
template <bool kC>
__device__ void phase_count(const ExploreArgs& A, int b, int nb, ExploreSmem* sm, int k) {
  ExploreCtl* ctl = A.ctl;
  const IterState* cur = &ctl->st[k & 1];
  const int64_t C = ld64(&cur->group_cands);
  const int32_t g = ld32(&cur->group_size);
  const int32_t i = ld32(&cur->iter);
  const int32_t parity = k & 1;
  const int64_t base = ld64(&ctl->n_plans);
  int64_t c0, c1;
  chunk(C, b, nb, &c0, &c1);
  const bool fits = c1 - c0 <= kCandCap;
  int32_t cnt = 0, bmin = kNoBucket;
  for (int jl = threadIdx.x; jl < (int)(c1 - c0); jl += kT) {
    const Cand q = local_cand<kC>(A, sm, fits, c0, jl, g);
    const bool keep = q.pc < A.kmax && !dominated(A, q.x, q.pc, q.cost);
    const int32_t eff = keep ? eff_bucket(A, q.cost, i) : -1;
    if (kC && fits) sm->ceff[jl] = eff;
    if (keep) {
      ++cnt;
      bmin = min(bmin, eff);
    }
  }
  int64_t a0, a1;
  chunk(base, b, nb, &a0, &a1);
  const bool ofits = a1 - a0 <= kOldCap;
  for (int64_t p = a0 + threadIdx.x; p < a1; p += kT) {
    const int32_t eff = old_eff(A, p);
    if (kC && ofits) sm->oeff[p - a0] = eff;
    if (eff >= 0) bmin = min(bmin, eff);
  }
  // count by a block sum; group index by warp minima and one atomic per warp
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) bmin = min(bmin, __shfl_xor_sync(0xffffffffu, bmin, o));
  if ((threadIdx.x & 31) == 0 && bmin != kNoBucket) atomicMin(&ctl->next_bucket[parity], bmin);
  cnt = block_sum<int32_t>(cnt);
  if (threadIdx.x == 0) A.bcnt[b] = cnt;
}

// P3: survivors written at arena ids in candidate order; members of the next group counted
// (older plans first, then this iteration's survivors) with their out-degree sums.
template <bool kC>
__device__ void phase_write(const ExploreArgs& A, int b, int nb, ExploreSmem* sm, int k) {
  ExploreCtl* ctl = A.ctl;
  const IterState* cur = &ctl->st[k & 1];
  const int64_t C = ld64(&cur->group_cands);
  const int32_t g = ld32(&cur->group_size);
  const int32_t i = ld32(&cur->iter);
  const int32_t nbk = ld32(&ctl->next_bucket[k & 1]);
  const int64_t base = ld64(&ctl->n_plans);
  int32_t before, total;
  block_prefix_of<int32_t>(A.bcnt, b, nb, &before, &total);
  if (base + total > A.cap) {
    if (b == 0 && threadIdx.x == 0) atomicExch(&ctl->status, (int)PUMP_ERR_CAPACITY);
    return;
  }
  int64_t c0, c1;
  chunk(C, b, nb, &c0, &c1);
  const bool fits = c1 - c0 <= kCandCap;
  int32_t cnt_n = 0, stop = 0;
  int64_t deg_n = 0;
  int64_t run = base + before;
  for (int t0 = 0; t0 < (int)(c1 - c0); t0 += kT) {
    const int jl = t0 + threadIdx.x;
    bool keep = false;
    int32_t eff = -1;
    Cand q;
    if (jl < (int)(c1 - c0)) {
      q = local_cand<kC>(A, sm, fits, c0, jl, g);
      if (kC && fits) {
        eff = sm->ceff[jl];
        keep = eff >= 0;
      } else {
        keep = q.pc < A.kmax && !dominated(A, q.x, q.pc, q.cost);
        eff = keep ? eff_bucket(A, q.cost, i) : -1;
      }
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
      if (A.is_goal[q.x]) {
        const int slot = atomicAdd(&ctl->n_goal_all, 1);
        A.goal_all[slot] = (int32_t)id;
      }
      if (kC && fits) sm->cedge[jl] = (int32_t)id;
      if (eff == nbk) {
        ++cnt_n;
        deg_n += deg_of(A, q.x);
        if (A.is_goal[q.x] && q.pc < A.kmin) stop = 1;
      }
    }
    run += tile_total;
  }
  int32_t cnt_o = 0;
  int64_t deg_o = 0;
  int64_t a0, a1;
  chunk(base, b, nb, &a0, &a1);
  const bool ofits = a1 - a0 <= kOldCap;
  if (nbk != kNoBucket) {
    for (int64_t p = a0 + threadIdx.x; p < a1; p += kT) {
      const int32_t eff = (kC && ofits) ? sm->oeff[p - a0] : old_eff(A, p);
      if (eff != nbk) continue;
      const int32_t x = ld32(A.head + p);
      ++cnt_o;
      deg_o += deg_of(A, x);
      if (A.is_goal[x] && ld32(A.popc + p) < A.kmin) stop = 1;
    }
  }
  int64_t red[3] = {pack_cd(cnt_o, deg_o), pack_cd(cnt_n, deg_n), stop};
  block_sums<3>(red);
  if (threadIdx.x == 0) {
    A.bdeg[b] = red[0];
    A.bdeg[kMaxBlocks + b] = red[1];
    if (red[2]) atomicOr(&ctl->stop_next, 1);
  }
  if (b == 0 && threadIdx.x == 0) ctl->survivors = total;
}

// P4: the next group in ascending id (older plans, then new survivors) and its candidate
// offsets; block 0 advances the control block.
template <bool kC>
__device__ void phase_select_write(const ExploreArgs& A, int b, int nb, ExploreSmem* sm, int k) {
  ExploreCtl* ctl = A.ctl;
  const IterState* cur = &ctl->st[k & 1];
  const int64_t C = ld64(&cur->group_cands);
  const int32_t i = ld32(&cur->iter);
  const int32_t nbk = ld32(&ctl->next_bucket[k & 1]);
  const int64_t base = ld64(&ctl->n_plans);
  // prefixes over blocks of: old-plan (count, degree), survivor (count, degree), survivor count
  int64_t red[6] = {0, 0, 0, 0, 0, 0};
  for (int q = threadIdx.x; q < nb; q += blockDim.x) {
    const int64_t po = ld64(A.bdeg + q), pn = ld64(A.bdeg + kMaxBlocks + q), sc = ld32(A.bcnt + q);
    red[1] += po;
    red[3] += pn;
    red[5] += sc;
    if (q < b) {
      red[0] += po;
      red[2] += pn;
      red[4] += sc;
    }
  }
  block_sums<6>(red);
  const int32_t before_o = pack_c(red[0]), total_o = pack_c(red[1]);
  const int64_t dbefore_o = pack_d(red[0]), dtotal_o = pack_d(red[1]);
  const int32_t before_n = pack_c(red[2]), total_n = pack_c(red[3]);
  const int64_t dbefore_n = pack_d(red[2]), dtotal_n = pack_d(red[3]);
  const int32_t before_s = (int32_t)red[4];
  if (nbk != kNoBucket) {
    // older plans
    int64_t a0, a1;
    chunk(base, b, nb, &a0, &a1);
    const bool ofits = a1 - a0 <= kOldCap;
    int32_t run = before_o;
    int64_t drun = dbefore_o;
    for (int64_t t0 = a0; t0 < a1; t0 += kT) {
      const int64_t p = t0 + threadIdx.x;
      bool sel = false;
      int32_t d = 0;
      int4 gi = make_int4(0, 0, 0, 0);
      if (p < a1) {
        const int32_t eff = (kC && ofits) ? sm->oeff[p - a0] : old_eff(A, p);
        sel = eff == nbk;
        if (sel) {
          const int32_t x = ld32(A.head + p);
          const int32_t r0 = A.row_ptr[x];
          d = A.row_ptr[x + 1] - r0;
          gi = make_int4((int32_t)p, x, r0, __float_as_int(ldf(A.cost + p)));
        }
      }
      int64_t tpk;
      const int64_t rpk = block_scan<int64_t>(sel ? pack_cd(1, d) : 0, &tpk);
      if (sel) {
        A.group[run + pack_c(rpk)] = (int32_t)p;
        A.ginfo[run + pack_c(rpk)] = gi;
        A.goff[run + pack_c(rpk)] = drun + pack_d(rpk);
      }
      run += pack_c(tpk);
      drun += pack_d(tpk);
    }
    // this iteration's survivors: this block's are arena ids [base + before_s, + its count); the
    // group list being written here must not be read, so they are taken from shared memory or
    // from the arena records P3 wrote
    int64_t c0, c1;
    chunk(C, b, nb, &c0, &c1);
    const bool fits = c1 - c0 <= kCandCap;
    run = total_o + before_n;
    drun = dtotal_o + dbefore_n;
    if (kC && fits) {
      for (int t0 = 0; t0 < (int)(c1 - c0); t0 += kT) {
        const int jl = t0 + threadIdx.x;
        bool sel = false;
        int32_t d = 0, id = -1;
        int4 gi = make_int4(0, 0, 0, 0);
        if (jl < (int)(c1 - c0)) {
          const int32_t eff = sm->ceff[jl];
          sel = eff >= 0 && eff == nbk;
          if (sel) {
            id = sm->cedge[jl];
            const int32_t x = sm->cx[jl];
            const int32_t r0 = A.row_ptr[x];
            d = A.row_ptr[x + 1] - r0;
            gi = make_int4(id, x, r0, __float_as_int(sm->ccost[jl]));
          }
        }
        int64_t tpk;
        const int64_t rpk = block_scan<int64_t>(sel ? pack_cd(1, d) : 0, &tpk);
        if (sel) {
          A.group[run + pack_c(rpk)] = id;
          A.ginfo[run + pack_c(rpk)] = gi;
          A.goff[run + pack_c(rpk)] = drun + pack_d(rpk);
        }
        run += pack_c(tpk);
        drun += pack_d(tpk);
      }
    } else {
      const int32_t mine = ld32(A.bcnt + b);
      const int64_t id0 = base + before_s;
      for (int t0 = 0; t0 < mine; t0 += kT) {
        const int k = t0 + threadIdx.x;
        bool sel = false;
        int32_t d = 0;
        int4 gi = make_int4(0, 0, 0, 0);
        if (k < mine) {
          const float c = ldf(A.cost + id0 + k);
          sel = eff_bucket(A, c, i) == nbk;
          if (sel) {
            const int32_t x = ld32(A.head + id0 + k);
            const int32_t r0 = A.row_ptr[x];
            d = A.row_ptr[x + 1] - r0;
            gi = make_int4((int32_t)(id0 + k), x, r0, __float_as_int(c));
          }
        }
        int64_t tpk;
        const int64_t rpk = block_scan<int64_t>(sel ? pack_cd(1, d) : 0, &tpk);
        if (sel) {
          A.group[run + pack_c(rpk)] = (int32_t)(id0 + k);
          A.ginfo[run + pack_c(rpk)] = gi;
          A.goff[run + pack_c(rpk)] = drun + pack_d(rpk);
        }
        run += pack_c(tpk);
        drun += pack_d(tpk);
      }
    }
  }
  if (b == 0 && threadIdx.x == 0) {
    IterState* nxt = &ctl->st[(k + 1) & 1];
    const int32_t gsize = nbk != kNoBucket ? total_o + total_n : 0;
    const int64_t gc = nbk != kNoBucket ? dtotal_o + dtotal_n : 0;
    nxt->group_size = gsize;
    nxt->group_cands = gc;
    A.goff[gsize] = gc;
    nxt->iter = nbk != kNoBucket ? nbk : i + 1;
    nxt->stop = A.early_stop ? ld32(&ctl->stop_next) : 0;
    ctl->stop_next = 0;
    ctl->next_bucket[(k + 1) & 1] = kNoBucket;
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
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ExploreSmem* sm = reinterpret_cast<ExploreSmem*>(smem_raw);
  const int b = blockIdx.x, nb = gridDim.x;
  ExploreCtl* ctl = A.ctl;
  int k = 0;
  for (;; ++k) {
    const IterState* cur = &ctl->st[k & 1];
    const int32_t g = ld32(&cur->group_size);
    const int32_t stop = ld32(&cur->stop);
    const int32_t it = ld32(&cur->iter);
    const int32_t st = ld32(&ctl->status);
    if (st || stop || g == 0) break;
    if (it >= A.max_iter) {
      if (b == 0 && threadIdx.x == 0) atomicExch(&ctl->status, (int)PUMP_ERR_TIMEOUT);
      break;
    }
    phase_expand<true>(A, b, nb, sm, k);
    if (!grid_sync(ctl, nb, A.spin_limit)) return;
    phase_count<true>(A, b, nb, sm, k);
    if (!grid_sync(ctl, nb, A.spin_limit)) return;
    phase_write<true>(A, b, nb, sm, k);
    if (!grid_sync(ctl, nb, A.spin_limit)) return;
    if (ld32(&ctl->status)) break;
    phase_select_write<true>(A, b, nb, sm, k);
    if (!grid_sync(ctl, nb, A.spin_limit)) return;
  }
  if (b == 0 && threadIdx.x == 0) ctl->k_exit = k;
}

__global__ void __launch_bounds__(kT) k_phase(ExploreArgs A, int which, int k) {
  switch (which) {
    case 1: phase_expand<false>(A, blockIdx.x, gridDim.x, nullptr, k); break;
    case 2: phase_count<false>(A, blockIdx.x, gridDim.x, nullptr, k); break;
    case 3: phase_write<false>(A, blockIdx.x, gridDim.x, nullptr, k); break;
    case 4: phase_select_write<false>(A, blockIdx.x, gridDim.x, nullptr, k); break;
  }
}

__global__ void k_fill_u32(uint32_t* p, int64_t n, uint32_t v) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) p[k] = v;
}

__global__ void k_explore_init(ExploreArgs A, int32_t start) { explore_init_thread(A, start); }

// End of a run: commit the last survivors and record the final group index.  k < 0 takes the
// iteration count the persistent kernel stored.
__global__ void k_explore_commit(ExploreCtl* c, int k) {
  if (k < 0) k = c->k_exit;
  c->n_plans += c->survivors;
  c->survivors = 0;
  c->iter = c->st[k & 1].iter;
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

int plan_explore_cluster(const ExploreArgs& A, int* nr, bool* dsm);
int run_explore_cluster(pump_graph* g, const ExploreArgs& A, int nr, bool dsm, cudaStream_t s);
int run_explore_fused(pump_graph* g, const ExploreArgs& A, int nr, bool dsm, cudaStream_t s, bool* launched);

// Explore kernels for one run.  mode 0: the thread-block cluster kernel (explore_cluster.cu)
// where the device can co-schedule one, else the grid kernel; 1: the grid kernel; 2: the
// phases as separate launches.
int run_explore_kernels(pump_graph* g, const ExploreArgs& A, int mode, cudaStream_t s, bool masks_pending) {
  const bool stepwise = mode == 2;
  int cl_nr = 0;
  bool cl_dsm = false;
  if (mode == 0) {
    const int rc = plan_explore_cluster(A, &cl_nr, &cl_dsm);
    if (rc) return rc;
  }
  g->last_fused = false;
  if (masks_pending && !(cl_nr > 0 && cl_dsm)) {  // the fused form needs the on-chip cluster form
    const int rc = compute_edge_masks(g, s);
    if (rc) return rc;
    masks_pending = false;
  }
  if (!(cl_nr > 0 && cl_dsm)) {  // the cluster kernel keeps mbest on chip and fills it itself
    const int64_t mb = (int64_t)g->n * A.kstride;
    k_fill_u32<<<256, 256, 0, s>>>(A.mbest, mb, 0x7f800000u);
    note_launch();
  }
  if (cl_nr > 0 && masks_pending) {
    // the fused launch initialises the run and orders P_goal itself
    bool launched = false;
    int rc = run_explore_fused(g, A, cl_nr, cl_dsm, s, &launched);
    if (rc) return rc;
    if (launched) {
      g->last_fused = true;
      return PUMP_OK;
    }
    rc = compute_edge_masks(g, s);  // the device cannot run the fused form
    if (rc) return rc;
  }
  k_explore_init<<<1, 1, 0, s>>>(A, g->start);
  note_launch();
  PUMP_CUDA_TRY(cudaGetLastError());
  int dev = 0;
  PUMP_CUDA_TRY(cudaGetDevice(&dev));
  int coop = 0;
  PUMP_CUDA_TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  const int sms = num_sms();
  if (cl_nr > 0) {
    const int rc = run_explore_cluster(g, A, cl_nr, cl_dsm, s);
    if (rc) return rc;
    PUMP_CUDA_TRY(cudaGetLastError());
    return PUMP_OK;
  }
  if (!stepwise && coop) {
    const size_t smem = sizeof(ExploreSmem);
    PUMP_CUDA_TRY(cudaFuncSetAttribute(k_explore_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    PUMP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_explore_persistent, kT, smem));
    const int max_nb = sms * (per_sm < 1 ? 1 : per_sm);
    int nb = explore_blocks();
    if (nb <= 0) nb = sms;
    if (nb > max_nb) nb = max_nb;
    if (nb > kMaxBlocks) nb = kMaxBlocks;
    ExploreArgs a = A;
    void* args[] = {&a};
    PUMP_CUDA_TRY(cudaLaunchCooperativeKernel((void*)k_explore_persistent, dim3(nb), dim3(kT), args, smem, s));
    note_launch();
    k_explore_commit<<<1, 1, 0, s>>>(A.ctl, -1);
    note_launch();
    PUMP_CUDA_TRY(cudaGetLastError());
    return PUMP_OK;
  }
  // stepwise: phases as separate launches, host reads the control block
  const int nb = sms < kMaxBlocks ? sms : kMaxBlocks;
  ExploreCtl h;
  int k = 0;
  for (;; ++k) {
    PUMP_CUDA_TRY(cudaMemcpyAsync(&h, A.ctl, sizeof(h), cudaMemcpyDeviceToHost, s));
    PUMP_CUDA_TRY(cudaStreamSynchronize(s));
    const IterState& cur = h.st[k & 1];
    if (h.status || cur.stop || cur.group_size == 0) break;
    if (cur.iter >= A.max_iter) {
      int st = PUMP_ERR_TIMEOUT;
      PUMP_CUDA_TRY(cudaMemcpyAsync(&A.ctl->status, &st, sizeof(int), cudaMemcpyHostToDevice, s));
      break;
    }
    for (int ph = 1; ph <= 4; ++ph) {
      k_phase<<<nb, kT, 0, s>>>(A, ph, k);
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
  k_explore_commit<<<1, 1, 0, s>>>(A.ctl, k);
  note_launch();
  PUMP_CUDA_TRY(cudaGetLastError());
  return PUMP_OK;
}

}  // namespace pump
