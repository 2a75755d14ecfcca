// Explore (Algorithm 4) inside one thread-block cluster.
//
// Why a cluster.  The search is a chain of dependent groups, and one group is
// small (hundreds of plans, thousands of candidates), so its cost is latency:
// the barriers between the steps of an iteration and the dependent loads
// inside them.  A grid-wide barrier built on global-memory atomics costs
// microseconds; the hardware barrier of a thread-block cluster costs well
// under one, and distributed shared memory lets the CTAs hand each other
// counts and the next group's members without a round trip through L2.  One
// cluster of CL CTAs (16 where the device can co-schedule them, else 8 or 4)
// runs the whole search.
//
// State.  The plan arena, the group list (ginfo, goff) and the goal list are
// in global memory as for the grid kernel (explore.cu).  The table mbest[x][k]
// (least cost ever inserted at node x with popcount k, float bits) is
// partitioned over the CTAs' shared memory by node (x mod CL) when it fits,
// else it stays in global memory.  The argument that "dominated by a plan ever
// inserted at x" equals "dominated by a plan in P(x)" is in explore.cu.
//
// One iteration (group i) is three phases, each closed by a cluster barrier:
//   A expand.  CTA r takes candidates [r per, (r+1) per) of the group (members
//     in ascending id, out-edges in ascending target; per = ceil(C / CL)), a
//     warp per member: cost, mask OR, popcount, CP cutoff, atomicMin into
//     mbest.  Members are stamped expanded (e = i).  The members of the chunk
//     were placed in the CTA's shared memory by their writers (phase C).
//   B filter.  Each cached candidate is tested against mbest (strict cost,
//     non-strict popcount) and gets its group index max(bucket, i + 1).
//     Recent plans that may still be open are re-tested the same way.  The
//     CTA counts survivors; for each group index i+1 .. i+kWin, members from
//     older plans and from survivors with their out-degree sums; goal-stop
//     bits; the least group index; the least id of an older open plan.  It
//     copies these counts into every CTA's shared memory.
//   C write.  Every CTA derives from the same counts the next group index,
//     arena ids (survivors numbered in candidate order: CTA by CTA, then by
//     position) and next-group positions (older plans first, then survivors,
//     each in id order).  It writes its survivors to the arena and its members
//     to the group list with candidate offsets, and copies each member into
//     the shared memory of every CTA whose next chunk holds its candidates.  A
//     next group index beyond the window takes one more counting round.
//
// Older plans.  A plan whose group index is at most i was expanded (it was a
// member of that group) or was dominated when that group was formed or
// skipped, and removal is permanent because mbest only decreases; a plan with
// a larger group index has not been expanded.  So an older plan is open and
// undominated iff its group index exceeds i and mbest does not dominate it,
// and only ids from the least id of an older open plan upward are re-tested.
//
// Every value that decides control flow (group size, candidate count, group
// index, stop, status) is computed identically by every CTA from the same
// counts, so all CTAs take the same number of barriers.
//
// Fused form (k_explore_fused).  The edge masks of a query and Explore share
// one cooperative launch: cluster 0 runs Explore, the CTAs of every other
// cluster compute masks (the per-edge routine of mask_dev.cuh) for the edges
// in a fixed order, rows by increasing shortest-path cost from the start, and
// count the finished edges of each row.  A plan of group i costs at most
// thr_{i+1}, so its node lies within that cost of the start, and the rows a
// group expands come early in the order; phase A waits (bounded) for the row
// count of each member to reach its degree before reading the row's masks.
// The Explore cluster computes the first positions of the order itself (one
// edge per warp) before it starts, so the first groups find their rows done.
// Masks are read through L2 (the workers write them during the launch).  A
// wait that runs out sets an error flag that phase B publishes, and every CTA
// ends the run with PUMP_ERR_TIMEOUT after the same phase C.  Counts are not
// cleared between runs: run e expects (e - 1) x degree + degree.  Each worker
// warp also counts itself when done; a CTA that sees every worker warp done
// (phase B, an unordered read made an acquire by a fence) skips the waits.
// The launch is the whole explore-only query: cluster 0 also initialises the
// run before its first barrier and orders P_goal after its last one.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <mutex>
#include <vector>

#include "mask_dev.cuh"
#include "pump_internal.cuh"

namespace cg = cooperative_groups;

namespace pump {
namespace {

#ifndef PUMP_CLUSTER_THREADS
#define PUMP_CLUSTER_THREADS 1024
#endif
constexpr int kCT = PUMP_CLUSTER_THREADS;  // threads per CTA
constexpr int kCW = kCT / 32;              // warps per CTA (at most 32: one warp scans the warp totals)
static_assert(kCT % 32 == 0 && kCW <= 32 && kCT >= 64, "CTA size");
constexpr int kCCap = 2048;       // candidates a CTA keeps in shared memory
constexpr int kOCap = 1024;       // older plans a CTA keeps in shared memory
constexpr int kMemCap = 512;      // next-chunk members a CTA receives in shared memory
constexpr int kWin = 32;          // group indices ahead counted in phase B
constexpr int kThr = 64;          // group thresholds thr_i .. thr_{i+63} kept per iteration
constexpr int kMaxCluster = 16;
constexpr uint32_t kGoalBit = 0x80000000u;
constexpr size_t kSmemLimit = 227 * 1024;
constexpr size_t kDynSmemMax = kSmemLimit - 2048;  // dynamic part (the kernel's static part is < 1 KiB)

__device__ __forceinline__ int32_t ld32(const int32_t* p) { return __ldcg(p); }
__device__ __forceinline__ int64_t ld64(const int64_t* p) { return __ldcg(reinterpret_cast<const long long*>(p)); }
__device__ __forceinline__ float ldf(const float* p) { return __ldcg(p); }
__device__ __forceinline__ uint32_t ldu(const uint32_t* p) { return __ldcg(p); }

// Asynchronous global -> shared copies (no register staging; the issuing thread waits for its own
// copies with cp_async_wait, and a barrier after that makes them visible to the CTA).
template <int kBytes>
__device__ __forceinline__ void cp_async(void* smem_dst, const void* gmem_src) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
  if constexpr (kBytes == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gmem_src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(d), "l"(gmem_src), "n"(kBytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Launch shape a cluster kernel was sized for on the host: CTAs per cluster (the on-chip
// dominance table is partitioned over exactly that many CTAs) and dynamic shared memory bytes.
struct LaunchShape {
  int32_t nr;
  uint32_t smem;
};

// True iff the kernel runs with the launch shape the host sized it for.  A launch of the same
// kernel with another cluster size or less shared memory would index the partitioned table and
// the staging arrays out of range; the kernels check this on entry and refuse such a launch
// (PUMP_ERR_CUDA in the control block) before touching shared memory.
__device__ __forceinline__ bool launch_shape_ok(const LaunchShape& ls) {
  uint32_t nct, dsz;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(nct));
  asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dsz));
  return nct == (uint32_t)ls.nr && (ls.nr & (ls.nr - 1)) == 0 && dsz >= ls.smem && blockDim.x == (unsigned)kCT &&
         blockDim.y == 1 && blockDim.z == 1 && gridDim.x % (unsigned)ls.nr == 0;
}

// Cluster sizes are powers of two (the host picks 16, 8 or 4 and the launch-shape check refuses
// others), so per-CTA shares and the node -> (CTA, row) split of the dominance table are shifts
// and masks instead of integer divisions on the phases' dependent chains.
__device__ __forceinline__ int log2_nr(int nr) { return __ffs(nr) - 1; }

// Counts toward one group index: older and new plans, and their out-degree sums.
struct PubQ {
  unsigned long long odeg, ndeg;
  int32_t ocnt, ncnt;
};
// Counts one CTA publishes after phase B (every CTA reads them in phase C).  16-byte aligned: the
// end of phase B copies the record's prefix up to entry qn into every CTA's shared memory with
// vector stores; entries from qn on are zero in the owner's record and not read by anyone.
struct alignas(16) Pub {
  int32_t surv;      // survivors of the CTA's chunk
  int32_t minb;      // least group index of an open undominated plan seen by the CTA
  int32_t min_open;  // least id of an older open undominated plan (INT_MAX if none)
  uint32_t stop;     // bit q: a member of group i+1+q is a goal plan with popc < K_min
  int32_t err;       // a wait for a row's masks ran out (fused form)
  int32_t qn;        // entries q[0 .. qn) may be nonzero (the last counted group index + 1)
  int32_t pad[2];
  PubQ q[kWin];
};
constexpr int kPubVec = (int)(sizeof(Pub) / 16);
constexpr int kPubHead = (int)(offsetof(Pub, q));  // bytes before the entries
constexpr int kPubErrWord = (int)(offsetof(Pub, err) / 4);  // 32-bit word of the error flag
static_assert(sizeof(Pub) % 16 == 0, "Pub copies as 16-byte words");
// Counts for one group index beyond the window (extra round).
struct PubS {
  int32_t ocnt, ncnt;
  unsigned long long odeg, ndeg;
  uint32_t stop, pad;
};

// Loop state, the same in every CTA of the cluster (kept in shared memory; thread 0 writes it
// between barriers).
struct St {
  int64_t C;      // candidates of the group
  int64_t base;   // arena size before the group's survivors
  int64_t lo;     // least id that may still be an open plan
  int64_t ncand;  // candidates over the run
  int32_t g;      // group size
  int32_t i;      // group index
  int32_t stop;
  int32_t status;
  int32_t n_groups;
  int32_t k;      // iteration (loop count)
  // this CTA's share of the iteration (set with the state; per-CTA values)
  int64_t c0, c1; // candidates [c0, c1) of the group
  int64_t a0, a1; // older plans [a0, a1) re-tested
  int32_t big;    // the group's chunks exceed the candidate cache
};

struct CSmem {
  St st;
  float thr[kThr];  // thr[q] = float((i + q) lambda r), the same rounding as bucket_of
  uint4 cmask[kCCap];   // OR'd mask words of a candidate (w <= 4)
  uint4 omask[kOCap];   // mask words of an older open plan (w <= 4)
  uint4 mt_mask[kMemCap];
  int4 mt_info[kMemCap];       // member: plan id, head node, row start, cost bits
  long long mt_off[kMemCap];   // member: first candidate offset
  int32_t mt_deg[kMemCap];     // member: out-degree
  int32_t mt_tag[kMemCap];     // member: group position
  int32_t mt_gen[kMemCap];     // member: iteration it belongs to (entry valid iff tag and gen match)
  int32_t cx[kCCap], cpar[kCCap], cedge[kCCap], ceff[kCCap], cr0[kCCap];
  uint32_t cdg[kCCap];  // target out-degree | goal bit
  float ccost[kCCap];
  int16_t cpc[kCCap];
  int32_t oeff[kOCap], ox[kOCap], or0[kOCap];
  uint32_t odg[kOCap];
  float ocost[kOCap];
  int16_t opc[kOCap];
  // an older plan's record, copied in during phase A (cp.async) when the arena keeps plan rows
  int32_t opf[kOCap], otc[kOCap];  // popcount, creation index
  int2 orw[kOCap];                  // row start, degree | goal bit
  Pub pub;     // this CTA's counts (accumulated in phase B)
  Pub pub_all[kMaxCluster];  // every CTA's counts (copied here by their owners at the end of phase B)
  PubS pubs_s; // the same for a group index beyond the window (read remotely in phase C)
  // cluster-wide values of phase C, derived by warp 0 and read by the whole CTA
  int32_t b_nbk, b_min_open, b_before_s, b_total_s, b_before_o, b_total_o, b_before_n, b_total_n, b_stop, b_fast, b_err;
  int32_t werr;        // this CTA: a wait for a row's masks ran out (fused form)
  int32_t rows_ready;  // this CTA saw every worker warp finished: no more waits (fused form)
  int32_t ready_row;   // a row whose masks are complete from the first group on, or -1 (fused form)
  long long b_dbefore_o, b_dtotal_o, b_dbefore_n, b_dtotal_n;
  ExploreArgs args;  // the query's arguments (batched form)
  int32_t qnext;     // query index taken by the cluster (batched form; written by CTA 0)
  int32_t slot0;     // member holding the first candidate of this CTA's chunk (set by its writer)
  int32_t slot_end;  // member holding the last candidate of this CTA's chunk (set by its writer)
  long long kept; // candidates under the CP cutoff, this CTA, whole run
};

__device__ __forceinline__ void chunk(int64_t total, int r, int nr, int64_t* lo, int64_t* hi) {
  const int64_t per = (total + nr - 1) >> log2_nr(nr);
  *lo = min(total, (int64_t)r * per);
  *hi = min(total, *lo + per);
}

// Whether iteration k runs on state S (the loop's exit tests; every CTA decides alike).
__device__ __forceinline__ bool iter_runs(const St& S, const ExploreArgs& A, int k) {
  return !(S.status || S.stop || S.g == 0) && !(S.i >= A.max_iter || k >= A.max_iter);
}

// Thread 0: this CTA's share of iteration k (set where the previous state is final, so the cluster
// barrier that follows publishes it and the loop needs no CTA barrier of its own).
__device__ __forceinline__ void iter_setup(St& S, int k, int r, int nr) {
  S.k = k;
  S.ncand += S.C;
  ++S.n_groups;
  chunk(S.C, r, nr, &S.c0, &S.c1);
  chunk(S.base - S.lo, r, nr, &S.a0, &S.a1);
  S.a0 += S.lo;
  S.a1 += S.lo;
  S.big = ((S.C + nr - 1) >> log2_nr(nr)) > kCCap ? 1 : 0;
}

// Exclusive block scan over kCT threads; returns the prefix and writes the total.
template <typename T>
__device__ T cscan(T v, T* total) {
  __shared__ T ws[kCW];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[warp] = x;
  __syncthreads();
  if (warp == 0) {
    T s = lane < kCW ? ws[lane] : T(0);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const T y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < kCW) ws[lane] = s;
  }
  __syncthreads();
  const T pre = (warp > 0 ? ws[warp - 1] : T(0)) + x - v;
  *total = ws[kCW - 1];
  __syncthreads();
  return pre;
}

// Two exclusive block scans in one shared-memory round: warp 0 scans the warp totals of the
// first values, warp 1 those of the second.  Returns the first prefix; *pb is the second.  Its
// shared words are rewritten only by the next call, so the caller needs a CTA barrier between
// two calls.
static_assert(kCW >= 2, "two warps scan the warp totals");
template <typename T>
__device__ T cscan2(T a, T b, T* ta, T* tb, T* pb) {
  __shared__ T ws2[2][kCW];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T x = a, y = b;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T u = __shfl_up_sync(0xffffffffu, x, o);
    const T w = __shfl_up_sync(0xffffffffu, y, o);
    if (lane >= o) {
      x += u;
      y += w;
    }
  }
  if (lane == 31) {
    ws2[0][warp] = x;
    ws2[1][warp] = y;
  }
  __syncthreads();
  if (warp < 2) {
    T s = lane < kCW ? ws2[warp][lane] : T(0);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const T u = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += u;
    }
    if (lane < kCW) ws2[warp][lane] = s;
  }
  __syncthreads();
  const T pa = (warp > 0 ? ws2[0][warp - 1] : T(0)) + x - a;
  *pb = (warp > 0 ? ws2[1][warp - 1] : T(0)) + y - b;
  *ta = ws2[0][kCW - 1];
  *tb = ws2[1][kCW - 1];
  return pa;  // no trailing barrier: one call per phase, and a barrier follows before the next
}

__device__ __forceinline__ long long csum_ll(long long v) {
  __shared__ long long s[kCW];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) s[warp] = v;
  __syncthreads();
  v = lane < kCW ? s[lane] : 0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  return v;
}

// Packed scan fields: survivor count in bits 52..63, member count in bits 40..51, member
// out-degree sum in bits 0..39 (a tile holds at most kCT items of each).
constexpr int kPackShift = 40;
__device__ __forceinline__ int64_t pack_cd(int64_t c, int64_t d) { return (c << kPackShift) | d; }
__device__ __forceinline__ int32_t pack_c(int64_t x) { return (int32_t)((x >> kPackShift) & 0xFFF); }
__device__ __forceinline__ int32_t pack_k(int64_t x) { return (int32_t)(x >> 52); }
__device__ __forceinline__ int64_t pack_d(int64_t x) { return x & ((int64_t(1) << kPackShift) - 1); }

// mbest row of node x: in the owning CTA's shared memory, or in global memory.
template <bool kDsm>
__device__ __forceinline__ uint32_t* mb_row(const ExploreArgs& A, cg::cluster_group& cl, uint32_t* mbl, int32_t x) {
  if (kDsm) {
    const int nr = (int)cl.num_blocks();
    return cl.map_shared_rank(mbl + (size_t)(x >> log2_nr(nr)) * A.kstride, (unsigned)(x & (nr - 1)));
  }
  return A.mbest + (size_t)x * A.kstride;
}

// mbest[x][k] = min(mbest[x][k], v) without waiting for the old value: a cluster-scope reduction
// into the owning CTA's shared memory (or a global one).  The cluster barrier closing phase A
// orders every reduction before phase B reads the table.
template <bool kDsm>
__device__ __forceinline__ void mb_min(const ExploreArgs& A, cg::cluster_group& cl, uint32_t* mbl, int32_t x, int k,
                                       uint32_t v) {
  if (kDsm) {
    const int nr = (int)cl.num_blocks();
    const uint32_t local = (uint32_t)__cvta_generic_to_shared(mbl + (size_t)(x >> log2_nr(nr)) * A.kstride + k);
    uint32_t remote;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(local), "r"((unsigned)(x & (nr - 1))));
    asm volatile("red.relaxed.cluster.shared::cluster.min.u32 [%0], %1;" ::"r"(remote), "r"(v) : "memory");
  } else {
    asm volatile("red.relaxed.gpu.global.min.u32 [%0], %1;" ::"l"(A.mbest + (size_t)x * A.kstride + k), "r"(v)
                 : "memory");
  }
}

template <bool kDsm>
__device__ __forceinline__ uint32_t mb_ld(const uint32_t* p) {
  if (kDsm) return *reinterpret_cast<const volatile uint32_t*>(p);
  return __ldcg(p);
}

// Dominated: some entry k <= pc of x's row holds a cost strictly below c.  Up to four entries
// are loaded at once.
template <bool kDsm>
__device__ __forceinline__ bool dominated_c(const ExploreArgs& A, cg::cluster_group& cl, uint32_t* mbl, int32_t x,
                                            int pc, float c) {
  const uint32_t* row = mb_row<kDsm>(A, cl, mbl, x);
  for (int k0 = 0; k0 <= pc; k0 += 4) {
    uint32_t v[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) v[j] = k0 + j <= pc ? mb_ld<kDsm>(row + k0 + j) : 0x7f800000u;
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (__uint_as_float(v[j]) < c) return true;
  }
  return false;
}

struct CCand {
  int32_t x, parent, edge, pc, r0;
  uint32_t dg;
  float cost;
};

// Release add: the warp's mask writes (ordered before it by the warp barrier) are visible to a
// thread whose acquire observes the new count.
__device__ __forceinline__ void red_release_add(uint32_t* p, uint32_t v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Fused form: waits until the mask workers have finished the deg edges of row x in this run
// (count - (epoch_m1 x deg) reaches deg, mod 2^32; every calling thread acquires the count
// itself).  After limit polls it sets *err and returns; once *err is set (a wait of this CTA ran
// out) it returns at once, so one lost row costs one limit.
__device__ __noinline__ void row_wait(const uint32_t* rowcnt, int32_t x, uint32_t deg, uint32_t epoch_m1,
                                      long long limit, int32_t* err) {
  volatile int32_t* verr = err;
  const uint32_t base = epoch_m1 * deg;
  long long it = 0;
  while (ld_acquire_u32(rowcnt + x) - base < deg) {
    if (*verr || ++it > limit) {
      *verr = 1;
      return;
    }
    __nanosleep(128);
  }
}

// Target of edge e: node, cost bits, row start, out-degree | goal bit.
__device__ __forceinline__ int4 edge_target(const ExploreArgs& A, int32_t e) {
  if (A.etgt) return __ldg(A.etgt + e);
  const int32_t x = A.col[e];
  const int32_t r0 = A.row_ptr[x];
  const uint32_t dg = (uint32_t)(A.row_ptr[x + 1] - r0) | (A.is_goal[x] ? kGoalBit : 0u);
  return make_int4(x, __float_as_int(A.ecost[e]), r0, (int32_t)dg);
}

// Candidate c of the current group, recomputed from the group list (chunks that do not fit).
__device__ __noinline__ CCand cand_at_c(const ExploreArgs& A, int64_t c, int32_t g, int32_t* err) {
  int lo = 0, hi = g;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (ld64(A.goff + mid) <= c) lo = mid; else hi = mid;
  }
  CCand q;
  const int4 gi = __ldcg(A.ginfo + lo);
  const int64_t off = ld64(A.goff + lo);
  if (A.rowcnt) row_wait(A.rowcnt, gi.y, (uint32_t)(ld64(A.goff + lo + 1) - off), A.epoch_m1, A.spin_limit, err);
  const int32_t e = gi.z + (int32_t)(c - off);
  const int4 t = edge_target(A, e);
  q.x = t.x;
  q.parent = gi.x;
  q.edge = e;
  q.cost = __fadd_rn(__int_as_float(gi.w), __int_as_float(t.y));
  q.r0 = t.z;
  q.dg = (uint32_t)t.w;
  int pc = 0;
  const uint32_t* pm = A.mask + (size_t)gi.x * A.w;
  const uint32_t* em = A.emask + (size_t)e * A.w;
  for (int j = 0; j < A.w; ++j) pc += __popc(ldu(pm + j) | ldu(em + j));
  q.pc = pc;
  return q;
}

__device__ __forceinline__ uint4 load_mask4(const uint32_t* p, int w) {
  return make_uint4(ldu(p), w > 1 ? ldu(p + 1) : 0u, w > 2 ? ldu(p + 2) : 0u, w > 3 ? ldu(p + 3) : 0u);
}

// Warp-aggregated count of a plan (an older one or a new one) toward group index i+1+q (q in
// [0, kWin)).
__device__ __forceinline__ void bucket_add(bool on, int q, int deg, bool goal_stop, bool older, Pub* pub) {
  const bool in = on && q >= 0 && q < kWin;
  const unsigned act = __ballot_sync(0xffffffffu, in);
  if (!in) return;
  const unsigned peers = __match_any_sync(act, q);
  const unsigned ds = __reduce_add_sync(peers, (unsigned)deg);
  const bool st = __any_sync(peers, goal_stop);
  if ((threadIdx.x & 31) == __ffs(peers) - 1) {
    PubQ& e = pub->q[q];
    atomicAdd(older ? &e.ocnt : &e.ncnt, __popc(peers));
    atomicAdd(older ? &e.odeg : &e.ndeg, (unsigned long long)ds);
    if (st) atomicOr(&pub->stop, 1u << q);
    atomicMax(&pub->qn, q + 1);
  }
}

// Group index past the threshold table (rare; kept out of line).
__device__ __noinline__ int32_t bucket_far(float c, double lr) { return bucket_of(c, lr); }

// Group index from the iteration's threshold table (float compares; bucket_of's double
// arithmetic is far slower on this part).  bucket_gt(c, a): least j > i + a with
// c <= thr_j, given c > thr_{i+a}; past the table it falls back to bucket_of (same result).
__device__ __forceinline__ int32_t bucket_gt(const CSmem* sm, const ExploreArgs& A, int32_t i, float c, int a) {
  int b = kThr - 1;
  if (!(c <= sm->thr[b])) return bucket_far(c, A.lr);
  while (b - a > 1) {
    const int m = (a + b) >> 1;
    if (c <= sm->thr[m]) b = m; else a = m;
  }
  return i + b;
}

// Group index of a survivor of group i: max(bucket(c), i + 1).
__device__ __forceinline__ int32_t eff_new(const CSmem* sm, const ExploreArgs& A, int32_t i, float c) {
  return c <= sm->thr[1] ? i + 1 : bucket_gt(sm, A, i, c, 1);
}

// ---------------------------------------------------------------- phase A
template <bool kDsm>
__device__ void c_expand(const ExploreArgs& A, CSmem* sm, uint32_t* mbl, cg::cluster_group& cl, const St& S) {
  const int r = (int)cl.block_rank(), nr = (int)cl.num_blocks();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // this CTA's counts for phase B (the copies other CTAs hold are separate)
  if (threadIdx.x < kWin) {
    sm->pub.q[threadIdx.x].ocnt = 0;
    sm->pub.q[threadIdx.x].ncnt = 0;
    sm->pub.q[threadIdx.x].odeg = 0;
    sm->pub.q[threadIdx.x].ndeg = 0;
  }
  if (threadIdx.x == 0) {
    sm->pub.stop = 0;
    sm->pub.qn = 0;
    sm->pub.surv = 0;
    sm->pub.minb = kNoBucket;
    sm->pub.min_open = INT_MAX;
  }
  if (threadIdx.x < kThr) sm->thr[threadIdx.x] = group_thr(S.i + (int32_t)threadIdx.x, A.lr);
  // the older plans phase B re-tests: their records copied into shared memory now, behind the
  // expansion, so that phase B only looks up their dominance (the same decision as phase B's)
  const bool pf = A.prow != nullptr && S.a1 - S.a0 <= kOCap;
  if (pf) {
    const int no = (int)(S.a1 - S.a0);
    for (int o = threadIdx.x; o < no; o += kCT) {
      const int64_t p = S.a0 + o;
      cp_async<4>(&sm->ox[o], A.head + p);
      cp_async<4>(&sm->ocost[o], A.cost + p);
      cp_async<4>(&sm->opf[o], A.popc + p);
      cp_async<4>(&sm->otc[o], A.tcre + p);
      cp_async<8>(&sm->orw[o], A.prow + p);
      if (A.w == 4) {
        cp_async<16>(&sm->omask[o], A.mask + (size_t)p * 4);
      } else if (A.w < 4) {
        uint32_t* om = reinterpret_cast<uint32_t*>(&sm->omask[o]);
        for (int j = 0; j < 4; ++j) {
          if (j < A.w)
            cp_async<4>(om + j, A.mask + (size_t)p * A.w + j);
          else
            om[j] = 0u;
        }
      }
    }
    cp_async_commit();
  }
  for (int64_t s = (int64_t)r * kCT + threadIdx.x; s < S.g; s += (int64_t)nr * kCT)
    A.eexp[ld32(&A.ginfo[s].x)] = S.i;
  const int64_t c0 = S.c0, c1 = S.c1;
  const int64_t n = c1 - c0;
  long long kept = 0;
  if (n > 0 && n <= kCCap) {
    const int w = A.w;
    const int32_t s_end = min(sm->slot_end, S.g - 1);
    for (int32_t s = sm->slot0 + warp; s <= s_end; s += kCW) {
      const int slot = s % kMemCap;
      int64_t lo_s, hi_s;
      int4 gi;
      uint4 pmv = make_uint4(0u, 0u, 0u, 0u);
      const bool local = sm->mt_tag[slot] == s && sm->mt_gen[slot] == S.k;
      if (local) {
        lo_s = sm->mt_off[slot];
        hi_s = lo_s + sm->mt_deg[slot];
        gi = sm->mt_info[slot];
        pmv = sm->mt_mask[slot];
      } else {
        lo_s = ld64(A.goff + s);
        hi_s = ld64(A.goff + s + 1);
        gi = __ldcg(A.ginfo + s);
      }
      if (lo_s >= c1) break;
      const int64_t lo = max(lo_s, c0), hi = min(hi_s, c1);
      if (lo >= hi) continue;
      const int32_t p = gi.x, r0 = gi.z;
      if (A.rowcnt && !sm->rows_ready && gi.y != sm->ready_row)
        row_wait(A.rowcnt, gi.y, (uint32_t)(hi_s - lo_s), A.epoch_m1, A.spin_limit, &sm->werr);
      const float pcost = __int_as_float(gi.w);
      const uint32_t* pm = A.mask + (size_t)p * w;
      if (!local && w <= 4) {
        const uint32_t pmw = lane < w ? ldu(pm + lane) : 0u;
        pmv.x = __shfl_sync(0xffffffffu, pmw, 0);
        pmv.y = __shfl_sync(0xffffffffu, pmw, 1);
        pmv.z = __shfl_sync(0xffffffffu, pmw, 2);
        pmv.w = __shfl_sync(0xffffffffu, pmw, 3);
      }
      // w <= 4: two candidates per lane per round, both edges' targets and masks loaded before
      // either is used (their L2 round trips overlap)
      if (w <= 4) {
        auto em_load = [&](int32_t e) -> uint4 {
          if (w == 4) return __ldcg(reinterpret_cast<const uint4*>(A.emask) + e);
          const uint32_t* ep = A.emask + (size_t)e * w;
          return make_uint4(ldu(ep), w > 1 ? ldu(ep + 1) : 0u, w > 2 ? ldu(ep + 2) : 0u, 0u);
        };
        auto put = [&](int64_t c, int32_t e, const int4& t, const uint4& em) {
          const float cost = __fadd_rn(pcost, __int_as_float(t.y));
          const int jl = (int)(c - c0);
          const uint4 m = make_uint4(pmv.x | em.x, pmv.y | em.y, pmv.z | em.z, pmv.w | em.w);
          const int pc = __popc(m.x) + __popc(m.y) + __popc(m.z) + __popc(m.w);
          sm->cmask[jl] = m;
          sm->cx[jl] = t.x;
          sm->cpar[jl] = p;
          sm->cedge[jl] = e;
          sm->ccost[jl] = cost;
          sm->cpc[jl] = (int16_t)pc;
          sm->cr0[jl] = t.z;
          sm->cdg[jl] = (uint32_t)t.w;
          if (pc < A.kmax) {
            mb_min<kDsm>(A, cl, mbl, t.x, pc, __float_as_uint(cost));
            ++kept;
          }
        };
        for (int64_t c = lo + lane; c < hi; c += 64) {
          const int64_t c2 = c + 32;
          const bool two = c2 < hi;
          const int32_t e = r0 + (int32_t)(c - lo_s), e2 = r0 + (int32_t)(c2 - lo_s);
          const int4 t = edge_target(A, e);
          const int4 t2 = two ? edge_target(A, e2) : make_int4(0, 0, 0, 0);
          const uint4 em = em_load(e);
          const uint4 em2 = two ? em_load(e2) : make_uint4(0u, 0u, 0u, 0u);
          put(c, e, t, em);
          if (two) put(c2, e2, t2, em2);
        }
        continue;
      }
      for (int64_t c = lo + lane; c < hi; c += 32) {
        const int32_t e = r0 + (int32_t)(c - lo_s);
        const int4 t = edge_target(A, e);
        const float cost = __fadd_rn(pcost, __int_as_float(t.y));
        const int jl = (int)(c - c0);
        int pc = 0;
        if (w <= 4) {
          uint4 em;
          if (w == 4) {
            em = __ldcg(reinterpret_cast<const uint4*>(A.emask) + e);
          } else {
            const uint32_t* ep = A.emask + (size_t)e * w;
            em.x = ldu(ep);
            em.y = w > 1 ? ldu(ep + 1) : 0u;
            em.z = w > 2 ? ldu(ep + 2) : 0u;
            em.w = 0u;
          }
          const uint4 m = make_uint4(pmv.x | em.x, pmv.y | em.y, pmv.z | em.z, pmv.w | em.w);
          pc = __popc(m.x) + __popc(m.y) + __popc(m.z) + __popc(m.w);
          sm->cmask[jl] = m;
        } else {
          const uint32_t* em = A.emask + (size_t)e * w;
          for (int j = 0; j < w; ++j) pc += __popc(ldu(pm + j) | ldu(em + j));
        }
        sm->cx[jl] = t.x;
        sm->cpar[jl] = p;
        sm->cedge[jl] = e;
        sm->ccost[jl] = cost;
        sm->cpc[jl] = (int16_t)pc;
        sm->cr0[jl] = t.z;
        sm->cdg[jl] = (uint32_t)t.w;
        if (pc < A.kmax) {
          mb_min<kDsm>(A, cl, mbl, t.x, pc, __float_as_uint(cost));
          ++kept;
        }
      }
    }
  } else if (n > 0) {
    for (int64_t c = c0 + threadIdx.x; c < c1; c += kCT) {
      const CCand q = cand_at_c(A, c, S.g, &sm->werr);
      if (q.pc < A.kmax) {
        mb_min<kDsm>(A, cl, mbl, q.x, q.pc, __float_as_uint(q.cost));
        ++kept;
      }
    }
  }
  if (pf) cp_async_wait();  // the cluster barrier that closes the phase publishes the copies
  // the run's count of kept candidates (a statistic read after the loop): warp sums, one
  // shared-memory atomic per warp
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) kept += __shfl_xor_sync(0xffffffffu, kept, o);
  if (lane == 0 && kept) atomicAdd(reinterpret_cast<unsigned long long*>(&sm->kept), (unsigned long long)kept);
}

// Group index of an older plan (head x, cost c, popcount pc, created in group t) if it is open and
// undominated, else -1 (see the header on older plans).
template <bool kDsm>
__device__ __forceinline__ int32_t old_eff_vals(const ExploreArgs& A, const CSmem* sm, cg::cluster_group& cl,
                                                uint32_t* mbl, int32_t x, float c, int32_t pc, int32_t t, int32_t i) {
  // bucket(c) <= i iff c <= thr_i; above it the table gives the bucket
  const int32_t b = c <= sm->thr[0] ? (t + 1 <= i ? -1 : bucket_far(c, A.lr)) : bucket_gt(sm, A, i, c, 0);
  if (b < 0) return -1;
  const int32_t eff = max(b, t + 1);
  if (eff <= i) return -1;
  if (dominated_c<kDsm>(A, cl, mbl, x, pc, c)) return -1;
  return eff;
}

// Older plan p: its group index if open and undominated, else -1.
template <bool kDsm>
__device__ __forceinline__ int32_t old_eff_c(const ExploreArgs& A, const CSmem* sm, cg::cluster_group& cl,
                                             uint32_t* mbl, int64_t p, int32_t i, int32_t* x_out, float* c_out,
                                             int32_t* pc_out) {
  const int32_t x = ld32(A.head + p);
  const float c = ldf(A.cost + p);
  const int32_t pc = ld32(A.popc + p);
  const int32_t t = ld32(A.tcre + p);
  *x_out = x;
  *c_out = c;
  *pc_out = pc;
  return old_eff_vals<kDsm>(A, sm, cl, mbl, x, c, pc, t, i);
}

// ---------------------------------------------------------------- phase B
// Candidate jl of the CTA's chunk: dominance test, group index; keeps its counts.
template <bool kDsm>
__device__ __forceinline__ void filter_cand(const ExploreArgs& A, CSmem* sm, uint32_t* mbl, cg::cluster_group& cl,
                                            const St& S, int jl, bool fits, int32_t& surv, int32_t& minb, bool& keep,
                                            int32_t& eff, int32_t& deg, bool& gstop) {
  CCand q;
  if (fits) {
    q.x = sm->cx[jl];
    q.pc = sm->cpc[jl];
    q.cost = sm->ccost[jl];
    q.dg = sm->cdg[jl];
  } else {
    q = cand_at_c(A, S.c0 + jl, S.g, &sm->werr);
  }
  keep = q.pc < A.kmax && !dominated_c<kDsm>(A, cl, mbl, q.x, q.pc, q.cost);
  if (keep) {
    eff = eff_new(sm, A, S.i, q.cost);
    deg = (int32_t)(q.dg & ~kGoalBit);
    ++surv;
    minb = min(minb, eff);
    gstop = (q.dg & kGoalBit) && q.pc < A.kmin;
  }
  if (fits) sm->ceff[jl] = eff;
}

// Older plan p (ids [a0, a1) of the CTA): open and undominated, and its group index; keeps its
// counts and, when the range fits, its record for phase C.
template <bool kDsm>
__device__ __forceinline__ void filter_old(const ExploreArgs& A, CSmem* sm, uint32_t* mbl, cg::cluster_group& cl,
                                           const St& S, int64_t p, int64_t a0, bool ofits, int32_t& minb,
                                           int32_t& min_open, int32_t& eff, int32_t& pc, int32_t& deg, bool& goal) {
  if (A.prow != nullptr && ofits) {
    // the record was copied into shared memory during phase A
    const int o = (int)(p - a0);
    const int32_t x = sm->ox[o], pcp = sm->opf[o];
    const int2 rw = sm->orw[o];
    eff = old_eff_vals<kDsm>(A, sm, cl, mbl, x, sm->ocost[o], pcp, sm->otc[o], S.i);
    pc = pcp;
    sm->oeff[o] = eff;
    if (eff >= 0) {
      deg = (int32_t)((uint32_t)rw.y & ~kGoalBit);
      goal = ((uint32_t)rw.y & kGoalBit) != 0;
      minb = min(minb, eff);
      min_open = min(min_open, (int32_t)p);
      sm->or0[o] = rw.x;
      sm->odg[o] = (uint32_t)rw.y;
      sm->opc[o] = (int16_t)pcp;
    }
    return;
  }
  int32_t x = 0, r0 = 0;
  float c = 0.f;
  // the plan's row, goal flag and mask are loaded with its record, before the dominance test
  // (distributed shared memory), so the two round trips overlap
  const int32_t xp = ld32(A.head + p);
  const int32_t r0p = A.row_ptr[xp], r1p = A.row_ptr[xp + 1];
  const bool goalp = A.is_goal[xp] != 0;
  const uint4 mp = (ofits && A.w <= 4) ? load_mask4(A.mask + (size_t)p * A.w, A.w) : make_uint4(0u, 0u, 0u, 0u);
  eff = old_eff_c<kDsm>(A, sm, cl, mbl, p, S.i, &x, &c, &pc);
  if (eff >= 0) {
    r0 = r0p;
    deg = r1p - r0p;
    goal = goalp;
    minb = min(minb, eff);
    min_open = min(min_open, (int32_t)p);
  }
  if (ofits) {
    const int o = (int)(p - a0);
    sm->oeff[o] = eff;
    if (eff >= 0) {
      sm->ox[o] = x;
      sm->ocost[o] = c;
      sm->or0[o] = r0;
      sm->odg[o] = (uint32_t)deg | (goal ? kGoalBit : 0u);
      sm->opc[o] = (int16_t)pc;
      if (A.w <= 4) sm->omask[o] = mp;
    }
  }
}

template <bool kDsm>
__device__ void c_filter(const ExploreArgs& A, CSmem* sm, uint32_t* mbl, cg::cluster_group& cl, const St& S) {
  const int r = (int)cl.block_rank(), nr = (int)cl.num_blocks();
  const int64_t c0 = S.c0, c1 = S.c1;
  const int n = (int)(c1 - c0);
  const bool fits = n <= kCCap;
  int32_t surv = 0, minb = kNoBucket, min_open = INT_MAX;
  // fused form: whether every worker warp has finished, read without ordering now (its latency
  // hides behind this phase) and made an acquire by a fence below if so
  uint32_t done_seen = 0;
  const bool poll_done = A.done && threadIdx.x == 0 && !sm->rows_ready;
  if (poll_done) done_seen = *reinterpret_cast<const volatile uint32_t*>(A.done);
  // A cached chunk of two passes (kCT < n <= kCCap) loads both passes' dominance rows before
  // testing either (one distributed-shared-memory round trip instead of two); the tests and the
  // counts are the same as pass by pass.
  const bool two = fits && n > kCT && A.kmax <= 4;
  const int64_t a0 = S.a0, a1 = S.a1;
  const bool ofits = a1 - a0 <= kOCap;
  // candidates and older plans in one pass when both fit it: disjoint threads, so their dependent
  // load chains overlap (the counts are sums, independent of the order)
  const bool merged = fits && !two && (int64_t)n + (a1 - a0) <= kCT;
  if (merged) {
    const int t = threadIdx.x;
    bool keep = false, gstop = false, goal = false;
    int32_t eff = -1, deg = 0, oeff = -1, opc = 0, odeg = 0;
    if (t < n)
      filter_cand<kDsm>(A, sm, mbl, cl, S, t, true, surv, minb, keep, eff, deg, gstop);
    else if (t < n + (int)(a1 - a0))
      filter_old<kDsm>(A, sm, mbl, cl, S, a0 + (t - n), a0, ofits, minb, min_open, oeff, opc, odeg, goal);
    bucket_add(keep, eff - S.i - 1, deg, gstop, false, &sm->pub);
    bucket_add(oeff >= 0, oeff - S.i - 1, odeg, goal && opc < A.kmin, true, &sm->pub);
  }
  for (int t0 = 0; t0 < n && !merged; t0 += two ? 2 * kCT : kCT) {
    const int jl = t0 + threadIdx.x, jl2 = jl + kCT;
    bool keep = false, keep2 = false;
    int32_t eff = -1, deg = 0, eff2 = -1, deg2 = 0;
    bool gstop = false, gstop2 = false;
    if (two) {
      // rows of both candidates (popc < kmax <= 4: entries 0 .. popc of one 4-entry row)
      const bool on1 = jl < n, on2 = jl2 < n;
      const int32_t x1 = on1 ? sm->cx[jl] : 0, pc1 = on1 ? sm->cpc[jl] : A.kmax;
      const int32_t x2 = on2 ? sm->cx[jl2] : 0, pc2 = on2 ? sm->cpc[jl2] : A.kmax;
      const float cc1 = on1 ? sm->ccost[jl] : 0.f, cc2 = on2 ? sm->ccost[jl2] : 0.f;
      const bool t1 = pc1 < A.kmax, t2 = pc2 < A.kmax;
      uint32_t v1[4], v2[4];
      const uint32_t* row1 = mb_row<kDsm>(A, cl, mbl, t1 ? x1 : 0);
      const uint32_t* row2 = mb_row<kDsm>(A, cl, mbl, t2 ? x2 : 0);
#pragma unroll
      for (int j = 0; j < 4; ++j) v1[j] = t1 && j <= pc1 ? mb_ld<kDsm>(row1 + j) : 0x7f800000u;
#pragma unroll
      for (int j = 0; j < 4; ++j) v2[j] = t2 && j <= pc2 ? mb_ld<kDsm>(row2 + j) : 0x7f800000u;
      bool d1 = false, d2 = false;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        d1 = d1 || __uint_as_float(v1[j]) < cc1;
        d2 = d2 || __uint_as_float(v2[j]) < cc2;
      }
      keep = t1 && !d1;
      keep2 = t2 && !d2;
      if (keep) {
        const uint32_t dg = sm->cdg[jl];
        eff = eff_new(sm, A, S.i, cc1);
        deg = (int32_t)(dg & ~kGoalBit);
        ++surv;
        minb = min(minb, eff);
        gstop = (dg & kGoalBit) && pc1 < A.kmin;
      }
      if (keep2) {
        const uint32_t dg = sm->cdg[jl2];
        eff2 = eff_new(sm, A, S.i, cc2);
        deg2 = (int32_t)(dg & ~kGoalBit);
        ++surv;
        minb = min(minb, eff2);
        gstop2 = (dg & kGoalBit) && pc2 < A.kmin;
      }
      if (on1) sm->ceff[jl] = eff;
      if (on2) sm->ceff[jl2] = eff2;
      bucket_add(keep, eff - S.i - 1, deg, gstop, false, &sm->pub);
      bucket_add(keep2, eff2 - S.i - 1, deg2, gstop2, false, &sm->pub);
      continue;
    }
    if (jl < n) filter_cand<kDsm>(A, sm, mbl, cl, S, jl, fits, surv, minb, keep, eff, deg, gstop);
    bucket_add(keep, eff - S.i - 1, deg, gstop, false, &sm->pub);
  }
  for (int64_t t0 = a0; t0 < a1 && !merged; t0 += kCT) {
    const int64_t p = t0 + threadIdx.x;
    int32_t eff = -1, pc = 0, deg = 0;
    bool goal = false;
    if (p < a1) filter_old<kDsm>(A, sm, mbl, cl, S, p, a0, ofits, minb, min_open, eff, pc, deg, goal);
    bucket_add(eff >= 0, eff - S.i - 1, deg, goal && pc < A.kmin, true, &sm->pub);
  }
  if (poll_done && done_seen == A.done_target) {
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
    sm->rows_ready = 1;  // read by phase A after this phase's barriers
  }
  // the CTA's survivor count and minima: warp reductions, then one shared-memory atomic per warp
  // into the record (reset in phase A)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    surv += __shfl_xor_sync(0xffffffffu, surv, o);
    minb = min(minb, __shfl_xor_sync(0xffffffffu, minb, o));
    min_open = min(min_open, __shfl_xor_sync(0xffffffffu, min_open, o));
  }
  if ((threadIdx.x & 31) == 0) {
    if (surv) atomicAdd(&sm->pub.surv, surv);
    if (minb != kNoBucket) atomicMin(&sm->pub.minb, minb);
    if (min_open != INT_MAX) atomicMin(&sm->pub.min_open, min_open);
  }
  __syncthreads();
  // the record into slot r of every CTA (the cluster barrier that closes this phase orders the
  // stores before phase C reads them; slot r is rewritten only after two more barriers), with the
  // error flag as it stands after the barrier above (every wait of this phase has ended)
  const uint4* src = reinterpret_cast<const uint4*>(&sm->pub);
  const uint32_t werr = (uint32_t)sm->werr;
  const int len = (kPubHead + (int)sizeof(PubQ) * sm->pub.qn + 15) / 16;  // 16-byte words pushed
  for (int t = threadIdx.x; t < len * nr; t += kCT) {
    const int dr = t / len, wv = t - dr * len;
    uint4* dst = reinterpret_cast<uint4*>(cl.map_shared_rank(&sm->pub_all[r], (unsigned)dr));
    uint4 v = src[wv];
    if (wv == kPubErrWord / 4) reinterpret_cast<uint32_t*>(&v)[kPubErrWord % 4] = werr;
    dst[wv] = v;
  }
}

// Warp 0: exclusive prefix over CTAs (lanes) of v for this CTA, and the total.
template <typename T>
__device__ __forceinline__ void lane_prefix(T v, int r, T* before, T* total) {
  const int lane = threadIdx.x & 31;
  T x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  *total = __shfl_sync(0xffffffffu, x, 31);
  const T incl = __shfl_sync(0xffffffffu, x, r);
  const T mine = __shfl_sync(0xffffffffu, v, r);
  *before = incl - mine;
}

// Recount for a next group index beyond the window (uniform decision; one extra barrier).
template <bool kDsm>
__device__ __noinline__ void c_recount(const ExploreArgs& A, CSmem* sm, uint32_t* mbl, cg::cluster_group& cl, const St& S,
                          int32_t nbk) {
  const int r = (int)cl.block_rank(), nr = (int)cl.num_blocks();
  const int64_t c0 = S.c0, c1 = S.c1;
  const int n = (int)(c1 - c0);
  const bool fits = n <= kCCap;
  long long nc = 0, nd = 0, oc = 0, od = 0;
  int32_t stop = 0;
  for (int jl = threadIdx.x; jl < n; jl += kCT) {
    int32_t eff, pc;
    uint32_t dg;
    if (fits) {
      eff = sm->ceff[jl];
      dg = sm->cdg[jl];
      pc = sm->cpc[jl];
    } else {
      const CCand q = cand_at_c(A, c0 + jl, S.g, &sm->werr);
      const bool keep = q.pc < A.kmax && !dominated_c<kDsm>(A, cl, mbl, q.x, q.pc, q.cost);
      eff = keep ? eff_new(sm, A, S.i, q.cost) : -1;
      dg = q.dg;
      pc = q.pc;
    }
    if (eff == nbk) {
      ++nc;
      nd += dg & ~kGoalBit;
      if ((dg & kGoalBit) && pc < A.kmin) stop = 1;
    }
  }
  const int64_t a0 = S.a0, a1 = S.a1;
  const bool ofits = a1 - a0 <= kOCap;
  for (int64_t p = a0 + threadIdx.x; p < a1; p += kCT) {
    int32_t eff, x = 0, pc = 0;
    uint32_t dg = 0;
    float c = 0.f;
    if (ofits) {
      eff = sm->oeff[p - a0];
      if (eff == nbk) {
        dg = sm->odg[p - a0];
        pc = sm->opc[p - a0];
      }
    } else {
      eff = old_eff_c<kDsm>(A, sm, cl, mbl, p, S.i, &x, &c, &pc);
      if (eff == nbk) dg = (uint32_t)(A.row_ptr[x + 1] - A.row_ptr[x]) | (A.is_goal[x] ? kGoalBit : 0u);
    }
    if (eff == nbk) {
      ++oc;
      od += dg & ~kGoalBit;
      if ((dg & kGoalBit) && pc < A.kmin) stop = 1;
    }
  }
  nc = csum_ll(nc);
  nd = csum_ll(nd);
  oc = csum_ll(oc);
  od = csum_ll(od);
  stop = __syncthreads_or(stop);
  if (threadIdx.x == 0) {
    sm->pubs_s.ncnt = (int32_t)nc;
    sm->pubs_s.ndeg = (unsigned long long)nd;
    sm->pubs_s.ocnt = (int32_t)oc;
    sm->pubs_s.odeg = (unsigned long long)od;
    sm->pubs_s.stop = stop ? 1u : 0u;
    sm->pubs_s.pad = 0u;
  }
}

// Copies a next-group member (iteration gen) into the shared memory of every CTA whose next
// chunk [rr per, min((rr+1) per, Cn)) holds some of its candidates [off, off + deg), and tells
// the CTAs whose chunk starts or ends inside it.  A member without edges goes to the CTA whose
// range holds its offset.
__device__ __forceinline__ void send_member(CSmem* sm, cg::cluster_group& cl, int64_t Cn, int64_t per, int32_t gen,
                                            int32_t pos, int4 info, int64_t off, int32_t deg, uint4 mask) {
  if (per <= 0) return;
  const int nr = (int)cl.num_blocks();
  const int slot = pos % kMemCap;
  int64_t first, last;
  const int64_t end = deg > 0 ? off + deg - 1 : off;
  if (end < (int64_t)INT_MAX && per < (int64_t)INT_MAX) {
    first = (uint32_t)off / (uint32_t)per;
    last = (uint32_t)end / (uint32_t)per;
  } else {
    first = off / per;
    last = end / per;
  }
  for (int64_t rr = first; rr <= last && rr < nr; ++rr) {
    CSmem* d = cl.map_shared_rank(sm, (unsigned)rr);
    d->mt_info[slot] = info;
    d->mt_off[slot] = off;
    d->mt_deg[slot] = deg;
    d->mt_mask[slot] = mask;
    d->mt_tag[slot] = pos;
    d->mt_gen[slot] = gen;
    if (deg > 0) {
      const int64_t lo = rr * per, hi = min((rr + 1) * per, Cn);
      if (lo >= off) d->slot0 = pos;                      // the chunk starts inside this member
      if (hi - 1 < off + deg && hi > lo) d->slot_end = pos;  // and ends inside it
    }
  }
}

// Arena record of survivor q at id; its mask from the candidate cache (slot jl) when the chunk is
// cached and w <= 4, else the parent's mask OR the edge's.  Returns the mask words (w <= 4).
__device__ __forceinline__ uint4 put_survivor(const ExploreArgs& A, CSmem* sm, int64_t id, const CCand& q, int jl,
                                              bool cached, int32_t i) {
  A.head[id] = q.x;
  A.parent[id] = q.parent;
  A.pedge[id] = q.edge;
  A.cost[id] = q.cost;
  A.popc[id] = q.pc;
  A.tcre[id] = i;
  A.eexp[id] = -1;
  if (A.prow) A.prow[id] = make_int2(q.r0, (int32_t)q.dg);
  uint32_t* om = A.mask + (size_t)id * A.w;
  uint4 m = make_uint4(0u, 0u, 0u, 0u);
  if (cached && A.w <= 4) {
    m = sm->cmask[jl];
    if (A.w == 4) {
      *reinterpret_cast<uint4*>(om) = m;
    } else {
      om[0] = m.x;
      if (A.w > 1) om[1] = m.y;
      if (A.w > 2) om[2] = m.z;
    }
  } else {
    const uint32_t* pm = A.mask + (size_t)q.parent * A.w;
    const uint32_t* em = A.emask + (size_t)q.edge * A.w;
    for (int j = 0; j < A.w; ++j) om[j] = ldu(pm + j) | ldu(em + j);
  }
  if (q.dg & kGoalBit) {
    const int slot = atomicAdd(&A.ctl->n_goal_all, 1);
    A.goal_all[slot] = (int32_t)id;
  }
  return m;
}

// Member at position pos of the next group: its record in the group list, and its copy to the
// CTAs whose candidate chunks it feeds.
__device__ __forceinline__ void put_member(const ExploreArgs& A, CSmem* sm, cg::cluster_group& cl, int64_t Cn,
                                           int64_t per, int32_t gen, int64_t pos, int64_t off, int32_t id, int32_t x,
                                           int32_t r0, float c, int32_t deg, uint4 m) {
  const int4 info = make_int4(id, x, r0, __float_as_int(c));
  A.ginfo[pos] = info;
  A.goff[pos] = off;
  send_member(sm, cl, Cn, per, gen, (int32_t)pos, info, off, deg, m);
}

// ---------------------------------------------------------------- phase C
template <bool kDsm>
__device__ void c_write(const ExploreArgs& A, CSmem* sm, uint32_t* mbl, cg::cluster_group& cl, St& S) {
  const int r = (int)cl.block_rank(), nr = (int)cl.num_blocks();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // Warps 0-3 read every CTA's counts (lane l from CTA l) and derive the cluster-wide values:
  // each the least group index, then warp 0 the survivors' and older plans' prefixes, warp 1 the
  // new plans', warps 2 and 3 the degree sums of the older and the new ones.
  if (warp < 4) {
    const bool on = lane < nr;
    const Pub* rp = &sm->pub_all[on ? lane : 0];
    int32_t minb = on ? rp->minb : kNoBucket;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) minb = min(minb, __shfl_xor_sync(0xffffffffu, minb, o));
    const int32_t q = minb == kNoBucket ? -1 : minb - S.i - 1;
    const bool fast = minb == kNoBucket || (q >= 0 && q < kWin);
    const bool has = minb != kNoBucket && fast && on && q < rp->qn;  // entries from qn on were not pushed
    if (warp == 0) {
      int32_t mo = on ? rp->min_open : INT_MAX;
      const int32_t sv = on ? rp->surv : 0;
      const bool werr = __any_sync(0xffffffffu, on && rp->err != 0);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mo = min(mo, __shfl_xor_sync(0xffffffffu, mo, o));
      int32_t bs, ts, bo, to;
      lane_prefix<int32_t>(sv, r, &bs, &ts);
      lane_prefix<int32_t>(has ? rp->q[q].ocnt : 0, r, &bo, &to);
      const bool stp = minb != kNoBucket && fast && __any_sync(0xffffffffu, on && ((rp->stop >> q) & 1u));
      if (lane == 0) {
        sm->b_nbk = minb;
        sm->b_min_open = mo;
        sm->b_before_s = bs;
        sm->b_total_s = ts;
        sm->b_fast = fast ? 1 : 0;
        sm->b_before_o = bo;
        sm->b_total_o = to;
        sm->b_stop = stp ? 1 : 0;
        sm->b_err = werr ? 1 : 0;
      }
    } else if (warp == 1) {
      int32_t bn, tn;
      lane_prefix<int32_t>(has ? rp->q[q].ncnt : 0, r, &bn, &tn);
      if (lane == 0) {
        sm->b_before_n = bn;
        sm->b_total_n = tn;
      }
    } else {
      long long db, dt;
      const bool older = warp == 2;
      lane_prefix<long long>(has ? (long long)(older ? rp->q[q].odeg : rp->q[q].ndeg) : 0, r, &db, &dt);
      if (lane == 0) {
        if (older) {
          sm->b_dbefore_o = db;
          sm->b_dtotal_o = dt;
        } else {
          sm->b_dbefore_n = db;
          sm->b_dtotal_n = dt;
        }
      }
    }
  }
  __syncthreads();
  const int32_t nbk = sm->b_nbk;
  if (!sm->b_fast) {
    // every CTA takes this branch together: nbk is the same everywhere
    c_recount<kDsm>(A, sm, mbl, cl, S, nbk);
    cl.sync();
    if (warp == 0) {
      const bool on = lane < nr;
      const PubS* rs = cl.map_shared_rank(&sm->pubs_s, (unsigned)(on ? lane : 0));
      const int32_t oc = on ? rs->ocnt : 0, nc = on ? rs->ncnt : 0;
      const long long od = on ? (long long)rs->odeg : 0, nd = on ? (long long)rs->ndeg : 0;
      const bool sb = on && rs->stop;
      int32_t bo, to, bn, tn;
      long long dbo, dto, dbn, dtn;
      lane_prefix<int32_t>(oc, r, &bo, &to);
      lane_prefix<int32_t>(nc, r, &bn, &tn);
      lane_prefix<long long>(od, r, &dbo, &dto);
      lane_prefix<long long>(nd, r, &dbn, &dtn);
      const bool stp = __any_sync(0xffffffffu, sb);
      if (lane == 0) {
        sm->b_before_o = bo;
        sm->b_total_o = to;
        sm->b_before_n = bn;
        sm->b_total_n = tn;
        sm->b_dbefore_o = dbo;
        sm->b_dtotal_o = dto;
        sm->b_dbefore_n = dbn;
        sm->b_dtotal_n = dtn;
        sm->b_stop = stp ? 1 : 0;
      }
    }
    __syncthreads();
  }
  const int32_t total_s = sm->b_total_s, before_s = sm->b_before_s;
  const int32_t total_o = sm->b_total_o, before_o = sm->b_before_o;
  const int32_t total_n = sm->b_total_n, before_n = sm->b_before_n;
  const long long dtotal_o = sm->b_dtotal_o, dbefore_o = sm->b_dbefore_o;
  const long long dtotal_n = sm->b_dtotal_n, dbefore_n = sm->b_dbefore_n;
  const bool stop_any = sm->b_stop != 0;
  const int32_t min_open = sm->b_min_open;
  if (S.base + total_s > A.cap) {
    __syncthreads();
    if (threadIdx.x == 0) S.status = PUMP_ERR_CAPACITY;
    __syncthreads();
    return;
  }
  const bool has_next = nbk != kNoBucket;
  const int64_t Cn = has_next ? dtotal_o + dtotal_n : 0;
  const int64_t per_n = (Cn + nr - 1) >> log2_nr(nr);  // the next group's candidates per CTA
  const bool small_w = A.w <= 4;
  // survivors to the arena, members among them to the group list
  const int64_t c0 = S.c0, c1 = S.c1;
  const int n = (int)(c1 - c0);
  const bool fits = n <= kCCap;
  // Chunks larger than the cache recompute their candidates from the group list, which this
  // phase overwrites with the next group: then survivors are written first, and after a barrier
  // (taken by every CTA: `big` is the same everywhere) the members are read back from the arena.
  const bool big = S.big != 0;
  const int64_t a0 = S.a0, a1 = S.a1;
  const int no = (int)min(a1 - a0, (int64_t)kCT + 1);
  int64_t run = S.base + before_s;
  int64_t mrun = total_o + before_n;
  int64_t drun = dtotal_o + dbefore_n;
  const bool one_pass = !big && has_next && n + no <= kCT;
  if (one_pass) {
    // cached survivors (threads below n) and cached older plans (threads n .. n + no - 1) in one
    // pass, both lists' positions from one scan round; the state fields used after the scan are
    // read before it, so thread 0 may rewrite the state without a barrier of its own at the end
    const int t = threadIdx.x;
    const int32_t Si = S.i, k1 = S.k + 1;
    bool keep = false, sel = false;
    int32_t eff = -1, x = 0, r0 = 0, odeg = 0;
    float c = 0.f;
    uint4 m = make_uint4(0u, 0u, 0u, 0u);
    CCand q;
    q.x = q.parent = q.edge = q.pc = q.r0 = 0;
    q.dg = 0u;
    q.cost = 0.f;
    if (t < n) {
      eff = sm->ceff[t];
      keep = eff >= 0;
      if (keep) {
        q.x = sm->cx[t];
        q.parent = sm->cpar[t];
        q.edge = sm->cedge[t];
        q.cost = sm->ccost[t];
        q.pc = sm->cpc[t];
        q.r0 = sm->cr0[t];
        q.dg = sm->cdg[t];
      }
    } else if (t < n + no) {
      const int o = t - n;
      sel = sm->oeff[o] == nbk;
      if (sel) {
        x = sm->ox[o];
        c = sm->ocost[o];
        r0 = sm->or0[o];
        odeg = (int32_t)(sm->odg[o] & ~kGoalBit);
        if (small_w) m = sm->omask[o];
      }
    }
    const int32_t deg = (int32_t)(q.dg & ~kGoalBit);
    const bool member = keep && eff == nbk;
    int64_t tk, tpk, rpk;
    const int64_t rk = cscan2<int64_t>((keep ? (int64_t(1) << 52) : 0) | (member ? pack_cd(1, deg) : 0),
                                       sel ? pack_cd(1, odeg) : 0, &tk, &tpk, &rpk);
    if (keep) {
      const int64_t id = run + pack_k(rk);
      const uint4 sm4 = put_survivor(A, sm, id, q, t, true, Si);
      if (member)
        put_member(A, sm, cl, Cn, per_n, k1, mrun + pack_c(rk), drun + pack_d(rk), (int32_t)id, q.x, q.r0, q.cost, deg,
                   sm4);
    }
    if (sel)
      put_member(A, sm, cl, Cn, per_n, k1, before_o + pack_c(rpk), dbefore_o + pack_d(rpk),
                 (int32_t)(a0 + (t - n)), x, r0, c, odeg, m);
  } else {
    for (int t0 = 0; t0 < n; t0 += kCT) {
      const int jl = t0 + threadIdx.x;
      bool keep = false;
      int32_t eff = -1;
      CCand q;
      q.x = q.parent = q.edge = q.pc = q.r0 = 0;
      q.dg = 0u;
      q.cost = 0.f;
      if (jl < n) {
        if (fits) {
          eff = sm->ceff[jl];
          keep = eff >= 0;
          if (keep) {
            q.x = sm->cx[jl];
            q.parent = sm->cpar[jl];
            q.edge = sm->cedge[jl];
            q.cost = sm->ccost[jl];
            q.pc = sm->cpc[jl];
            q.r0 = sm->cr0[jl];
            q.dg = sm->cdg[jl];
          }
        } else {
          q = cand_at_c(A, c0 + jl, S.g, &sm->werr);
          keep = q.pc < A.kmax && !dominated_c<kDsm>(A, cl, mbl, q.x, q.pc, q.cost);
          if (keep) eff = eff_new(sm, A, S.i, q.cost);
        }
      }
      const int32_t deg = (int32_t)(q.dg & ~kGoalBit);
      const bool member = !big && keep && eff == nbk;
      int64_t tk;
      const int64_t rk = cscan<int64_t>((keep ? (int64_t(1) << 52) : 0) | (member ? pack_cd(1, deg) : 0), &tk);
      if (keep) {
        const int64_t id = run + pack_k(rk);
        const uint4 m = put_survivor(A, sm, id, q, jl, fits, S.i);
        if (member)
          put_member(A, sm, cl, Cn, per_n, S.k + 1, mrun + pack_c(rk), drun + pack_d(rk), (int32_t)id, q.x, q.r0,
                     q.cost, deg, m);
      }
      run += pack_k(tk);
      mrun += pack_c(tk);
      drun += pack_d(tk);
    }
    if (big) {
      cl.sync();
      const int32_t mine = sm->pub.surv;
      const int64_t id0 = S.base + before_s;
      for (int t0 = 0; t0 < mine; t0 += kCT) {
        const int k = t0 + threadIdx.x;
        bool sel = false;
        int32_t x = 0, r0 = 0, deg = 0;
        float c = 0.f;
        if (k < mine) {
          c = ldf(A.cost + id0 + k);
          sel = has_next && eff_new(sm, A, S.i, c) == nbk;
          if (sel) {
            x = ld32(A.head + id0 + k);
            r0 = A.row_ptr[x];
            deg = A.row_ptr[x + 1] - r0;
          }
        }
        int64_t tm;
        const int64_t mr = cscan<int64_t>(sel ? pack_cd(1, deg) : 0, &tm);
        if (sel) {
          const uint4 m = small_w ? load_mask4(A.mask + (size_t)(id0 + k) * A.w, A.w) : make_uint4(0u, 0u, 0u, 0u);
          put_member(A, sm, cl, Cn, per_n, S.k + 1, mrun + pack_c(mr), drun + pack_d(mr), (int32_t)(id0 + k), x, r0, c,
                     deg, m);
        }
        mrun += pack_c(tm);
        drun += pack_d(tm);
      }
    }
    // older members (ids below every survivor's) come first in the next group
    if (has_next) {
      const bool ofits = a1 - a0 <= kOCap;
      int64_t orun = before_o, odrun = dbefore_o;
      for (int64_t t0 = a0; t0 < a1; t0 += kCT) {
        const int64_t p = t0 + threadIdx.x;
        bool sel = false;
        int32_t x = 0, r0 = 0, deg = 0;
        float c = 0.f;
        uint4 m = make_uint4(0u, 0u, 0u, 0u);
        if (p < a1) {
          int32_t eff;
          if (ofits) {
            const int o = (int)(p - a0);
            eff = sm->oeff[o];
            if (eff == nbk) {
              x = sm->ox[o];
              c = sm->ocost[o];
              r0 = sm->or0[o];
              deg = (int32_t)(sm->odg[o] & ~kGoalBit);
              if (small_w) m = sm->omask[o];
            }
          } else {
            int32_t pc;
            eff = old_eff_c<kDsm>(A, sm, cl, mbl, p, S.i, &x, &c, &pc);
            if (eff == nbk) {
              r0 = A.row_ptr[x];
              deg = A.row_ptr[x + 1] - r0;
              if (small_w) m = load_mask4(A.mask + (size_t)p * A.w, A.w);
            }
          }
          sel = eff == nbk;
        }
        int64_t tpk;
        const int64_t rpk = cscan<int64_t>(sel ? pack_cd(1, deg) : 0, &tpk);
        if (sel)
          put_member(A, sm, cl, Cn, per_n, S.k + 1, orun + pack_c(rpk), odrun + pack_d(rpk), (int32_t)p, x, r0, c, deg,
                     m);
        orun += pack_c(tpk);
        odrun += pack_d(tpk);
      }
    }
  }
  const int32_t gn = has_next ? total_o + total_n : 0;
  if (r == 0 && threadIdx.x == 0) A.goff[gn] = Cn;
  // next state (the same in every CTA of the cluster) and, if it runs, the next iteration's share;
  // the cluster barrier after this phase publishes both
  if (!one_pass) __syncthreads();
  if (threadIdx.x == 0) {
    S.lo = min((int64_t)min_open, S.base);
    S.base += total_s;
    S.g = gn;
    S.C = Cn;
    S.i = has_next ? nbk : S.i + 1;
    S.stop = A.early_stop && stop_any ? 1 : 0;
    if (sm->b_err) S.status = PUMP_ERR_TIMEOUT;
    if (iter_runs(S, A, S.k + 1)) iter_setup(S, S.k + 1, r, nr);
  }
}

// Dominance table of this CTA's nodes: +inf, and the root's entry (start, 0) = 0.
template <bool kDsm>
__device__ void explore_table_init(const ExploreArgs& A, int32_t start, uint32_t* mbl, int r, int nr) {
  if (!kDsm) return;
  const int rows = (A.n + nr - 1) / nr;
  for (int k = threadIdx.x; k < rows * A.kstride; k += kCT) mbl[k] = 0x7f800000u;  // +inf
  __syncthreads();
  if ((start & (nr - 1)) == r && threadIdx.x == 0) mbl[(size_t)(start >> log2_nr(nr)) * A.kstride] = 0u;
}

// The CTA's search state before group 0.  fresh: the run starts from the root alone (the state
// explore_init_thread writes), derived here instead of read back, and the root is this CTA's
// local member; otherwise the state comes from the control block.
template <bool kDsm>
__device__ void explore_state_init(const ExploreArgs& A, int32_t start, CSmem* sm, int r, int nr, bool fresh,
                                   int32_t ready_row) {
  for (int k = threadIdx.x; k < kMemCap; k += kCT) {
    sm->mt_tag[k] = -1;
    sm->mt_gen[k] = -1;
  }
  __syncthreads();
  St& S = sm->st;
  if (threadIdx.x == 0) {
    sm->slot0 = 0;  // group 0 is the root alone
    sm->slot_end = 0;
    sm->kept = 0;
    sm->werr = 0;
    sm->rows_ready = A.rowcnt ? 0 : 1;
    sm->ready_row = ready_row;
    if (fresh) {
      const int32_t r0 = A.row_ptr[start];
      const int64_t d0 = A.row_ptr[start + 1] - r0;
      S.C = d0;
      S.g = 1;
      S.i = 0;
      S.stop = (A.early_stop && A.is_goal[start] && 0 < A.kmin) ? 1 : 0;
      S.base = 1;
      sm->mt_info[0] = make_int4(0, start, r0, __float_as_int(0.f));
      sm->mt_off[0] = 0;
      sm->mt_deg[0] = (int32_t)d0;
      sm->mt_mask[0] = make_uint4(0u, 0u, 0u, 0u);
      sm->mt_tag[0] = 0;
      sm->mt_gen[0] = 0;
    } else {
      ExploreCtl* ctl = A.ctl;
      S.C = ld64(&ctl->st[0].group_cands);
      S.g = ld32(&ctl->st[0].group_size);
      S.i = ld32(&ctl->st[0].iter);
      S.stop = ld32(&ctl->st[0].stop);
      S.base = ld64(&ctl->n_plans);
    }
    S.lo = 0;
    S.ncand = 0;
    S.status = 0;
    S.n_groups = 0;
    S.k = 0;
    if (iter_runs(S, A, 0)) iter_setup(S, 0, r, nr);
  }
}

// The group loop and the run's results; starts after a cluster barrier that follows the table
// and state initialisation, ends with one.
template <bool kDsm>
__device__ void explore_loop(const ExploreArgs& A, CSmem* sm, uint32_t* mbl, cg::cluster_group& cl) {
  const int r = (int)cl.block_rank();
  ExploreCtl* ctl = A.ctl;
  St& S = sm->st;
  int k = 0;
  for (;; ++k) {
    if (S.status || S.stop || S.g == 0) break;
    // every iteration expands at least one plan that no later group holds, so k is also
    // bounded by the arena; both caps end the run with the same status
    if (S.i >= A.max_iter || k >= A.max_iter) {
      __syncthreads();
      if (threadIdx.x == 0) S.status = PUMP_ERR_TIMEOUT;
      __syncthreads();
      break;
    }
    c_expand<kDsm>(A, sm, mbl, cl, S);
    cl.sync();
    c_filter<kDsm>(A, sm, mbl, cl, S);
    cl.sync();
    c_write<kDsm>(A, sm, mbl, cl, S);
    cl.sync();
  }
  if (threadIdx.x == 0) atomicAdd(reinterpret_cast<unsigned long long*>(&ctl->n_kept), (unsigned long long)sm->kept);
  if (r == 0 && threadIdx.x == 0) {
    ctl->n_plans = S.base;
    ctl->n_candidates = S.ncand;
    ctl->n_groups = S.n_groups;
    ctl->status = S.status;
    ctl->iter = S.i;
    ctl->survivors = 0;
    ctl->k_exit = k;
  }
  cl.sync();  // no CTA leaves (or starts another run) while another may still touch its shared memory
}

// One Explore run by the whole cluster.  Starts and ends with a cluster barrier, so a cluster
// can run several in a row (batched form).
template <bool kDsm>
__device__ void explore_one(const ExploreArgs& A, int32_t start, CSmem* sm, uint32_t* mbl, cg::cluster_group& cl) {
  const int r = (int)cl.block_rank(), nr = (int)cl.num_blocks();
  explore_table_init<kDsm>(A, start, mbl, r, nr);
  explore_state_init<kDsm>(A, start, sm, r, nr, false, -1);
  cl.sync();
  explore_loop<kDsm>(A, sm, mbl, cl);
}

template <bool kDsm>
__global__ void __launch_bounds__(kCT, 1) k_explore_cluster(ExploreArgs A, int32_t start, LaunchShape ls) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (!launch_shape_ok(ls)) {  // every CTA sees the same shape: all leave here
    if (blockIdx.x == 0 && threadIdx.x == 0) A.ctl->status = PUMP_ERR_CUDA;
    return;
  }
  CSmem* sm = reinterpret_cast<CSmem*>(smem_raw);
  uint32_t* mbl = reinterpret_cast<uint32_t*>(smem_raw + ((sizeof(CSmem) + 15) & ~size_t(15)));
  cg::cluster_group cl = cg::this_cluster();
  explore_one<kDsm>(A, start, sm, mbl, cl);
}

// Batched form: every cluster takes the next query from *next (a device counter starting at 0)
// until none is left; query q runs with As[q] and starts[q], exactly as the single-query kernel.
template <bool kDsm>
__global__ void __launch_bounds__(kCT, 1) k_explore_cluster_batch(const ExploreArgs* __restrict__ As,
                                                                  const int32_t* __restrict__ starts, int32_t nq,
                                                                  int32_t* next, LaunchShape ls) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (!launch_shape_ok(ls)) {
    if (blockIdx.x == 0)
      for (int q = threadIdx.x; q < nq; q += kCT) As[q].ctl->status = PUMP_ERR_CUDA;
    return;
  }
  CSmem* sm = reinterpret_cast<CSmem*>(smem_raw);
  uint32_t* mbl = reinterpret_cast<uint32_t*>(smem_raw + ((sizeof(CSmem) + 15) & ~size_t(15)));
  cg::cluster_group cl = cg::this_cluster();
  const int r = (int)cl.block_rank(), nr = (int)cl.num_blocks();
  constexpr int kArgWords = sizeof(ExploreArgs) / 4;
  static_assert(sizeof(ExploreArgs) % 4 == 0, "argument copy");
  for (;;) {
    if (r == 0 && threadIdx.x == 0) {
      const int32_t q = atomicAdd(next, 1);
      for (int rr = 0; rr < nr; ++rr) *cl.map_shared_rank(&sm->qnext, (unsigned)rr) = q;
    }
    cl.sync();
    const int32_t q = sm->qnext;
    if (q >= nq) break;
    const uint32_t* src = reinterpret_cast<const uint32_t*>(As + q);
    for (int t = threadIdx.x; t < kArgWords; t += kCT) reinterpret_cast<uint32_t*>(&sm->args)[t] = src[t];
    __syncthreads();
    explore_one<kDsm>(sm->args, starts[q], sm, mbl, cl);
  }
  cl.sync();  // the last query index was read everywhere before any CTA leaves
}

// ---------------------------------------------------------------- fused form
// Mask workers' arguments: the query pass's inputs and the order they take the edges in.
struct FuseArgs {
  const float4* xp;          // pair-major normals (maskdev::pair_count)
  const float* phi;          // E x 4
  const float* L;            // E x 3
  const float* nom;          // E x W x 3
  const float* linf;         // 3
  const float* ibox;         // E x 6
  const unsigned int* dmax;  // E
  const float* boxes;        // nb x 6
  const int2* eorder;        // E: (edge, source row) in the order the workers take them
  uint32_t* emask;           // E x w (written)
  uint32_t* rowcnt;          // n + 1: finished edges per row, then worker warps finished (both
                             // accumulated over runs)
  unsigned long long* wctr;  // positions taken by the workers, accumulated over runs
  int32_t N, W, nb, E, w, n;
  int32_t xi_smem;           // the normals fit in shared memory next to the boxes
  int32_t hold_row;          // test hook: this row is never counted (-1: none)
  int32_t* goal_sorted;      // P_goal in PlanSelection order (written after Explore, CTA 0)
};

// Shared memory a worker CTA uses (boxes, per-warp scratch, normals when they fit).
__host__ __device__ constexpr size_t worker_smem(int nb, int N, int W, bool xi_smem) {
  return maskdev::fixed_smem(nb, kCW) +
         (xi_smem ? sizeof(float4) * (size_t)(W + 1) * 3 * maskdev::pair_count(N / 32) * 32 : 0);
}

#ifndef PUMP_FUSED_MASK_NP
#define PUMP_FUSED_MASK_NP 1  // word pairs side by side per pass in the fused kernel (1: no spills beside Explore)
#endif
constexpr int kWorkChunk = 2;  // positions a worker warp takes at a time

// Mask of the edge at position q of the order, then its count toward its row by a release add
// after the warp barrier.
__device__ __forceinline__ void mask_position(const FuseArgs& F, const float4* xp, const float (&linf)[3],
                                              const float* boxes, int* my_cand, uint32_t* wm, int lane, long long q) {
  const int2 ex = __ldg(F.eorder + q);
  maskdev::edge_mask_one<PUMP_FUSED_MASK_NP>(ex.x, xp, F.N, F.W, F.phi, F.L, F.nom, linf, F.ibox, F.dmax, boxes,
                                             F.nb, F.w, my_cand, wm, lane, F.emask);
  __syncwarp();
  if (lane == 0 && ex.y != F.hold_row) red_release_add(F.rowcnt + ex.y, 1u);
}

// Prologue of the fused launch (Explore cluster, before group 0): positions [0, head) of the order,
// which are the start row's edges r0s, r0s + 1, ... (its row comes first), position q on CTA
// q mod nr, each of its word pairs on its own warp (half a warp's chain per task for N = 128),
// the CTA's positions counted toward the start row after its tasks are done.
__device__ __forceinline__ void mask_prologue(const FuseArgs& F, unsigned char* smem, long long head, int32_t start,
                                              int32_t r0s, int r, int nr) {
  float* boxes = reinterpret_cast<float*>(smem);
  int* cand = reinterpret_cast<int*>(boxes + maskdev::kBoxStride * F.nb);
  uint32_t* wmask_all = reinterpret_cast<uint32_t*>(cand + kCW * maskdev::kCandCap);
  float4* xp_s = reinterpret_cast<float4*>(smem + maskdev::fixed_smem(F.nb, kCW));
  const int xp_n = (F.W + 1) * 3 * maskdev::pair_count(F.w) * 32;
  maskdev::stage(F.boxes, F.nb, boxes, F.xp, F.xi_smem ? xp_s : nullptr, xp_n);
  __syncthreads();
  const float4* xp = F.xi_smem ? xp_s : F.xp;
  const float linf[3] = {F.linf[0], F.linf[1], F.linf[2]};
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int* my_cand = cand + warp * maskdev::kCandCap;
  uint32_t* wm = wmask_all + warp * kMaxWaypoints;
  const int npair = maskdev::pair_count(F.w);
  const long long mine = head > r ? (head - r + nr - 1) / nr : 0;  // positions r, r + nr, ... below head
  for (long long t = warp; t < mine * npair; t += kCW) {
    const long long q = r + (t / npair) * nr;
    const int pr = (int)(t % npair);
    maskdev::edge_mask_one<PUMP_FUSED_MASK_NP>(r0s + q, xp, F.N, F.W, F.phi, F.L, F.nom, linf, F.ibox, F.dmax, boxes,
                                               F.nb, F.w, my_cand, wm, lane, F.emask, pr, pr + 1);
  }
  __syncthreads();
  if (threadIdx.x == 0 && mine > 0 && start != F.hold_row) {
    __threadfence();
    red_release_add(F.rowcnt + start, (uint32_t)mine);
  }
}

// The block stages the boxes (and the normals, when they fit) in shared memory.  Then either
// positions q0 + v, q0 + v + V, ... below q1 (warp v of V; `dynamic` false), or, with `dynamic`,
// chunks of kWorkChunk positions from [q0, q1) in increasing order from the run's counter: run e
// of a graph takes increments (e - 1) x per_run onward, per_run being the increments every run
// makes (each worker warp takes chunks until one starts at or past q1).  A worker warp counts
// itself done at the end.
__device__ __forceinline__ void mask_positions(const FuseArgs& F, unsigned char* smem, long long q0, long long q1,
                                               long long v, long long V, bool dynamic, uint32_t epoch_m1,
                                               long long n_workers) {
  float* boxes = reinterpret_cast<float*>(smem);
  int* cand = reinterpret_cast<int*>(boxes + maskdev::kBoxStride * F.nb);
  uint32_t* wmask_all = reinterpret_cast<uint32_t*>(cand + kCW * maskdev::kCandCap);
  float4* xp_s = reinterpret_cast<float4*>(smem + maskdev::fixed_smem(F.nb, kCW));
  const int xp_n = (F.W + 1) * 3 * maskdev::pair_count(F.w) * 32;
  maskdev::stage(F.boxes, F.nb, boxes, F.xp, F.xi_smem ? xp_s : nullptr, xp_n);
  __syncthreads();
  const float4* xp = F.xi_smem ? xp_s : F.xp;
  const float linf[3] = {F.linf[0], F.linf[1], F.linf[2]};
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int* my_cand = cand + warp * maskdev::kCandCap;
  uint32_t* wm = wmask_all + warp * kMaxWaypoints;
  if (!dynamic) {
    for (long long q = q0 + v; q < q1; q += V) mask_position(F, xp, linf, boxes, my_cand, wm, lane, q);
    return;
  }
  const unsigned long long chunks = (unsigned long long)((max(q1 - q0, 0ll) + kWorkChunk - 1) / kWorkChunk);
  const unsigned long long per_run = (chunks + (unsigned long long)n_workers) * kWorkChunk;
  const unsigned long long base = (unsigned long long)epoch_m1 * per_run;
  for (;;) {
    unsigned long long t = 0;
    if (lane == 0) t = atomicAdd(F.wctr, (unsigned long long)kWorkChunk);
    t = __shfl_sync(0xffffffffu, t, 0) - base;
    const long long qa = q0 + (long long)t;
    if (t >= (unsigned long long)(q1 - q0) || qa >= q1) break;
    const long long qb = min(q1, qa + kWorkChunk);
    for (long long q = qa; q < qb; ++q) mask_position(F, xp, linf, boxes, my_cand, wm, lane, q);
  }
  if (lane == 0) red_release_add(F.rowcnt + F.n, 1u);  // this warp's edges are counted
}

// Masks and Explore in one cooperative launch: cluster 0 runs Explore (A.rowcnt set), the
// other clusters are mask workers.  The first positions of the order (the start row, one edge per
// warp on different SMs) are computed by the Explore cluster itself before it starts, so group 0
// does not wait for the workers' first edges; the workers take the rest.
// Cluster 0 also writes the run's initial state first and P_goal's order last.
template <bool kDsm>
__global__ void __launch_bounds__(kCT, 1) k_explore_fused(ExploreArgs A, int32_t start, FuseArgs F, LaunchShape ls) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (!launch_shape_ok(ls)) {  // refused before any shared memory or count is touched
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      explore_init_thread(A, start);
      A.ctl->status = PUMP_ERR_CUDA;
    }
    return;
  }
  cg::cluster_group cl = cg::this_cluster();
  const int nr = (int)cl.num_blocks();
  // positions [0, head) (the start row's out-degree: the start's row comes first in the order)
  // are computed by the Explore cluster before group 0, the rest by the workers
  const int32_t r0s = __ldg(A.row_ptr + start);
  const long long head = min((long long)F.E, (long long)(__ldg(A.row_ptr + start + 1) - r0s));
  if ((int)blockIdx.x < nr) {
    const int r = (int)cl.block_rank();
    CSmem* sm = reinterpret_cast<CSmem*>(smem_raw);
    const size_t mbl_off = (sizeof(CSmem) + 15) & ~size_t(15);
    uint32_t* mbl = reinterpret_cast<uint32_t*>(smem_raw + mbl_off);
    // shared memory serves as the prologue's mask scratch first (from offset 0); when that ends
    // below the dominance table, the table is set up before the prologue and one cluster barrier
    // closes both, every CTA deriving the root state itself (the start row's masks are complete
    // at that barrier, so group 0 does not wait for them)
    const size_t pro_end = maskdev::fixed_smem(F.nb, kCW) +
                           (F.xi_smem ? sizeof(float4) * (size_t)(F.W + 1) * 3 * maskdev::pair_count(F.w) * 32 : 0);
    const bool early = pro_end <= mbl_off;
    if (early) explore_table_init<kDsm>(A, start, mbl, r, nr);
    // the run's initial state in global memory (root plan, control block), read after a barrier
    if (blockIdx.x == 0 && threadIdx.x == 0) explore_init_thread(A, start);
    mask_prologue(F, smem_raw, head, start, r0s, r, nr);
    if (early) {
      __syncthreads();
    } else {
      cl.sync();
      explore_table_init<kDsm>(A, start, mbl, r, nr);
    }
    // (the test hook that withholds a row's count keeps that row's waits)
    explore_state_init<kDsm>(A, start, sm, r, nr, early, early && start != F.hold_row ? start : -1);
    cl.sync();
    explore_loop<kDsm>(A, sm, mbl, cl);
    // P_goal in PlanSelection order (the loop ends with a cluster barrier: every plan written)
    if (blockIdx.x == 0) goal_finalize_block(A, A.group, F.goal_sorted);
    return;
  }
  const long long nwb = (long long)gridDim.x - nr;
  mask_positions(F, smem_raw, head, F.E, 0, 0, true, A.epoch_m1, nwb * kCW);
}

// Row order of the fused form.  Shortest-path cost from the start over the graph's edges
// (float sums; an ordering key only), by label-correcting rounds inside one thread-block cluster
// (hardware cluster barriers between rounds): a warp per node whose cost fell in the previous
// round relaxes its out-edges (atomicMin on the float bits, which order like the non-negative
// costs).  changed[r mod 3] says whether round r has work; every thread reads it after the same
// barrier, so all leave together.  At most max_rounds rounds (rows still unreached sort last).
__global__ void __launch_bounds__(1024, 1) k_sssp(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                                  const float* __restrict__ ecost, int32_t n, int32_t start,
                                                  uint32_t* dist, uint8_t* fa, uint8_t* fb, int32_t* changed,
                                                  int32_t max_rounds) {
  cg::cluster_group cl = cg::this_cluster();
  const long long tid = (long long)cl.block_rank() * blockDim.x + threadIdx.x;
  const long long nt = (long long)cl.num_blocks() * blockDim.x;
  for (long long x = tid; x < n; x += nt) {
    dist[x] = x == start ? 0u : 0x7f800000u;
    fa[x] = x == start ? 1 : 0;
    fb[x] = 0;
  }
  if (tid < 3) changed[tid] = tid == 0 ? 1 : 0;
  cl.sync();
  const int lane = threadIdx.x & 31;
  const long long gw = tid >> 5, nw = nt >> 5;
  for (int r = 0; r < max_rounds; ++r) {
    if (__ldcg(changed + r % 3) == 0) break;
    uint8_t* cur = (r & 1) ? fb : fa;
    uint8_t* nxt = (r & 1) ? fa : fb;
    bool any = false;
    // a warp takes 32 consecutive nodes at a time: their flags and row bounds in one load each
    for (long long b = gw * 32; b < n; b += nw * 32) {
      const long long xl = b + lane;
      const bool on = xl < n && __ldcg(cur + xl) != 0;
      const int32_t r0l = on ? row_ptr[xl] : 0, r1l = on ? row_ptr[xl + 1] : 0;
      const float dl = on ? __uint_as_float(__ldcg(dist + xl)) : 0.f;
      if (on) cur[xl] = 0;
      // the flagged nodes' out-edges as one list (warp scan of their degrees); lanes take list
      // positions k, k + 32, ... so the loads of all of them are in flight together
      const int32_t degl = r1l - r0l;
      int32_t incl = degl;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      const int32_t total = __shfl_sync(0xffffffffu, incl, 31);
      for (int32_t k0 = 0; k0 < total; k0 += 32) {
        const int32_t k = k0 + lane;
        // source lane: the least lane whose inclusive prefix exceeds k
        int lo = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
          const int32_t v = __shfl_sync(0xffffffffu, incl, lo + step - 1);
          if (v <= k) lo += step;
        }
        const int32_t before = __shfl_sync(0xffffffffu, incl - degl, lo);
        const int32_t e0 = __shfl_sync(0xffffffffu, r0l, lo);
        const float dx = __shfl_sync(0xffffffffu, dl, lo);
        if (k < total) {
          const int32_t e = e0 + (k - before);
          const int32_t y = col[e];
          const uint32_t nd = __float_as_uint(__fadd_rn(dx, ecost[e]));
          if (nd < atomicMin(dist + y, nd)) {
            nxt[y] = 1;
            any = true;
          }
        }
      }
    }
    if (__any_sync(0xffffffffu, any) && lane == 0) changed[(r + 1) % 3] = 1;
    if (tid == 0) changed[(r + 2) % 3] = 0;
    cl.sync();
  }
}

constexpr int kOrderBuckets = 4096;
constexpr int kSsspRounds = 64;  // label-correcting rounds of the row order (converged in 11 on the indoor graph)
constexpr int kOrderThreads = 1024;

// Exclusive prefix of one value per thread over a kOrderThreads block; *tot gets the sum.
__device__ int32_t order_scan(int32_t v, int32_t* wsum, int32_t* tot) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int32_t w = wsum[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    wsum[lane] = w;
  }
  __syncthreads();
  const int32_t pre = (warp > 0 ? wsum[warp - 1] : 0) + x - v;
  *tot = wsum[31];
  __syncthreads();
  return pre;
}

// Rows by increasing cost (the start's row alone first, then a counting sort on the cost quantised
// to kOrderBuckets - 2 levels over [0, largest finite cost]; unreachable rows last; order inside a
// level unspecified), and the exclusive prefix of their out-degrees (n + 1 entries).  One block of
// kOrderThreads threads.
__global__ void __launch_bounds__(kOrderThreads) k_row_order(const uint32_t* __restrict__ dist,
                                                             const int32_t* __restrict__ row_ptr, int32_t n,
                                                             int32_t start, int32_t* __restrict__ order,
                                                             int32_t* __restrict__ epos) {
  __shared__ int32_t hist[kOrderBuckets];
  __shared__ float s_max[32];
  __shared__ int32_t wsum[32];
  constexpr int kPer = kOrderBuckets / kOrderThreads;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  float m = 0.f;
  for (int32_t x = t; x < n; x += kOrderThreads) {
    const float d = __uint_as_float(dist[x]);
    if (d < __int_as_float(0x7f800000)) m = fmaxf(m, d);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) s_max[warp] = m;
  for (int b = t; b < kOrderBuckets; b += kOrderThreads) hist[b] = 0;
  __syncthreads();
  m = 0.f;
  for (int k = 0; k < 32; ++k) m = fmaxf(m, s_max[k]);
  const float scale = m > 0.f ? (float)(kOrderBuckets - 3) / m : 0.f;
  auto level = [&](int32_t x) {
    if (x == start) return 0;
    const float d = __uint_as_float(dist[x]);
    if (!(d < __int_as_float(0x7f800000))) return kOrderBuckets - 1;
    return 1 + min(kOrderBuckets - 3, (int)(d * scale));
  };
  for (int32_t x = t; x < n; x += kOrderThreads) atomicAdd(&hist[level(x)], 1);
  __syncthreads();
  {  // exclusive prefix over the levels, kPer consecutive levels per thread
    int32_t c[kPer], sum = 0;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      c[k] = hist[t * kPer + k];
      sum += c[k];
    }
    int32_t tot;
    int32_t run = order_scan(sum, wsum, &tot);
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      hist[t * kPer + k] = run;
      run += c[k];
    }
  }
  __syncthreads();
  for (int32_t x = t; x < n; x += kOrderThreads) order[atomicAdd(&hist[level(x)], 1)] = x;
  __syncthreads();
  // exclusive prefix of the out-degrees in that order, kOrderThreads rows at a time
  int32_t carry = 0;
  for (int32_t j0 = 0; j0 < n; j0 += kOrderThreads) {
    const int32_t j = j0 + t;
    const int32_t deg = j < n ? row_ptr[order[j] + 1] - row_ptr[order[j]] : 0;
    int32_t tot;
    const int32_t pre = order_scan(deg, wsum, &tot);
    if (j < n) epos[j] = carry + pre;
    carry += tot;
  }
  if (t == 0) epos[n] = carry;
}

// Edge order: row order[j]'s edges at positions epos[j] .. epos[j+1] - 1, a warp per row.
__global__ void k_edge_order(const int32_t* __restrict__ order, const int32_t* __restrict__ epos,
                             const int32_t* __restrict__ row_ptr, int32_t n, int2* __restrict__ eorder) {
  const int lane = threadIdx.x & 31;
  for (long long j = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < n;
       j += ((long long)gridDim.x * blockDim.x) >> 5) {
    const int32_t x = order[j];
    const int32_t r0 = row_ptr[x], deg = row_ptr[x + 1] - r0, base = epos[j];
    for (int32_t k = lane; k < deg; k += 32) eorder[base + k] = make_int2(r0 + k, x);
  }
}

// Per edge: target node, edge cost bits, target row start, target out-degree | goal bit.
__global__ void k_edge_targets(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                               const float* __restrict__ ecost, const uint8_t* __restrict__ is_goal, int32_t E,
                               int4* __restrict__ out) {
  for (int32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < E; e += gridDim.x * blockDim.x) {
    const int32_t x = col[e];
    const int32_t r0 = row_ptr[x];
    const uint32_t dg = (uint32_t)(row_ptr[x + 1] - r0) | (is_goal[x] ? kGoalBit : 0u);
    out[e] = make_int4(x, __float_as_int(ecost[e]), r0, (int32_t)dg);
  }
}

size_t cluster_smem_bytes(int n, int kstride, int nr, bool dsm) {
  size_t b = (sizeof(CSmem) + 15) & ~size_t(15);
  if (dsm) b += sizeof(uint32_t) * (size_t)((n + nr - 1) / nr) * kstride;
  return b;
}

template <bool kDsm>
int try_cluster_size(int nr, size_t smem, cudaStream_t s, cudaLaunchConfig_t* cfg, cudaLaunchAttribute* attr) {
  auto kern = k_explore_cluster<kDsm>;
  auto bkern = k_explore_cluster_batch<kDsm>;
  if (cudaFuncSetAttribute(bkern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDynSmemMax) != cudaSuccess ||
      cudaFuncSetAttribute(bkern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  // one ceiling for every configuration (the attribute belongs to the kernel, not to a launch)
  if (smem > kDynSmemMax ||
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDynSmemMax) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (nr > 8 && cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  cfg->gridDim = dim3(nr);
  cfg->blockDim = dim3(kCT);
  cfg->dynamicSmemBytes = smem;
  cfg->stream = s;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = nr;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg->attrs = attr;
  cfg->numAttrs = 1;
  int nclusters = 0;
  if (cudaOccupancyMaxActiveClusters(&nclusters, kern, cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nclusters;
}

// Cluster size: PUMP_EXPLORE_CLUSTER overrides (0 disables the cluster kernel), and
// PUMP_EXPLORE_MBEST_GLOBAL=1 keeps the dominance table in global memory.  Both are read on
// every call (tuning and tests).
int cluster_env() {
  const char* e = getenv("PUMP_EXPLORE_CLUSTER");
  return e ? atoi(e) : -1;
}

bool mbest_global_env() {
  const char* e = getenv("PUMP_EXPLORE_MBEST_GLOBAL");
  return e && atoi(e) != 0;
}

// Cluster form for a run: size and where mbest lives.  The device check (attributes and the
// occupancy query) is done once per device and configuration and remembered.
struct ClusterChoice {
  int dev, nr, kstride_rows;  // key: device, cluster size, mbest words per CTA (0: global)
  size_t smem;
  int ok;
};

std::mutex g_choice_mu;
std::vector<ClusterChoice> g_choices;

int cluster_ok(int dev, int nr, bool dsm, size_t smem, int words) {
  {
    std::lock_guard<std::mutex> lk(g_choice_mu);
    for (const auto& c : g_choices)
      if (c.dev == dev && c.nr == nr && c.kstride_rows == (dsm ? words : 0) && c.smem == smem) return c.ok;
  }
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  const int ok = (dsm ? try_cluster_size<true>(nr, smem, 0, &cfg, attr) : try_cluster_size<false>(nr, smem, 0, &cfg, attr)) >= 1;
  std::lock_guard<std::mutex> lk(g_choice_mu);
  g_choices.push_back({dev, nr, dsm ? words : 0, smem, ok ? 1 : 0});
  return ok;
}

}  // namespace

// Edge targets of a graph (computed once; the graph's arrays do not change afterwards).
int ensure_edge_targets(pump_graph* g, cudaStream_t s) {
  if (g->etgt || g->E == 0) return PUMP_OK;
  g->etgt = (int4*)graph_alloc(g, sizeof(int4) * (size_t)g->E, s);
  if (!g->etgt) return PUMP_ERR_OOM;
  const int blocks = (int)std::min<int64_t>(((int64_t)g->E + 255) / 256, 4096);
  k_edge_targets<<<blocks, 256, 0, s>>>(g->row_ptr, g->col, g->ecost, g->is_goal, g->E, g->etgt);
  note_launch();
  PUMP_CUDA_TRY(cudaGetLastError());
  return PUMP_OK;
}

// Picks the cluster form: *nr = cluster size (0 when no cluster form fits the device) and *dsm =
// mbest in distributed shared memory, for tables of n nodes x kstride.  want_nr > 0 asks for one
// size (0: 16, else 8, else 4; the PUMP_EXPLORE_CLUSTER environment variable overrides it) and
// want_global keeps mbest in global memory.
int plan_cluster_form(int32_t n, int32_t kstride, int want_nr, bool want_global, int* nr_out, bool* dsm_out,
                      size_t* smem_out) {
  *nr_out = 0;
  *dsm_out = false;
  const int env = cluster_env();
  if (env == 0) return PUMP_OK;
  int sizes[3] = {16, 8, 4};
  int n_sizes = 3;
  const int want = env > 0 ? env : want_nr;
  if (want > 0) {
    if (want > kMaxCluster || (want & (want - 1))) return PUMP_OK;  // the kernels need a power of two
    sizes[0] = want;
    n_sizes = 1;
  }
  int dev = 0;
  PUMP_CUDA_TRY(cudaGetDevice(&dev));
  const size_t fixed = cluster_smem_bytes(n, kstride, 1, false);
  for (int t = 0; t < n_sizes; ++t) {
    const int nr = sizes[t];
    const int words = ((n + nr - 1) / nr) * kstride;
    const bool dsm = !want_global && !mbest_global_env() && fixed + sizeof(uint32_t) * (size_t)words + 4096 <= kSmemLimit;
    const size_t smem = cluster_smem_bytes(n, kstride, nr, dsm);
    if (cluster_ok(dev, nr, dsm, smem, words)) {
      *nr_out = nr;
      *dsm_out = dsm;
      if (smem_out) *smem_out = smem;
      return PUMP_OK;
    }
  }
  return PUMP_OK;
}

int plan_explore_cluster(const ExploreArgs& A, int* nr_out, bool* dsm_out) {
  return plan_cluster_form(A.n, A.kstride, 0, false, nr_out, dsm_out, nullptr);
}

static void cluster_config(cudaLaunchConfig_t* cfg, cudaLaunchAttribute* attr, int nr, int n_clusters, size_t smem,
                           cudaStream_t s) {
  *cfg = cudaLaunchConfig_t{};
  cfg->gridDim = dim3(nr * n_clusters);
  cfg->blockDim = dim3(kCT);
  cfg->dynamicSmemBytes = smem;
  cfg->stream = s;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = nr;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg->attrs = attr;
  cfg->numAttrs = 1;
}

// Launches the cluster kernel in the form plan_explore_cluster chose.
int run_explore_cluster(pump_graph* g, const ExploreArgs& A, int nr, bool dsm, cudaStream_t s) {
  const size_t smem = cluster_smem_bytes(A.n, A.kstride, nr, dsm);
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  cluster_config(&cfg, attr, nr, 1, smem, s);
  const int32_t start = g->start;
  cudaError_t e;
  const LaunchShape ls{nr, (uint32_t)smem};
  if (dsm)
    e = cudaLaunchKernelEx(&cfg, k_explore_cluster<true>, A, start, ls);
  else
    e = cudaLaunchKernelEx(&cfg, k_explore_cluster<false>, A, start, ls);
  note_launch();
  return e == cudaSuccess ? PUMP_OK : PUMP_ERR_CUDA;
}

// Clusters of the batched kernel that fit on the device at once for this form.
int cluster_capacity(int nr, bool dsm, size_t smem, int* out) {
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  *out = dsm ? try_cluster_size<true>(nr, smem, 0, &cfg, attr) : try_cluster_size<false>(nr, smem, 0, &cfg, attr);
  return PUMP_OK;
}

// Batched launch: n_clusters clusters of nr CTAs take queries from *next until nq are done.
int run_explore_cluster_batch(const ExploreArgs* As_dev, const int32_t* starts_dev, int32_t nq, int nr, bool dsm,
                              size_t smem, int n_clusters, int32_t* next_dev, cudaStream_t s) {
  PUMP_CUDA_TRY(cudaMemsetAsync(next_dev, 0, sizeof(int32_t), s));
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  cluster_config(&cfg, attr, nr, n_clusters, smem, s);
  cudaError_t e;
  const LaunchShape ls{nr, (uint32_t)smem};
  if (dsm)
    e = cudaLaunchKernelEx(&cfg, k_explore_cluster_batch<true>, As_dev, starts_dev, nq, next_dev, ls);
  else
    e = cudaLaunchKernelEx(&cfg, k_explore_cluster_batch<false>, As_dev, starts_dev, nq, next_dev, ls);
  note_launch();
  return e == cudaSuccess ? PUMP_OK : PUMP_ERR_CUDA;
}

bool fused_masks_env() {
  const char* e = getenv("PUMP_FUSED_MASKS");
  return !(e && atoi(e) == 0);
}

// Side stream of the calling host thread (one per device, highest priority, so its blocks are
// placed first when the graph build's own kernels become ready with them) and its two events.
struct SideStream {
  int dev = -1;
  cudaStream_t s = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
};
static SideStream* side_stream() {
  struct Holder {
    std::vector<SideStream> v;
    ~Holder() {  // the thread ends (a server worker): release its streams and events
      for (auto& x : v) {
        int cur = 0;
        if (cudaGetDevice(&cur) != cudaSuccess) break;
        cudaSetDevice(x.dev);
        cudaEventDestroy(x.fork);
        cudaEventDestroy(x.join);
        cudaStreamDestroy(x.s);
        cudaSetDevice(cur);
      }
      cudaGetLastError();
    }
  };
  thread_local Holder h;
  std::vector<SideStream>& v = h.v;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  for (auto& x : v)
    if (x.dev == dev) return &x;
  SideStream x;
  x.dev = dev;
  int lo = 0, hi = 0;
  if (cudaDeviceGetStreamPriorityRange(&lo, &hi) != cudaSuccess ||
      cudaStreamCreateWithPriority(&x.s, cudaStreamNonBlocking, hi) != cudaSuccess ||
      cudaEventCreateWithFlags(&x.fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&x.join, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  v.push_back(x);
  return &v.back();
}

// Row order of the fused form, once per graph (its arrays do not change afterwards): costs from
// the start (k_sssp, one cluster), rows sorted by them, edges in that row order.  The kernels
// run on stream `ks`; the memory comes from stream s.  row_order_begin starts them (on the
// calling thread's side stream when `overlap`, after the work already on s), row_order_end
// makes s wait for them and keeps the result.  Where the device cannot run the cluster pass,
// nothing is kept and the fused form is not used.
int row_order_begin(pump_graph* g, cudaStream_t s, bool overlap) {
  if (g->eorder || g->order_scratch || g->E == 0 || g->hsmc) return PUMP_OK;
  const int32_t n = g->n;
  // one graph allocation (edge order, then the counts) and one scratch allocation: an allocator
  // call can cost more than these kernels
  const size_t eo_bytes = (sizeof(int2) * (size_t)g->E + 255) & ~size_t(255);
  unsigned char* keep = (unsigned char*)graph_alloc(g, eo_bytes + sizeof(uint32_t) * ((size_t)n + 1), s);
  const size_t n4 = ((size_t)n + 64) & ~size_t(63);  // 4-byte words per n-sized part, padded
  uint32_t* scratch = (uint32_t*)dev_alloc(sizeof(uint32_t) * (3 * n4 + 64) + 2 * n4 + 64, s);
  if (!keep || !scratch) {
    if (scratch) dev_free(scratch, s);
    return PUMP_ERR_OOM;
  }
  int2* eo = reinterpret_cast<int2*>(keep);
  uint32_t* dist = scratch;
  int32_t* order = reinterpret_cast<int32_t*>(scratch + n4);
  int32_t* epos = reinterpret_cast<int32_t*>(scratch + 2 * n4);
  int32_t* changed = reinterpret_cast<int32_t*>(scratch + 3 * n4);
  uint8_t* fa = reinterpret_cast<uint8_t*>(scratch + 3 * n4 + 64);
  uint8_t* fb = fa + n;
  SideStream* side = overlap ? side_stream() : nullptr;
  cudaStream_t ks = s;
  if (side && cudaEventRecord(side->fork, s) == cudaSuccess && cudaStreamWaitEvent(side->s, side->fork, 0) == cudaSuccess)
    ks = side->s;
  cudaGetLastError();
  int32_t nn = n, start = g->start, max_rounds = kSsspRounds;
  // one cluster: 16 CTAs where the device co-schedules them, else 8
  cudaError_t e = cudaErrorUnknown;
  for (int nr : {16, 8}) {
    if (nr > 8 && cudaFuncSetAttribute(k_sssp, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.gridDim = dim3(nr);
    cfg.blockDim = dim3(1024);
    cfg.stream = ks;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = nr;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, k_sssp, g->row_ptr, g->col, g->ecost, nn, start, dist, fa, fb, changed, max_rounds);
    if (e == cudaSuccess) break;
    cudaGetLastError();
  }
  if (e == cudaSuccess) {
    note_launch();
    k_row_order<<<1, kOrderThreads, 0, ks>>>(dist, g->row_ptr, n, g->start, order, epos);
    note_launch();
    const int eb = (int)std::min<int64_t>(((int64_t)n * 32 + 255) / 256, 4096);
    k_edge_order<<<eb, 256, 0, ks>>>(order, epos, g->row_ptr, n, eo);
    note_launch();
  }
  const bool launched = e == cudaSuccess && cudaGetLastError() == cudaSuccess;
  if (ks != s) {  // s waits for the side stream at row_order_end (the scratch stays until then)
    PUMP_CUDA_TRY(cudaEventRecord(side->join, ks));
    g->order_join = side->join;
  }
  g->order_scratch = scratch;
  g->order_keep = launched ? keep : nullptr;
  return PUMP_OK;
}

int row_order_end(pump_graph* g, cudaStream_t s) {
  if (!g->order_scratch) return PUMP_OK;
  if (g->order_join) PUMP_CUDA_TRY(cudaStreamWaitEvent(s, g->order_join, 0));
  g->order_join = nullptr;
  dev_free(g->order_scratch, s);
  g->order_scratch = nullptr;
  if (g->order_keep) {
    const size_t eo_bytes = (sizeof(int2) * (size_t)g->E + 255) & ~size_t(255);
    g->eorder = reinterpret_cast<int2*>(g->order_keep);
    g->rowcnt = reinterpret_cast<uint32_t*>(static_cast<unsigned char*>(g->order_keep) + eo_bytes);
    g->order_keep = nullptr;
  }
  return PUMP_OK;
}

// The order for a graph that has none yet (on s).
static int ensure_row_order(pump_graph* g, cudaStream_t s, bool* ok) {
  int rc = row_order_begin(g, s, false);
  if (!rc) rc = row_order_end(g, s);
  *ok = g->eorder != nullptr;
  return rc;
}

// Fused form per device and shared-memory size: clusters the kernel can keep resident at once
// (0: the form does not apply), found once.
struct FusedChoice {
  int dev;
  size_t smem;
  int clusters;
};
std::mutex g_fused_mu;
std::vector<FusedChoice> g_fused;

static int fused_clusters(int dev, int nr, size_t smem) {
  {
    std::lock_guard<std::mutex> lk(g_fused_mu);
    for (const auto& c : g_fused)
      if (c.dev == dev && c.smem == smem) return c.clusters;
  }
  int ncl = 0;
  auto kern = k_explore_fused<true>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDynSmemMax) == cudaSuccess &&
      cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    cluster_config(&cfg, attr, nr, 1, smem, 0);
    if (cudaOccupancyMaxActiveClusters(&ncl, kern, &cfg) != cudaSuccess) ncl = 0;
  }
  cudaGetLastError();
  if (ncl < 2) ncl = 0;
  std::lock_guard<std::mutex> lk(g_fused_mu);
  g_fused.push_back({dev, smem, ncl});
  return ncl;
}

static void fused_disable(int dev, size_t smem) {
  std::lock_guard<std::mutex> lk(g_fused_mu);
  for (auto& c : g_fused)
    if (c.dev == dev && c.smem == smem) c.clusters = 0;
}

// Masks and Explore in one cooperative launch (k_explore_fused): cluster 0 explores, every other
// co-resident cluster computes masks.  *launched = false, with nothing of the run enqueued,
// where the form does not apply (box masks, mbest on chip, a second cluster resident, the edge
// order available); the caller then runs the separate launches.
int run_explore_fused(pump_graph* g, const ExploreArgs& A0, int nr, bool dsm, cudaStream_t s, bool* launched) {
  *launched = false;
  if (!dsm || g->hsmc || g->E == 0 || !g->has_geometry) return PUMP_OK;
  const bool xi_smem = worker_smem(g->n_boxes, g->N, g->W, true) <= kDynSmemMax;
  const size_t smem = std::max(cluster_smem_bytes(A0.n, A0.kstride, nr, dsm),
                               worker_smem(g->n_boxes, g->N, g->W, xi_smem));
  if (smem > kDynSmemMax) return PUMP_OK;
  int dev = 0;
  PUMP_CUDA_TRY(cudaGetDevice(&dev));
  const int ncl = fused_clusters(dev, nr, smem);
  if (ncl < 2) return PUMP_OK;
  bool ok = false;
  int rc = ensure_row_order(g, s, &ok);
  if (rc || !ok) return rc;
  // counts accumulate over runs (no clearing per run); zeroed after a run that may have left
  // them short
  if (g->rowcnt_dirty) {
    PUMP_CUDA_TRY(cudaMemsetAsync(g->rowcnt, 0, sizeof(uint32_t) * ((size_t)g->n + 1), s));
    PUMP_CUDA_TRY(cudaMemsetAsync(g->wctr + 1, 0, sizeof(unsigned long long), s));
    g->fuse_epoch = 0;
    g->rowcnt_dirty = false;
  }
  const uint32_t epoch = ++g->fuse_epoch;
  const uint32_t worker_warps = (uint32_t)((ncl - 1) * nr * kCW);
  ExploreArgs A = A0;
  A.rowcnt = g->rowcnt;
  A.epoch_m1 = epoch - 1;
  A.done = g->rowcnt + g->n;
  A.done_target = epoch * worker_warps;
  // test hooks (bounded-wait path): PUMP_TEST_FUSED_HOLD_ROW names a row whose count never
  // completes, PUMP_TEST_SPIN_LIMIT shortens the waits
  const char* hold = getenv("PUMP_TEST_FUSED_HOLD_ROW");
  const char* lim = getenv("PUMP_TEST_SPIN_LIMIT");
  if (lim && atoll(lim) > 0) A.spin_limit = atoll(lim);
  FuseArgs F;
  F.xp = g->xi_p;
  F.wctr = g->wctr + 1;
  F.phi = g->phi;
  F.L = g->L;
  F.nom = g->nom;
  F.linf = g->linf_dev;
  F.ibox = g->ibox;
  F.dmax = g->dmax;
  F.boxes = g->boxes;
  F.eorder = g->eorder;
  F.emask = g->emask;
  F.rowcnt = g->rowcnt;
  F.N = g->N;
  F.W = g->W;
  F.nb = g->n_boxes;
  F.E = g->E;
  F.w = g->n_words;
  F.n = g->n;
  F.xi_smem = xi_smem ? 1 : 0;
  F.hold_row = hold ? atoi(hold) : -1;
  if (F.hold_row >= 0) g->rowcnt_dirty = true;  // that row's count stays short
  F.goal_sorted = g->ex.goal_sorted;
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[2];
  cluster_config(&cfg, attr, nr, ncl, smem, s);
  attr[1].id = cudaLaunchAttributeCooperative;
  attr[1].val.cooperative = 1;
  cfg.numAttrs = 2;
  const int32_t start = g->start;
  const LaunchShape ls{nr, (uint32_t)smem};
  if (cudaLaunchKernelEx(&cfg, k_explore_fused<true>, A, start, F, ls) != cudaSuccess) {
    cudaGetLastError();
    fused_disable(dev, smem);
    g->rowcnt_dirty = true;
    return PUMP_OK;
  }
  note_launch();
  g->masks_ready = true;
  *launched = true;
  return PUMP_OK;
}

}  // namespace pump
