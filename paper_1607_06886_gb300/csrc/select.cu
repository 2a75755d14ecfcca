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
// The first min(|P_goal|, 32) plans are certified in one batch up front, which
// settles any P_goal of up to 32 plans with a single host synchronisation.
//
// MC(p).  Rollout m, step s draws one Philox4x32-10 block with counter
// (m, s lo, 0, s hi) and key (seed lo, seed hi); its 128 bits give six 21-bit
// uniforms u in (0,1) (mc_normals), and Box-Muller gives
// sqrt(-2 ln u1) (cos 2 pi u2, sin 2 pi u2) in float for (xi0, xi1).  The
// deviation starts at Linf xi (step 0) and is carried over the plan's
// connections; each waypoint interval takes `substeps` steps of
// hs = (tau / W) / substeps with Phi(hs), L(hs) and the nominal position at
// t = ((k-1) substeps + s) hs.  A rollout collides iff a step position lies in
// a closed box.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "pump_internal.cuh"

namespace pump {
namespace {


__global__ void k_goal_finalize(ExploreArgs A, int32_t* removed, int32_t* sorted) { goal_finalize_block(A, removed, sorted); }

// Selection state (device): bisection indices and the outcome.
struct SelState {
  int32_t l, u, m, phase, last_m, need, done, status, chosen, n_probes, n_cert, G;
  long long last_c, chosen_c;
  int32_t path_len, popc;
  float cost;
  int32_t err;
};

constexpr int kCertMax = 32;  // plans certified per batch

// Prepare a batch: on the first call (want < 0) the first min(G, kCertMax) plans of
// P_goal in selection order, else the single index `want`.  An Explore error or an empty
// P_goal ends the selection at once.
__global__ void k_sel_prepare(const ExploreCtl* __restrict__ ctl, SelState* st, const int32_t* __restrict__ sorted,
                              long long* by_index, int32_t* batch_idx, int32_t* batch_plan, int want) {
  SelState s = *st;
  if (want < 0) {
    s = SelState{};
    s.G = ctl->status ? 0 : ctl->n_goal;
    s.chosen = -1;
    s.need = -1;
    if (ctl->status) {
      s.done = 1;
      s.status = ctl->status;
    } else if (s.G == 0) {
      s.done = 1;
      s.status = PUMP_ERR_INFEASIBLE;
    }
    s.n_cert = s.done ? 0 : min(s.G, kCertMax);
    for (int k = 0; k < s.n_cert; ++k) {
      batch_idx[k] = k;
      batch_plan[k] = sorted[k];
    }
  } else {
    s.n_cert = 1;
    batch_idx[0] = want;
    batch_plan[0] = sorted[want];
  }
  *st = s;
}

__global__ void k_clear_index(const SelState* __restrict__ st, long long* by_index) {
  const int G = st->G;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < G; k += gridDim.x * blockDim.x) by_index[k] = -1;
}

// Path of each plan: node ids from x_init and the edge ids between them.
__global__ void k_mc_paths(const SelState* __restrict__ st, const int32_t* __restrict__ plans,
                           const int32_t* __restrict__ parent, const int32_t* __restrict__ pedge,
                           const int32_t* __restrict__ head, int32_t* plen, int32_t* pedges, int32_t* pnodes,
                           int32_t* err) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= st->n_cert) return;
  int len = 0;
  for (int32_t q = plans[k]; parent[q] >= 0; q = parent[q]) {
    if (++len > kMaxPathEdges) {
      atomicExch(err, 1);
      plen[k] = 0;
      return;
    }
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

// Per path edge: Phi(hs) (4), L(hs) (3), the bits of the boxes its particles can reach (1), then
// W*S*3 nominal positions.  Plan k's table starts at k * kMaxPathEdges * stride.  A block per
// path edge: its threads take the sample positions (double cubic, rounded to float) while the
// last thread computes Phi and L; min/max of the positions by warp and block reduction.
constexpr int kPrepThreads = 128;
__global__ void __launch_bounds__(kPrepThreads) k_mc_prep(const int32_t* __restrict__ n_cert_p,
                                                          const int32_t* __restrict__ plen,
                                                          const int32_t* __restrict__ pedges,
                                                          const int32_t* __restrict__ pnodes,
                                                          const float* __restrict__ states,
                                                          const float* __restrict__ tau, int W, int S, float sigma,
                                                          const float* __restrict__ boxes, int nb, float B,
                                                          float* table) {
  const int k = blockIdx.y;
  if (k >= *n_cert_p) return;
  const int L = plen[k];
  const int stride = 8 + W * S * 3;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  constexpr int kWarpsP = kPrepThreads / 32;
  constexpr int kModel = kPrepThreads - 1;  // the thread computing Phi and L
  __shared__ Cubic cq[3];
  __shared__ float s_lo[kWarpsP][3], s_hi[kWarpsP][3];
  for (int j = blockIdx.x; j < L; j += gridDim.x) {
    const int e = pedges[(size_t)k * kMaxPathEdges + j];
    const int v = pnodes[(size_t)k * (kMaxPathEdges + 1) + j], u = pnodes[(size_t)k * (kMaxPathEdges + 1) + j + 1];
    float* T = table + ((size_t)k * kMaxPathEdges + j) * stride;
    const float t32 = tau[e];
    const float h = __fdiv_rn(t32, (float)W);
    const float hs = __fdiv_rn(h, (float)S);
    if (t < 3) {
      double xv[6], xu[6];
      for (int q = 0; q < 6; ++q) {
        xv[q] = (double)states[6 * v + q];
        xu[q] = (double)states[6 * u + q];
      }
      cq[t] = cubic_dev(xv, xu, (double)t32, t);
    }
    __syncthreads();
    float lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
      lo[a] = __int_as_float(0x7f800000);
      hi[a] = -lo[a];
    }
    if (t == kModel) {
      double Phi[4], Lm[3], Linf[3];
      model_dev((double)sigma, (double)hs, Phi, Lm, Linf);
      for (int q = 0; q < 4; ++q) T[q] = __double2float_rn(Phi[q]);
      for (int q = 0; q < 3; ++q) T[4 + q] = __double2float_rn(Lm[q]);
    } else {
      const int WS = W * S;
      for (int q = t; q < WS; q += kPrepThreads - 1) {
        const double tq = (double)(q + 1) * (double)hs;  // sample s of waypoint interval kk: (kk-1) S + s
        for (int a = 0; a < 3; ++a) {
          const float pv = __double2float_rn(cubic_at(cq[a], tq));
          T[8 + q * 3 + a] = pv;
          lo[a] = fminf(lo[a], pv);
          hi[a] = fmaxf(hi[a], pv);
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
      for (int a = 0; a < 3; ++a) {
        lo[a] = fminf(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
        hi[a] = fmaxf(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
      }
    if (lane == 0)
      for (int a = 0; a < 3; ++a) {
        s_lo[warp][a] = lo[a];
        s_hi[warp][a] = hi[a];
      }
    __syncthreads();
    if (warp == 0) {
      for (int a = 0; a < 3; ++a) {
        lo[a] = s_lo[0][a];
        hi[a] = s_hi[0][a];
        for (int r = 1; r < kWarpsP; ++r) {
          lo[a] = fminf(lo[a], s_lo[r][a]);
          hi[a] = fmaxf(hi[a], s_hi[r][a]);
        }
        lo[a] = __fsub_rn(lo[a], B);
        hi[a] = __fadd_rn(hi[a], B);
      }
      // boxes that can hold a position nominal + d0 with |d0| <= B on every axis (lane o: box o)
      bool ov = false;
      if (lane < nb && lane < 32) {
        const float* b = boxes + 6 * lane;
        ov = b[0] <= hi[0] && lo[0] <= b[3] && b[1] <= hi[1] && lo[1] <= b[4] && b[2] <= hi[2] && lo[2] <= b[5];
      }
      const unsigned bits = __ballot_sync(0xffffffffu, ov);
      if (lane == 0) T[7] = __uint_as_float(bits);
    }
    __syncthreads();  // cq and the reduction buffers are reused by the next path edge
  }
}

// Normals of rollout m, step s for the three axes: one Philox4x32-10 call, counter
// (m, s lo, 0, s hi), key (seed lo, seed hi), its words w0..w3 cut into six 21-bit fields: the
// top 21 bits of each word, then the low 11 bits of w0 followed by bits 10..1 of w1, and the same
// from w2 and w3; axis j takes u1 from field 2j and u2 from field 2j + 1, u = (b + 1/2) 2^-21
// (exact in float).
__device__ __forceinline__ void mc_normals(uint64_t seed, uint64_t m, uint64_t s, float* z) {
  uint32_t w[4];
  philox4x32((uint32_t)m, (uint32_t)s, 0u, (uint32_t)(s >> 32), (uint32_t)seed, (uint32_t)(seed >> 32), w);
  const uint32_t b[6] = {w[0] >> 11, w[1] >> 11, w[2] >> 11, w[3] >> 11,
                         ((w[0] & 0x7FFu) << 10) | ((w[1] & 0x7FFu) >> 1),
                         ((w[2] & 0x7FFu) << 10) | ((w[3] & 0x7FFu) >> 1)};
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const float u1 = ((float)b[2 * j] + 0.5f) * 4.76837158203125e-07f;
    const float u2 = ((float)b[2 * j + 1] + 0.5f) * 4.76837158203125e-07f;
    // hardware log2 and sine/cosine approximations (absolute error ~2^-21); the clamp keeps r
    // real where the approximate log of a u1 just below 1 comes out positive
    const float r = sqrtf(fmaxf(-2.0f * __logf(u1), 0.0f));
    float sn, cs;
    __sincosf(6.28318530717958648f * u2, &sn, &cs);
    z[2 * j] = r * cs;
    z[2 * j + 1] = r * sn;
  }
}

constexpr int kMcThreads = 128;
constexpr int kMcTableSmem = 4096;  // floats of a plan's table staged in shared memory (larger: read from L2)

// Box test of a position: with nb <= 32 and every |d0| <= B only the path edge's candidate
// boxes (bits) can hold it; otherwise all boxes are tested.
__device__ __forceinline__ bool mc_hit(const float* p, const float* d0, float B, uint32_t bits, const float* boxes,
                                       int nb) {
  if (nb <= 32 && fabsf(d0[0]) <= B && fabsf(d0[1]) <= B && fabsf(d0[2]) <= B) {
    while (bits) {
      const int o = __ffs(bits) - 1;
      bits &= bits - 1u;
      if (in_box_dev(p[0], p[1], p[2], boxes + 6 * o)) return true;
    }
    return false;
  }
  for (int o = 0; o < nb; ++o)
    if (in_box_dev(p[0], p[1], p[2], boxes + 6 * o)) return true;
  return false;
}

__device__ __forceinline__ void mc_update(const float* z, float P0, float P1, float P2, float P3, float L0, float L1,
                                          float L2, const float* nomq, float* d0, float* d1, float* p) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float n0 = __fmul_rn(L0, z[2 * a]);
    const float n1 = fmaf(L1, z[2 * a], __fmul_rn(L2, z[2 * a + 1]));
    const float e0 = fmaf(P0, d0[a], fmaf(P1, d1[a], n0));
    const float e1 = fmaf(P2, d0[a], fmaf(P3, d1[a], n1));
    d0[a] = e0;
    d1[a] = e1;
    p[a] = __fadd_rn(nomq[a], e0);
  }
}

// kMcLanes lanes per rollout (1 or 2); plan k = blockIdx.x / bpp.  The normals of a step depend only on
// (seed, rollout, step), so the lanes of a rollout draw the normals of consecutive steps in
// parallel (lane j takes steps j, j + kMcLanes, ...; Philox4x64 dominates the work) and pass
// them round by group shuffles; every lane of the group then applies the same updates in step
// order, so all of them hold the same deviation and the same hit flag.
template <int kMcLanes>
__global__ void __launch_bounds__(kMcThreads) k_mc_rollout(const int32_t* __restrict__ n_cert_p, int bpp,
                                                            const int32_t* __restrict__ plen,
                                                            const float* __restrict__ table, int W, int S,
                                                            const float* __restrict__ linf_g,
                                                            const float* __restrict__ boxes_g, int nb, int n_mc,
                                                            uint64_t seed, float B, unsigned long long* counts) {
  extern __shared__ float sm[];
  const int k = blockIdx.x / bpp;
  if (k >= *n_cert_p) return;
  const int L = plen[k];
  const int stride = 8 + W * S * 3;
  const int tfl = L * stride;
  const bool tab_smem = tfl <= kMcTableSmem;
  float* boxes = sm;
  float* tab = sm + 6 * nb;
  const float* T0 = table + (size_t)k * kMaxPathEdges * stride;
  for (int q = threadIdx.x; q < 6 * nb; q += blockDim.x) boxes[q] = boxes_g[q];
  if (tab_smem)
    for (int q = threadIdx.x; q < tfl; q += blockDim.x) tab[q] = T0[q];
  __syncthreads();
  const float* T = tab_smem ? tab : T0;
  const int lane = threadIdx.x & 31;
  const int j = lane % kMcLanes;                        // lane within the rollout's group
  const int g0 = lane - j;                              // first lane of the group
  const unsigned gmask = ((1u << kMcLanes) - 1u) << g0;
  const int m = (blockIdx.x % bpp) * (kMcThreads / kMcLanes) + threadIdx.x / kMcLanes;
  bool hit = false;
  if (m < n_mc) {
    float z[6], d0[3], d1[3], p[3];
    mc_normals(seed, (uint64_t)m, 0ull, z);
    const float l0 = linf_g[0], l1 = linf_g[1], l2 = linf_g[2];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      d0[a] = __fmul_rn(l0, z[2 * a]);
      d1[a] = fmaf(l1, z[2 * a], __fmul_rn(l2, z[2 * a + 1]));
    }
    const int WS = W * S;
    uint64_t step = 0;  // steps taken before this edge
    for (int e = 0; e < L && !hit; ++e) {
      const float* Te = T + (size_t)e * stride;
      const float P0 = Te[0], P1 = Te[1], P2 = Te[2], P3 = Te[3], L0 = Te[4], L1 = Te[5], L2 = Te[6];
      const uint32_t bits = __float_as_uint(Te[7]);
      for (int q0 = 0; q0 < WS && !hit; q0 += kMcLanes) {
        float zj[6];
        if (q0 + j < WS) {
          mc_normals(seed, (uint64_t)m, step + (uint64_t)(q0 + j) + 1ull, zj);
        } else {
#pragma unroll
          for (int c = 0; c < 6; ++c) zj[c] = 0.f;
        }
        const int nq = min(kMcLanes, WS - q0);
#pragma unroll
        for (int t = 0; t < kMcLanes; ++t) {
          if (t >= nq || hit) break;
#pragma unroll
          for (int c = 0; c < 6; ++c) z[c] = __shfl_sync(gmask, zj[c], g0 + t);
          mc_update(z, P0, P1, P2, P3, L0, L1, L2, Te + 8 + (q0 + t) * 3, d0, d1, p);
          hit = mc_hit(p, d0, B, bits, boxes, nb);
        }
      }
      step += (uint64_t)WS;
    }
  }
  const unsigned bal = __ballot_sync(0xffffffffu, hit && j == 0);
  if (lane == 0 && bal) atomicAdd(counts + k, (unsigned long long)__popc(bal));
}

constexpr int kMcScanSteps = 8;  // steps per lane per chunk: a chunk is 32 x 8 steps of one rollout
constexpr int kMcScanThreads = 256;

// MC(p) with a warp per rollout.  The deviation recurrence d_s = Phi_e d_{s-1} + n_s (per axis,
// n_s = L_e (z0, z1)_s, e the step's edge) is affine in d, so a chunk of 32 x 8 steps runs in
// parallel: lane j draws the normals of its 8 steps and composes their maps, an inclusive scan
// over the lanes gives every lane the deviation at the start of its steps, and each lane walks its
// steps from there and tests their positions.  A rollout collides when any step's position lies
// in a box, whatever the order the steps are tested in.  Work items (plan k, rollout m) are spread
// over the warps of the grid.  Against walking the steps one after another the deviations differ
// only by the float rounding of the composed maps (relative ~1e-7); lane 0 of the first chunk
// reproduces the one-after-another values exactly.
__global__ void __launch_bounds__(kMcScanThreads) k_mc_scan(const int32_t* __restrict__ n_cert_p,
                                                             const int32_t* __restrict__ plen,
                                                             const float* __restrict__ table, int W, int S,
                                                             const float* __restrict__ linf_g,
                                                             const float* __restrict__ boxes_g, int nb, int n_mc,
                                                             uint64_t seed, float B, unsigned long long* counts) {
  extern __shared__ float boxes[];
  for (int q = threadIdx.x; q < 6 * nb; q += blockDim.x) boxes[q] = boxes_g[q];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const long long items = (long long)(*n_cert_p) * n_mc;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const int stride = 8 + W * S * 3, WS = W * S;
  const float l0 = linf_g[0], l1 = linf_g[1], l2 = linf_g[2];
  for (long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < items; w += nwarps) {
    const int k = (int)(w / n_mc), m = (int)(w % n_mc);
    const float* T = table + (size_t)k * kMaxPathEdges * stride;
    const int Ls = plen[k] * WS;
    float z[6], d0[3], d1[3];
    mc_normals(seed, (uint64_t)m, 0ull, z);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      d0[a] = __fmul_rn(l0, z[2 * a]);
      d1[a] = fmaf(l1, z[2 * a], __fmul_rn(l2, z[2 * a + 1]));
    }
    bool hit = false;
    for (int base = 0; base < Ls && !hit; base += 32 * kMcScanSteps) {
      const int s0 = base + lane * kMcScanSteps + 1;  // first step of this lane
      int e = s0 <= Ls ? (s0 - 1) / WS : 0, q = s0 <= Ls ? (s0 - 1) - e * WS : 0;
      // 1. the lane's steps: normals, noise terms and the composed map (M, v): d -> M d + v
      float n0[kMcScanSteps][3], n1[kMcScanSteps][3];
      float M00 = 1.f, M01 = 0.f, M10 = 0.f, M11 = 1.f, v0[3] = {0.f, 0.f, 0.f}, v1[3] = {0.f, 0.f, 0.f};
      {
        int ee = e, qq = q;
#pragma unroll
        for (int c = 0; c < kMcScanSteps; ++c) {
          const int s = s0 + c;
          if (s <= Ls) {
            const float* Te = T + (size_t)ee * stride;
            const float P0 = Te[0], P1 = Te[1], P2 = Te[2], P3 = Te[3], L0 = Te[4], L1 = Te[5], L2 = Te[6];
            mc_normals(seed, (uint64_t)m, (uint64_t)s, z);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
              n0[c][a] = __fmul_rn(L0, z[2 * a]);
              n1[c][a] = fmaf(L1, z[2 * a], __fmul_rn(L2, z[2 * a + 1]));
              const float t0 = fmaf(P0, v0[a], fmaf(P1, v1[a], n0[c][a]));
              const float t1 = fmaf(P2, v0[a], fmaf(P3, v1[a], n1[c][a]));
              v0[a] = t0;
              v1[a] = t1;
            }
            const float a00 = fmaf(P0, M00, __fmul_rn(P1, M10)), a01 = fmaf(P0, M01, __fmul_rn(P1, M11));
            const float a10 = fmaf(P2, M00, __fmul_rn(P3, M10)), a11 = fmaf(P2, M01, __fmul_rn(P3, M11));
            M00 = a00;
            M01 = a01;
            M10 = a10;
            M11 = a11;
            if (++qq == WS) {
              qq = 0;
              ++ee;
            }
          } else {
#pragma unroll
            for (int a = 0; a < 3; ++a) n0[c][a] = n1[c][a] = 0.f;
          }
        }
      }
      // 2. inclusive scan over the lanes: (M, v) after the maps of every lower lane, lower first
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const float u00 = __shfl_up_sync(0xffffffffu, M00, off), u01 = __shfl_up_sync(0xffffffffu, M01, off);
        const float u10 = __shfl_up_sync(0xffffffffu, M10, off), u11 = __shfl_up_sync(0xffffffffu, M11, off);
        float w0[3], w1[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          w0[a] = __shfl_up_sync(0xffffffffu, v0[a], off);
          w1[a] = __shfl_up_sync(0xffffffffu, v1[a], off);
        }
        if (lane >= off) {
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            const float t0 = fmaf(M00, w0[a], fmaf(M01, w1[a], v0[a]));
            const float t1 = fmaf(M10, w0[a], fmaf(M11, w1[a], v1[a]));
            v0[a] = t0;
            v1[a] = t1;
          }
          const float a00 = fmaf(M00, u00, __fmul_rn(M01, u10)), a01 = fmaf(M00, u01, __fmul_rn(M01, u11));
          const float a10 = fmaf(M10, u00, __fmul_rn(M11, u10)), a11 = fmaf(M10, u01, __fmul_rn(M11, u11));
          M00 = a00;
          M01 = a01;
          M10 = a10;
          M11 = a11;
        }
      }
      // 3. the deviation at the start of this lane's steps (exclusive prefix) and at the chunk's end
      float x0[3], x1[3];
      {
        float e00 = __shfl_up_sync(0xffffffffu, M00, 1), e01 = __shfl_up_sync(0xffffffffu, M01, 1);
        float e10 = __shfl_up_sync(0xffffffffu, M10, 1), e11 = __shfl_up_sync(0xffffffffu, M11, 1);
        const float f00 = __shfl_sync(0xffffffffu, M00, 31), f01 = __shfl_sync(0xffffffffu, M01, 31);
        const float f10 = __shfl_sync(0xffffffffu, M10, 31), f11 = __shfl_sync(0xffffffffu, M11, 31);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          float y0 = __shfl_up_sync(0xffffffffu, v0[a], 1), y1 = __shfl_up_sync(0xffffffffu, v1[a], 1);
          if (lane == 0) {
            x0[a] = d0[a];
            x1[a] = d1[a];
          } else {
            x0[a] = fmaf(e00, d0[a], fmaf(e01, d1[a], y0));
            x1[a] = fmaf(e10, d0[a], fmaf(e11, d1[a], y1));
          }
          const float g0 = __shfl_sync(0xffffffffu, v0[a], 31), g1 = __shfl_sync(0xffffffffu, v1[a], 31);
          const float c0 = fmaf(f00, d0[a], fmaf(f01, d1[a], g0));
          const float c1 = fmaf(f10, d0[a], fmaf(f11, d1[a], g1));
          d0[a] = c0;
          d1[a] = c1;
        }
        (void)e00;
        (void)e01;
        (void)e10;
        (void)e11;
      }
      // 4. walk the lane's steps and test the positions
      bool h = false;
#pragma unroll
      for (int c = 0; c < kMcScanSteps; ++c) {
        const int s = s0 + c;
        if (s <= Ls && !h) {
          const float* Te = T + (size_t)e * stride;
          const float P0 = Te[0], P1 = Te[1], P2 = Te[2], P3 = Te[3];
          const uint32_t bits = __float_as_uint(Te[7]);
          const float* nomq = Te + 8 + q * 3;
          float p[3];
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            const float t0 = fmaf(P0, x0[a], fmaf(P1, x1[a], n0[c][a]));
            const float t1 = fmaf(P2, x0[a], fmaf(P3, x1[a], n1[c][a]));
            x0[a] = t0;
            x1[a] = t1;
            p[a] = __fadd_rn(nomq[a], t0);
          }
          h = mc_hit(p, x0, B, bits, boxes, nb);
          if (++q == WS) {
            q = 0;
            ++e;
          }
        }
      }
      hit = __any_sync(0xffffffffu, h);
    }
    if (lane == 0 && hit) atomicAdd(counts + k, 1ull);
  }
}

__global__ void k_counts_store(const SelState* __restrict__ st, const unsigned long long* __restrict__ counts,
                               const int32_t* __restrict__ idx, long long* by_index) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < st->n_cert) by_index[idx[k]] = (long long)counts[k];
}

// Advance Algorithm 5's bisection as far as the known counts allow; when done, backtrack the
// chosen plan into `path` (x_init first) and record its cost and popcount.
__global__ void k_bisect_run(SelState* st, const int32_t* __restrict__ sorted, const long long* by_index, int n_mc,
                             double alpha, const int32_t* __restrict__ parent, const int32_t* __restrict__ head,
                             const float* __restrict__ cost, const int32_t* __restrict__ popc, int32_t* path,
                             int32_t path_cap) {
  SelState s = *st;
  s.need = -1;
  const int G = s.G;
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
      if (c < 0) {
        s.need = s.m - 1;
        break;
      }
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
        if (c < 0) {
          s.need = s.m - 1;
          break;
        }
        s.n_probes++;
      }
      s.chosen = sorted[s.m - 1];
      s.chosen_c = c;
      s.status = ((double)c / (double)n_mc > alpha) ? (int)PUMP_ERR_INFEASIBLE : (int)PUMP_OK;
      s.done = 1;
    }
  }
  if (s.done && s.chosen >= 0) {
    int len = 0;
    for (int32_t q = s.chosen; q >= 0; q = parent[q]) ++len;
    s.path_len = len;
    int k = len;
    for (int32_t q = s.chosen; q >= 0; q = parent[q]) {
      --k;
      if (k < path_cap) path[k] = head[q];
    }
    s.cost = cost[s.chosen];
    s.popc = popc[s.chosen];
  }
  *st = s;
}

}  // namespace

int ensure_mc(pump_graph* g, cudaStream_t s) {
  ExploreBufs& X = g->ex;
  if (X.mc_count) return PUMP_OK;
  const int cap = kCertMax;
  X.mc_count = (int64_t*)graph_alloc(g, sizeof(int64_t) * cap, s);
  X.mc_plan = (int32_t*)graph_alloc(g, sizeof(int32_t) * cap, s);
  X.mc_plen = (int32_t*)graph_alloc(g, sizeof(int32_t) * (cap + 1), s);
  X.mc_pedges = (int32_t*)graph_alloc(g, sizeof(int32_t) * (size_t)cap * kMaxPathEdges, s);
  X.path_buf = (int32_t*)graph_alloc(g, sizeof(int32_t) * (size_t)cap * (kMaxPathEdges + 1), s);
  X.sel_state = graph_alloc(g, sizeof(SelState), s);
  X.sel_err = (int32_t*)graph_alloc(g, sizeof(int32_t) * 2, s);
  X.sel_idx = (int32_t*)graph_alloc(g, sizeof(int32_t) * cap, s);
  if (!X.mc_count || !X.mc_plan || !X.mc_plen || !X.mc_pedges || !X.path_buf || !X.sel_state || !X.sel_err ||
      !X.sel_idx)
    return PUMP_ERR_OOM;
  X.mc_cap = cap;
  return PUMP_OK;
}

// Table for kCertMax plans of up to kMaxPathEdges connections each.
int ensure_table(pump_graph* g, int S, cudaStream_t s) {
  ExploreBufs& X = g->ex;
  const int64_t want = (int64_t)kCertMax * kMaxPathEdges * (8 + g->W * S * 3);
  if (want > X.mc_table_floats) {
    X.mc_table = (float*)graph_realloc(g, X.mc_table, sizeof(float) * want, s);
    if (!X.mc_table) {
      X.mc_table_floats = 0;
      return PUMP_ERR_OOM;
    }
    X.mc_table_floats = want;
  }
  return PUMP_OK;
}

// MC form by the batch's plan count (measured): the warp scan up to kMcScanMax plans, two lanes
// per rollout up to kMcTwoLaneMax, then one.  PUMP_MC_FORM (1, 2, 3) fixes one form (tuning).
#ifndef PUMP_MC_FORM
#define PUMP_MC_FORM 0
#endif
#ifndef PUMP_MC_SCAN_MAX
#define PUMP_MC_SCAN_MAX 2
#endif
#ifndef PUMP_MC_TWO_LANE_MAX
#define PUMP_MC_TWO_LANE_MAX 6
#endif
constexpr int kMcScanMax = PUMP_MC_SCAN_MAX;
constexpr int kMcTwoLaneMax = PUMP_MC_TWO_LANE_MAX;

// Dynamic shared memory ceiling of the Monte Carlo kernels, set once per device to the most any
// query can ask for (every box and a full staged table).  The attribute belongs to the kernel,
// not to a launch: a per-query value set by one host thread could lower the limit under another
// thread's launch between its own set and launch (the request server plans queries on several
// threads), and that launch would fail.
constexpr size_t kMcSmemMax = sizeof(float) * 6 * (size_t)kMaxBoxes + sizeof(float) * kMcTableSmem;
std::mutex g_mc_attr_mu;
std::vector<int> g_mc_attr_dev;

int mc_attributes() {
  int dev = 0;
  PUMP_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_mc_attr_mu);
  for (int d : g_mc_attr_dev)
    if (d == dev) return PUMP_OK;
  PUMP_CUDA_TRY(cudaFuncSetAttribute(k_mc_scan, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMcSmemMax));
  PUMP_CUDA_TRY(cudaFuncSetAttribute(k_mc_rollout<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMcSmemMax));
  PUMP_CUDA_TRY(cudaFuncSetAttribute(k_mc_rollout<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMcSmemMax));
  g_mc_attr_dev.push_back(dev);
  return PUMP_OK;
}

// Certify the plans of the current batch (n_cert read on the device from the state).
// n_cert: the batch's plan count, known on the host (the device copy n_cert_dev holds the same).
int mc_batch(pump_graph* g, const int32_t* n_cert_dev, int n_cert, int n_mc, int S, uint64_t seed,
             cudaStream_t s) {
  ExploreBufs& X = g->ex;
  dim3 grid(64, std::max(n_cert, 1));  // path edges j, j + 64, ... per block row
  // deviation bound for the box cull: 12 stationary position standard deviations (any B is exact)
  const double sq3 = 1.7320508075688772935;
  const float B = (float)(12.0 * (double)g->sigma * sqrt(1.0 / sq3 + 0.5 * sq3)) + 1e-6f;
  k_mc_prep<<<grid, kPrepThreads, 0, s>>>(n_cert_dev, X.mc_plen, X.mc_pedges, X.path_buf, g->states, g->tau, g->W, S,
                                g->sigma, g->boxes, g->n_boxes, B, X.mc_table);
  note_launch();
  PUMP_CUDA_TRY(cudaMemsetAsync(X.mc_count, 0, sizeof(int64_t) * std::max(n_cert, 1), s));
  // the form that measured fastest for this many plans: the warp scan while few rollouts are in
  // flight (one or two plans), then two and one lanes per rollout
  if (n_mc > 0 && n_cert > 0) {
    const int rca = mc_attributes();
    if (rca) return rca;
    const size_t smem_boxes = sizeof(float) * 6 * (size_t)std::max(g->n_boxes, 1);
    unsigned long long* counts = reinterpret_cast<unsigned long long*>(X.mc_count);
    const int form = PUMP_MC_FORM ? PUMP_MC_FORM : (n_cert <= kMcScanMax ? 1 : (n_cert <= kMcTwoLaneMax ? 2 : 3));
    if (form == 1) {
      k_mc_scan<<<num_sms() * 4, kMcScanThreads, smem_boxes, s>>>(n_cert_dev, X.mc_plen, X.mc_table, g->W, S,
                                                                  g->linf_dev, g->boxes, g->n_boxes, n_mc, seed, B,
                                                                  counts);
    } else {
      const size_t smem = smem_boxes + sizeof(float) * kMcTableSmem;
      if (form == 2) {
        const int bpp = (n_mc + kMcThreads / 2 - 1) / (kMcThreads / 2);
        k_mc_rollout<2><<<n_cert * bpp, kMcThreads, smem, s>>>(n_cert_dev, bpp, X.mc_plen, X.mc_table, g->W, S,
                                                               g->linf_dev, g->boxes, g->n_boxes, n_mc, seed, B, counts);
      } else {
        const int bpp = (n_mc + kMcThreads - 1) / kMcThreads;
        k_mc_rollout<1><<<n_cert * bpp, kMcThreads, smem, s>>>(n_cert_dev, bpp, X.mc_plen, X.mc_table, g->W, S,
                                                               g->linf_dev, g->boxes, g->n_boxes, n_mc, seed, B, counts);
      }
    }
    note_launch();
  }
  PUMP_CUDA_TRY(cudaGetLastError());
  return PUMP_OK;
}

// Pinned read-back area of PlanSelection, one per host thread (allocated once): the control
// block, the selection state, the error flag and the path arrive with one wait per round.
struct SelHost {
  ExploreCtl ctl;
  SelState hs;
  int32_t err;
  int32_t path[kMaxPathEdges + 1];
};
static SelHost* sel_host() {
  struct Buf {
    SelHost* p = nullptr;
    ~Buf() {
      if (p) cudaFreeHost(p);
    }
  };
  thread_local Buf b;
  if (!b.p && cudaHostAlloc((void**)&b.p, sizeof(SelHost), cudaHostAllocDefault) != cudaSuccess) b.p = nullptr;
  return b.p;
}

int run_select(pump_graph* g, const pump_plan_params* p, int32_t* path, int32_t path_cap, pump_plan_result* out,
               ExploreCtl* ctl_host, cudaStream_t s) {
  ExploreBufs& X = g->ex;
  const int S = p->mc_substeps;
  std::memset(ctl_host, 0, sizeof(ExploreCtl));
  int rc = ensure_mc(g, s);
  if (!rc) rc = ensure_table(g, S, s);
  if (!rc && X.sel_cap < X.cap) {
    X.sel_by_index = (long long*)graph_realloc(g, X.sel_by_index, sizeof(long long) * X.cap, s);
    X.sel_cap = X.sel_by_index ? (int32_t)X.cap : 0;
    if (!X.sel_by_index) rc = PUMP_ERR_OOM;
  }
  if (rc) return rc;
  SelState* st = (SelState*)X.sel_state;
  const int32_t* n_cert_dev = &st->n_cert;
  PUMP_CUDA_TRY(cudaMemsetAsync(X.sel_err, 0, sizeof(int32_t) * 2, s));
  SelHost* H = sel_host();
  if (!H) return PUMP_ERR_CUDA;
  // Explore's outcome on the host: the first batch's plan count picks the certification form
  PUMP_CUDA_TRY(cudaMemcpyAsync(&H->ctl, X.ctl, sizeof(ExploreCtl), cudaMemcpyDeviceToHost, s));
  PUMP_CUDA_TRY(cudaStreamSynchronize(s));
  *ctl_host = H->ctl;
  const int G0 = ctl_host->status ? 0 : ctl_host->n_goal;
  SelState hs;
  out->n_certified = 0;
  for (int round = 0; round < 256; ++round) {
    const int want = round == 0 ? -1 : hs.need;
    k_sel_prepare<<<1, 1, 0, s>>>(X.ctl, st, X.goal_sorted, X.sel_by_index, X.sel_idx, X.mc_plan, want);
    note_launch();
    if (round == 0) {
      k_clear_index<<<64, 256, 0, s>>>(st, X.sel_by_index);
      note_launch();
    }
    const int n_cert = round == 0 ? std::min(G0, kCertMax) : 1;
    k_mc_paths<<<1, kCertMax, 0, s>>>(st, X.mc_plan, X.parent, X.pedge, X.head, X.mc_plen, X.mc_pedges, X.path_buf,
                                      X.sel_err);
    note_launch();
    rc = mc_batch(g, n_cert_dev, n_cert, p->n_mc, S, p->mc_seed, s);
    if (rc) return rc;
    k_counts_store<<<1, kCertMax, 0, s>>>(st, reinterpret_cast<unsigned long long*>(X.mc_count), X.sel_idx,
                                          X.sel_by_index);
    note_launch();
    k_bisect_run<<<1, 1, 0, s>>>(st, X.goal_sorted, X.sel_by_index, p->n_mc, (double)p->alpha, X.parent, X.head,
                                 X.cost, X.popc, X.path_buf, kMaxPathEdges + 1);
    note_launch();
    PUMP_CUDA_TRY(cudaGetLastError());
    PUMP_CUDA_TRY(cudaMemcpyAsync(&H->hs, st, sizeof(SelState), cudaMemcpyDeviceToHost, s));
    PUMP_CUDA_TRY(cudaMemcpyAsync(&H->err, X.sel_err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    const int ncopy = std::min(path_cap, kMaxPathEdges + 1);
    if (path && ncopy > 0)
      PUMP_CUDA_TRY(cudaMemcpyAsync(H->path, X.path_buf, sizeof(int32_t) * ncopy, cudaMemcpyDeviceToHost, s));
    PUMP_CUDA_TRY(cudaStreamSynchronize(s));
    hs = H->hs;
    const int32_t err = H->err;
    if (path && ncopy > 0) std::memcpy(path, H->path, sizeof(int32_t) * ncopy);
    if (err) return PUMP_ERR_INVALID_ARG;
    out->n_certified += hs.n_cert;
    if (hs.done) break;
    if (hs.need < 0) return PUMP_ERR_CUDA;
  }
  if (!hs.done) return PUMP_ERR_TIMEOUT;
  if (hs.status != PUMP_OK && hs.status != PUMP_ERR_INFEASIBLE) return hs.status;
  out->chosen_plan = hs.chosen;
  out->mc_collisions = hs.chosen >= 0 ? hs.chosen_c : -1;
  out->cp_mc = (hs.chosen >= 0 && p->n_mc > 0) ? (double)hs.chosen_c / (double)p->n_mc : 0.0;
  out->status = hs.status;
  out->cost = hs.chosen >= 0 ? hs.cost : 0.f;
  out->popc = hs.chosen >= 0 ? hs.popc : 0;
  out->cp_hat = (float)out->popc / (float)g->N;
  out->path_len = hs.chosen >= 0 ? std::min(hs.path_len, path_cap) : 0;
  out->path_truncated = (hs.chosen >= 0 && hs.path_len > path_cap) ? 1 : 0;
  out->n_goal = hs.G;
  return PUMP_OK;
}

int run_goal_finalize(pump_graph* g, const ExploreArgs& A, cudaStream_t s) {
  // the group array is free after Explore and serves as scratch
  k_goal_finalize<<<1, 1024, 0, s>>>(A, A.group, g->ex.goal_sorted);
  note_launch();
  PUMP_CUDA_TRY(cudaGetLastError());
  return PUMP_OK;
}

__global__ void k_one_plan(SelState* st) {
  SelState s{};
  s.n_cert = 1;
  *st = s;
}

int run_certify_path(pump_graph* g, const int32_t* path_dev, int32_t path_len, int32_t n_mc, int32_t substeps,
                     uint64_t seed, int64_t* n_collide, cudaStream_t s) {
  int rc = ensure_mc(g, s);
  if (!rc) rc = ensure_table(g, substeps, s);
  if (rc) return rc;
  ExploreBufs& X = g->ex;
  SelState* st = (SelState*)X.sel_state;
  PUMP_CUDA_TRY(cudaMemsetAsync(X.sel_err, 0, sizeof(int32_t) * 2, s));
  k_one_plan<<<1, 1, 0, s>>>(st);
  note_launch();
  k_path_edges<<<(path_len + 63) / 64, 64, 0, s>>>(path_dev, path_len, g->row_ptr, g->col, X.mc_pedges, X.path_buf,
                                                   X.mc_plen, X.sel_err);
  note_launch();
  rc = mc_batch(g, &st->n_cert, 1, n_mc, substeps, seed, s);
  if (rc) return rc;
  long long c = 0;
  int32_t err = 0;
  PUMP_CUDA_TRY(cudaMemcpyAsync(&c, X.mc_count, sizeof(long long), cudaMemcpyDeviceToHost, s));
  PUMP_CUDA_TRY(cudaMemcpyAsync(&err, X.sel_err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  PUMP_CUDA_TRY(cudaStreamSynchronize(s));
  if (err) return PUMP_ERR_INVALID_ARG;
  *n_collide = c;
  return PUMP_OK;
}

}  // namespace pump
