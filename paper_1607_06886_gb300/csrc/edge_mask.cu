// Edge particle collision masks (Section III-B, with a direct particle-in-box
// test in place of the half-space test): the graph-build bound pass, the query
// pass over every edge (a warp per edge, the per-edge routine in mask_dev.cuh)
// and the Half-Space Monte Carlo forms.  The normals (xi_t[k][axis][i], or pair-major for the box
// masks) and the boxes sit in shared memory; the grids are persistent over the edges.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <mutex>
#include <vector>

#include "mask_dev.cuh"
#include "pump_internal.cuh"

namespace pump {
namespace {

constexpr int kWarps = 8;
constexpr int kHsStage = 128;  // HSMC: half-spaces of one edge staged in shared memory per warp

// Shared memory of the HSMC query pass before the normals: staged half-spaces and waypoint offsets.
__host__ __device__ constexpr size_t edge_mask_hs_fixed_smem() {
  return (sizeof(float4) * kWarps * kHsStage + sizeof(int32_t) * kWarps * (kMaxWaypoints + 1) + 15) & ~(size_t)15;
}

using maskdev::kBoxStride;

__host__ __device__ constexpr size_t edge_mask_fixed_smem(int nb) { return maskdev::fixed_smem(nb, kWarps); }

// Graph-build pass (obstacle independent): per edge the largest |d0| over all particles,
// waypoints and axes, as float bits.  A warp per edge, the edge's Phi and L loaded once: lane l
// runs the particles of NP word pairs (pair-major normals, one 16-byte load per pair and axis)
// in the halves of packed FP32x2 registers, with the arithmetic of the query pass; the warp's
// maximum is stored directly.  Particles past N have zero normals and add nothing.
template <int NP>
__device__ __forceinline__ float bound_pass(const float4* __restrict__ xp, int npair, int W,
                                            const unsigned long long (&P2)[4], const unsigned long long (&L2)[3],
                                            const unsigned long long (&I2)[3], int p0, int lane) {
  const float4* xq = xp + (size_t)p0 * 32 + lane;
  unsigned long long d0[NP][3], d1[NP][3];
#pragma unroll
  for (int j = 0; j < NP; ++j)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float4 x = xq[((size_t)a * npair + j) * 32];
      const unsigned long long X0 = maskdev::pk2(x.x, x.y), X1 = maskdev::pk2(x.z, x.w);
      d0[j][a] = maskdev::mul2(I2[0], X0);
      d1[j][a] = maskdev::fma2(I2[1], X0, maskdev::mul2(I2[2], X1));
    }
  float m = 0.f;
  for (int k = 1; k <= W; ++k) {
    const float4* xk = xq + (size_t)k * 3 * npair * 32;
#pragma unroll
    for (int j = 0; j < NP; ++j)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const float4 x = xk[((size_t)a * npair + j) * 32];
        const unsigned long long X0 = maskdev::pk2(x.x, x.y), X1 = maskdev::pk2(x.z, x.w);
        const unsigned long long m0 = maskdev::mul2(L2[0], X0);
        const unsigned long long m1 = maskdev::fma2(L2[1], X0, maskdev::mul2(L2[2], X1));
        const unsigned long long e0 = maskdev::fma2(P2[0], d0[j][a], maskdev::fma2(P2[1], d1[j][a], m0));
        const unsigned long long e1 = maskdev::fma2(P2[2], d0[j][a], maskdev::fma2(P2[3], d1[j][a], m1));
        d0[j][a] = e0;
        d1[j][a] = e1;
        float u, v;
        maskdev::upk2(e0, u, v);
        m = fmaxf(m, fmaxf(fabsf(u), fabsf(v)));
      }
  }
  return m;
}

template <bool kSmemXi>
__global__ void __launch_bounds__(kWarps * 32) k_edge_bound(const float4* __restrict__ xp_g, int npair, int W,
                                                            const float* __restrict__ phi,
                                                            const float* __restrict__ Lg,
                                                            const float* __restrict__ linf_g, int E,
                                                            unsigned int* __restrict__ dbound) {
  extern __shared__ __align__(16) unsigned char smem[];
  float4* xp_s = reinterpret_cast<float4*>(smem);
  const int xp_n = (W + 1) * 3 * npair * 32;
  if (kSmemXi)
    for (int k = threadIdx.x; k < xp_n; k += blockDim.x) xp_s[k] = xp_g[k];
  __syncthreads();
  const float4* xp = kSmemXi ? xp_s : xp_g;
  const unsigned long long I2[3] = {maskdev::pk2(linf_g[0], linf_g[0]), maskdev::pk2(linf_g[1], linf_g[1]),
                                    maskdev::pk2(linf_g[2], linf_g[2])};
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (long long e = (long long)blockIdx.x * kWarps + warp; e < E; e += (long long)gridDim.x * kWarps) {
    const float4 ph = *reinterpret_cast<const float4*>(phi + 4 * e);
    const float l0 = Lg[3 * e], l1 = Lg[3 * e + 1], l2 = Lg[3 * e + 2];
    const unsigned long long P2[4] = {maskdev::pk2(ph.x, ph.x), maskdev::pk2(ph.y, ph.y), maskdev::pk2(ph.z, ph.z),
                                      maskdev::pk2(ph.w, ph.w)};
    const unsigned long long L2[3] = {maskdev::pk2(l0, l0), maskdev::pk2(l1, l1), maskdev::pk2(l2, l2)};
    float m = 0.f;
    int p = 0;
    for (; p + 2 <= npair; p += 2) m = fmaxf(m, bound_pass<2>(xp, npair, W, P2, L2, I2, p, lane));
    if (p < npair) m = fmaxf(m, bound_pass<1>(xp, npair, W, P2, L2, I2, p, lane));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) dbound[e] = __float_as_uint(m);
  }
}

// Per edge: box holding every particle position, [min nominal - M, max nominal + M] per axis,
// rounded to nearest (float rounding is monotone, so fl(nominal + d0) stays inside).
__global__ void k_edge_ibox(const float* __restrict__ nom, const unsigned int* __restrict__ dbound, int E, int W,
                            float* __restrict__ ibox) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  const float M = __uint_as_float(dbound[e]);
  const float* nm = nom + (size_t)e * W * 3;
  for (int a = 0; a < 3; ++a) {
    float lo = nm[a], hi = nm[a];
    for (int k = 1; k < W; ++k) {
      lo = fminf(lo, nm[k * 3 + a]);
      hi = fmaxf(hi, nm[k * 3 + a]);
    }
    ibox[6 * (size_t)e + a] = __fsub_rn(lo, M);
    ibox[6 * (size_t)e + 3 + a] = __fadd_rn(hi, M);
  }
}

// Query pass: a warp per edge (maskdev::edge_mask_one), grid persistent over the edges; each warp
// takes the next kMaskChunk edges from a counter (edges differ widely in work: one whose position
// box meets no obstacle is a few instructions), so no SM idles while others hold long edges.
#ifndef PUMP_MASK_MIN_BLOCKS
#define PUMP_MASK_MIN_BLOCKS 3  // 80 registers: three 256-thread blocks per SM (batched and HSMC passes)
#endif
#ifndef PUMP_MASK_QUERY_MIN_BLOCKS
// the single-query passes at 64 registers, four blocks per SM where their staging fits: measured
// 5 % faster than three blocks at 80 registers (the batched pass spills at 64 and stays at three)
#define PUMP_MASK_QUERY_MIN_BLOCKS 4
#endif
constexpr int kMaskChunk = 4;  // default edges per take
template <bool kSmemXi, int kNP = 2>
__global__ void __launch_bounds__(kWarps * 32, PUMP_MASK_QUERY_MIN_BLOCKS) k_edge_mask(const float4* __restrict__ xp_g, int N, int W,
                                                           const float* __restrict__ phi, const float* __restrict__ Lg,
                                                           const float* __restrict__ nom, const float* __restrict__ linf_g,
                                                           const float* __restrict__ ibox_g,
                                                           const unsigned int* __restrict__ dmax,
                                                           const float* __restrict__ boxes_g, int nb, int E, int w,
                                                           unsigned long long* __restrict__ ctr, int chunk,
                                                           uint32_t* __restrict__ mask) {
  extern __shared__ __align__(16) unsigned char smem[];
  float* boxes = reinterpret_cast<float*>(smem);  // kBoxStride floats per box (16-byte aligned rows)
  int* cand = reinterpret_cast<int*>(boxes + kBoxStride * nb);
  uint32_t* wmask_all = reinterpret_cast<uint32_t*>(cand + kWarps * maskdev::kCandCap);
  float4* xp_s = reinterpret_cast<float4*>(smem + edge_mask_fixed_smem(nb));
  const int xp_n = (W + 1) * 3 * maskdev::pair_count(w) * 32;
  maskdev::stage(boxes_g, nb, boxes, xp_g, kSmemXi ? xp_s : nullptr, xp_n);
  __syncthreads();
  const float4* xp = kSmemXi ? xp_s : xp_g;
  const float linf[3] = {linf_g[0], linf_g[1], linf_g[2]};
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int* my_cand = cand + warp * maskdev::kCandCap;
  uint32_t* wm = wmask_all + warp * kMaxWaypoints;
  for (;;) {
    unsigned long long t = 0;
    if (lane == 0) t = atomicAdd(ctr, (unsigned long long)chunk);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= (unsigned long long)E) break;
    const long long e1 = min((long long)E, (long long)t + chunk);
    for (long long e = (long long)t; e < e1; ++e)
      maskdev::edge_mask_one<kNP, false>(e, xp, N, W, phi, Lg, nom, linf, ibox_g, dmax, boxes, nb, w, my_cand, wm, lane,
                                  mask);
  }
}

// Batched query pass: the box masks of many graphs in one persistent launch.  Their edges form one
// list of items (graph j's edges [i * span, (i + 1) * span) for i < ceil(E_j / span); graph j's
// items from item0[j] on).  A block takes the next item from one counter, stages the graph's boxes
// (and normals, when xi_smem) when the item belongs to another graph than its last one, and its
// warps take the item's edges, chunk at a time, from a shared counter.  Thread 0 keeps the graph
// index and moves it forward (items come in increasing order).
struct MaskJob {
  const float4* xp;
  const float* phi;
  const float* L;
  const float* nom;
  const float* linf;
  const float* ibox;
  const unsigned int* dmax;
  const float* boxes;
  uint32_t* emask;
  long long E;
  int32_t N, W, nb, w, xi_smem;
};

template <int kNP>
__global__ void __launch_bounds__(kWarps * 32, PUMP_MASK_MIN_BLOCKS)
    k_edge_mask_batch(const MaskJob* __restrict__ jobs, const long long* __restrict__ item0, int nq, int span,
                      int chunk, unsigned long long* __restrict__ ctr) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ long long s_item;
  __shared__ int s_job;
  __shared__ unsigned int s_next;
  const long long n_items = __ldg(item0 + nq);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int cur = -1, jq = 0;
  for (;;) {
    if (threadIdx.x == 0) {
      const long long it = (long long)atomicAdd(ctr, 1ull);
      if (it < n_items)
        while (jq + 1 < nq && __ldg(item0 + jq + 1) <= it) ++jq;
      s_item = it;
      s_job = jq;
      s_next = 0u;
    }
    __syncthreads();
    const long long it = s_item;
    if (it >= n_items) break;
    const int j = s_job;
    const MaskJob& J = jobs[j];
    const int nb = J.nb, W = J.W, w = J.w, N = J.N;
    float* boxes = reinterpret_cast<float*>(smem);
    int* cand = reinterpret_cast<int*>(boxes + kBoxStride * nb);
    uint32_t* wmask_all = reinterpret_cast<uint32_t*>(cand + kWarps * maskdev::kCandCap);
    float4* xp_s = reinterpret_cast<float4*>(smem + edge_mask_fixed_smem(nb));
    if (j != cur) {
      const int xp_n = (W + 1) * 3 * maskdev::pair_count(w) * 32;
      maskdev::stage(J.boxes, nb, boxes, J.xp, J.xi_smem ? xp_s : nullptr, xp_n);
      __syncthreads();
      cur = j;
    }
    const float4* xp = J.xi_smem ? xp_s : J.xp;
    const float linf[3] = {J.linf[0], J.linf[1], J.linf[2]};
    int* my_cand = cand + warp * maskdev::kCandCap;
    uint32_t* wm = wmask_all + warp * kMaxWaypoints;
    const long long e_begin = (it - __ldg(item0 + j)) * (long long)span;
    const long long e_end = min(J.E, e_begin + span);
    for (;;) {
      unsigned int t = 0u;
      if (lane == 0) t = atomicAdd(&s_next, (unsigned int)chunk);
      t = __shfl_sync(0xffffffffu, t, 0);
      const long long e0 = e_begin + (long long)t;
      if (e0 >= e_end) break;
      const long long e1 = min(e_end, e0 + chunk);
      for (long long e = e0; e < e1; ++e)
        maskdev::edge_mask_one<kNP>(e, xp, N, W, J.phi, J.L, J.nom, linf, J.ibox, J.dmax, boxes, nb, w, my_cand, wm,
                                    lane, J.emask);
    }
    __syncthreads();  // the item's edges are done: the staging and the shared counter are reused
  }
}

// Masks of a list of edges (repeats allowed): row j of out = the mask of edge elist[j], the
// per-(plan, edge) recomputation an expansion performs without the per-edge memo.  Warps take list
// positions from a counter like k_edge_mask; an id outside [0, E) leaves its row untouched and
// counts in *bad.
template <bool kSmemXi>
__global__ void __launch_bounds__(kWarps * 32, PUMP_MASK_QUERY_MIN_BLOCKS)
    k_edge_mask_list(const float4* __restrict__ xp_g, int N, int W, const float* __restrict__ phi,
                     const float* __restrict__ Lg, const float* __restrict__ nom, const float* __restrict__ linf_g,
                     const float* __restrict__ ibox_g, const unsigned int* __restrict__ dmax,
                     const float* __restrict__ boxes_g, int nb, int E, int w, const int32_t* __restrict__ elist,
                     long long n, unsigned long long* __restrict__ ctr, int chunk, uint32_t* __restrict__ out,
                     unsigned int* __restrict__ bad) {
  extern __shared__ __align__(16) unsigned char smem[];
  float* boxes = reinterpret_cast<float*>(smem);
  int* cand = reinterpret_cast<int*>(boxes + kBoxStride * nb);
  uint32_t* wmask_all = reinterpret_cast<uint32_t*>(cand + kWarps * maskdev::kCandCap);
  float4* xp_s = reinterpret_cast<float4*>(smem + edge_mask_fixed_smem(nb));
  const int xp_n = (W + 1) * 3 * maskdev::pair_count(w) * 32;
  maskdev::stage(boxes_g, nb, boxes, xp_g, kSmemXi ? xp_s : nullptr, xp_n);
  __syncthreads();
  const float4* xp = kSmemXi ? xp_s : xp_g;
  const float linf[3] = {linf_g[0], linf_g[1], linf_g[2]};
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int* my_cand = cand + warp * maskdev::kCandCap;
  uint32_t* wm = wmask_all + warp * kMaxWaypoints;
  for (;;) {
    unsigned long long t = 0;
    if (lane == 0) t = atomicAdd(ctr, (unsigned long long)chunk);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= (unsigned long long)n) break;
    const long long j1 = min(n, (long long)t + chunk);
    for (long long j = (long long)t; j < j1; ++j) {
      const int32_t e = __ldg(elist + j);
      if (e < 0 || e >= E) {
        if (lane == 0) atomicAdd(bad, 1u);
        continue;
      }
      maskdev::edge_mask_one<2, false>(e, xp, N, W, phi, Lg, nom, linf, ibox_g, dmax, boxes, nb, w, my_cand, wm, lane, out,
                                0, -1, j);
    }
  }
}

// ---------------------------------------------------------------- Half-Space Monte Carlo
//
// Local convex region of waypoint y (nominal position) with nominal velocity v, in the arithmetic
// the header states (float, each operation rounded as written, left to right).  Writes to `out`
// (when given) the half-spaces (a, b) a particle of the edge can fire: a.dy <= (|a0| + |a1| +
// |a2|) max |dy_j| <= (|a0| + |a1| + |a2|) M, so a half-space with (|a0| + |a1| + |a2|) M (1 +
// 2^-10) < b can never fire (the margin covers the test's rounding) and is left out.  Returns
// how many are kept.
__device__ int hs_region(const float* y, const float* v, const float* boxes, int nb, float M, float4* out) {
  uint32_t alive[kMaxBoxes / 32];
  const int nwords = (nb + 31) / 32;
  for (int q = 0; q < nwords; ++q) alive[q] = (q + 1) * 32 <= nb ? 0xffffffffu : ((1u << (nb - q * 32)) - 1u);
  const float vv = __fadd_rn(__fadd_rn(__fmul_rn(v[0], v[0]), __fmul_rn(v[1], v[1])), __fmul_rn(v[2], v[2]));
  int kept = 0;
  for (int count = 0; count < kHsMax; ++count) {
    int best = -1;
    float bestd = __int_as_float(0x7f800000), d0 = 0.f, d1 = 0.f, d2 = 0.f;
    for (int q = 0; q < nwords; ++q) {
      uint32_t bits = alive[q];
      while (bits) {
        const int o = q * 32 + __ffs(bits) - 1;
        bits &= bits - 1u;
        const float* b = boxes + 6 * o;
        const float e0 = __fsub_rn(fminf(fmaxf(y[0], b[0]), b[3]), y[0]);
        const float e1 = __fsub_rn(fminf(fmaxf(y[1], b[1]), b[4]), y[1]);
        const float e2 = __fsub_rn(fminf(fmaxf(y[2], b[2]), b[5]), y[2]);
        const float dd = __fadd_rn(__fadd_rn(__fmul_rn(e0, e0), __fmul_rn(e1, e1)), __fmul_rn(e2, e2));
        if (dd < bestd) {
          best = o;
          bestd = dd;
          d0 = e0;
          d1 = e1;
          d2 = e2;
        }
      }
    }
    if (best < 0 || !(bestd > 0.f)) break;
    float a0 = d0, a1 = d1, a2 = d2;
    if (vv > 0.f) {
      const float dv = __fadd_rn(__fadd_rn(__fmul_rn(d0, v[0]), __fmul_rn(d1, v[1])), __fmul_rn(d2, v[2]));
      const float f = __fdiv_rn(dv, vv);
      a0 = __fsub_rn(d0, __fmul_rn(f, v[0]));
      a1 = __fsub_rn(d1, __fmul_rn(f, v[1]));
      a2 = __fsub_rn(d2, __fmul_rn(f, v[2]));
    }
    const float bb = __fadd_rn(__fadd_rn(__fmul_rn(a0, a0), __fmul_rn(a1, a1)), __fmul_rn(a2, a2));
    if ((fabsf(a0) + fabsf(a1) + fabsf(a2)) * M * 1.0009765625f >= bb) {
      if (out) out[kept] = make_float4(a0, a1, a2, bb);
      ++kept;
    }
    alive[best >> 5] &= ~(1u << (best & 31));
    for (int q = 0; q < nwords; ++q) {
      uint32_t bits = alive[q];
      while (bits) {
        const int o = q * 32 + __ffs(bits) - 1;
        bits &= bits - 1u;
        const float* b = boxes + 6 * o;
        float m = 0.f;
        m = __fadd_rn(m, fminf(__fmul_rn(d0, __fsub_rn(b[0], y[0])), __fmul_rn(d0, __fsub_rn(b[3], y[0]))));
        m = __fadd_rn(m, fminf(__fmul_rn(d1, __fsub_rn(b[1], y[1])), __fmul_rn(d1, __fsub_rn(b[4], y[1]))));
        m = __fadd_rn(m, fminf(__fmul_rn(d2, __fsub_rn(b[2], y[2])), __fmul_rn(d2, __fsub_rn(b[5], y[2]))));
        if (m >= bestd) alive[q] &= ~(1u << (o & 31));
      }
    }
  }
  return kept;
}

// Graph build (HSMC): per waypoint (thread), the number of kept half-spaces, then their values.
template <bool kFill>
__global__ void k_hs_build(const float* __restrict__ nom, const float* __restrict__ nvel,
                           const unsigned int* __restrict__ dmax, const float* __restrict__ boxes_g, int nb, int E,
                           int W, int32_t* __restrict__ cnt, const int32_t* __restrict__ off, float4* __restrict__ ab) {
  extern __shared__ float hs_boxes[];
  for (int k = threadIdx.x; k < 6 * nb; k += blockDim.x) hs_boxes[k] = boxes_g[k];
  __syncthreads();
  const long long EW = (long long)E * W;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < EW; q += (long long)gridDim.x * blockDim.x) {
    const int e = (int)(q / W);
    const float M = __uint_as_float(dmax[e]);
    const float y[3] = {nom[3 * q], nom[3 * q + 1], nom[3 * q + 2]};
    const float v[3] = {nvel[3 * q], nvel[3 * q + 1], nvel[3 * q + 2]};
    if (kFill)
      hs_region(y, v, hs_boxes, nb, M, ab + off[q]);
    else
      cnt[q] = hs_region(y, v, hs_boxes, nb, M, nullptr);
  }
}

// Query pass (HSMC): a warp per edge; lane l advances the particles of NP pairs of mask words in
// packed FP32x2 registers (pair-major normals, as the box pass), and at waypoint k each particle
// tests the edge's kept half-spaces hs[off_k .. off_{k+1}): a . dy, the sums and products rounded
// as written, above b.  Packed FP32x2 arithmetic rounds each half as the scalar operation does, so
// the words equal the scalar evaluation's.
template <int NP>
__device__ __forceinline__ void pair_pass_hs(const float4* __restrict__ xp, int npair,
                                             const unsigned long long (&P2)[4], const unsigned long long (&L2)[3],
                                             const unsigned long long (&I2)[3], const int32_t* woff,
                                             const float4* hs, int k_last, int p0, int w, int lane, uint32_t* out) {
  using namespace maskdev;
  unsigned long long d0[NP][3], d1[NP][3];
  bool hit[NP][2];
  const float4* xq = xp + (size_t)p0 * 32 + lane;
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    hit[j][0] = hit[j][1] = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float4 x = xq[((size_t)a * npair + j) * 32];
      const unsigned long long X0 = pk2(x.x, x.y), X1 = pk2(x.z, x.w);
      d0[j][a] = mul2(I2[0], X0);
      d1[j][a] = fma2(I2[1], X0, mul2(I2[2], X1));
    }
  }
  for (int k = 1; k <= k_last; ++k) {
    const float4* xk = xq + (size_t)k * 3 * npair * 32;
#pragma unroll
    for (int j = 0; j < NP; ++j) {
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const float4 x = xk[((size_t)a * npair + j) * 32];
        const unsigned long long X0 = pk2(x.x, x.y), X1 = pk2(x.z, x.w);
        const unsigned long long m0 = mul2(L2[0], X0);
        const unsigned long long m1 = fma2(L2[1], X0, mul2(L2[2], X1));
        const unsigned long long e0 = fma2(P2[0], d0[j][a], fma2(P2[1], d1[j][a], m0));
        const unsigned long long e1 = fma2(P2[2], d0[j][a], fma2(P2[3], d1[j][a], m1));
        d0[j][a] = e0;
        d1[j][a] = e1;
      }
    }
    for (int h = woff[k - 1]; h < woff[k]; ++h) {
      const float4 q = hs[h];
      const unsigned long long A0 = pk2(q.x, q.x), A1 = pk2(q.y, q.y), A2 = pk2(q.z, q.z);
#pragma unroll
      for (int j = 0; j < NP; ++j) {
        float s0, s1;
        upk2(fma2(A2, d0[j][2], fma2(A1, d0[j][1], mul2(A0, d0[j][0]))), s0, s1);
        hit[j][0] = hit[j][0] || s0 > q.w;
        hit[j][1] = hit[j][1] || s1 > q.w;
      }
    }
    bool done = true;
#pragma unroll
    for (int j = 0; j < NP; ++j) done = done && hit[j][0] && hit[j][1];
    if (__all_sync(0xffffffffu, done)) break;
  }
#pragma unroll
  for (int j = 0; j < NP; ++j)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int word = 2 * (p0 + j) + h;
      const unsigned bits = __ballot_sync(0xffffffffu, hit[j][h]);
      if (lane == 0 && word < w) out[word] = bits;
    }
}

// Warps take edges, kMaskChunk at a time, from a counter (edges differ widely in work).
template <bool kSmemXi>
__global__ void __launch_bounds__(kWarps * 32, PUMP_MASK_MIN_BLOCKS) k_edge_mask_hs(
    const float4* __restrict__ xp_g, int N, int W, const float* __restrict__ phi, const float* __restrict__ Lg,
    const float* __restrict__ linf_g, const int32_t* __restrict__ hs_off, const float4* __restrict__ hs_ab, int E,
    int w, unsigned long long* __restrict__ ctr, uint32_t* __restrict__ mask) {
  using namespace maskdev;
  extern __shared__ __align__(16) unsigned char smem[];
  float4* stage_all = reinterpret_cast<float4*>(smem);
  int32_t* woff_all = reinterpret_cast<int32_t*>(stage_all + kWarps * kHsStage);
  float4* xp_s = reinterpret_cast<float4*>(smem + edge_mask_hs_fixed_smem());
  const int npair = pair_count(w);
  const int xp_n = (W + 1) * 3 * npair * 32;
  if (kSmemXi)
    for (int k = threadIdx.x; k < xp_n; k += blockDim.x) xp_s[k] = xp_g[k];
  __syncthreads();
  const float4* xp = kSmemXi ? xp_s : xp_g;
  const unsigned long long I2[3] = {pk2(linf_g[0], linf_g[0]), pk2(linf_g[1], linf_g[1]), pk2(linf_g[2], linf_g[2])};
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float4* stage = stage_all + warp * kHsStage;
  int32_t* woff = woff_all + warp * (kMaxWaypoints + 1);
  for (;;) {
    unsigned long long t = 0;
    if (lane == 0) t = atomicAdd(ctr, (unsigned long long)kMaskChunk);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= (unsigned long long)E) break;
    const long long e1 = min((long long)E, (long long)t + kMaskChunk);
    for (long long e = (long long)t; e < e1; ++e) {
      const int32_t* off = hs_off + (size_t)e * W;
      const int32_t o0 = off[0], o1 = off[W];
      uint32_t* out = mask + (size_t)e * w;
      if (o0 == o1) {
        for (int word = lane; word < w; word += 32) out[word] = 0u;
        continue;
      }
      const float4 ph = *reinterpret_cast<const float4*>(phi + 4 * e);
      const float l0 = Lg[3 * e], l1 = Lg[3 * e + 1], l2 = Lg[3 * e + 2];
      // waypoint offsets relative to the edge's first half-space, and the last waypoint with one
      int k_last = 0;
      for (int k = lane; k <= W; k += 32) {
        woff[k] = off[k] - o0;
        if (k > 0 && off[k] > off[k - 1]) k_last = max(k_last, k);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) k_last = max(k_last, __shfl_xor_sync(0xffffffffu, k_last, o));
      const int nh = o1 - o0;
      const bool staged = nh <= kHsStage;
      if (staged)
        for (int h = lane; h < nh; h += 32) stage[h] = hs_ab[o0 + h];
      __syncwarp();
      const float4* hs = staged ? stage : hs_ab + o0;
      const unsigned long long P2[4] = {pk2(ph.x, ph.x), pk2(ph.y, ph.y), pk2(ph.z, ph.z), pk2(ph.w, ph.w)};
      const unsigned long long L2[3] = {pk2(l0, l0), pk2(l1, l1), pk2(l2, l2)};
      int p = 0;
      for (; p + 2 <= npair; p += 2) pair_pass_hs<2>(xp, npair, P2, L2, I2, woff, hs, k_last, p, w, lane, out);
      for (; p < npair; ++p) pair_pass_hs<1>(xp, npair, P2, L2, I2, woff, hs, k_last, p, w, lane, out);
      __syncwarp();
    }
  }
}

}  // namespace

size_t edge_mask_smem(int N, int W, int nb, bool xi_in_smem) {
  size_t b = edge_mask_fixed_smem(nb);
  if (xi_in_smem) b += sizeof(float4) * (size_t)(W + 1) * 3 * maskdev::pair_count(N / 32) * 32;
  return b;
}

struct OccEntry {
  const void* kernel;
  size_t smem;
  int dev, per_sm;
};
static std::mutex g_occ_mu;
static std::vector<OccEntry> g_occ;
constexpr size_t kMaskSmemMax = 200 * 1024;

// Blocks for `items` work items: resident blocks per SM (queried once per kernel, size and
// device) times the SMs, at most one block per items_per_block items.
template <typename K>
static int occupancy_grid(K kernel, size_t smem, long long items_per_block, long long items, int* grid) {
  if (smem > kMaskSmemMax) return PUMP_ERR_INVALID_ARG;
  int dev = 0;
  PUMP_CUDA_TRY(cudaGetDevice(&dev));
  int per_sm = -1;
  {
    std::lock_guard<std::mutex> lk(g_occ_mu);
    for (const auto& o : g_occ)
      if (o.kernel == (const void*)kernel && o.smem == smem && o.dev == dev) per_sm = o.per_sm;
  }
  if (per_sm < 0) {
    // one ceiling for every size (the attribute belongs to the kernel)
    PUMP_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaskSmemMax));
    PUMP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kWarps * 32, smem));
    std::lock_guard<std::mutex> lk(g_occ_mu);
    g_occ.push_back({(const void*)kernel, smem, dev, per_sm});
  }
  if (per_sm < 1) per_sm = 1;
  long long want = (items + items_per_block - 1) / items_per_block;
  long long gsz = (long long)num_sms() * per_sm;
  if (gsz > want) gsz = want;
  if (gsz < 1) gsz = 1;
  *grid = (int)gsz;
  return PUMP_OK;
}

// Obstacle-independent per-edge position boxes (graph build).
int compute_edge_bounds(pump_graph* g, cudaStream_t s) {
  if (g->E == 0) return PUMP_OK;
  g->dmax = (unsigned int*)graph_alloc(g, sizeof(unsigned int) * (size_t)g->E, s);
  unsigned int* dbound = g->dmax;
  if (!dbound) return PUMP_ERR_OOM;
  const int npair = maskdev::pair_count(g->n_words);
  const size_t smem_xi = sizeof(float4) * (size_t)(g->W + 1) * 3 * npair * 32;
  const bool use_smem = smem_xi <= 160 * 1024;
  const long long items = (long long)g->E;  // a warp per edge
  int grid = 1;
  if (use_smem) {
    {
      const int rco = occupancy_grid(k_edge_bound<true>, smem_xi, kWarps, items, &grid);
      if (rco) return rco;
    }
    k_edge_bound<true><<<grid, kWarps * 32, smem_xi, s>>>(g->xi_p, npair, g->W, g->phi, g->L, g->linf_dev, g->E,
                                                          dbound);
    note_launch();
  } else {
    {
      const int rco = occupancy_grid(k_edge_bound<false>, 16, kWarps, items, &grid);
      if (rco) return rco;
    }
    k_edge_bound<false><<<grid, kWarps * 32, 16, s>>>(g->xi_p, npair, g->W, g->phi, g->L, g->linf_dev, g->E,
                                                      dbound);
    note_launch();
  }
  k_edge_ibox<<<(g->E + 255) / 256, 256, 0, s>>>(g->nom, dbound, g->E, g->W, g->ibox);
  note_launch();
  PUMP_CUDA_TRY(cudaGetLastError());
  return PUMP_OK;
}

int scan_counts(const int32_t* in, int n, int32_t* out, cudaStream_t s);

// HSMC half-spaces of every waypoint (graph build, after the deviation bounds).
int build_halfspaces(pump_graph* g, cudaStream_t s) {
  const long long EW = (long long)g->E * g->W;
  if (EW > (long long)INT32_MAX - 1) return PUMP_ERR_INVALID_ARG;
  g->hs_off = (int32_t*)graph_alloc(g, sizeof(int32_t) * (size_t)(EW + 1), s);
  int32_t* cnt = (int32_t*)dev_alloc(sizeof(int32_t) * (size_t)(EW + 1), s);
  if (!g->hs_off || !cnt) return PUMP_ERR_OOM;
  const size_t smem = sizeof(float) * 6 * (size_t)std::max(g->n_boxes, 1);
  const int grid = (int)std::min<long long>((EW + 255) / 256, (long long)num_sms() * 8);
  if (EW > 0) {
    k_hs_build<false><<<grid, 256, smem, s>>>(g->nom, g->nvel, g->dmax, g->boxes, g->n_boxes, g->E, g->W, cnt,
                                              nullptr, nullptr);
    note_launch();
  }
  int rc = scan_counts(cnt, (int)EW, g->hs_off, s);
  int32_t total = 0;
  if (!rc && cudaMemcpyAsync(&total, g->hs_off + EW, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    rc = PUMP_ERR_CUDA;
  if (!rc && cudaStreamSynchronize(s) != cudaSuccess) rc = PUMP_ERR_CUDA;
  dev_free(cnt, s);
  if (rc) return rc;
  g->hs_ab = (float4*)graph_alloc(g, sizeof(float4) * (size_t)std::max(total, 1), s);
  if (!g->hs_ab) return PUMP_ERR_OOM;
  if (EW > 0 && total > 0) {
    k_hs_build<true><<<grid, 256, smem, s>>>(g->nom, g->nvel, g->dmax, g->boxes, g->n_boxes, g->E, g->W, nullptr,
                                             g->hs_off, g->hs_ab);
    note_launch();
  }
  PUMP_CUDA_TRY(cudaGetLastError());
  return PUMP_OK;
}

static int compute_edge_masks_hs(pump_graph* g, cudaStream_t s) {
  const size_t smem_xi = edge_mask_hs_fixed_smem() +
                         sizeof(float4) * (size_t)(g->W + 1) * 3 * maskdev::pair_count(g->n_words) * 32;
  const bool use_smem = smem_xi <= 160 * 1024;
  const size_t smem = use_smem ? smem_xi : edge_mask_hs_fixed_smem();
  PUMP_CUDA_TRY(cudaMemsetAsync(g->wctr, 0, sizeof(unsigned long long), s));
  int grid = 1;
  if (use_smem) {
    const int rco = occupancy_grid(k_edge_mask_hs<true>, smem, kWarps * (long long)kMaskChunk, g->E, &grid);
    if (rco) return rco;
    k_edge_mask_hs<true><<<grid, kWarps * 32, smem, s>>>(g->xi_p, g->N, g->W, g->phi, g->L, g->linf_dev, g->hs_off,
                                                         g->hs_ab, g->E, g->n_words, g->wctr, g->emask);
  } else {
    const int rco = occupancy_grid(k_edge_mask_hs<false>, smem, kWarps * (long long)kMaskChunk, g->E, &grid);
    if (rco) return rco;
    k_edge_mask_hs<false><<<grid, kWarps * 32, smem, s>>>(g->xi_p, g->N, g->W, g->phi, g->L, g->linf_dev, g->hs_off,
                                                          g->hs_ab, g->E, g->n_words, g->wctr, g->emask);
  }
  note_launch();
  PUMP_CUDA_TRY(cudaGetLastError());
  g->masks_ready = true;
  return PUMP_OK;
}

// Launch of the query pass with kNP word pairs per warp pass.
template <bool kSmemXi, int kNP>
static int launch_edge_mask(pump_graph* g, size_t smem, int chunk, cudaStream_t s) {
  int grid = 1;
  const int rco = occupancy_grid(k_edge_mask<kSmemXi, kNP>, smem, kWarps * (long long)chunk, g->E, &grid);
  if (rco) return rco;
  k_edge_mask<kSmemXi, kNP><<<grid, kWarps * 32, smem, s>>>(g->xi_p, g->N, g->W, g->phi, g->L, g->nom, g->linf_dev,
                                                            g->ibox, g->dmax, g->boxes, g->n_boxes, g->E,
                                                            g->n_words, g->wctr, chunk, g->emask);
  note_launch();
  return PUMP_OK;
}

// pairs: word pairs per warp pass (1 or 2; 0 = 2); chunk: edges a warp takes at a time (0 = 4).
int compute_edge_masks(pump_graph* g, cudaStream_t s, int pairs, int chunk) {
  if (g->E == 0) {
    g->masks_ready = true;
    return PUMP_OK;
  }
  if (g->hsmc) return compute_edge_masks_hs(g, s);
  const size_t smem_xi = edge_mask_smem(g->N, g->W, g->n_boxes, true);
  const bool use_smem = smem_xi <= 160 * 1024;
  const size_t smem = use_smem ? smem_xi : edge_mask_smem(g->N, g->W, g->n_boxes, false);
  if (chunk <= 0) chunk = kMaskChunk;
  PUMP_CUDA_TRY(cudaMemsetAsync(g->wctr, 0, sizeof(unsigned long long), s));
  int rc;
  if (pairs == 1)
    rc = use_smem ? launch_edge_mask<true, 1>(g, smem, chunk, s) : launch_edge_mask<false, 1>(g, smem, chunk, s);
  else
    rc = use_smem ? launch_edge_mask<true, 2>(g, smem, chunk, s) : launch_edge_mask<false, 2>(g, smem, chunk, s);
  if (rc) return rc;
  PUMP_CUDA_TRY(cudaGetLastError());
  g->masks_ready = true;
  return PUMP_OK;
}

// Masks of n listed edges into out (n x w words); *bad (device, may be null) counts ids outside
// [0, E).  Enqueued only.
int compute_edge_masks_list(pump_graph* g, const int32_t* elist, long long n, uint32_t* out, uint32_t* bad,
                            cudaStream_t s) {
  const size_t smem_xi = edge_mask_smem(g->N, g->W, g->n_boxes, true);
  const bool use_smem = smem_xi <= 160 * 1024;
  const size_t smem = use_smem ? smem_xi : edge_mask_smem(g->N, g->W, g->n_boxes, false);
  // the list's take counter, and a count of bad ids when the caller keeps none
  unsigned long long* scratch = (unsigned long long*)dev_alloc(2 * sizeof(unsigned long long), s);
  if (!scratch) return PUMP_ERR_OOM;
  unsigned int* badc = bad ? bad : reinterpret_cast<unsigned int*>(scratch + 1);
  int rc = PUMP_OK;
  if (cudaMemsetAsync(scratch, 0, 2 * sizeof(unsigned long long), s) != cudaSuccess ||
      (bad && cudaMemsetAsync(bad, 0, sizeof(unsigned int), s) != cudaSuccess))
    rc = PUMP_ERR_CUDA;
  int grid = 1;
  if (!rc && n > 0)
    rc = use_smem ? occupancy_grid(k_edge_mask_list<true>, smem, kWarps * (long long)kMaskChunk, n, &grid)
                  : occupancy_grid(k_edge_mask_list<false>, smem, kWarps * (long long)kMaskChunk, n, &grid);
  if (!rc && n > 0) {
    if (use_smem)
      k_edge_mask_list<true><<<grid, kWarps * 32, smem, s>>>(g->xi_p, g->N, g->W, g->phi, g->L, g->nom, g->linf_dev,
                                                             g->ibox, g->dmax, g->boxes, g->n_boxes, (int)g->E,
                                                             g->n_words, elist, n, scratch, kMaskChunk, out, badc);
    else
      k_edge_mask_list<false><<<grid, kWarps * 32, smem, s>>>(g->xi_p, g->N, g->W, g->phi, g->L, g->nom, g->linf_dev,
                                                              g->ibox, g->dmax, g->boxes, g->n_boxes, (int)g->E,
                                                              g->n_words, elist, n, scratch, kMaskChunk, out, badc);
    note_launch();
    if (cudaGetLastError() != cudaSuccess) rc = PUMP_ERR_CUDA;
  }
  dev_free(scratch, s);
  return rc;
}

// Box masks of several graphs in one launch of k_edge_mask_batch (HSMC graphs and graphs without
// edges take their own path).  span: edges per item (0 = 1024); pairs and chunk as above.
int compute_edge_masks_batch(pump_graph* const* gs, int nq, cudaStream_t s, int pairs, int chunk, int span) {
  if (chunk <= 0) chunk = kMaskChunk;
  if (span <= 0) span = 1024;
  std::vector<MaskJob> jobs;
  std::vector<long long> item0(1, 0);
  std::vector<pump_graph*> done;
  size_t smem_fixed = 0, smem_xi = 0;
  for (int q = 0; q < nq; ++q) {
    pump_graph* g = gs[q];
    if (g->E == 0 || g->hsmc) {
      const int rc = compute_edge_masks(g, s, pairs, chunk);
      if (rc) return rc;
      continue;
    }
    smem_fixed = std::max(smem_fixed, edge_mask_smem(g->N, g->W, g->n_boxes, false));
    smem_xi = std::max(smem_xi, edge_mask_smem(g->N, g->W, g->n_boxes, true));
  }
  // one allocation for every job: the normals of a job stay in shared memory when its staging
  // fits the launch's (the largest that fits 160 KiB)
  const size_t smem = smem_xi <= 160 * 1024 ? smem_xi : std::max(smem_fixed, (size_t)160 * 1024);
  for (int q = 0; q < nq; ++q) {
    pump_graph* g = gs[q];
    if (g->E == 0 || g->hsmc) continue;
    MaskJob J;
    J.xp = g->xi_p;
    J.phi = g->phi;
    J.L = g->L;
    J.nom = g->nom;
    J.linf = g->linf_dev;
    J.ibox = g->ibox;
    J.dmax = g->dmax;
    J.boxes = g->boxes;
    J.emask = g->emask;
    J.E = g->E;
    J.N = g->N;
    J.W = g->W;
    J.nb = g->n_boxes;
    J.w = g->n_words;
    J.xi_smem = edge_mask_smem(g->N, g->W, g->n_boxes, true) <= smem ? 1 : 0;
    jobs.push_back(J);
    item0.push_back(item0.back() + (g->E + span - 1) / span);
    done.push_back(g);
  }
  const int nj = (int)jobs.size();
  if (nj == 0) return PUMP_OK;
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  const size_t b_jobs = al(sizeof(MaskJob) * (size_t)nj), b_item = al(sizeof(long long) * (size_t)(nj + 1));
  unsigned char* buf = (unsigned char*)dev_alloc(b_jobs + b_item + 256, s);
  if (!buf) return PUMP_ERR_OOM;
  MaskJob* jobs_dev = reinterpret_cast<MaskJob*>(buf);
  long long* item0_dev = reinterpret_cast<long long*>(buf + b_jobs);
  unsigned long long* ctr = reinterpret_cast<unsigned long long*>(buf + b_jobs + b_item);
  int rc = PUMP_OK;
  if (cudaMemcpyAsync(jobs_dev, jobs.data(), sizeof(MaskJob) * nj, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(item0_dev, item0.data(), sizeof(long long) * (nj + 1), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemsetAsync(ctr, 0, sizeof(unsigned long long), s) != cudaSuccess)
    rc = PUMP_ERR_CUDA;
  int grid = 1;
  if (!rc)
    rc = pairs == 1 ? occupancy_grid(k_edge_mask_batch<1>, smem, 1, item0.back(), &grid)
                    : occupancy_grid(k_edge_mask_batch<2>, smem, 1, item0.back(), &grid);
  if (!rc) {
    if (pairs == 1)
      k_edge_mask_batch<1><<<grid, kWarps * 32, smem, s>>>(jobs_dev, item0_dev, nj, span, chunk, ctr);
    else
      k_edge_mask_batch<2><<<grid, kWarps * 32, smem, s>>>(jobs_dev, item0_dev, nj, span, chunk, ctr);
    note_launch();
    if (cudaGetLastError() != cudaSuccess) rc = PUMP_ERR_CUDA;
  }
  dev_free(buf, s);
  if (rc) return rc;
  for (pump_graph* g : done) g->masks_ready = true;
  return PUMP_OK;
}

}  // namespace pump
