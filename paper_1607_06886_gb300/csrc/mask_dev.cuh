// Particle collision mask of one edge (Section III-B, with a direct particle-in-box test in
// place of the half-space test): the per-edge work of the query pass, shared by the stand-alone
// mask kernel (edge_mask.cu) and the mask workers of the fused Explore launch
// (explore_cluster.cu).
//
// The particle deviations of an edge depend on its step h and the common normals, not on the
// obstacles.  Graph build records, per edge, a box holding every particle position (nominal
// waypoints widened by the largest |d0| of any particle).  A warp takes one edge: lanes test the
// obstacle boxes against that box, and an edge with no box left gets zero mask words without
// running its particles.  Otherwise lane l runs particle 32*word + l through the recurrence once
// per word and tests the left boxes; the mask word is the warp ballot of the per-particle OR over
// waypoints and boxes.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "pump_internal.cuh"

namespace pump {
namespace maskdev {

constexpr int kCandCap = 64;
// floats per box in shared memory, each coordinate twice (one packed FP32x2 operand):
// lo x x y y | lo z z, hi x x | hi y y z z, with -0 stored as +0
constexpr int kBoxStride = 12;

// Shared memory of one block of the query pass before the normals: boxes, per-warp candidate
// lists and per-warp waypoint box masks (16-byte aligned end).
__host__ __device__ constexpr size_t fixed_smem(int nb, int warps) {
  return (sizeof(float) * kBoxStride * (size_t)nb + sizeof(int) * warps * kCandCap +
          sizeof(uint32_t) * warps * kMaxWaypoints + 15) & ~(size_t)15;
}

// The particle deviation recurrence (Section III-B), per axis with normals (x0, x1): at step 0
// d0 = Linf0 x0, d1 = fma(Linf1, x0, Linf2 x1); at each step k, with the edge's Phi and L,
// n0 = L0 x0, n1 = fma(L1, x0, L2 x1), d0' = fma(P0, d0, fma(P1, d1, n0)),
// d1' = fma(P2, d0, fma(P3, d1, n1)), every product and fused multiply-add rounded to nearest in
// this order; the position offset at waypoint k is the new d0.  The passes below run it on two
// particles per packed register.

// Two floats in one 64-bit register and the packed FP32x2 operations of sm_100-class parts: each
// half is rounded exactly as the scalar __fmul_rn / fmaf, so pairs of particles advance with
// the same arithmetic in half the instructions.
__device__ __forceinline__ unsigned long long pk2(float a, float b) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void upk2(unsigned long long r, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b, unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ unsigned long long mul2(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

__device__ __forceinline__ unsigned long long sub2(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ unsigned long long add2(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

// Pair-major normals.  xi_p[((k * 3 + a) * npair + jp) * 32 + l] = (xi0 of particle 64 jp + l,
// xi0 of particle 64 jp + 32 + l, xi1 of the first, xi1 of the second) for waypoint step k, axis
// a: one 16-byte load gives a lane both halves of its particle pair (zeros past N).
__host__ __device__ constexpr int pair_count(int w) { return (w + 1) / 2; }

// NP pairs of mask words (pairs p0 .. p0 + NP - 1, i.e. words 2 p0 .. 2 (p0 + NP) - 1 below w):
// lane l advances particles 64 jp + l and 64 jp + 32 + l in the two halves of packed FP32x2
// registers (each half rounds exactly as the scalar recurrence above and the position add),
// through waypoints 1..k_last, and tests the boxes left at each.  The words are the warp ballots
// of each half.  The warp stops early once every lane's particles have hit.
//
// Box test on packed positions: lo <= p iff p - lo has its sign bit clear, and p <= hi iff hi - p
// has, for finite values with no -0 on either side (a difference of equal values is +0; only
// -0 - +0 gives -0).  Boxes are staged with -0 as +0, and the nominal waypoint is taken the same
// way, so no position is -0 (p = nominal + deviation is -0 only when both are).  Six packed
// subtractions and the OR of their sign bits test two particles against one box.  kStaged loads
// the box's three 16-byte rows one at a time beside their tests (fewer live registers); otherwise
// all three first.
template <int NP, bool kStaged>
__device__ __forceinline__ void pair_pass(const float4* __restrict__ xp, int npair, const unsigned long long (&P2)[4],
                                          const unsigned long long (&L2)[3], const unsigned long long (&I2)[3],
                                          const float* __restrict__ nm, int k_last, bool narrow, const uint32_t* wm,
                                          const int* my_cand, bool all, int nc, const float* boxes, int p0, int w,
                                          int lane, uint32_t* out) {
  unsigned long long d0[NP][3], d1[NP][3];
  unsigned long long acc[NP];  // the sign bit of each half: that particle has hit a box
  const float4* xq = xp + (size_t)p0 * 32 + lane;
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    acc[j] = 0ull;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float4 x = xq[((size_t)a * npair + j) * 32];
      const unsigned long long X0 = pk2(x.x, x.y), X1 = pk2(x.z, x.w);
      d0[j][a] = mul2(I2[0], X0);
      d1[j][a] = fma2(I2[1], X0, mul2(I2[2], X1));
    }
  }
  for (int k = 1; k <= k_last; ++k) {
    const float n0 = __fadd_rn(nm[(k - 1) * 3], 0.f), n1 = __fadd_rn(nm[(k - 1) * 3 + 1], 0.f),
                n2 = __fadd_rn(nm[(k - 1) * 3 + 2], 0.f);  // -0 as +0
    const unsigned long long N2[3] = {pk2(n0, n0), pk2(n1, n1), pk2(n2, n2)};
    const float4* xk = xq + (size_t)k * 3 * npair * 32;
    unsigned long long p[NP][3];  // positions, both halves
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
        p[j][a] = add2(N2[a], e0);
      }
    }
    unsigned bits = narrow ? wm[k - 1] : 0u;
    int c = 0;
    for (;;) {
      int o;
      if (narrow) {
        if (!bits) break;
        const int b = __ffs(bits) - 1;
        bits &= bits - 1u;
        o = my_cand[b];
      } else {
        if (c >= nc) break;
        o = all ? c : my_cand[c];
        ++c;
      }
      const ulonglong2* bq = reinterpret_cast<const ulonglong2*>(boxes + kBoxStride * o);
      if (kStaged) {
        unsigned long long ob[NP];
        const ulonglong2 q0 = bq[0];  // lo x, lo y
#pragma unroll
        for (int j = 0; j < NP; ++j) ob[j] = sub2(p[j][0], q0.x) | sub2(p[j][1], q0.y);
        const ulonglong2 q1 = bq[1];  // lo z, hi x
#pragma unroll
        for (int j = 0; j < NP; ++j) ob[j] |= sub2(p[j][2], q1.x) | sub2(q1.y, p[j][0]);
        const ulonglong2 q2 = bq[2];  // hi y, hi z
#pragma unroll
        for (int j = 0; j < NP; ++j) acc[j] |= ~(ob[j] | sub2(q2.x, p[j][1]) | sub2(q2.y, p[j][2]));
      } else {
        const ulonglong2 q0 = bq[0], q1 = bq[1], q2 = bq[2];
#pragma unroll
        for (int j = 0; j < NP; ++j)
          acc[j] |= ~(sub2(p[j][0], q0.x) | sub2(q1.y, p[j][0]) | sub2(p[j][1], q0.y) | sub2(q2.x, p[j][1]) |
                      sub2(p[j][2], q1.x) | sub2(q2.y, p[j][2]));
      }
    }
    unsigned long long all_hit = ~0ull;
#pragma unroll
    for (int j = 0; j < NP; ++j) all_hit &= acc[j];
    const bool done = (all_hit & 0x8000000080000000ull) == 0x8000000080000000ull;
    if (__all_sync(0xffffffffu, done)) break;
  }
#pragma unroll
  for (int j = 0; j < NP; ++j)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int word = 2 * (p0 + j) + h;
      const unsigned bits = __ballot_sync(0xffffffffu, ((acc[j] >> (32 * h + 31)) & 1ull) != 0);
      if (lane == 0 && word < w) out[word] = bits;
    }
}

// Stages the boxes in shared memory (kBoxStride floats per box) and, when given, the normals.
template <typename T>
__device__ __forceinline__ void stage(const float* __restrict__ boxes_g, int nb, float* boxes,
                                      const T* __restrict__ xi_g, T* xi_s, int xi_n) {
  for (int k = threadIdx.x; k < kBoxStride * nb; k += blockDim.x) {
    const int o = k / kBoxStride, c = k - o * kBoxStride;
    boxes[k] = __fadd_rn(boxes_g[6 * o + (c >> 1)], 0.f);  // -0 becomes +0, every other value stays
  }
  if (xi_s)
    for (int k = threadIdx.x; k < xi_n; k += blockDim.x) xi_s[k] = xi_g[k];
}

// The w mask words of edge e, written by the calling warp.  Boxes that miss the edge's position
// box cannot hold any of its particle positions; an edge with none left gets zero mask words
// without running the particles.  With at most 32 boxes left, the warp narrows them per waypoint:
// at waypoint k every particle position lies in [nominal_k - M, nominal_k + M] (M = the edge's
// largest |d0|, rounded the way the positions are), so only boxes meeting that box are tested
// there, and the particles run only up to the last waypoint that has one.  Each 32-particle word
// then runs the recurrence once and its lanes stop testing when all of them have hit (up to
// kMaxNP word pairs side by side per pass: fewer live registers with 1).  With [p_first, p_last)
// only those word pairs are computed (an edge with no box left still gets all its words zeroed).
// my_cand (kCandCap ints) and wm (kMaxWaypoints words) are the warp's shared-memory scratch.
// The words go to row `row` of mask (row < 0: row e).
template <int kMaxNP = 2, bool kStaged = true>
__device__ __forceinline__ void edge_mask_one(long long e, const float4* __restrict__ xp, int N, int W,
                                              const float* __restrict__ phi, const float* __restrict__ Lg,
                                              const float* __restrict__ nom, const float (&linf)[3],
                                              const float* __restrict__ ibox_g, const unsigned int* __restrict__ dmax,
                                              const float* boxes, int nb, int w, int* my_cand, uint32_t* wm, int lane,
                                              uint32_t* __restrict__ mask, int p_first = 0, int p_last = -1,
                                              long long row = -1) {
  const float* ib = ibox_g + 6 * e;
  const float lo0 = ib[0], lo1 = ib[1], lo2 = ib[2], hi0 = ib[3], hi1 = ib[4], hi2 = ib[5];
  int n_cand = 0;
  for (int base = 0; base < nb; base += 32) {
    const int o = base + lane;
    bool ov = false;
    if (o < nb) {
      const float* b = boxes + kBoxStride * o;
      ov = b[0] <= hi0 && lo0 <= b[6] && b[2] <= hi1 && lo1 <= b[8] && b[4] <= hi2 && lo2 <= b[10];
    }
    const unsigned bal = __ballot_sync(0xffffffffu, ov);
    const int pos = n_cand + __popc(bal & ((1u << lane) - 1u));
    if (ov && pos < kCandCap) my_cand[pos] = o;
    n_cand += __popc(bal);
  }
  __syncwarp();
  if (n_cand == 0) {
    for (int word = lane; word < w; word += 32) mask[(size_t)(row < 0 ? e : row) * w + word] = 0u;
    __syncwarp();
    return;
  }
  // the live edge's other reads issued together: the narrowing and the passes would otherwise
  // wait for them one after another
  const float M = __uint_as_float(dmax[e]);
  const float4 ph = *reinterpret_cast<const float4*>(phi + 4 * e);
  const float l0 = Lg[3 * e], l1 = Lg[3 * e + 1], l2 = Lg[3 * e + 2];
  const float* nm = nom + (size_t)e * W * 3;
  asm volatile("prefetch.global.L1 [%0];" ::"l"(nm));
  asm volatile("prefetch.global.L1 [%0];" ::"l"(nm + (W * 3 - 1)));
  int k_last = W;
  const bool narrow = n_cand <= 32;
  if (narrow) {
    // boxes per waypoint: lane c tests candidate c against waypoint k's position box
    const float* bc = boxes + kBoxStride * my_cand[lane < n_cand ? lane : 0];
    k_last = 0;
    for (int k = 1; k <= W; ++k) {
      const float n0 = nm[(k - 1) * 3], n1 = nm[(k - 1) * 3 + 1], n2 = nm[(k - 1) * 3 + 2];
      const bool ov = lane < n_cand && bc[0] <= __fadd_rn(n0, M) && __fsub_rn(n0, M) <= bc[6] &&
                      bc[2] <= __fadd_rn(n1, M) && __fsub_rn(n1, M) <= bc[8] &&
                      bc[4] <= __fadd_rn(n2, M) && __fsub_rn(n2, M) <= bc[10];
      const unsigned m = __ballot_sync(0xffffffffu, ov);
      if (lane == 0) wm[k - 1] = m;
      if (m) k_last = k;
    }
    __syncwarp();
  }
  if (k_last == 0) {
    for (int word = lane; word < w; word += 32) mask[(size_t)(row < 0 ? e : row) * w + word] = 0u;
    __syncwarp();
    return;
  }
  const bool all = n_cand > kCandCap;
  const int nc = all ? nb : n_cand;
  const unsigned long long P2[4] = {pk2(ph.x, ph.x), pk2(ph.y, ph.y), pk2(ph.z, ph.z), pk2(ph.w, ph.w)};
  const unsigned long long L2[3] = {pk2(l0, l0), pk2(l1, l1), pk2(l2, l2)};
  const unsigned long long I2[3] = {pk2(linf[0], linf[0]), pk2(linf[1], linf[1]), pk2(linf[2], linf[2])};
  const int npair = pair_count(w);
  const int pe = p_last < 0 ? npair : min(p_last, npair);
  uint32_t* out = mask + (size_t)(row < 0 ? e : row) * w;
  int p = p_first;
  if (kMaxNP >= 2)
    for (; p + 2 <= pe; p += 2)
      pair_pass<2, kStaged>(xp, npair, P2, L2, I2, nm, k_last, narrow, wm, my_cand, all, nc, boxes, p, w, lane, out);
  for (; p < pe; ++p) pair_pass<1, kStaged>(xp, npair, P2, L2, I2, nm, k_last, narrow, wm, my_cand, all, nc, boxes, p, w, lane, out);
  __syncwarp();
}

}  // namespace maskdev
}  // namespace pump
