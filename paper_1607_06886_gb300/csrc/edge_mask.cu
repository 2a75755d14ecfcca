// Edge particle collision masks (Section III-B, with a direct particle-in-box
// test in place of the half-space test).
//
// One warp handles one (edge, 32-particle word): lane l is particle
// 32*word + l.  The common normals xi_t[k][axis][i] and the boxes are staged
// in shared memory once per block; the grid is persistent over the
// (edge, word) items.  Pass 1 runs the particle recurrence and reduces the
// warp's exact position bounding box; boxes that miss it cannot hold any of
// the warp's positions and are culled.  Pass 2 re-runs the (deterministic)
// recurrence only when some box survives and tests the survivors; the mask
// word is the warp ballot of the per-particle OR over waypoints and boxes.
#include <cuda_runtime.h>

#include "pump_internal.cuh"

namespace pump {
namespace {

constexpr int kWarps = 8;
constexpr int kCandCap = 64;

__device__ __forceinline__ void dev_init(const float* linf, float2 x, float& d0, float& d1) {
  d0 = __fmul_rn(linf[0], x.x);
  d1 = fmaf(linf[1], x.x, __fmul_rn(linf[2], x.y));
}

__device__ __forceinline__ void dev_step(const float* P, const float* L, float2 x, float& d0, float& d1) {
  float n0 = __fmul_rn(L[0], x.x);
  float n1 = fmaf(L[1], x.x, __fmul_rn(L[2], x.y));
  float e0 = fmaf(P[0], d0, fmaf(P[1], d1, n0));
  float e1 = fmaf(P[2], d0, fmaf(P[3], d1, n1));
  d0 = e0;
  d1 = e1;
}

template <bool kSmemXi>
__global__ void __launch_bounds__(kWarps * 32) k_edge_mask(const float2* __restrict__ xi_g, int N, int W,
                                                           const float* __restrict__ phi, const float* __restrict__ Lg,
                                                           const float* __restrict__ nom, const float* __restrict__ linf_g,
                                                           const float* __restrict__ boxes_g, int nb, int E, int w,
                                                           uint32_t* __restrict__ mask) {
  extern __shared__ __align__(16) unsigned char smem[];
  float* boxes = reinterpret_cast<float*>(smem);
  int* cand = reinterpret_cast<int*>(boxes + 6 * nb);
  float2* xi_s = reinterpret_cast<float2*>(cand + kWarps * kCandCap);
  for (int k = threadIdx.x; k < 6 * nb; k += blockDim.x) boxes[k] = boxes_g[k];
  const int xi_n = (W + 1) * 3 * N;
  if (kSmemXi)
    for (int k = threadIdx.x; k < xi_n; k += blockDim.x) xi_s[k] = xi_g[k];
  __syncthreads();
  const float2* xi = kSmemXi ? xi_s : xi_g;
  const float linf[3] = {linf_g[0], linf_g[1], linf_g[2]};
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int* my_cand = cand + warp * kCandCap;
  const long long items = (long long)E * w;
  for (long long it = (long long)blockIdx.x * kWarps + warp; it < items; it += (long long)gridDim.x * kWarps) {
    const int e = (int)(it / w), word = (int)(it % w);
    const int i = word * 32 + lane;
    const float P[4] = {phi[4 * (size_t)e], phi[4 * (size_t)e + 1], phi[4 * (size_t)e + 2], phi[4 * (size_t)e + 3]};
    const float L[3] = {Lg[3 * (size_t)e], Lg[3 * (size_t)e + 1], Lg[3 * (size_t)e + 2]};
    const float* nm = nom + (size_t)e * W * 3;
    // pass 1: bounding box of the warp's positions
    float d0[3], d1[3], lo[3], hi[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      dev_init(linf, xi[(size_t)a * N + i], d0[a], d1[a]);
      lo[a] = __int_as_float(0x7f800000);
      hi[a] = -lo[a];
    }
    for (int k = 1; k <= W; ++k) {
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        dev_step(P, L, xi[((size_t)k * 3 + a) * N + i], d0[a], d1[a]);
        float p = __fadd_rn(nm[(k - 1) * 3 + a], d0[a]);
        lo[a] = fminf(lo[a], p);
        hi[a] = fmaxf(hi[a], p);
      }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        lo[a] = fminf(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
        hi[a] = fmaxf(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
      }
    }
    // cull: boxes overlapping the bounding box (closed intervals)
    int n_cand = 0;
    for (int base = 0; base < nb; base += 32) {
      int o = base + lane;
      bool ov = false;
      if (o < nb) {
        const float* b = boxes + 6 * o;
        ov = b[0] <= hi[0] && lo[0] <= b[3] && b[1] <= hi[1] && lo[1] <= b[4] && b[2] <= hi[2] && lo[2] <= b[5];
      }
      unsigned bal = __ballot_sync(0xffffffffu, ov);
      int pos = n_cand + __popc(bal & ((1u << lane) - 1u));
      if (ov && pos < kCandCap) my_cand[pos] = o;
      n_cand += __popc(bal);
    }
    __syncwarp();
    uint32_t word_bits = 0;
    if (n_cand > 0) {
      const bool all = n_cand > kCandCap;
      const int nc = all ? nb : n_cand;
      bool hit = false;
#pragma unroll
      for (int a = 0; a < 3; ++a) dev_init(linf, xi[(size_t)a * N + i], d0[a], d1[a]);
      for (int k = 1; k <= W; ++k) {
        float p[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          dev_step(P, L, xi[((size_t)k * 3 + a) * N + i], d0[a], d1[a]);
          p[a] = __fadd_rn(nm[(k - 1) * 3 + a], d0[a]);
        }
        for (int c = 0; c < nc && !hit; ++c) {
          const int o = all ? c : my_cand[c];
          hit = in_box_dev(p[0], p[1], p[2], boxes + 6 * o);
        }
      }
      word_bits = __ballot_sync(0xffffffffu, hit);
    }
    if (lane == 0) mask[(size_t)e * w + word] = word_bits;
    __syncwarp();
  }
}

}  // namespace

size_t edge_mask_smem(int N, int W, int nb, bool xi_in_smem) {
  size_t b = sizeof(float) * 6 * (size_t)nb + sizeof(int) * kWarps * kCandCap;
  b = (b + 15) & ~(size_t)15;
  if (xi_in_smem) b += sizeof(float2) * (size_t)(W + 1) * 3 * N;
  return b;
}

int compute_edge_masks(pump_graph* g, cudaStream_t s) {
  if (g->E == 0) {
    g->masks_ready = true;
    return PUMP_OK;
  }
  const size_t smem_xi = edge_mask_smem(g->N, g->W, g->n_boxes, true);
  const bool use_smem = smem_xi <= 160 * 1024;
  const size_t smem = use_smem ? smem_xi : edge_mask_smem(g->N, g->W, g->n_boxes, false);
  int blocks_per_sm = 0;
  if (use_smem) {
    PUMP_CUDA_TRY(cudaFuncSetAttribute(k_edge_mask<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    PUMP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, k_edge_mask<true>, kWarps * 32, smem));
  } else {
    PUMP_CUDA_TRY(cudaFuncSetAttribute(k_edge_mask<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    PUMP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, k_edge_mask<false>, kWarps * 32, smem));
  }
  if (blocks_per_sm < 1) blocks_per_sm = 1;
  long long items = (long long)g->E * g->n_words;
  long long want = (items + kWarps - 1) / kWarps;
  long long grid = (long long)num_sms() * blocks_per_sm;
  if (grid > want) grid = want;
  if (use_smem) {
    k_edge_mask<true><<<(int)grid, kWarps * 32, smem, s>>>(g->xi_t, g->N, g->W, g->phi, g->L, g->nom, g->linf_dev,
                                                           g->boxes, g->n_boxes, g->E, g->n_words, g->emask);
    note_launch();
  } else {
    k_edge_mask<false><<<(int)grid, kWarps * 32, smem, s>>>(g->xi_t, g->N, g->W, g->phi, g->L, g->nom, g->linf_dev,
                                                            g->boxes, g->n_boxes, g->E, g->n_words, g->emask);
    note_launch();
  }
  PUMP_CUDA_TRY(cudaGetLastError());
  g->masks_ready = true;
  return PUMP_OK;
}

}  // namespace pump
