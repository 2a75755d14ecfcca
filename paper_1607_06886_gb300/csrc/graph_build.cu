// BuildGraph (Algorithm 3) on the device: SampleFree validity, Near with the
// optimal steering cost, Collision on the nominal connection, and the per-edge
// values the exploration uses (cost, duration, waypoint step, closed-loop
// Phi(h), noise factor L(h), nominal waypoints).  Compiled without FMA
// contraction so double-precision expressions round as written.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "pump_internal.cuh"

namespace pump {
namespace {

constexpr int kBlock = 256;

__global__ void k_node_flags(const float* __restrict__ states, int n, const float* __restrict__ boxes, int nb,
                             const int32_t* __restrict__ goal_idx, int n_goal, uint8_t* valid, uint8_t* is_goal) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < n) {
    float x = states[6 * v], y = states[6 * v + 1], z = states[6 * v + 2];
    bool in = false;
    for (int o = 0; o < nb && !in; ++o) in = in_box_dev(x, y, z, boxes + 6 * o);
    valid[v] = in ? 0 : 1;
    is_goal[v] = 0;
  }
}

__global__ void k_goal_flags(const int32_t* __restrict__ goal_idx, int n_goal, uint8_t* is_goal) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n_goal) is_goal[goal_idx[k]] = 1;
}

// Exact necessary conditions for float(Cost(v,u)) < r, evaluated in float with
// a 1e-4 relative margin (float rounding here is below 1e-6 relative):
//   Cost >= 2 |dv|                       (time term + velocity-change energy)
//   |dp| < |vbar| r + (3/32) r^2         (position energy 12|dp - vbar t|^2/t^3 < r - t, t < r)
__device__ inline bool prefilter(const float* sv, const float* su, float r) {
  float dv2 = 0.f, dp2 = 0.f, vb2 = 0.f;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    float dv = su[3 + j] - sv[3 + j], dp = su[j] - sv[j], vb = 0.5f * (su[3 + j] + sv[3 + j]);
    dv2 += dv * dv;
    dp2 += dp * dp;
    vb2 += vb * vb;
  }
  const float m = 1.0001f;
  if (2.f * sqrtf(dv2) >= r * m) return false;
  if (sqrtf(dp2) >= (sqrtf(vb2) * r + 0.09375f * r * r) * m + 1e-6f) return false;
  return true;
}

// A uniform grid over the valid nodes' positions, so that a source scans only the cells its
// prefilter bound can reach.  Cell index per axis: min(G - 1, floor((p - lo) * inv)), monotone in
// p, so every target within the bound of a source lies in the cells between the indices of the
// bound's two ends.
constexpr int kGridMax = 32;  // cells per axis at most
struct Grid {
  float lo[3], inv[3];
  int G[3];
  float vmax;  // largest |velocity| of a valid node
};
__device__ __forceinline__ int grid_cell(const Grid& gr, int a, float p) {
  const float t = floorf(__fmul_rn(__fsub_rn(p, gr.lo[a]), gr.inv[a]));
  return t < 0.f ? 0 : (t >= (float)(gr.G[a] - 1) ? gr.G[a] - 1 : (int)t);
}
// Half-width of the position window a pair with source speed |v_v| = vv can pass: the prefilter's
// position threshold with |vbar| <= (vmax + vv) / 2, widened by 1e-4 relative and 1e-6 absolute
// (the float rounding of the prefilter's sums and square roots is below 1e-6 relative).
__device__ __forceinline__ float grid_bound(const Grid& gr, float vv, float r) {
  return ((0.5f * (gr.vmax + vv) * r + 0.09375f * r * r) * 1.0001f + 1e-6f) * 1.0001f + 1e-6f;
}

// One block: bounding box and largest speed of the valid nodes, then the grid (cells about a
// quarter of the widest bound per side, at most kGridMax per axis).
__global__ void k_grid_setup(const float* __restrict__ states, const uint8_t* __restrict__ valid, int n, float r,
                             Grid* out) {
  __shared__ float s_lo[3][32], s_hi[3][32], s_v[32];
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY}, vm = 0.f;
  for (int v = threadIdx.x; v < n; v += blockDim.x) {
    if (!valid[v]) continue;
    const float* x = states + 6 * v;
    for (int a = 0; a < 3; ++a) {
      lo[a] = fminf(lo[a], x[a]);
      hi[a] = fmaxf(hi[a], x[a]);
    }
    vm = fmaxf(vm, sqrtf(x[3] * x[3] + x[4] * x[4] + x[5] * x[5]));
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    for (int a = 0; a < 3; ++a) {
      lo[a] = fminf(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
      hi[a] = fmaxf(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
    }
    vm = fmaxf(vm, __shfl_xor_sync(0xffffffffu, vm, o));
  }
  if (lane == 0) {
    for (int a = 0; a < 3; ++a) {
      s_lo[a][warp] = lo[a];
      s_hi[a][warp] = hi[a];
    }
    s_v[warp] = vm;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nwarp = (int)(blockDim.x >> 5);
    Grid gr;
    gr.vmax = 0.f;
    for (int w = 0; w < nwarp; ++w) gr.vmax = fmaxf(gr.vmax, s_v[w]);
    gr.vmax *= 1.0001f;
    const float cell = fmaxf(0.25f * ((gr.vmax * r + 0.09375f * r * r) * 1.0001f + 1e-6f), 1e-30f);
    for (int a = 0; a < 3; ++a) {
      float l = INFINITY, h = -INFINITY;
      for (int w = 0; w < nwarp; ++w) {
        l = fminf(l, s_lo[a][w]);
        h = fmaxf(h, s_hi[a][w]);
      }
      if (!(h >= l)) {  // no valid node
        l = 0.f;
        h = 0.f;
      }
      const float ext = h - l;
      int G = (int)fminf((float)kGridMax, fmaxf(1.f, ceilf(ext / cell)));
      gr.lo[a] = l;
      gr.G[a] = G;
      gr.inv[a] = ext > 0.f ? (float)G / ext : 0.f;
    }
    *out = gr;
  }
}

__global__ void k_grid_count(const float* __restrict__ states, const uint8_t* __restrict__ valid, int n,
                             const Grid* __restrict__ grid, int32_t* __restrict__ cnt) {
  const Grid gr = *grid;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    if (!valid[v]) continue;
    const float* x = states + 6 * v;
    const int c = (grid_cell(gr, 2, x[2]) * gr.G[1] + grid_cell(gr, 1, x[1])) * gr.G[0] + grid_cell(gr, 0, x[0]);
    atomicAdd(cnt + c, 1);
  }
}

// Nodes by cell (cells in z, y, x order; the order inside a cell is not fixed, and nothing
// downstream depends on it: kept pairs are placed by their rank in the keep bitmap).
__global__ void k_grid_scatter(const float* __restrict__ states, const uint8_t* __restrict__ valid, int n,
                               const Grid* __restrict__ grid, const long long* __restrict__ off,
                               int32_t* __restrict__ cursor, int32_t* __restrict__ sorted,
                               float* __restrict__ sorted_states) {
  const Grid gr = *grid;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    if (!valid[v]) continue;
    const float* x = states + 6 * v;
    const int c = (grid_cell(gr, 2, x[2]) * gr.G[1] + grid_cell(gr, 1, x[1])) * gr.G[0] + grid_cell(gr, 0, x[0]);
    const long long i = off[c] + atomicAdd(cursor + c, 1);
    sorted[i] = v;
    for (int j = 0; j < 6; ++j) sorted_states[6 * i + j] = x[j];  // the states in cell order too
  }
}

// Exclusive scan of the grid's cell counts into 64-bit offsets (the cell count read from the grid).
__global__ void k_grid_scan(const int32_t* __restrict__ in, const Grid* __restrict__ grid, long long* __restrict__ out);

// The pairs (v, u), v != u, both valid, that pass the prefilter, row by row: a warp per source v
// scans the grid rows (y, z) its bound reaches, each row's cells [x0, x1] one contiguous slice of
// the sorted nodes, 32 targets at a time.  Pass 1 counts each row's pairs, an exclusive scan gives
// the row offsets, and pass 2 writes each row's pairs from its offset (the same targets in the
// same order as pass 1 counted them): no atomics.
template <bool kWrite>
__global__ void k_prefilter(const float* __restrict__ states, const uint8_t* __restrict__ valid, int n, float r,
                            const Grid* __restrict__ grid, const long long* __restrict__ coff,
                            const int32_t* __restrict__ sorted, const float* __restrict__ sorted_states,
                            int32_t* __restrict__ cnt, const long long* __restrict__ off, int2* __restrict__ list) {
  const Grid gr = *grid;
  const int lane = threadIdx.x & 31;
  const int warps = (int)(((long long)gridDim.x * blockDim.x) >> 5);
  for (int v = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5); v < n; v += warps) {
    int c = 0;
    if (valid[v]) {
      float sv[6];
#pragma unroll
      for (int j = 0; j < 6; ++j) sv[j] = states[6 * v + j];
      const float R = grid_bound(gr, sqrtf(sv[3] * sv[3] + sv[4] * sv[4] + sv[5] * sv[5]), r);
      int c0[3], c1[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        // the window's ends, widened by their own rounding (relative to the coordinate's size)
        const float w = R + (fabsf(sv[a]) + R) * 1e-6f;
        c0[a] = grid_cell(gr, a, __fsub_rn(sv[a], w));
        c1[a] = grid_cell(gr, a, __fadd_rn(sv[a], w));
      }
      long long base = kWrite ? off[v] : 0;
      const int ny = c1[1] - c0[1] + 1, nrows = ny * (c1[2] - c0[2] + 1);
      for (int rb = 0; rb < nrows; rb += 32) {
        // the slices of up to 32 grid rows (y, z), one per lane, loaded together
        long long sa = 0, se = 0;
        if (rb + lane < nrows) {
          const int q = rb + lane, cz = c0[2] + q / ny, cy = c0[1] + q % ny;
          const int row = (cz * gr.G[1] + cy) * gr.G[0];
          sa = coff[row + c0[0]];
          se = coff[row + c1[0] + 1];
        }
        const int nb = min(32, nrows - rb);
        for (int t = 0; t < nb; ++t) {
          const long long ia = __shfl_sync(0xffffffffu, sa, t), ie = __shfl_sync(0xffffffffu, se, t);
          for (long long i0 = ia; i0 < ie; i0 += 32) {
            const long long i = i0 + lane;
            const bool in = i < ie;
            const int u = in ? sorted[i] : v;
            const bool ok = in && u != v && prefilter(sv, sorted_states + 6 * (in ? i : ia), r);
            const unsigned bl = __ballot_sync(0xffffffffu, ok);
            if (kWrite && ok) list[base + c + __popc(bl & ((1u << lane) - 1u))] = make_int2(v, u);
            c += __popc(bl);
          }
        }
      }
    }
    if (!kWrite && lane == 0) cnt[v] = c;
  }
}

// Exclusive scan of n int32 counts into 64-bit offsets out[0..n] (out[n] = total); one block.
__global__ void k_scan_ll(const int32_t* __restrict__ in, int n, long long* __restrict__ out) {
  __shared__ long long part[1024];
  const int t = threadIdx.x, T = blockDim.x;
  const int per = (n + T - 1) / T;
  const int b0 = min(n, t * per), b1 = min(n, b0 + per);
  long long sum = 0;
  for (int i = b0; i < b1; ++i) sum += in[i];
  part[t] = sum;
  __syncthreads();
  for (int d = 1; d < T; d <<= 1) {
    const long long add = t >= d ? part[t - d] : 0;
    __syncthreads();
    part[t] += add;
    __syncthreads();
  }
  long long run = part[t] - sum;  // exclusive prefix of this thread's chunk
  for (int i = b0; i < b1; ++i) {
    out[i] = run;
    run += in[i];
  }
  if (t == T - 1) out[n] = part[T - 1];
}

__global__ void k_grid_scan(const int32_t* __restrict__ in, const Grid* __restrict__ grid, long long* __restrict__ out) {
  __shared__ long long part[1024];
  const int n = grid->G[0] * grid->G[1] * grid->G[2];
  const int t = threadIdx.x, T = blockDim.x;
  const int per = (n + T - 1) / T;
  const int b0 = min(n, t * per), b1 = min(n, b0 + per);
  long long sum = 0;
  for (int i = b0; i < b1; ++i) sum += in[i];
  part[t] = sum;
  __syncthreads();
  for (int d = 1; d < T; d <<= 1) {
    const long long add = t >= d ? part[t - d] : 0;
    __syncthreads();
    part[t] += add;
    __syncthreads();
  }
  long long run = part[t] - sum;
  for (int i = b0; i < b1; ++i) {
    out[i] = run;
    run += in[i];
  }
  if (t == T - 1) out[n] = part[T - 1];
}

// Float estimate of Cost(v,u), used only to skip pairs far above the radius.  Same monotone
// pieces as steer_dev; J is evaluated as tau + |dv|^2/tau + 12|dp - vbar tau|^2/tau^3, a sum
// of non-negative terms (no cancellation), at the float roots.  J(tau) >= Cost for every tau,
// and a minimum float cannot resolve is no deeper than float rounding, so a pair whose
// estimate exceeds r by 0.1 % is not a neighbour.  Returns false when undecided.
__device__ inline float st32_f(float a, float b, float c, float t) { return ((t * t - 4.f * a) * t + 24.f * b) * t - 36.f * c; }
__device__ inline float st32_fp(float a, float b, float t) { return (4.f * t * t - 8.f * a) * t + 24.f * b; }
__device__ inline float st32_root(float a, float b, float c, int which, float lo, float hi, bool inc) {
  float x = 0.5f * (lo + hi);
  for (int it = 0; it < 80; ++it) {
    const float gx = which == 0 ? st32_f(a, b, c, x) : st32_fp(a, b, x);
    if (gx == 0.f) return x;
    const bool right = inc ? (gx < 0.f) : (gx > 0.f);
    if (right) lo = x; else hi = x;
    const float dg = which == 0 ? st32_fp(a, b, x) : (12.f * x * x - 8.f * a);
    float xn = x - gx / dg;
    if (!(xn > lo && xn < hi)) xn = 0.5f * (lo + hi);
    const float step = fabsf(xn - x);
    x = xn;
    if (step <= 2.4e-7f * fabsf(x) || !(hi - lo > 1.2e-7f * fabsf(hi))) break;
  }
  return x;
}
__device__ inline bool steer_estimate(const float* xv, const float* xu, float* J_out, float* tmin = nullptr,
                                      int* n_min = nullptr, float* Jmin = nullptr) {
  float a = 0.f, b = 0.f, c = 0.f, dv2 = 0.f;
  float dp[3], vb[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    dp[j] = xu[j] - xv[j];
    const float v0 = xv[3 + j], v1 = xu[3 + j];
    vb[j] = 0.5f * (v0 + v1);
    a += v0 * v0 + v0 * v1 + v1 * v1;
    b += dp[j] * (v0 + v1);
    c += dp[j] * dp[j];
    dv2 += (v1 - v0) * (v1 - v0);
  }
  if (!(c > 0.f)) return false;
  const float tc = sqrtf(2.f * a / 3.f);
  const float hi_f = 1.f + fmaxf(4.f * a, fmaxf(24.f * fabsf(b), 36.f * c));
  float lo_s[2], hi_s[2];
  int ns = 0;
  if (st32_fp(a, b, tc) >= 0.f) {
    lo_s[ns] = 0.f; hi_s[ns++] = hi_f;
  } else {
    const float hi_fp = fmaxf(1.f + fmaxf(2.f * a, 6.f * fabsf(b)), tc * 2.f + 1.f);
    const float tb = st32_root(a, b, c, 1, tc, hi_fp, true);
    if (b > 0.f) {
      lo_s[ns] = 0.f; hi_s[ns++] = st32_root(a, b, c, 1, 0.f, tc, false);
    }
    lo_s[ns] = tb; hi_s[ns++] = fmaxf(hi_f, tb * 2.f + 1.f);
  }
  float best = __int_as_float(0x7f800000);
  bool any = false;
  for (int q = 0; q < ns; ++q) {
    if (!(st32_f(a, b, c, lo_s[q]) < 0.f && st32_f(a, b, c, hi_s[q]) > 0.f)) continue;
    const float t = st32_root(a, b, c, 0, lo_s[q], hi_s[q], true);
    if (!(t > 0.f)) continue;
    float r2 = 0.f;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const float d = dp[j] - vb[j] * t;
      r2 += d * d;
    }
    const float J = t + dv2 / t + 12.f * r2 / (t * t * t);
    if (tmin) {
      tmin[*n_min] = t;
      Jmin[*n_min] = J;
      ++*n_min;
    }
    best = fminf(best, J);
    any = true;
  }
  *J_out = best;
  return any;
}

// Collision(v, u): the nominal connection of duration tau (float) sampled at
// t_m = tau (m / 4W), m = 1..4W, positions (the double cubic at t_m) rounded to float, closed
// boxes; frac[m-1] = m / (4W) in double.  Evaluated in float with a rounding margin: the
// definition's sample position is the double cubic at t_m rounded to float; the float cubic
// (coefficients and Horner steps in float) is within eps of it, where eps bounds the rounding of
// every float step by 2^-15 (1 + M), M the largest |p0| + |v0| tau + |c2| tau^2 + |c3| tau^3 of
// the three axes (the actual error is below 2^-19 (1 + M)).  A sample more than eps outside a box
// on some axis misses it, one more than eps inside on every axis hits it; only samples within eps
// of a face are evaluated the definition's way, in double (k_collide).
// Near and Collision in passes over shrinking lists, so that each pass runs one uniform piece of
// work with full warps: k_steer_filter takes the float estimate of every listed pair and keeps the
// pairs it cannot reject (about one in four); k_steer_pairs refines their cost in double (FP64 is
// slow on this part, so it must not run on the few lanes of a warp whose pair survived) and
// passes the rare pairs that need the full analysis to k_steer_slow; k_collide tests the nominal
// connections of the pairs whose cost is below r in float, a warp per pair, and k_collide_exact
// settles the few pairs the float test leaves undecided.  Outputs are indexed by the
// pair and the keep bitmap is an OR, so the order of the lists does not matter.
__global__ void k_steer_filter(const float* __restrict__ states, const int2* __restrict__ list, long long n_list,
                               float r, uint2* __restrict__ one, unsigned long long* n_one, uint4* __restrict__ two,
                               unsigned long long* n_two, uint32_t* __restrict__ slow, unsigned long long* n_slow) {
  const int lane = threadIdx.x & 31;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long q0 = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); q0 < n_list; q0 += stride) {
    const long long q = q0 + lane;
    int kind = 0;  // 0 rejected, 1 one minimum, 2 two minima, 3 full analysis
    float tmin[2] = {0.f, 0.f};
    if (q < n_list) {
      const int2 vu = list[q];
      float fv[6], fu[6];
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        fv[j] = states[6 * vu.x + j];
        fu[j] = states[6 * vu.y + j];
      }
      float J32, Jmin[2];
      int nm = 0;
      const bool est = steer_estimate(fv, fu, &J32, tmin, &nm, Jmin);
      if (!(est && J32 > r * 1.001f)) {
        if (!est || nm < 1 || (nm == 2 && fabsf(Jmin[0] - Jmin[1]) <= 1e-4f * fmaxf(Jmin[0], Jmin[1])))
          kind = 3;
        else
          kind = nm;
      }
    }
    const unsigned b1 = __ballot_sync(0xffffffffu, kind == 1), b2 = __ballot_sync(0xffffffffu, kind == 2);
    const unsigned b3 = __ballot_sync(0xffffffffu, kind == 3);
    unsigned long long base1 = 0, base2 = 0, base3 = 0;
    if (lane == 0) {
      if (b1) base1 = atomicAdd(n_one, (unsigned long long)__popc(b1));
      if (b2) base2 = atomicAdd(n_two, (unsigned long long)__popc(b2));
      if (b3) base3 = atomicAdd(n_slow, (unsigned long long)__popc(b3));
    }
    base1 = __shfl_sync(0xffffffffu, base1, 0);
    base2 = __shfl_sync(0xffffffffu, base2, 0);
    base3 = __shfl_sync(0xffffffffu, base3, 0);
    const unsigned below = (1u << lane) - 1u;
    if (kind == 1) one[base1 + __popc(b1 & below)] = make_uint2((uint32_t)q, __float_as_uint(tmin[0]));
    if (kind == 2)
      two[base2 + __popc(b2 & below)] = make_uint4((uint32_t)q, __float_as_uint(tmin[0]), __float_as_uint(tmin[1]), 0u);
    if (kind == 3) slow[base3 + __popc(b3 & below)] = (uint32_t)q;
  }
}

// f and f' of the steering polynomial with fused multiply-adds for the refinement's Newton steps
// (this unit is compiled without contraction; the steps only need f's sign and an approximate
// quotient f / f', taken in float: its relative error (~1e-7) leaves the iteration converging to
// the same double root without a double division).
struct SteerFma {
  double a4, b24, c36, a8;
};
__device__ inline double st_f_fma(const SteerFma& k, double t) {
  return __fma_rn(__fma_rn(__fma_rn(t, t, -k.a4), t, k.b24), t, -k.c36);
}
__device__ inline double st_fp_fma(const SteerFma& k, double t) {
  return __fma_rn(__fma_rn(4.0 * t, t, -k.a8), t, k.b24);
}

// J(t) as t + |dv|^2 / t + 12 |dp - vbar t|^2 / t^3 (the same function as st_J, written as a sum of
// non-negative terms, one division).
__device__ inline double st_J_sum(const double* xv, const double* xu, double t) {
  const double u = 1.0 / t;
  double dv2 = 0.0, r2 = 0.0;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const double dv = xu[3 + j] - xv[3 + j], vb = 0.5 * (xv[3 + j] + xu[3 + j]);
    const double d = (xu[j] - xv[j]) - vb * t;
    dv2 += dv * dv;
    r2 += d * d;
  }
  return t + dv2 * u + 12.0 * r2 * (u * u * u);
}

// Append q to a list, one atomic per warp (every lane of the warp calls this).
__device__ inline void warp_append(bool take, uint32_t q, uint32_t* out, unsigned long long* n_out) {
  const int lane = threadIdx.x & 31;
  const unsigned b = __ballot_sync(0xffffffffu, take);
  if (!b) return;
  unsigned long long base = 0;
  if (lane == 0) base = atomicAdd(n_out, (unsigned long long)__popc(b));
  base = __shfl_sync(0xffffffffu, base, 0);
  if (take) out[base + __popc(b & ((1u << lane) - 1u))] = q;
}

// Pairs with NM float minimisers (one list per count, so a warp runs one shape of work): each
// minimiser brackets the double root (+-1e-5 relative, end signs checked in double), and three
// Newton steps from it (float quotient, f in double) reach the root to the last bit; a pair whose
// bracket or convergence check fails goes to k_steer_slow.  A pair with float(Cost) < r gets its
// duration and cost written and goes to the collision pass.
template <int NM>
__global__ void k_steer_pairs(const float* __restrict__ states, const int2* __restrict__ list,
                              const uint32_t* __restrict__ items, const unsigned long long* __restrict__ n_items,
                              float r, double* __restrict__ res_tau, float* __restrict__ res_cost,
                              uint32_t* __restrict__ slow, unsigned long long* n_slow, uint32_t* __restrict__ cand,
                              unsigned long long* n_cand) {
  constexpr int kW = NM == 1 ? 2 : 4;  // words per item
  const int lane = threadIdx.x & 31;
  const long long ns = (long long)*n_items;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long k0 = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); k0 < ns; k0 += stride) {
    const long long k = k0 + lane;
    bool to_slow = false, edge = false;
    uint32_t q = 0;
    if (k < ns) {
      q = items[k * kW];
      const int2 vu = list[q];
      double xv[6], xu[6];
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        xv[j] = (double)states[6 * vu.x + j];
        xu[j] = (double)states[6 * vu.y + j];
      }
      SteerCoef c{0.0, 0.0, 0.0};
      for (int j = 0; j < 3; ++j) {
        const double dp = xu[j] - xv[j], v0 = xv[3 + j], v1 = xu[3 + j];
        c.a += v0 * v0 + v0 * v1 + v1 * v1;
        c.b += dp * (v0 + v1);
        c.c += dp * dp;
      }
      const SteerFma kf{4.0 * c.a, 24.0 * c.b, 36.0 * c.c, 8.0 * c.a};
      double best_t = -1.0, best_J = 0.0;
#pragma unroll
      for (int m = 0; m < NM; ++m) {
        const double t0 = (double)__uint_as_float(items[k * kW + 1 + m]);
        const double lo = t0 * (1.0 - 1e-5), hi = t0 * (1.0 + 1e-5);
        if (!(st_f(c, lo) < 0.0 && st_f(c, hi) > 0.0)) to_slow = true;
        double x = t0, step = 0.0;
#pragma unroll
        for (int it = 0; it < 3; ++it) {
          step = (double)((float)st_f_fma(kf, x) / (float)st_fp_fma(kf, x));
          x -= step;
        }
        if (!(fabs(step) <= 4.0e-16 * fabs(x) && x > lo && x < hi)) to_slow = true;
        const double Jt = st_J_sum(xv, xu, x);
        if (best_t < 0.0 || Jt < best_J || (Jt == best_J && x < best_t)) {
          best_t = x;
          best_J = Jt;
        }
      }
      if (!to_slow && __double2float_rn(best_J) < r) {
        res_tau[q] = best_t;
        res_cost[q] = __double2float_rn(best_J);
        edge = true;
      }
    }
    warp_append(to_slow, q, slow, n_slow);
    warp_append(edge, q, cand, n_cand);
  }
}

// Survivors that need the full analysis of Cost(v,u) (steer_dev).
__global__ void k_steer_slow(const float* __restrict__ states, const int2* __restrict__ list,
                             const uint32_t* __restrict__ slow, const unsigned long long* __restrict__ n_slow, float r,
                             double* __restrict__ res_tau, float* __restrict__ res_cost, uint32_t* __restrict__ cand,
                             unsigned long long* n_cand) {
  const int lane = threadIdx.x & 31;
  const long long ns = (long long)*n_slow;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long k0 = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); k0 < ns; k0 += stride) {
    const long long k = k0 + lane;
    bool edge = false;
    uint32_t q = 0;
    if (k < ns) {
      q = slow[k];
      const int2 vu = list[q];
      double xv[6], xu[6];
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        xv[j] = (double)states[6 * vu.x + j];
        xu[j] = (double)states[6 * vu.y + j];
      }
      double tau, J;
      if (steer_dev(xv, xu, &tau, &J) && __double2float_rn(J) < r) {
        res_tau[q] = tau;
        res_cost[q] = __double2float_rn(J);
        edge = true;
      }
    }
    warp_append(edge, q, cand, n_cand);
  }
}

// Nominal-connection coefficients in float for Collision: the cubic per axis, the reach R of each
// axis (|v0| tau + |c2| tau^2 + |c3| tau^3) and the margin eps = 2^-15 (1 + M).
struct FloatConn {
  float p0[3], v0[3], c2[3], c3[3], R[3], eps;
};
__device__ inline FloatConn float_conn(const float* fv, const float* fu, float tau) {
  FloatConn c;
  float M = 0.f;
  for (int a = 0; a < 3; ++a) {
    c.p0[a] = fv[a];
    c.v0[a] = fv[3 + a];
    const float dp = fu[a] - c.p0[a] - c.v0[a] * tau, dv = fu[3 + a] - c.v0[a];
    c.c2[a] = (3.f * dp - dv * tau) / (tau * tau);
    c.c3[a] = (dv * tau - 2.f * dp) / (tau * tau * tau);
    c.R[a] = fabsf(c.v0[a]) * tau + fabsf(c.c2[a]) * tau * tau + fabsf(c.c3[a]) * tau * tau * tau;
    M = fmaxf(M, fabsf(c.p0[a]) + c.R[a]);
  }
  c.eps = (1.f + M) * 3.0517578125e-5f;
  return c;
}

// Collision(v, u) for the pairs whose cost is below r, a warp per pair, in float only: the lanes
// take the samples m (32 at a time) and test them against the boxes the connection can reach.  A
// sample more than eps inside a box on every axis is a hit and ends the pair; one more than eps
// outside on some axis misses that box.  A pair without a hit but with a sample within eps of a
// box is undecided in float and goes to k_collide_exact; a pair with neither is kept.
__global__ void k_collide(const float* __restrict__ states, const int2* __restrict__ list,
                          const uint32_t* __restrict__ cand, const unsigned long long* __restrict__ n_cand, int n,
                          int W, const float* __restrict__ boxes_g, int nb, const double* __restrict__ res_tau,
                          uint32_t* keep, uint32_t* __restrict__ undec, unsigned long long* n_undec) {
  extern __shared__ float smf[];
  float* fracf = smf;
  float* boxes = fracf + 4 * W;
  for (int k = threadIdx.x; k < 6 * nb; k += blockDim.x) boxes[k] = boxes_g[k];
  for (int m = threadIdx.x; m < 4 * W; m += blockDim.x) fracf[m] = __double2float_rn((double)(m + 1) / (double)(4 * W));
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int nw = (n + 31) / 32;
  const long long nc = (long long)*n_cand;
  const long long warps = ((long long)gridDim.x * blockDim.x) >> 5;
  const int S = 4 * W;
  for (long long k = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < nc; k += warps) {
    const uint32_t q = cand[k];
    const int2 vu = list[q];
    float fv[6], fu[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      fv[j] = states[6 * vu.x + j];
      fu[j] = states[6 * vu.y + j];
    }
    const float tau = __double2float_rn(res_tau[q]);
    const FloatConn c = float_conn(fv, fu, tau);
    const float eps = c.eps;
    // boxes the connection can reach (the first 64; beyond that every box is tested)
    unsigned long long cb = 0ull;
    for (int o0 = 0; o0 < 64 && o0 < nb; o0 += 32) {
      const int o = o0 + lane;
      bool ov = false;
      if (o < nb) {
        const float* b = boxes + 6 * o;
        ov = true;
        for (int a = 0; a < 3; ++a) ov = ov && b[a] <= c.p0[a] + c.R[a] + eps && c.p0[a] - c.R[a] - eps <= b[3 + a];
      }
      cb |= (unsigned long long)__ballot_sync(0xffffffffu, ov) << o0;
    }
    const bool rest = nb > 64;
    bool hit = false, und = false;
    if (cb || rest) {
      for (int m0 = 1; m0 <= S && !hit; m0 += 32) {
        const int m = m0 + lane;
        bool h = false, u = false;
        if (m <= S) {
          const float t = tau * fracf[m - 1];
          float p[3];
          for (int a = 0; a < 3; ++a) p[a] = fmaf(fmaf(fmaf(c.c3[a], t, c.c2[a]), t, c.v0[a]), t, c.p0[a]);
          unsigned long long bits = cb;
          int o = -1;
          for (;;) {
            if (bits) {
              o = __ffsll((long long)bits) - 1;
              bits &= bits - 1ull;
            } else if (rest && o < 64) {
              o = 64;
            } else if (rest && o >= 64 && o + 1 < nb) {
              ++o;
            } else {
              break;
            }
            const float* b = boxes + 6 * o;
            bool out = false, in = true;
            for (int a = 0; a < 3; ++a) {
              out = out || p[a] < b[a] - eps || p[a] > b[3 + a] + eps;
              in = in && p[a] >= b[a] + eps && p[a] <= b[3 + a] - eps;
            }
            if (out) continue;
            if (in) {
              h = true;
              break;
            }
            u = true;
          }
        }
        hit = __any_sync(0xffffffffu, h);
        und = __any_sync(0xffffffffu, u) || und;
      }
    }
    if (lane == 0 && !hit) {
      if (und)
        undec[atomicAdd(n_undec, 1ull)] = q;
      else
        atomicOr(keep + (size_t)vu.x * nw + (vu.y >> 5), 1u << (vu.y & 31));
    }
  }
}

// Pairs k_collide could not decide, a warp per pair: the same float test per sample and box, and
// for a sample within eps of a box the definition's evaluation (double cubic at t_m, rounded to
// float, closed box).
__global__ void k_collide_exact(const float* __restrict__ states, const int2* __restrict__ list,
                                const uint32_t* __restrict__ undec, const unsigned long long* __restrict__ n_undec,
                                int n, int W, const float* __restrict__ boxes, int nb, const double* __restrict__ res_tau,
                                uint32_t* keep) {
  const int lane = threadIdx.x & 31;
  const int nw = (n + 31) / 32;
  const long long nu = (long long)*n_undec;
  const long long warps = ((long long)gridDim.x * blockDim.x) >> 5;
  const int S = 4 * W;
  for (long long k = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < nu; k += warps) {
    const uint32_t q = undec[k];
    const int2 vu = list[q];
    float fv[6], fu[6];
    double xv[6], xu[6];
    for (int j = 0; j < 6; ++j) {
      fv[j] = states[6 * vu.x + j];
      fu[j] = states[6 * vu.y + j];
      xv[j] = (double)fv[j];
      xu[j] = (double)fu[j];
    }
    const float tau = __double2float_rn(res_tau[q]);
    const double td = (double)tau;
    const FloatConn c = float_conn(fv, fu, tau);
    const float eps = c.eps;
    Cubic cx[3];
    for (int a = 0; a < 3; ++a) cx[a] = cubic_dev(xv, xu, td, a);
    bool hit = false;
    for (int m0 = 1; m0 <= S && !hit; m0 += 32) {
      const int m = m0 + lane;
      bool h = false;
      if (m <= S) {
        const double fr = (double)m / (double)S;
        const float t = tau * __double2float_rn(fr);
        float p[3];
        for (int a = 0; a < 3; ++a) p[a] = fmaf(fmaf(fmaf(c.c3[a], t, c.c2[a]), t, c.v0[a]), t, c.p0[a]);
        for (int o = 0; o < nb && !h; ++o) {
          const float* b = boxes + 6 * o;
          bool out = false, in = true;
          for (int a = 0; a < 3; ++a) {
            out = out || p[a] < b[a] - eps || p[a] > b[3 + a] + eps;
            in = in && p[a] >= b[a] + eps && p[a] <= b[3 + a] - eps;
          }
          if (out) continue;
          if (in) {
            h = true;
            break;
          }
          const double te = td * fr;
          h = in_box_dev((float)cubic_at(cx[0], te), (float)cubic_at(cx[1], te), (float)cubic_at(cx[2], te), b);
        }
      }
      hit = __any_sync(0xffffffffu, h);
    }
    if (!hit && lane == 0) atomicOr(keep + (size_t)vu.x * nw + (vu.y >> 5), 1u << (vu.y & 31));
  }
}

__global__ void k_row_counts(const uint32_t* __restrict__ keep, int n, int32_t* deg) {
  const int nw = (n + 31) / 32;
  int v = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  int lane = threadIdx.x & 31;
  if (v >= n) return;
  int c = 0;
  for (int k = lane; k < nw; k += 32) c += __popc(keep[(size_t)v * nw + k]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if (lane == 0) deg[v] = c;
}

// Exclusive scan of n int32 into out[0..n], out[n] = total; one block.
__global__ void k_scan_single(const int32_t* __restrict__ in, int n, int32_t* out) {
  __shared__ int64_t part[1024];
  int T = blockDim.x, t = threadIdx.x;
  int per = (n + T - 1) / T;
  int lo = min(n, t * per), hi = min(n, lo + per);
  int64_t s = 0;
  for (int k = lo; k < hi; ++k) s += in[k];
  part[t] = s;
  __syncthreads();
  for (int off = 1; off < T; off <<= 1) {
    int64_t v = t >= off ? part[t - off] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  int64_t run = part[t] - s;
  for (int k = lo; k < hi; ++k) {
    out[k] = (int32_t)run;
    run += in[k];
  }
  if (t == T - 1) out[n] = (int32_t)part[T - 1];
}

// Edge index of the first kept pair of each keep word: row start + kept pairs before it in the
// row (a warp per row, 32 words at a time).
__global__ void k_word_prefix(const uint32_t* __restrict__ keep, int n, const int32_t* __restrict__ row_ptr,
                              int32_t* __restrict__ wpre) {
  const int nw = (n + 31) / 32;
  const int v = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (v >= n) return;
  int run = row_ptr[v];
  for (int k0 = 0; k0 < nw; k0 += 32) {
    const int k = k0 + lane;
    const int c = k < nw ? __popc(keep[(size_t)v * nw + k]) : 0;
    int x = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (k < nw) wpre[(size_t)v * nw + k] = run + x - c;
    run += __shfl_sync(0xffffffffu, x, 31);
  }
}

// Kept pairs to their CSR slots (targets ascending within a row).
__global__ void k_scatter_edges(const int2* __restrict__ list, long long n_list, int n,
                                const uint32_t* __restrict__ keep, const int32_t* __restrict__ wpre,
                                const double* __restrict__ res_tau, const float* __restrict__ res_cost,
                                int32_t* __restrict__ src, int32_t* __restrict__ col, double* __restrict__ etau,
                                float* __restrict__ ecost) {
  const int nw = (n + 31) / 32;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n_list;
       q += (long long)gridDim.x * blockDim.x) {
    const int2 vu = list[q];
    const size_t wi = (size_t)vu.x * nw + (vu.y >> 5);
    const uint32_t word = keep[wi];
    const uint32_t bit = 1u << (vu.y & 31);
    if (!(word & bit)) continue;
    const int e = wpre[wi] + __popc(word & (bit - 1u));
    src[e] = vu.x;
    col[e] = vu.y;
    etau[e] = res_tau[q];
    ecost[e] = res_cost[q];
  }
}

// Per edge: float duration, waypoint step h = tau/W, Phi(h), L(h), nominal waypoints at t = k h.
// Float-float (a pair of floats, ~48 significant bits; Dekker's and Knuth's exact sum and the
// fused-multiply-add exact product) evaluation of the nominal cubic.  A value is rounded to float
// from its float-float form only when that form lies farther than 2^-40 S from both float
// rounding midpoints around it (S: the sum of the terms' magnitudes; the float-float error is
// below 0.16 x 2^-40 S and the double evaluation's below 0.001 x 2^-40 S), so the float equals
// the one the double evaluation rounds to; otherwise the double evaluation is taken.
struct FF {
  float hi, lo;
};
__device__ __forceinline__ FF ff_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b), bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ FF ff_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ FF ff_from_double(double x) {
  const float hi = __double2float_rn(x);
  return {hi, __double2float_rn(x - (double)hi)};
}
__device__ __forceinline__ FF ff_add(FF a, FF b) {
  FF s = ff_two_sum(a.hi, b.hi);
  const FF t = ff_two_sum(a.lo, b.lo);
  s.lo = __fadd_rn(s.lo, t.hi);
  s = ff_fast_two_sum(s.hi, s.lo);
  s.lo = __fadd_rn(s.lo, t.lo);
  return ff_fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ FF ff_mul(FF a, FF b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return ff_fast_two_sum(p, e);
}
// The float nearest to v.hi + v.lo, or NaN where that value lies within M of a rounding midpoint.
__device__ __forceinline__ float ff_round_checked(FF v, float M) {
  const float f = __fadd_rn(v.hi, v.lo);
  const float d = __fadd_rn(__fsub_rn(v.hi, f), v.lo);  // v - f (v.hi - f is exact)
  const float up = __fsub_rn(nextafterf(f, __int_as_float(0x7f800000)), f);
  const float dn = __fsub_rn(f, nextafterf(f, __int_as_float(0xff800000)));
  if (f == 0.f || !(up < __int_as_float(0x7f800000)) || !(dn < __int_as_float(0x7f800000))) return __int_as_float(0x7fc00000);
  return fabsf(d) + M < 0.4995f * fminf(up, dn) ? f : __int_as_float(0x7fc00000);
}

__global__ void k_fill_edges(const float* __restrict__ states, int E, int W, float sigma,
                             const int32_t* __restrict__ src, const int32_t* __restrict__ col,
                             const double* __restrict__ etau, float* tau_o, float* h_o, float* phi_o, float* L_o,
                             float* nom_o, float* nvel_o) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  const int v = src[e], u = col[e];
  double xv[6], xu[6];
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    xv[j] = (double)states[6 * v + j];
    xu[j] = (double)states[6 * u + j];
  }
  const float t32 = __double2float_rn(etau[e]);
  const float h = __fdiv_rn(t32, (float)W);
  tau_o[e] = t32;
  h_o[e] = h;
  double Phi[4], L[3], Linf[3];
  model_dev((double)sigma, (double)h, Phi, L, Linf);
#pragma unroll
  for (int q = 0; q < 4; ++q) phi_o[4 * (size_t)e + q] = __double2float_rn(Phi[q]);
#pragma unroll
  for (int q = 0; q < 3; ++q) L_o[3 * (size_t)e + q] = __double2float_rn(L[q]);
  const double td = (double)t32;
  for (int j = 0; j < 3; ++j) {
    const Cubic c = cubic_dev(xv, xu, td, j);
    // the cubic's terms in float-float (kk h has at most 30 significant bits: t is exact)
    const FF p0 = ff_from_double(c.p0), v0 = ff_from_double(c.v0), c2 = ff_from_double(c.c2),
             c3 = ff_from_double(c.c3), c2x2 = ff_from_double(2.0 * c.c2), c3x3 = ff_from_double(3.0 * c.c3);
    const float a0 = fabsf(p0.hi), a1 = fabsf(v0.hi), a2 = fabsf(c2.hi), a3 = fabsf(c3.hi);
    for (int kk = 1; kk <= W; ++kk) {
      const double tk = (double)kk * (double)h;
      const FF t = ff_from_double(tk);
      const float tf = fabsf(t.hi);
      // nominal position p0 + v0 t + c2 t t + c3 t t t, in the double evaluation's association
      const FF pos = ff_add(ff_add(ff_add(p0, ff_mul(v0, t)), ff_mul(ff_mul(c2, t), t)),
                            ff_mul(ff_mul(ff_mul(c3, t), t), t));
      const float Sp = 1.0001f * (a0 + tf * (a1 + tf * (a2 + tf * a3)));
      float fp = ff_round_checked(pos, Sp * 0x1p-40f);
      if (fp != fp) fp = __double2float_rn(cubic_at(c, tk));
      nom_o[((size_t)e * W + (kk - 1)) * 3 + j] = fp;
      // nominal velocity v0 + 2 c2 t + 3 c3 t t
      const FF vel = ff_add(ff_add(v0, ff_mul(c2x2, t)), ff_mul(ff_mul(c3x3, t), t));
      const float Sv = 1.0001f * (a1 + tf * (2.0f * a2 + 3.0f * tf * a3));
      float fv = ff_round_checked(vel, Sv * 0x1p-40f);
      if (fv != fv) fv = __double2float_rn(c.v0 + 2.0 * c.c2 * tk + 3.0 * c.c3 * tk * tk);
      nvel_o[((size_t)e * W + (kk - 1)) * 3 + j] = fv;
    }
  }
}

// xi[i][k][axis][c] -> xi_t[k][axis][i] as float2 (lane-contiguous particles).
__global__ void k_transpose_xi(const float* __restrict__ xi, int N, int W, float2* xi_t) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  int total = N * (W + 1) * 3;
  if (q >= total) return;
  int i = q / ((W + 1) * 3);
  int rem = q % ((W + 1) * 3);
  int k = rem / 3, a = rem % 3;
  xi_t[((size_t)k * 3 + a) * N + i] = make_float2(xi[2 * (size_t)q], xi[2 * (size_t)q + 1]);
}

// xi_t -> pair-major xi_p[((k * 3 + a) * npair + jp) * 32 + l] = (xi0 of particles 64 jp + l and
// 64 jp + 32 + l, then their xi1; zeros past N).
__global__ void k_pair_xi(const float2* __restrict__ xi_t, int N, int W, int npair, float4* xi_p) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long total = (long long)(W + 1) * 3 * npair * 32;
  if (q >= total) return;
  const int l = (int)(q & 31);
  const long long r = q >> 5;
  const int jp = (int)(r % npair);
  const long long ka = r / npair;  // k * 3 + a
  const int i0 = 64 * jp + l, i1 = i0 + 32;
  const float2 x0 = i0 < N ? xi_t[ka * N + i0] : make_float2(0.f, 0.f);
  const float2 x1 = i1 < N ? xi_t[ka * N + i1] : make_float2(0.f, 0.f);
  xi_p[q] = make_float4(x0.x, x1.x, x0.y, x1.y);
}

__global__ void k_linf(float sigma, float* out) {
  double Phi[4], L[3], Linf[3];
  model_dev((double)sigma, 1.0, Phi, L, Linf);
  out[0] = __double2float_rn(Linf[0]);
  out[1] = __double2float_rn(Linf[1]);
  out[2] = __double2float_rn(Linf[2]);
}

// What the build reads back at its end, in one copy: out[0] the valid node count (atomics onto a
// zeroed word), out[1] the start's validity, out[2..4] the bits of L_inf.
__global__ void k_build_summary(const uint8_t* __restrict__ valid, int n, int32_t start,
                                const float* __restrict__ linf, int32_t* out) {
  int c = 0;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) c += valid[v];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, c);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    out[1] = valid[start];
    for (int a = 0; a < 3; ++a) out[2 + a] = __float_as_int(linf[a]);
  }
}

}  // namespace

// Expects g->states, g->boxes, g->valid, g->is_goal, xi (raw, device) staged.
int build_graph_device(pump_graph* g, int32_t start_idx, bool* start_valid, cudaStream_t s) {
  const int n = g->n;
  const int nw = (n + 31) / 32;
  const int sms = num_sms();
  // node flags (validity) and goal flags were filled by the caller's kernels
  // prefilter: count per row, scan, allocate, list
  unsigned long long* d_count = (unsigned long long*)dev_alloc(sizeof(unsigned long long) * 5, s);
  int32_t* rcnt = (int32_t*)dev_alloc(sizeof(int32_t) * (size_t)n, s);
  long long* roff = (long long*)dev_alloc(sizeof(long long) * (size_t)(n + 1), s);
  if (!d_count || !rcnt || !roff) return PUMP_ERR_OOM;
  PUMP_CUDA_TRY(cudaMemsetAsync(d_count, 0, sizeof(unsigned long long) * 5, s));
  // the valid nodes on a position grid: cell counts, offsets, the nodes in cell order
  constexpr int kCells = kGridMax * kGridMax * kGridMax;
  Grid* d_grid = (Grid*)dev_alloc(sizeof(Grid), s);
  int32_t* ccnt = (int32_t*)dev_alloc(sizeof(int32_t) * 2 * (size_t)kCells, s);  // counts, then cursors
  long long* coff = (long long*)dev_alloc(sizeof(long long) * ((size_t)kCells + 1), s);
  int32_t* sorted = (int32_t*)dev_alloc(sizeof(int32_t) * (size_t)std::max(n, 1), s);
  float* sorted_states = (float*)dev_alloc(sizeof(float) * 6 * (size_t)std::max(n, 1), s);
  if (!d_grid || !ccnt || !coff || !sorted || !sorted_states) return PUMP_ERR_OOM;
  PUMP_CUDA_TRY(cudaMemsetAsync(ccnt, 0, sizeof(int32_t) * 2 * (size_t)kCells, s));
  const int gnodes = std::max(1, std::min((n + kBlock - 1) / kBlock, sms * 8));
  k_grid_setup<<<1, 1024, 0, s>>>(g->states, g->valid, n, g->radius, d_grid);
  note_launch();
  k_grid_count<<<gnodes, kBlock, 0, s>>>(g->states, g->valid, n, d_grid, ccnt);
  note_launch();
  k_grid_scan<<<1, 1024, 0, s>>>(ccnt, d_grid, coff);
  note_launch();
  k_grid_scatter<<<gnodes, kBlock, 0, s>>>(g->states, g->valid, n, d_grid, coff, ccnt + kCells, sorted,
                                           sorted_states);
  note_launch();
  const int grid = (int)std::min<long long>(((long long)n * 32 + kBlock - 1) / kBlock, (long long)sms * 16);
  k_prefilter<false><<<grid, kBlock, 0, s>>>(g->states, g->valid, n, g->radius, d_grid, coff, sorted, sorted_states,
                                             rcnt, nullptr, nullptr);
  note_launch();
  k_scan_ll<<<1, 1024, 0, s>>>(rcnt, n, roff);
  note_launch();
  long long n_list_ll = 0;
  PUMP_CUDA_TRY(cudaMemcpyAsync(&n_list_ll, roff + n, sizeof(n_list_ll), cudaMemcpyDeviceToHost, s));
  PUMP_CUDA_TRY(cudaStreamSynchronize(s));
  const unsigned long long n_list = (unsigned long long)n_list_ll;
  int2* list = nullptr;
  if (n_list) {
    list = (int2*)dev_alloc(sizeof(int2) * n_list, s);
    if (!list) { dev_free(d_count, s); return PUMP_ERR_OOM; }
    k_prefilter<true><<<grid, kBlock, 0, s>>>(g->states, g->valid, n, g->radius, d_grid, coff, sorted, sorted_states,
                                              nullptr, roff, list);
    note_launch();
  }
  dev_free(sorted_states, s);
  dev_free(sorted, s);
  dev_free(coff, s);
  dev_free(ccnt, s);
  dev_free(d_grid, s);
  uint32_t* keep = (uint32_t*)dev_alloc(sizeof(uint32_t) * (size_t)n * nw, s);
  int32_t* deg = (int32_t*)dev_alloc(sizeof(int32_t) * (size_t)std::max(n + 1, 8), s);
  int32_t* wpre = (int32_t*)dev_alloc(sizeof(int32_t) * (size_t)n * nw, s);
  double* res_tau = (double*)dev_alloc(sizeof(double) * (n_list ? n_list : 1), s);
  float* res_cost = (float*)dev_alloc(sizeof(float) * (n_list ? n_list : 1), s);
  if (!keep || !deg || !wpre || !res_tau || !res_cost) return PUMP_ERR_OOM;
  PUMP_CUDA_TRY(cudaMemsetAsync(keep, 0, sizeof(uint32_t) * (size_t)n * nw, s));
  long long list_blocks = ((long long)n_list + kBlock - 1) / kBlock;
  const int glist = (int)(list_blocks < (long long)sms * 16 ? (list_blocks > 0 ? list_blocks : 1) : (long long)sms * 16);
  uint32_t* surv = nullptr;
  if (n_list) {
    if (n_list > 0xFFFFFFFFull) return PUMP_ERR_CAPACITY;
    // word offsets: slow [0, n), cand [n, 2n), one (uint2, 8-byte aligned), two (uint4, 16-byte aligned)
    const unsigned long long off_one = (3 * n_list + 1) & ~1ull;
    const unsigned long long off_two = (off_one + 2 * n_list + 3) & ~3ull;
    surv = (uint32_t*)dev_alloc(sizeof(uint32_t) * (off_two + 4 * n_list), s);
    if (!surv) return PUMP_ERR_OOM;
    uint32_t* surv_slow = surv + n_list;
    uint32_t* cand = surv + 2 * n_list;
    uint2* one = reinterpret_cast<uint2*>(surv + off_one);
    uint4* two = reinterpret_cast<uint4*>(surv + off_two);
    k_steer_filter<<<glist, kBlock, 0, s>>>(g->states, list, (long long)n_list, g->radius, one, d_count, two,
                                            d_count + 4, surv_slow, d_count + 1);
    note_launch();
    k_steer_pairs<1><<<sms * 4, kBlock, 0, s>>>(g->states, list, reinterpret_cast<const uint32_t*>(one), d_count,
                                                g->radius, res_tau, res_cost, surv_slow, d_count + 1, cand, d_count + 2);
    note_launch();
    k_steer_pairs<2><<<sms * 4, kBlock, 0, s>>>(g->states, list, reinterpret_cast<const uint32_t*>(two), d_count + 4,
                                                g->radius, res_tau, res_cost, surv_slow, d_count + 1, cand, d_count + 2);
    note_launch();
    k_steer_slow<<<sms, kBlock, 0, s>>>(g->states, list, surv_slow, d_count + 1, g->radius, res_tau, res_cost, cand,
                                        d_count + 2);
    note_launch();
    const size_t smem = sizeof(float) * 4 * g->W + sizeof(float) * 6 * (g->n_boxes > 0 ? g->n_boxes : 1);
    uint32_t* undec = surv_slow;  // the slow list is consumed by now
    k_collide<<<sms * 8, kBlock, smem, s>>>(g->states, list, cand, d_count + 2, n, g->W, g->boxes, g->n_boxes, res_tau,
                                            keep, undec, d_count + 3);
    note_launch();
    k_collide_exact<<<sms, kBlock, 0, s>>>(g->states, list, undec, d_count + 3, n, g->W, g->boxes, g->n_boxes, res_tau,
                                        keep);
    note_launch();
  }
  k_row_counts<<<(n + 7) / 8, kBlock, 0, s>>>(keep, n, deg);
  note_launch();
  g->row_ptr = (int32_t*)graph_alloc(g, sizeof(int32_t) * (size_t)(n + 1), s);
  if (!g->row_ptr) return PUMP_ERR_OOM;
  k_scan_single<<<1, 1024, 0, s>>>(deg, n, g->row_ptr);
  note_launch();
  int32_t E = 0;
  PUMP_CUDA_TRY(cudaMemcpyAsync(&E, g->row_ptr + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  PUMP_CUDA_TRY(cudaStreamSynchronize(s));
  g->E = E;
  size_t Es = E > 0 ? (size_t)E : 1;
  g->col = (int32_t*)graph_alloc(g, sizeof(int32_t) * Es, s);
  g->ecost = (float*)graph_alloc(g, sizeof(float) * Es, s);
  g->tau = (float*)graph_alloc(g, sizeof(float) * Es, s);
  g->h = (float*)graph_alloc(g, sizeof(float) * Es, s);
  g->phi = (float*)graph_alloc(g, sizeof(float) * 4 * Es, s);
  g->L = (float*)graph_alloc(g, sizeof(float) * 3 * Es, s);
  g->nom = (float*)graph_alloc(g, sizeof(float) * 3 * (size_t)g->W * Es, s);
  g->emask = (uint32_t*)graph_alloc(g, sizeof(uint32_t) * (size_t)g->n_words * Es, s);
  g->ibox = (float*)graph_alloc(g, sizeof(float) * 6 * Es, s);
  g->nvel = (float*)graph_alloc(g, sizeof(float) * 3 * (size_t)g->W * Es, s);
  if (!g->col || !g->ecost || !g->tau || !g->h || !g->phi || !g->L || !g->nom || !g->emask || !g->ibox || !g->nvel)
    return PUMP_ERR_OOM;
  if (E > 0) {
    int32_t* src = (int32_t*)dev_alloc(sizeof(int32_t) * Es, s);
    double* etau = (double*)dev_alloc(sizeof(double) * Es, s);
    if (!src || !etau) return PUMP_ERR_OOM;
    k_word_prefix<<<(n + 7) / 8, kBlock, 0, s>>>(keep, n, g->row_ptr, wpre);
    note_launch();
    k_scatter_edges<<<glist, kBlock, 0, s>>>(list, (long long)n_list, n, keep, wpre, res_tau, res_cost, src, g->col,
                                             etau, g->ecost);
    note_launch();
    // the adjacency and costs are final: the fused form's edge order is laid out beside the
    // per-edge fill and the deviation bounds (a side stream; joined before the build returns)
    if (!g->hsmc && g->fuse_masks && fused_masks_env()) {
      const int rco = row_order_begin(g, s, true);
      if (rco) return rco;
    }
    k_fill_edges<<<(E + 127) / 128, 128, 0, s>>>(g->states, E, g->W, g->sigma, src, g->col, etau, g->tau, g->h,
                                                 g->phi, g->L, g->nom, g->nvel);
    note_launch();
    dev_free(src, s);
    dev_free(etau, s);
  }
  {
    const int rcb = compute_edge_bounds(g, s);
    if (rcb) return rcb;
  }
  if (g->hsmc) {
    const int rch = build_halfspaces(g, s);
    if (rch) return rch;
  }
  {
    const int rco = row_order_end(g, s);
    if (rco) return rco;
  }
  // valid node count (for export), the start's validity and L_inf: one read-back
  PUMP_CUDA_TRY(cudaMemsetAsync(deg, 0, sizeof(int32_t), s));
  k_build_summary<<<32, kBlock, 0, s>>>(g->valid, n, start_idx, g->linf_dev, deg);
  note_launch();
  int32_t summary[5] = {0, 0, 0, 0, 0};
  PUMP_CUDA_TRY(cudaMemcpyAsync(summary, deg, sizeof(summary), cudaMemcpyDeviceToHost, s));
  PUMP_CUDA_TRY(cudaGetLastError());
  PUMP_CUDA_TRY(cudaStreamSynchronize(s));
  g->n_valid = summary[0];
  *start_valid = summary[1] != 0;
  std::memcpy(g->linf, summary + 2, sizeof(float) * 3);
  dev_free(d_count, s);
  if (list) dev_free(list, s);
  if (surv) dev_free(surv, s);
  dev_free(rcnt, s);
  dev_free(roff, s);
  dev_free(keep, s);
  dev_free(deg, s);
  dev_free(wpre, s);
  dev_free(res_tau, s);
  dev_free(res_cost, s);
  return PUMP_OK;
}

// Exclusive scan of n counts into out[0..n] (out[n] = total).
int scan_counts(const int32_t* in, int n, int32_t* out, cudaStream_t s) {
  k_scan_single<<<1, 1024, 0, s>>>(in, n, out);
  note_launch();
  PUMP_CUDA_TRY(cudaGetLastError());
  return PUMP_OK;
}

int launch_node_flags(pump_graph* g, const int32_t* goal_dev, cudaStream_t s) {
  k_node_flags<<<(g->n + kBlock - 1) / kBlock, kBlock, 0, s>>>(g->states, g->n, g->boxes, g->n_boxes, goal_dev,
                                                              g->n_goal, g->valid, g->is_goal);
  note_launch();
  k_goal_flags<<<(g->n_goal + kBlock - 1) / kBlock, kBlock, 0, s>>>(goal_dev, g->n_goal, g->is_goal);
  note_launch();
  PUMP_CUDA_TRY(cudaGetLastError());
  return PUMP_OK;
}

int launch_transpose_xi(pump_graph* g, const float* xi_dev, cudaStream_t s) {
  int total = g->N * (g->W + 1) * 3;
  k_transpose_xi<<<(total + kBlock - 1) / kBlock, kBlock, 0, s>>>(xi_dev, g->N, g->W, g->xi_t);
  note_launch();
  const int npair = (g->N / 32 + 1) / 2;
  const long long ptot = (long long)(g->W + 1) * 3 * npair * 32;
  k_pair_xi<<<(unsigned)((ptot + kBlock - 1) / kBlock), kBlock, 0, s>>>(g->xi_t, g->N, g->W, npair, g->xi_p);
  note_launch();
  PUMP_CUDA_TRY(cudaGetLastError());
  return PUMP_OK;
}

int launch_linf(pump_graph* g, float* out_dev, cudaStream_t s) {
  k_linf<<<1, 1, 0, s>>>(g->sigma, out_dev);
  note_launch();
  PUMP_CUDA_TRY(cudaGetLastError());
  return PUMP_OK;
}

}  // namespace pump
