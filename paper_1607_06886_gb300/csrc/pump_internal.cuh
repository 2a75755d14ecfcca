// Internal declarations shared by the libpump translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <climits>
#include <vector>

#include "../../include/pump.h"

namespace pump {

constexpr int kMaxBoxes = 1024;
constexpr int kMaxWaypoints = 64;
constexpr int kMaxParticles = 1024;
constexpr int kMaxWords = kMaxParticles / 32;
constexpr int kMaxPathEdges = 4096;
constexpr int32_t kNoBucket = INT_MAX;

// ---------------------------------------------------------------------------
// Device allocation through the installed allocator; every buffer of a graph
// is tracked so pump_graph_destroy can release it.
void* dev_alloc(size_t bytes, cudaStream_t s);

// Count of kernels this library has launched (host-side, all devices).
void note_launch();
void dev_free(void* p, cudaStream_t s);

struct DevBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
};

// Per-iteration state of Explore, double-buffered by iteration parity: iteration k
// reads slot k & 1 and its last phase writes slot (k + 1) & 1, so no block reads a
// field another block of the same phase is changing.
struct IterState {
  int64_t group_cands;  // candidates of the group
  int32_t group_size;   // |G|
  int32_t iter;         // group index i
  int32_t stop;         // the group holds a goal plan with popc < K_min
  int32_t pad;
};

// Control block of one Explore run (device resident).
struct ExploreCtl {
  IterState st[2];
  int64_t n_plans;        // committed arena size
  int64_t n_candidates;   // partial plans evaluated so far
  int64_t n_kept;         // candidates under the CP cutoff
  int32_t next_bucket[2]; // least group index among open undominated plans, by parity
  int32_t stop_next;
  int32_t status;         // pump_status of the run (CAPACITY, TIMEOUT)
  int32_t n_groups;       // non-empty groups expanded
  int32_t survivors;      // survivors of the last expansion (committed at the next P1)
  int32_t n_goal_all;     // arena plans at goal nodes (unfiltered)
  int32_t n_goal;         // |P_goal|
  int32_t k_exit;         // iteration count when the loop ended
  int32_t iter;           // final group index (set when the run ends)
  uint32_t bar_count;     // grid barrier arrivals
  uint32_t bar_gen;       // grid barrier generation
};

struct ExploreArgs {
  // graph
  const int32_t* row_ptr;
  const int32_t* col;
  const float* ecost;
  const uint32_t* emask;
  const uint8_t* is_goal;
  int32_t n;
  int32_t w;       // mask words
  int32_t kmax;    // popc < kmax survives the CP cutoff
  int32_t kstride; // row length of mbest (max(kmax, 1))
  int32_t kmin;    // goal plan with popc < kmin stops the search
  double lr;       // lambda * r in double
  int32_t max_iter;
  int32_t early_stop;
  // arena
  int32_t* head;
  int32_t* parent;
  int32_t* pedge;
  int32_t* tcre;
  int32_t* eexp;
  float* cost;
  int32_t* popc;
  uint32_t* mask;
  int64_t cap;
  // search state
  uint32_t* mbest;  // n x kmax float bits: least cost of any plan inserted at (node, popc)
  int32_t* group;
  int4* ginfo;      // per group slot: plan id, head node, row start, cost bits
  int64_t* goff;    // group_size + 1 candidate offsets
  const int4* etgt; // per edge: target node, cost bits, target row start, degree | goal bit (or null)
  int2* prow = nullptr;  // per plan: its head's row start, degree | goal bit (cluster forms; or null)
  int32_t* bcnt;    // per-block survivor / selection counts
  int64_t* bdeg;    // per-block degree sums
  int32_t* goal_all;
  ExploreCtl* ctl;
  long long spin_limit;
  // fused form: finished edges per row, counted by the mask workers of the same launch (a
  // member's row is read once its count reaches the row's degree); null when the masks are ready.
  // Counts accumulate over runs: run e (from 1) starts at (e - 1) x degree (mod 2^32).
  const uint32_t* rowcnt = nullptr;
  uint32_t epoch_m1 = 0;            // e - 1
  const uint32_t* done = nullptr;   // worker warps finished, accumulated over runs
  uint32_t done_target = 0;         // its value once every worker warp of run e has finished
};

struct ExploreBufs {
  int64_t cap = 0;
  int32_t kmax_alloc = 0;
  int32_t w_alloc = 0;
  int32_t* head = nullptr;
  int32_t* parent = nullptr;
  int32_t* pedge = nullptr;
  int32_t* tcre = nullptr;
  int32_t* eexp = nullptr;
  float* cost = nullptr;
  int32_t* popc = nullptr;
  uint32_t* mask = nullptr;
  uint32_t* mbest = nullptr;
  int32_t* group = nullptr;
  int4* ginfo = nullptr;
  int64_t* goff = nullptr;
  int32_t* bcnt = nullptr;
  int64_t* bdeg = nullptr;
  int32_t* goal_all = nullptr;
  int32_t* goal_sorted = nullptr;
  int2* prow = nullptr;
  ExploreCtl* ctl = nullptr;
  // selection / certification scratch
  void* sel_state = nullptr;      // bisection state
  long long* sel_by_index = nullptr;  // MC count per P_goal index (-1 unknown)
  int32_t sel_cap = 0;
  int64_t* sel_toff = nullptr;    // table offsets per certified plan
  int32_t* sel_err = nullptr;     // path error flag, path length
  int32_t* sel_idx = nullptr;     // P_goal indices being certified
  int64_t* mc_count = nullptr;    // per certified plan
  int32_t* mc_plan = nullptr;     // plan ids being certified
  int32_t* mc_plen = nullptr;     // path edge counts
  int32_t* mc_pedges = nullptr;   // n_cert x kMaxPathEdges edge ids
  float* mc_table = nullptr;      // per path edge: Phi(4), L(3), nominal (W*S*3)
  int64_t mc_table_floats = 0;
  int32_t mc_cap = 0;
  int32_t* path_buf = nullptr;    // backtracked node ids
  std::vector<DevBuf> bufs;
};

}  // namespace pump

struct pump_graph {
  int32_t n = 0, E = 0, N = 0, W = 0, n_words = 0, n_boxes = 0, n_goal = 0, start = 0;
  int32_t n_valid = 0;
  float radius = 0.f, sigma = 0.f;
  bool has_geometry = false;
  bool masks_ready = false;
  int device = 0;
  float linf[3] = {0, 0, 0};
  float* linf_dev = nullptr; // 3 floats: Cholesky factor of the stationary covariance
  float* states = nullptr;   // n x 6
  float* boxes = nullptr;    // n_boxes x 6 (lo, hi)
  float2* xi_t = nullptr;    // [(W+1)][3][N] (xi0, xi1) pairs
  float4* xi_p = nullptr;    // pair-major normals of the box masks (maskdev::pair_count)
  unsigned long long* wctr = nullptr;  // edge counters of the mask passes: [0] stand-alone kernel
                                       // (zeroed per launch), [1] fused workers (over runs)
  uint8_t* valid = nullptr;
  uint8_t* is_goal = nullptr;
  int32_t* row_ptr = nullptr;
  int32_t* col = nullptr;
  float* ecost = nullptr;
  float* tau = nullptr;
  float* h = nullptr;
  float* phi = nullptr;      // E x 4
  float* L = nullptr;        // E x 3
  float* nom = nullptr;      // E x W x 3
  uint32_t* emask = nullptr; // E x n_words
  float* ibox = nullptr;     // E x 6: box holding every particle position of the edge
  int4* etgt = nullptr;      // E: target node, cost bits, target row start, degree | goal bit
  unsigned int* dmax = nullptr;  // E: largest |d0| of the edge's particles (float bits)
  float* nvel = nullptr;     // E x W x 3: nominal velocity at the waypoints
  bool hsmc = false;         // masks by Half-Space Monte Carlo
  int32_t* hs_off = nullptr; // E*W + 1: first half-space of waypoint (e, k) (HSMC)
  float4* hs_ab = nullptr;   // half-spaces (a xyz, b) that a particle of the edge can fire (HSMC)
  // fused masks + Explore: edges in the order the mask workers take them (edge, source row),
  // rows by increasing shortest-path cost from the start; finished edges per row
  int2* eorder = nullptr;
  uint32_t* rowcnt = nullptr;       // n + 1: finished edges per row, then worker warps finished
  uint32_t fuse_epoch = 0;          // fused runs since the counts were last zeroed
  void* order_scratch = nullptr;    // edge order being laid out (graph build): its scratch,
  void* order_keep = nullptr;       // the order's own allocation,
  cudaEvent_t order_join = nullptr; // and the side stream's event to wait for
  bool rowcnt_dirty = true;         // counts must be zeroed before the next fused run
  bool fuse_masks = true;    // pump_plan may run the masks inside the Explore launch
  bool last_fused = false;   // the last Explore run computed the masks in its launch
  std::vector<pump::DevBuf> bufs;
  pump::ExploreBufs ex;
  // last explore
  bool explored = false;
  int64_t last_plans = 0;
  int32_t last_goal = 0;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  pump::ExploreCtl* ctl_host = nullptr;  // pinned copy of Explore's control block (pump_plan; the
                                         // calling thread's, not owned by the graph)
};

namespace pump {

void* graph_alloc(pump_graph* g, size_t bytes, cudaStream_t s);
void* graph_realloc(pump_graph* g, void* old, size_t bytes, cudaStream_t s);

// status helpers
#define PUMP_CUDA_TRY(expr)                        \
  do {                                             \
    cudaError_t _e = (expr);                       \
    if (_e != cudaSuccess) return PUMP_ERR_CUDA;   \
  } while (0)

int build_graph_device(pump_graph* g, int32_t start_idx, bool* start_valid, cudaStream_t s);
// Edge order of the fused form (explore_cluster.cu): begun during the graph build (on a side
// stream when `overlap`), completed on s before the build returns.
int row_order_begin(pump_graph* g, cudaStream_t s, bool overlap);
int row_order_end(pump_graph* g, cudaStream_t s);
int build_halfspaces(pump_graph* g, cudaStream_t s);
constexpr int kHsMax = 8;  // half-spaces per waypoint (HSMC)
int compute_edge_masks(pump_graph* g, cudaStream_t s, int pairs = 0, int chunk = 0);
int compute_edge_masks_list(pump_graph* g, const int32_t* elist, long long n, uint32_t* out, uint32_t* bad,
                            cudaStream_t s);
int compute_edge_masks_batch(pump_graph* const* gs, int nq, cudaStream_t s, int pairs = 0, int chunk = 0, int span = 0);
int compute_edge_bounds(pump_graph* g, cudaStream_t s);
int run_explore(pump_graph* g, const pump_plan_params* p, float radius, pump_plan_result* stats,
                cudaStream_t s, bool collect, bool masks_pending = false);
void fill_explore_stats(pump_graph* g, const ExploreCtl& h, pump_plan_result* st);
int run_select(pump_graph* g, const pump_plan_params* p, int32_t* path, int32_t path_cap,
               pump_plan_result* out, ExploreCtl* ctl_host, cudaStream_t s);
int run_certify_path(pump_graph* g, const int32_t* path_host, int32_t path_len, int32_t n_mc,
                     int32_t substeps, uint64_t seed, int64_t* n_collide, cudaStream_t s);
int ensure_explore_bufs(pump_graph* g, int64_t cap, int32_t kmax, cudaStream_t s);
// masks_pending: the query's edge masks are not computed yet; the run computes them, inside the
// Explore launch where the fused form applies (explore_cluster.cu), else before it.
int run_explore_kernels(pump_graph* g, const ExploreArgs& A, int mode, cudaStream_t s, bool masks_pending = false);
// Fused masks + Explore allowed by the environment (PUMP_FUSED_MASKS=0 turns it off).
bool fused_masks_env();
int ensure_edge_targets(pump_graph* g, cudaStream_t s);
int prepare_explore_args(pump_graph* g, const pump_plan_params* p, float radius, ExploreArgs* out, cudaStream_t s);
int check_plan_params(const pump_plan_params* p);
int make_events(pump_graph* g);
void destroy_on_stream(pump_graph* g, cudaStream_t s);
// Explore kernel form from pump_plan_params.flags (see run_explore_kernels).
inline int explore_mode(int32_t flags) {
  return (flags & PUMP_STEPWISE) ? 2 : ((flags & PUMP_EXPLORE_GRID) ? 1 : 0);
}
int num_sms();

// ---------------------------------------------------------------------------
// Device helpers.

// Closed-loop model of one axis: LQR gain K = [1, sqrt(3)] (Q = I, R = 1) on
// the double integrator gives A = [[0, 1], [-1, -sqrt(3)]] with eigenvalues
// -sqrt(3)/2 +- i/2, so e^{A h} = e^{-sqrt(3) h/2} [cos(h/2) I + 2 sin(h/2) (A + sqrt(3)/2 I)].
// With V_c = sigma^2 I the stationary covariance S solves A S + S A^T + V_c = 0:
//   S12 = -sigma^2/2, S22 = sigma^2 / sqrt(3), S11 = S22 + sqrt(3) sigma^2 / 2,
// and the step noise covariance is Q(h) = S - e^{Ah} S e^{A^T h}.
__host__ __device__ inline void model_dev(double sigma, double h, double* Phi, double* L, double* Linf) {
  const double sq3 = 1.7320508075688772935;
  double ex = exp(-0.5 * sq3 * h);
  double sn = sin(0.5 * h), cs = cos(0.5 * h);
  Phi[0] = ex * (cs + sq3 * sn);
  Phi[1] = ex * (2.0 * sn);
  Phi[2] = -ex * (2.0 * sn);
  Phi[3] = ex * (cs - sq3 * sn);
  double s2 = sigma * sigma;
  double S12 = -0.5 * s2, S22 = s2 / sq3, S11 = S22 + 0.5 * sq3 * s2;
  // P S P^T
  double a = Phi[0], b = Phi[1], c = Phi[2], d = Phi[3];
  double t00 = a * S11 + b * S12, t01 = a * S12 + b * S22;
  double t10 = c * S11 + d * S12, t11 = c * S12 + d * S22;
  double r00 = t00 * a + t01 * b, r01 = t00 * c + t01 * d, r11 = t10 * c + t11 * d;
  double q00 = S11 - r00, q01 = S12 - r01, q11 = S22 - r11;
  double l00 = q00 > 0.0 ? sqrt(q00) : 0.0;
  double l10 = l00 > 0.0 ? q01 / l00 : 0.0;
  double rr = q11 - l10 * l10;
  L[0] = l00;
  L[1] = l10;
  L[2] = rr > 0.0 ? sqrt(rr) : 0.0;
  double i00 = S11 > 0.0 ? sqrt(S11) : 0.0;
  double i10 = i00 > 0.0 ? S12 / i00 : 0.0;
  double ir = S22 - i10 * i10;
  Linf[0] = i00;
  Linf[1] = i10;
  Linf[2] = ir > 0.0 ? sqrt(ir) : 0.0;
}

// Steering cost of the double integrator with c = integral (1 + |u|^2) dt.
// J(tau) = tau + 4a/tau - 12b/tau^2 + 12c/tau^3 with a = |v0|^2 + v0.v1 + |v1|^2,
// b = dp.(v0 + v1), c = |dp|^2; J' = f/tau^4, f = tau^4 - 4a tau^2 + 24b tau - 36c.
// Local minima are the roots where f crosses upward.  f' = 4 tau^3 - 8a tau + 24b
// is convex on tau > 0 with its minimum at tc = sqrt(2a/3); its positive roots
// split (0, inf) into monotone pieces of f.  Each root is found by Newton's
// method safeguarded by bisection on its bracket.
struct SteerCoef {
  double a, b, c;
};

__device__ inline double st_f(const SteerCoef& k, double t) { return ((t * t - 4.0 * k.a) * t + 24.0 * k.b) * t - 36.0 * k.c; }
__device__ inline double st_fp(const SteerCoef& k, double t) { return (4.0 * t * t - 8.0 * k.a) * t + 24.0 * k.b; }
__device__ inline double st_fpp(const SteerCoef& k, double t) { return 12.0 * t * t - 8.0 * k.a; }
__device__ inline double st_J(const SteerCoef& k, double t) {
  return t + (4.0 * k.a) / t - (12.0 * k.b) / (t * t) + (12.0 * k.c) / (t * t * t);
}

// which = 0: root of f, 1: root of f'.  `inc`: the function increases on [lo, hi].
__device__ inline double st_root(const SteerCoef& k, int which, double lo, double hi, bool inc) {
  double x = 0.5 * (lo + hi);
  for (int it = 0; it < 300; ++it) {
    double gx = which == 0 ? st_f(k, x) : st_fp(k, x);
    if (gx == 0.0) return x;
    bool right = inc ? (gx < 0.0) : (gx > 0.0);
    if (right) lo = x; else hi = x;
    double dg = which == 0 ? st_fp(k, x) : st_fpp(k, x);
    double xn = x - gx / dg;
    if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
    double step = fabs(xn - x);
    x = xn;
    if (step <= 4.0e-16 * fabs(x) || !(hi - lo > 2.5e-16 * fabs(hi))) break;
  }
  return x;
}

// Returns false for identical states (no connection).
__device__ inline bool steer_dev(const double* x0, const double* x1, double* tau_out, double* J_out) {
  SteerCoef k{0.0, 0.0, 0.0};
  for (int j = 0; j < 3; ++j) {
    double dp = x1[j] - x0[j], v0 = x0[3 + j], v1 = x1[3 + j];
    k.a += v0 * v0 + v0 * v1 + v1 * v1;
    k.b += dp * (v0 + v1);
    k.c += dp * dp;
  }
  if (k.c == 0.0 && k.a == 0.0) return false;
  double tc = sqrt(2.0 * k.a / 3.0);
  double hi_f = 1.0 + fmax(4.0 * k.a, fmax(24.0 * fabs(k.b), 36.0 * k.c));
  double lo_s[2], hi_s[2];
  int ns = 0;
  if (st_fp(k, tc) >= 0.0) {
    lo_s[ns] = 0.0; hi_s[ns++] = hi_f;
  } else {
    double hi_fp = 1.0 + fmax(2.0 * k.a, 6.0 * fabs(k.b));
    hi_fp = fmax(hi_fp, tc * 2.0 + 1.0);
    double tb = st_root(k, 1, tc, hi_fp, true);
    if (k.b > 0.0) {
      double ta = st_root(k, 1, 0.0, tc, false);
      lo_s[ns] = 0.0; hi_s[ns++] = ta;
    }
    lo_s[ns] = tb; hi_s[ns++] = fmax(hi_f, tb * 2.0 + 1.0);
  }
  double best_t = -1.0, best_J = __longlong_as_double(0x7ff0000000000000ll);
  for (int s = 0; s < ns; ++s) {
    double lo = lo_s[s], hi = hi_s[s];
    if (!(st_f(k, lo) < 0.0 && st_f(k, hi) > 0.0)) continue;
    double t = st_root(k, 0, lo, hi, true);
    double J = st_J(k, t);
    if (J < best_J || (J == best_J && t < best_t)) {
      best_J = J;
      best_t = t;
    }
  }
  if (!(best_t > 0.0)) return false;
  *tau_out = best_t;
  *J_out = best_J;
  return true;
}

// Position of the optimal connection of duration tau at time t, one axis: the cubic
// p0 + v0 t + c2 t^2 + c3 t^3 matching both end states.
struct Cubic {
  double p0, v0, c2, c3;
};
__device__ inline Cubic cubic_dev(const double* x0, const double* x1, double tau, int j) {
  Cubic q;
  q.p0 = x0[j];
  q.v0 = x0[3 + j];
  double dp = x1[j] - q.p0 - q.v0 * tau, dv = x1[3 + j] - q.v0;
  q.c2 = (3.0 * dp - dv * tau) / (tau * tau);
  q.c3 = (dv * tau - 2.0 * dp) / (tau * tau * tau);
  return q;
}
__device__ inline double cubic_at(const Cubic& q, double t) { return q.p0 + q.v0 * t + q.c2 * t * t + q.c3 * t * t * t; }

__device__ inline bool in_box_dev(float x, float y, float z, const float* b) {
  return b[0] <= x && x <= b[3] && b[1] <= y && y <= b[4] && b[2] <= z && z <= b[5];
}

// Group index of a cost: least i >= 0 with cost <= float(i * lr).
__device__ inline float group_thr(int32_t i, double lr) { return __double2float_rn(__dmul_rn((double)i, lr)); }
__device__ inline int32_t bucket_of(float cost, double lr) {
  double q = ceil((double)cost / lr);
  int32_t i = q < 0.0 ? 0 : (q > 2.0e9 ? 2000000000 : (int32_t)q);
  while (i > 0 && cost <= group_thr(i - 1, lr)) --i;
  while (cost > group_thr(i, lr)) ++i;
  return i;
}

// Explore's starting state, one thread: the root plan (id 0) at the start node, mbest entry
// (start, 0) = 0, group 0 = {root} with its candidate offsets, and the control block.
__device__ __forceinline__ void explore_init_thread(const ExploreArgs& A, int32_t start) {
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
  A.ginfo[0] = make_int4(0, start, A.row_ptr[start], __float_as_int(0.f));
  const int64_t d0 = A.row_ptr[start + 1] - A.row_ptr[start];
  A.goff[0] = 0;
  A.goff[1] = d0;
  if (A.prow) A.prow[0] = make_int2(A.row_ptr[start], (int32_t)((uint32_t)d0 | (A.is_goal[start] ? 0x80000000u : 0u)));
  c->n_plans = 1;
  c->n_candidates = 0;
  c->n_kept = 0;
  c->st[0].group_cands = d0;
  c->st[0].group_size = 1;
  c->st[0].iter = 0;
  c->st[0].stop = (A.early_stop && A.is_goal[start] && 0 < A.kmin) ? 1 : 0;
  c->st[1].group_cands = 0;
  c->st[1].group_size = 0;
  c->st[1].iter = 0;
  c->st[1].stop = 0;
  c->next_bucket[0] = kNoBucket;
  c->next_bucket[1] = kNoBucket;
  c->stop_next = 0;
  c->status = 0;
  c->n_groups = 0;
  c->survivors = 0;
  c->n_goal_all = 0;
  c->n_goal = 0;
  c->k_exit = 0;
  c->iter = 0;
  c->bar_count = 0;
  c->bar_gen = 0;
  if (A.is_goal[start]) {
    A.goal_all[0] = 0;
    c->n_goal_all = 1;
  }
}

// P_goal order: popc ascending, then cost descending, then id ascending.
__device__ __forceinline__ bool key_less(const ExploreArgs& A, int32_t a, int32_t b) {
  const int32_t pa = A.popc[a], pb = A.popc[b];
  if (pa != pb) return pa < pb;
  const float ca = A.cost[a], cb = A.cost[b];
  if (ca != cb) return ca > cb;
  return a < b;
}

// P_goal from the goal plans Explore recorded (one block): drops the plans RemoveDominated removed
// (settled from creation / expansion stamps) and sorts the rest in PlanSelection order.
__device__ __forceinline__ void goal_finalize_block(const ExploreArgs& A, int32_t* removed, int32_t* sorted) {
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

// Philox4x32-10 (Salmon et al., SC'11): one 32 x 32 -> 64-bit product per lane of the round.
__device__ inline void philox4x32(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1,
                                  uint32_t* o) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)M0 * c0, p1 = (uint64_t)M1 * c2;
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0, n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    c1 = (uint32_t)p1;
    c3 = (uint32_t)p0;
    c0 = n0;
    c2 = n2;
    k0 += W0;
    k1 += W1;
  }
  o[0] = c0; o[1] = c1; o[2] = c2; o[3] = c3;
}

// Philox4x64-10 (Salmon et al., SC'11).
__device__ inline void philox4x64(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3, uint64_t k0, uint64_t k1,
                                  uint64_t* o) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint64_t hi0 = __umul64hi(M0, c0), lo0 = M0 * c0;
    uint64_t hi1 = __umul64hi(M1, c2), lo1 = M1 * c2;
    uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += W0; k1 += W1;
  }
  o[0] = c0; o[1] = c1; o[2] = c2; o[3] = c3;
}

}  // namespace pump
