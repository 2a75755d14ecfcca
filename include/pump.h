/*
 * pump.h - C interface of libpump, a GB300 (sm_103a) implementation of the
 * multiobjective exploration of PUMP (Parallel Uncertainty-aware
 * Multiobjective Planning; Ichter, Schmerling, Agha-mohammadi, Pavone,
 * "Real-Time Stochastic Kinodynamic Motion Planning via Multiobjective Search
 * on GPUs").
 *
 * Conventions for every entry point:
 *  - Returns a pump_status code; no exception or device trap crosses this
 *    interface.  Output arguments are written only when PUMP_OK is returned,
 *    except where stated.
 *  - Array arguments may be host or device pointers (the library inspects
 *    each one); host arrays are copied to the device on the given stream.
 *    The caller keeps ownership of everything it passes in.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *    enqueued on it; calls that return results on the host synchronise it.
 *  - A pump_graph is used by one stream at a time.
 *  - Device memory comes from the allocator installed with
 *    pump_set_allocator (default: cudaMallocAsync on the call's stream).
 *
 * Problem model (Section II, Eq. (1)-(3); Section V-A): 6D double integrator
 * (3D position, velocity), state x = (p, v).  Obstacles are closed
 * axis-aligned boxes (Section V-C).  A plan's approximate collision
 * probability is popcount(mask) / N where mask ORs, over the plan's
 * connections, which of N particles collide (Section III-B).
 */
#ifndef PUMP_H_
#define PUMP_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PUMP_OK = 0,
  PUMP_ERR_INVALID_ARG = 1, /* bad size, pointer or parameter                    */
  PUMP_ERR_OOM = 2,         /* the allocator returned NULL                         */
  PUMP_ERR_CUDA = 3,        /* a CUDA runtime call failed                          */
  PUMP_ERR_CAPACITY = 4,    /* plan arena full: raise pump_plan_params.max_plans   */
  PUMP_ERR_TIMEOUT = 5,     /* iteration cap reached, or a device wait gave up     */
  PUMP_ERR_INFEASIBLE = 6   /* Algorithm 5 found no plan with MC CP <= alpha       */
} pump_status;

/* pump_plan_params.flags */
#define PUMP_NO_EARLY_STOP 1 /* Explore runs until P_open is empty (testing)        */
#define PUMP_EXPLORE_ONLY 2  /* pump_plan stops after Explore (no PlanSelection)    */
#define PUMP_STEPWISE 4      /* run Explore's phases as separate launches           */
#define PUMP_EXPLORE_GRID 8  /* run Explore as one grid-wide cooperative kernel
                                instead of one thread-block cluster                 */
#define PUMP_NO_WAIT 16      /* with PUMP_EXPLORE_ONLY: pump_plan enqueues the query
                                and returns at once (see pump_plan_collect)         */

typedef struct pump_graph pump_graph;

/* Closed box lo <= p <= hi on all three axes. */
typedef struct {
  float lo[3];
  float hi[3];
} pump_aabb;

typedef struct {
  float radius;        /* r_n: edge v->u iff float(Cost(v,u)) < radius (Section IV, Near) */
  int32_t n_particles; /* N, a multiple of 32 in [32, 1024]; masks have N/32 words       */
  int32_t n_waypoints; /* W >= 1 waypoints per connection                                */
  float sigma;         /* process-noise standard deviation, V_c = sigma^2 I (Eq. (1))    */
  int32_t flags;       /* 0, or PUMP_GRAPH_HSMC | PUMP_GRAPH_SEPARATE_MASKS               */
} pump_graph_params;

/* Particle collision masks by Half-Space Monte Carlo (the paper's CP approximation, section
 * "Half-Space Monte Carlo", Eq. (eq:hs)) instead of the particle-in-box test.  Per waypoint the
 * graph build forms the local convex region of the nominal position y with nominal velocity v:
 * repeatedly the remaining box closest to y (closest point c, ties to the lower box index),
 * d = c - y, a half-space recorded and every remaining box lying in {z : d.(z - y) >= d.d}
 * pruned (the closest box always), at most 8 half-spaces; each half-space is turned away from
 * the direction of travel, a = d - ((d.v)/(v.v)) v (a = d if v = 0), b = a.a.  A particle with
 * position deviation dy fires it iff fma(a2, dy2, fma(a1, dy1, a0 dy0)) > b; its mask bit is the
 * OR over waypoints 1..W and half-spaces.  All of it in float, each operation rounded as
 * written, left to right (a waypoint on or inside a box ends its region). */
#define PUMP_GRAPH_HSMC 1
/* The graph's queries keep the edge masks in their own launch (pump_plan never fuses them into
 * the Explore launch), so the build lays out no edge order for the fused form.  For callers that
 * run many queries on the device at once (the request server), where a launch holding most of
 * the device would stop the others from overlapping. */
#define PUMP_GRAPH_SEPARATE_MASKS 2

typedef struct {
  float alpha;            /* CP target (Eq. (3))                                          */
  float eta;              /* CP approximation factor: alpha_min = alpha/eta, alpha_max = eta*alpha (Algorithm 2) */
  float lambda;           /* group cost factor in (0, 1] (Algorithm 2, Algorithm 4)        */
  int32_t n_mc;           /* Monte Carlo rollouts per certification (Section III-A)       */
  int32_t mc_substeps;    /* rollout sub-steps per waypoint interval (>= 1)                */
  uint64_t mc_seed;       /* Philox4x32-10 key (lo, hi words) of the rollout normals       */
  int64_t max_plans;      /* plan arena capacity; more survivors -> PUMP_ERR_CAPACITY      */
  int32_t max_iterations; /* cap on Explore's group index; exceeded -> PUMP_ERR_TIMEOUT    */
  int32_t flags;          /* PUMP_NO_EARLY_STOP | PUMP_EXPLORE_ONLY | PUMP_STEPWISE |
                             PUMP_EXPLORE_GRID | PUMP_NO_WAIT                         */
} pump_plan_params;

typedef struct {
  int32_t status;         /* pump_status of the plan (PUMP_ERR_INFEASIBLE possible)        */
  int32_t chosen_plan;    /* arena id of the selected plan, -1 if none                     */
  float cost;             /* its cost                                                      */
  int32_t popc;           /* its particle-collision count; CP-hat = popc / N               */
  float cp_hat;           /* popc / N                                                      */
  double cp_mc;           /* Monte Carlo CP of the selected plan                           */
  int64_t mc_collisions;  /* colliding rollouts of the selected plan                       */
  int64_t n_candidates;   /* partial plans evaluated (Algorithm 4, candidate creation)     */
  int64_t n_kept;         /* candidates under the CP cutoff                                */
  int64_t n_plans;        /* plans in the arena (root + surviving candidates)              */
  int32_t n_iterations;   /* final group index i of Algorithm 4                            */
  int32_t n_groups;       /* non-empty groups expanded                                     */
  int32_t n_goal;         /* |P_goal|                                                      */
  int32_t n_certified;    /* plans certified by Monte Carlo                                */
  int32_t path_len;       /* node ids of the selected plan written to `path`               */
  int32_t path_truncated; /* 1 if path_len exceeded path_cap (path holds the first path_cap) */
  float ms_masks;         /* device time of the edge-mask step                             */
  float ms_explore;       /* device time of Explore                                        */
  float ms_select;        /* device time of PlanSelection                                  */
  int32_t fused;          /* 1: the edge masks ran inside the Explore launch (ms_masks then
                             covers only what precedes it, ms_explore both)               */
} pump_plan_result;

/* --------------------------------------------------------------------------
 * pump_set_allocator: install device-memory callbacks used for every later
 * allocation (graph buffers and plan scratch).  alloc(bytes, stream, ctx)
 * returns a device pointer or NULL; free_(ptr, stream, ctx) releases it.
 * Passing alloc == NULL restores the default (cudaMallocAsync/cudaFreeAsync).
 * Not thread-safe with concurrent library calls.  Returns PUMP_OK.
 * No counterpart in the paper (runtime plumbing).
 */
int pump_set_allocator(void* (*alloc)(size_t bytes, void* stream, void* ctx),
                       void (*free_)(void* ptr, void* stream, void* ctx), void* ctx);

/* --------------------------------------------------------------------------
 * pump_build_graph: BuildGraph (Algorithm 3) plus the obstacle-dependent
 * edge geometry the exploration needs.
 *  states  : n x 6 float (p, v) row-major; x_init = states[start_idx].
 *  goal_idx: n_goal node ids forming X_goal (at least one; Algorithm 3 keeps
 *            one sample of X_goal in V).
 *  boxes   : n_boxes closed AABBs (0 <= n_boxes <= 1024).
 *  xi      : N x (W+1) x 3 x 2 float standard normals (common random numbers
 *            of the particles: xi[i][0] draws the initial deviation from the
 *            stationary covariance, xi[i][k] drives step k).  The normals are
 *            an input rather than a seed: they are the random numbers the
 *            method draws (Section III-B), and taking them from the caller
 *            lets any generator supply them and lets an independent
 *            implementation consume exactly the same particles, so masks can
 *            be compared bit for bit.
 * Computes: node validity (outside every box), directed edges v->u for
 * valid v != u with float(Cost(v,u)) < radius whose nominal connection,
 * sampled at 4W uniform times in (0, tau], stays outside the boxes; edges of
 * each source sorted by target id; per edge the float cost, duration tau,
 * waypoint step h = tau/W, the closed-loop transition Phi(h) and noise
 * factor L(h), and the W nominal waypoints at t = k h.  Cost is the optimal
 * cost of the connection under c = integral (1 + u^T u) dt (Section II).
 * Errors: INVALID_ARG (n < 2, start/goal ids out of range or start inside
 * a box, N not a multiple of 32 or > 1024, W < 1 or > 64, radius <= 0,
 * sigma < 0), OOM, CUDA.  On success *out owns device memory; release with
 * pump_graph_destroy.  Synchronises `stream`.
 */
int pump_build_graph(const float* states, int32_t n, int32_t start_idx, const int32_t* goal_idx,
                     int32_t n_goal, const pump_aabb* boxes, int32_t n_boxes, const float* xi,
                     const pump_graph_params* params, void* stream, pump_graph** out);
/* pump_graph_build: former name of pump_build_graph (same arguments, same behaviour). */
int pump_graph_build(const float* states, int32_t n, int32_t start_idx, const int32_t* goal_idx,
                     int32_t n_goal, const pump_aabb* boxes, int32_t n_boxes, const float* xi,
                     const pump_graph_params* params, void* stream, pump_graph** out);

/* --------------------------------------------------------------------------
 * pump_graph_from_csr: import a precomputed graph with its edge masks (the
 * paper caches neighbours and edge controls offline, Section V-A).
 *  row_ptr : n+1 int32, col: E int32 targets (ascending within a row, no self
 *            loops), ecost: E float edge costs (>= 0), emask: E x (N/32) uint32.
 *  start_idx, goal_idx: as in pump_build_graph.
 * The graph has no geometry: pump_edge_masks and pump_certify return
 * INVALID_ARG on it.  Errors: INVALID_ARG, OOM, CUDA.  Synchronises.
 */
int pump_graph_from_csr(int32_t n, const int32_t* row_ptr, const int32_t* col, const float* ecost,
                        const uint32_t* emask, int32_t n_particles, int32_t start_idx,
                        const int32_t* goal_idx, int32_t n_goal, void* stream, pump_graph** out);

/* --------------------------------------------------------------------------
 * pump_edge_masks: particle collision mask of every edge (Section III-B with
 * a direct particle-in-box test).  Particle i of edge e starts at deviation
 * Linf xi[i][0] (Linf the Cholesky factor of the stationary covariance) and
 * steps d <- Phi(h) d + L(h) xi[i][k], k = 1..W, per axis in float with the
 * fixed fused-multiply-add order
 *   n0 = L00 xi0;  n1 = fma(L10, xi0, L11 xi1);
 *   d0 = fma(Phi00, d0, fma(Phi01, d1, n0));  d1 = fma(Phi10, d0_old, fma(Phi11, d1, n1));
 * its position at waypoint k is nominal_k + d0 (float add).  Bit i of the
 * mask is set iff some waypoint position lies in some box.  Masks are kept
 * in the graph (E x N/32 words, bit i%32 of word i/32).  Enqueued on
 * `stream`, no synchronisation.  Errors: INVALID_ARG (NULL graph, imported
 * graph), CUDA.
 */
int pump_edge_masks(pump_graph* g, void* stream);

/* pump_edge_masks_list: the same masks for a list of edges, repeats allowed:
 * row j of out_masks (device, n x N/32 words, caller-owned) is the mask of
 * edge edges[j] (device int32 ids in [0, E)).  This is the per-(plan, edge)
 * recomputation that an expansion performs when it evaluates the collision
 * probability per candidate, as Algorithm 4's expansion is written; the
 * library's own path computes each edge's mask once per query instead (a
 * mask does not depend on the plan).  The call exists for that comparison
 * and for callers that want candidate masks directly.  Box graphs only.
 * An id outside [0, E) leaves its row untouched and is counted in *bad_ids
 * (device uint32, caller-owned, zeroed by the call; may be NULL).  Enqueued on
 * `stream`, no synchronisation.  Errors: INVALID_ARG (NULL, imported or HSMC
 * graph, n < 0), OOM, CUDA.
 */
int pump_edge_masks_list(pump_graph* g, const int32_t* edges, int64_t n, uint32_t* out_masks, uint32_t* bad_ids,
                         void* stream);

/* --------------------------------------------------------------------------
 * pump_explore: Explore (Algorithm 4) on the graph's current edge masks.
 * Starts from the root plan (x_init, {}, 0, 0); groups G_i = open plans with
 * cost <= float(i * (lambda * r)) (product in double; r = the graph's radius,
 * or the `radius` argument for imported graphs); each group plan is extended
 * along every out-edge (cost = float sum, mask = OR); candidates with
 * popc >= K_max are cut (K_max = #{k >= 0 : k < (eta*alpha) N}); every open
 * plan dominated at its node (another plan there with strictly lower cost
 * and no larger popc) is removed; the search stops when a group holds a goal
 * plan with popc < K_min (K_min = #{k >= 0 : k < (alpha/eta) N}) or no open
 * plan remains.  Surviving candidates get consecutive arena ids in candidate
 * order (group plans by ascending id, then out-edges by target id).
 * `radius` is used only for graphs from pump_graph_from_csr (pass 0 for
 * built graphs).  Results stay in the graph (pump_export); counters in
 * `stats` (only the Explore fields are written).  Synchronises.
 * Errors: INVALID_ARG, OOM, CUDA, CAPACITY (arena full), TIMEOUT.
 */
int pump_explore(pump_graph* g, const pump_plan_params* params, float radius, pump_plan_result* stats,
                 void* stream);

/* --------------------------------------------------------------------------
 * pump_plan: PUMP (Algorithm 2) on a built graph: edge masks, Explore, and
 * PlanSelection (Algorithm 5): P_goal sorted by ascending CP-hat, ties by
 * descending cost then ascending id; 1-based bisection with MC(P_m) > alpha
 * moving u = m - 1, else l = m; failure if the final MC(P_m) > alpha.
 * Smoothing is not applied.  `path` (host, capacity path_cap) receives the
 * node ids of the selected plan from x_init.  The box masks run inside the
 * Explore launch where the device allows it (out->fused); the graph's first
 * such query also lays out its edge order (rows by shortest-path cost from
 * the start), which later queries reuse.  The environment variable
 * PUMP_FUSED_MASKS=0 keeps the masks in their own launch.  Results are the
 * same either way.  `out` is written on PUMP_OK
 * and on PUMP_ERR_INFEASIBLE (out->status tells which).  Synchronises,
 * except with PUMP_EXPLORE_ONLY | PUMP_NO_WAIT: the query (masks and
 * Explore) is only enqueued on `stream` and out->status, out->fused are
 * written, no counters or times; read the counters with pump_plan_collect.
 * Queries enqueued back to back on one graph run in stream order; a device
 * error (a timed-out wait) in one may make the next ones fail as well.
 * Errors: those of pump_explore, plus INFEASIBLE (no certified plan);
 * INVALID_ARG for PUMP_NO_WAIT without PUMP_EXPLORE_ONLY.
 */
int pump_plan(pump_graph* g, const pump_plan_params* params, int32_t* path, int32_t path_cap,
              pump_plan_result* out, void* stream);

/* --------------------------------------------------------------------------
 * pump_plan_collect: waits for `stream` and writes the Explore counters of
 * the graph's last query to `out` (as pump_explore does); afterwards
 * pump_export reads that query's arena.  For queries enqueued with
 * PUMP_NO_WAIT.  No counterpart in the paper (runtime plumbing).  Returns the
 * query's status.  Errors: INVALID_ARG (NULL, or no query ran), CUDA, and
 * the query's own CAPACITY / TIMEOUT.
 */
int pump_plan_collect(pump_graph* g, pump_plan_result* out, void* stream);

/* --------------------------------------------------------------------------
 * pump_plan_batch: pump_plan for n_queries independent queries, one per
 * built graph, with the box masks of all queries in one persistent launch and
 * the Explore runs of all queries in another (no counterpart in the paper: a
 * throughput form of Algorithm 2 for many problems at once).  graphs[q] (distinct, built by pump_build_graph) is
 * planned with params[q]; results[q] receives what pump_plan would write for
 * it (the selected path is left in the graph: pump_export of the plan arrays
 * and goal plans), except that ms_masks / ms_explore / ms_select are the
 * whole batch's phase times.  Each result equals the single-query result:
 * every query runs exactly the single-query algorithm, only concurrently.
 * `config` (may be NULL) chooses the form of the Explore launch and of the
 * edge-mask launches (results are the same in every form):
 */
typedef struct {
  int32_t cluster_size; /* CTAs per query: 16, 8 or 4; 0 = the largest the device co-schedules */
  int32_t mbest_global; /* 1: dominance tables in global memory instead of on chip             */
  int32_t max_clusters; /* queries in flight at once; 0 = as many as fit on the device          */
  int32_t mask_pairs;   /* particle block of the mask pass: mask-word pairs a warp advances side
                           by side (1 or 2; 0 = 2)                                             */
  int32_t mask_chunk;   /* edges a warp of the mask pass takes at a time (1 .. 64; 0 = 4)       */
  int32_t mask_span;    /* edges of one graph a block of the mask pass takes at a time (a
                           multiple of 32, 32 .. 65536; 0 = 1024)                              */
} pump_batch_config;
/* Queries whose params set PUMP_EXPLORE_ONLY stop after Explore; the others
 * run PlanSelection one after another.  Synchronises.
 * Errors: INVALID_ARG (null or repeated graph, imported graph, bad params or
 * config), OOM, CUDA; a query's own Explore or selection error is returned in
 * results[q].status (and the call returns the first such error).
 */
int pump_plan_batch(pump_graph* const* graphs, int32_t n_queries, const pump_plan_params* params,
                    const pump_batch_config* config, pump_plan_result* results, void* stream);

/* --------------------------------------------------------------------------
 * Serving: a request loop with continuous batching (no counterpart in the
 * paper; a deployment form of Algorithm 2 for a stream of queries).
 *
 * A server owns `max_slots` slots, each a CUDA stream with a worker thread on
 * the device current at creation.  Submitted requests wait in arrival order
 * and are admitted as soon as a slot is free and their estimated device memory
 * fits in `device_bytes` next to the admitted ones (a request larger than the
 * whole budget runs alone).  An admitted request builds its graph from its
 * arrays (pump_build_graph), plans (pump_plan) and frees the graph; requests in
 * different slots run concurrently on the device.  Every result equals the
 * result of the same calls made alone.  Device memory comes from the installed
 * allocator (pump_set_allocator), called from the worker threads.
 */
typedef struct pump_server pump_server;
typedef struct {
  const float* states;      /* n x 6, as pump_build_graph (host)            */
  int32_t n;
  int32_t start_idx;
  const int32_t* goal_idx;  /* n_goal node ids (host)                       */
  int32_t n_goal;
  const pump_aabb* boxes;   /* n_boxes (host)                               */
  int32_t n_boxes;
  const float* xi;          /* N x (W+1) x 3 x 2 (host)                      */
  pump_graph_params graph;
  pump_plan_params plan;
} pump_request;

/* Creates a server.  max_slots in [1, 64]; device_bytes > 0.
 * Errors: INVALID_ARG, CUDA. */
int pump_server_create(int32_t max_slots, int64_t device_bytes, pump_server** out);

/* Queues a request (its arrays are copied before the call returns) and
 * writes its ticket.  Errors: INVALID_ARG (bad arrays or sizes, server
 * stopping), OOM (host memory). */
int pump_server_submit(pump_server* s, const pump_request* req, int64_t* ticket);

/* Waits up to timeout_s seconds for a ticket.  On completion writes the
 * result (as pump_plan writes it), up to path_cap path node ids, the
 * latency from submission to completion in milliseconds, returns the
 * request's status, and forgets the ticket.  Returns PUMP_ERR_TIMEOUT if the
 * request is not done yet (the ticket stays valid), INVALID_ARG for an
 * unknown ticket. */
int pump_server_wait(pump_server* s, int64_t ticket, double timeout_s, pump_plan_result* out, int32_t* path,
                     int32_t path_cap, double* latency_ms);

/* Counters: submitted, admitted, completed, queued, running, peak running,
 * estimated bytes in use, peak estimated bytes (8 int64). */
int pump_server_stats(pump_server* s, int64_t* counters);

/* Stops the server: requests not yet admitted are dropped, admitted ones
 * finish; then the workers exit and the streams are released. */
void pump_server_destroy(pump_server* s);

/* --------------------------------------------------------------------------
 * pump_certify: MC(p) (Section III-A) for the plan visiting `path`
 * (path_len >= 1 node ids, consecutive ones joined by graph edges).  n_mc
 * rollouts of the closed loop: deviation drawn from the stationary
 * covariance at x_init and carried across connections; each waypoint
 * interval split into `substeps` steps of h/substeps; a rollout collides
 * iff a sub-step position lies in a box.  Rollout m, step s takes one
 * Philox4x32-10 call, counter (m, s lo, 0, s hi) and key (seed lo, seed hi);
 * its words w0..w3 give six 21-bit fields (the top 21 bits of each word,
 * then the low 11 bits of w0 followed by bits 10..1 of w1, and the same from
 * w2 and w3), and axis j draws its two normals by Box-Muller from fields 2j
 * and 2j+1, u = (b + 1/2) 2^-21.  Writes the colliding count and
 * count / n_mc.
 * Errors: INVALID_ARG (imported graph, path not along edges), OOM, CUDA.
 * Synchronises.
 */
int pump_certify(pump_graph* g, const int32_t* path, int32_t path_len, int32_t n_mc, int32_t substeps,
                 uint64_t seed, int64_t* n_collide, double* cp, void* stream);

/* --------------------------------------------------------------------------
 * pump_export: copy one array of the graph or of the last Explore into host
 * memory `host_buf` of `cap` bytes; *needed receives the byte size (always
 * written).  Returns INVALID_ARG if cap < needed or `what` is unknown.
 * Synchronises.  No counterpart in the paper (inspection and testing).
 */
enum {
  PUMP_EXPORT_COUNTS = 0,     /* int64[8]: n, E, n_plans, n_goal, N, W, n_words, valid nodes */
  PUMP_EXPORT_NODE_VALID = 1, /* uint8[n]                        */
  PUMP_EXPORT_ROW_PTR = 2,    /* int32[n+1]                      */
  PUMP_EXPORT_COL = 3,        /* int32[E]                        */
  PUMP_EXPORT_ECOST = 4,      /* float[E]                        */
  PUMP_EXPORT_TAU = 5,        /* float[E]                        */
  PUMP_EXPORT_H = 6,          /* float[E]                        */
  PUMP_EXPORT_PHI = 7,        /* float[E][4]                     */
  PUMP_EXPORT_L = 8,          /* float[E][3]                     */
  PUMP_EXPORT_NOMINAL = 9,    /* float[E][W][3]                  */
  PUMP_EXPORT_LINF = 10,      /* float[3]                        */
  PUMP_EXPORT_MASKS = 11,     /* uint32[E][N/32]                 */
  PUMP_EXPORT_PLAN_HEAD = 12, /* int32[n_plans]                  */
  PUMP_EXPORT_PLAN_PARENT = 13,
  PUMP_EXPORT_PLAN_COST = 14,    /* float[n_plans]                  */
  PUMP_EXPORT_PLAN_MASK = 15,    /* uint32[n_plans][N/32]           */
  PUMP_EXPORT_PLAN_POPC = 16,    /* int32[n_plans]                  */
  PUMP_EXPORT_PLAN_CREATED = 17, /* int32[n_plans] group index that created the plan (-1 root) */
  PUMP_EXPORT_PLAN_EXPANDED = 18, /* int32[n_plans] group index that expanded it, -1 if never */
  PUMP_EXPORT_GOAL_PLANS = 19,    /* int32[n_goal] P_goal ids in PlanSelection order */
  PUMP_EXPORT_EDGE_BOX = 20,      /* float[E][6] lo xyz, hi xyz: box holding every particle
                                     position of the edge (graph build; pump_edge_masks skips
                                     the obstacles it misses) */
  PUMP_EXPORT_NOMINAL_VEL = 21,   /* float[E][W][3] nominal velocity at the waypoints */
  PUMP_EXPORT_EDGE_ORDER = 22     /* int32[E][2] (edge, source row) in the order the masks of
                                     the fused launch are computed: rows by increasing
                                     shortest-path cost from the start, a row's edges in order
                                     (set by the first pump_plan that fuses; INVALID_ARG before) */
};
int pump_export(pump_graph* g, int32_t what, void* host_buf, size_t cap, size_t* needed);

/* --------------------------------------------------------------------------
 * pump_explore_noalloc: pump_explore for callers that cannot allocate device
 * memory while they plan: a robot's real-time control loop that reserves its
 * device memory at start-up (an allocation inside the loop can block for an
 * unbounded time, or fail once memory is fragmented), an embedded runtime
 * with a fixed memory budget, or a process whose device allocator belongs to
 * a host framework that must not be re-entered from this library.  No
 * counterpart in the paper: it is the same Explore run as pump_explore on an
 * imported graph, with the same results, but it calls no cudaMalloc,
 * cudaFree or other allocating routine.
 *  Inputs (device pointers on the current device, or managed memory):
 *  row_ptr n+1, col E, ecost E, emask E x N/32 (as for pump_graph_from_csr,
 *  which the caller must already satisfy: no checks are made on their
 *  contents), is_goal n bytes (nonzero = in X_goal).
 *  Outputs (same kind of pointers, `capacity` entries each; plan_mask
 *  capacity x N/32 words): the plan arena as pump_export would return it,
 *  and goal_plans (P_goal in PlanSelection order, stats->n_goal entries).
 *  stats receives the Explore counters.  The arena used holds
 *  C = min(capacity, params->max_plans) plans; more -> PUMP_ERR_CAPACITY.
 *  The kernels' scratch lives in a file-scope device array of 32 MiB that
 *  every GPU loading the library holds until the process exits.  A call
 *  needs 48 KiB + 4 n max(K_max, 1) + 36 C bytes (rounded up per buffer to
 *  256 B); larger problems return PUMP_ERR_INVALID_ARG, as do host pointers
 *  and pointers to another device's memory.  The first call on a device looks
 *  up the array's device address (cudaGetSymbolAddress) with that device
 *  current; make that first call before any stream capture.  All calls on a
 *  device share the array and it keeps the last call's contents (each call
 *  initialises what it reads): calls whose work overlaps on the GPU race and
 *  must be serialised by the caller.  Synchronises `stream` before it returns,
 *  on failure too.  Errors: INVALID_ARG, CUDA, CAPACITY, TIMEOUT.
 */
int pump_explore_noalloc(int32_t n, const int32_t* row_ptr, const int32_t* col, const float* ecost,
                         const uint32_t* emask, int32_t n_particles, int32_t start_idx, const uint8_t* is_goal,
                         float radius, const pump_plan_params* params, int64_t capacity, int32_t* plan_head,
                         int32_t* plan_parent, float* plan_cost, uint32_t* plan_mask, int32_t* plan_popc,
                         int32_t* plan_created, int32_t* plan_expanded, int32_t* goal_plans,
                         pump_plan_result* stats, void* stream);

/* ------------------------------------------------------------------------ */
/* Learned sampling proposal.  Not in the paper, which draws SampleFree      */
/* uniformly (Algorithm 3); an extension that learns where solution paths    */
/* run and proposes part of the samples there.                               */
/*                                                                          */
/* Network: dims[0] -> ... -> dims[L] (every width a multiple of 16, at most  */
/* 4096), ReLU after every layer but the last.  Products take BF16 operands  */
/* (inputs, weights, hidden activations rounded to nearest even) on the      */
/* tensor cores with FP32 sums; weights, biases and Adam's moments are FP32. */
/* An input row is [features (F floats), eight standard normals, zeros].     */
/* The first six outputs o are squashed into the state box: position         */
/* 0.5 + 0.5 tanh(o_j), velocity vmax tanh(o_j).  Loss (pump_mlp_set_loss):  */
/* winner takes all over the row's targets, or path-indexed; batch mean.     */
/* Optimiser: Adam (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected).       */
/* Parameter vector layout (FP32): per layer W (out x in, row-major) then b. */
/*                                                                          */
/* Draws: row r of draw set (t, stream) takes its normals from Philox4x64-10 */
/* (Salmon et al., SC'11) with counter (t, r, stream, 0) and key (seed, 1):  */
/* word j gives normals 2j, 2j+1 by Box-Muller on bits 63..40 and 39..16.    */
/* A training row's environment comes from counter (t, r, stream + 1, 0):    */
/* floor((word0 >> 32) n_env / 2^32).  Training step t (t = steps taken so   */
/* far) uses stream 0; proposals use t = 0, stream 2.                        */
/*                                                                          */
/* Every call below runs on the model's own stream, ordered after `stream`   */
/* (NULL: the legacy default stream), and returns when its work is done.     */
/* Pointer arguments may be host or device memory unless stated.  A model    */
/* is not thread-safe.  Errors: INVALID_ARG for bad sizes or NULL pointers,  */
/* OOM, CUDA.                                                               */
/* ------------------------------------------------------------------------ */
typedef struct pump_mlp pump_mlp;

/* pump_mlp_create: a model with n_layers layers of widths dims[0..n_layers],
 * He-uniform weights drawn from `seed`, zero biases, Adam state cleared. */
int pump_mlp_create(int32_t n_layers, const int32_t* dims, uint64_t seed, pump_mlp** out);

/* pump_mlp_param_count: length of the parameter vector (-1 for NULL). */
int64_t pump_mlp_param_count(const pump_mlp* m);

/* pump_mlp_set_params / pump_mlp_get_params: copy the FP32 parameter vector
 * in or out (count must equal pump_mlp_param_count).  Setting clears Adam's
 * moments and step count; getting also returns the step count (may be NULL). */
int pump_mlp_set_params(pump_mlp* m, const float* params, int64_t count);
int pump_mlp_get_params(pump_mlp* m, float* params, int64_t count, int64_t* steps);

/* pump_mlp_forward: outputs y (B x dims[L], FP32) of inputs x (B x dims[0],
 * FP32, rounded to BF16 on entry). */
int pump_mlp_forward(pump_mlp* m, const float* x, int32_t B, float* y, void* stream);

/* pump_mlp_gradients: gradient of sum(dy * y) with respect to every
 * parameter (vector layout; dy B x dims[L] FP32, rounded to BF16 like the
 * loss gradient) at inputs x.  Leaves the parameters unchanged. */
int pump_mlp_gradients(pump_mlp* m, const float* x, int32_t B, const float* dy, float* grads, int64_t count,
                       void* stream);

/* pump_mlp_train_step: one Adam step on explicit rows: inputs x (B x dims[0])
 * and per-row targets (B x T x 6, row r using its first n_targets[r]; a row
 * with none adds nothing).  Writes the batch's mean loss before the step. */
int pump_mlp_train_step(pump_mlp* m, const float* x, int32_t B, const float* targets, const int32_t* n_targets,
                        int32_t T, float lr, float vmax, float* mean_loss, void* stream);

/* pump_mlp_set_loss: the training loss.  kind 0 (default): winner takes all,
 * min over the row's targets of |s - y_p|^2.  kind 1: path-indexed, the
 * targets read as a polyline in path order and the target taken at fraction
 * u = Phi(x[latent_col]) of it by node index (Phi the standard normal CDF, x
 * the row's BF16 input): a = u (n - 1), i = min(floor(a), n - 2),
 * y = y_i + (a - i)(y_{i+1} - y_i), or y_0 when n = 1.  Errors: INVALID_ARG
 * for another kind or a column outside [0, dims[0]). */
int pump_mlp_set_loss(pump_mlp* m, int32_t kind, int32_t latent_col);

/* pump_mlp_set_data: copy a training set into the model: per environment e,
 * features feat[e] (F floats, F + 8 <= dims[0]) and targets (n_env x T x 6)
 * of which the first n_targets[e] are used. */
int pump_mlp_set_data(pump_mlp* m, const float* feat, int32_t F, int32_t n_env, const float* targets,
                      const int32_t* n_targets, int32_t T);

/* pump_mlp_train: `steps` Adam steps of B rows each on the stored training
 * set, every row drawing its environment and normals (draw set (t, 0)).  One
 * step is captured as a CUDA graph on first use and replayed.  Writes the
 * mean loss of each step to loss_trace[0 .. steps) (may be NULL). */
int pump_mlp_train(pump_mlp* m, int32_t B, int32_t steps, float lr, float vmax, uint64_t seed, float* loss_trace,
                   void* stream);

/* pump_mlp_assemble: the inputs x (B x dims[0], FP32 values of the BF16
 * rows) and environments env (B, may be NULL) that training step t with
 * `seed` would use on the stored training set; no training happens. */
int pump_mlp_assemble(pump_mlp* m, int32_t B, int64_t t, uint64_t seed, float* x, int32_t* env);

/* pump_mlp_propose: `count` proposal states (count x 6) for one environment
 * with features feat (F floats), latent draws (0, r, 2) for rows r. */
int pump_mlp_propose(pump_mlp* m, const float* feat, int32_t F, int32_t count, uint64_t seed, float vmax,
                     float* states, void* stream);

/* pump_mlp_destroy: release a model (NULL is a no-op). */
void pump_mlp_destroy(pump_mlp* m);

/* pump_kernel_launches: number of kernels this library has launched in the
 * process so far (host-side counter, all devices; for launch accounting).
 * No counterpart in the paper. */
uint64_t pump_kernel_launches(void);

/* pump_graph_destroy: release a graph and its scratch (NULL is a no-op). */
void pump_graph_destroy(pump_graph* g);

/* pump_status_str: static description of a status code. */
const char* pump_status_str(int status);

#ifdef __cplusplus
}
#endif
#endif /* PUMP_H_ */
