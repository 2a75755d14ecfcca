/*
 * CPU oracle for PUMP (Ichter, Schmerling, Agha-mohammadi, Pavone,
 * "Real-Time Stochastic Kinodynamic Motion Planning via Multiobjective Search
 * on GPUs").
 *
 * TEST INFRASTRUCTURE.  This file is a plain, slow, single-threaded
 * restatement of what the planner computes (O4 and O5 also take a thread
 * count, used only to time the oracle on all host cores: the threads split
 * independent loops and the results are the single-thread results).  Only the test-suite, the smoke
 * check and the benchmark's CPU-baseline leg load it.  It shares no code with
 * the CUDA library: no headers, helpers or tables.  It must be compiled with
 * -ffp-contract=off so that the compiler does not fuse the float products and
 * sums written below.  Floating point is double except where the planner's
 * definition fixes float (graph values handed to the search, particle
 * recurrence, path-cost sums).
 *
 * Contents, each in the paper's order and notation:
 *   O1 steering cost  Cost(u,v)            Section II (cost c), Section IV
 *   O2 graph build    BuildGraph           Algorithm 3
 *   O3 tracking model and particles        Eq. (1), Eq. (2), Section III-B
 *   O4 edge particle collision masks       Section III-B (OR over time, count / N)
 *   O5 Explore                             Algorithm 4 and RemoveDominated, Section IV
 *   O6 PlanSelection and MC(p)             Algorithm 5, Section III-A
 *   Philox4x64-10 and Philox4x32-10        Salmon et al., SC'11 (MC normals:
 *      Philox4x32-10; proposal draws: Philox4x64-10)
 *   O7 draws of the learned sampling proposal (latents, batch rows); the
 *      proposal network itself is restated in oracle/mlp.py
 *
 * Readings of points the paper leaves open (cost weights, controller gains,
 * tie rules, thresholds) are stated beside the code that takes them.
 */
#include <math.h>
#include <pthread.h>
#include <stdatomic.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_INVALID_ARG 1
#define ORC_ERR_OOM 2
#define ORC_ERR_CAPACITY 4
#define ORC_ERR_TIMEOUT 5
#define ORC_ERR_INFEASIBLE 6

#define ORC_NO_EARLY_STOP 1

/* ========================================================================== */
/* O1  Steering cost.                                                           */
/*                                                                              */
/* Double integrator x'' = u per axis (Section V-A).  Cost of a connection of  */
/* duration tau: c = integral_0^tau (1 + u^T u) dt, the mixed time / control    */
/* effort cost the paper uses (Section II); unit weights are our reading.      */
/* For fixed tau the optimal control gives, with dp = p1 - p0,                 */
/*   J(tau) = tau + 4a/tau - 12b/tau^2 + 12c/tau^3,                             */
/*   a = |v0|^2 + v0.v1 + |v1|^2,  b = dp.(v0 + v1),  c = |dp|^2,              */
/* and Cost(u,v) = min over tau > 0 of J(tau).  dJ/dtau = f(tau)/tau^4 with    */
/*   f(tau) = tau^4 - 4a tau^2 + 24b tau - 36c,                                 */
/* so the minimisers are roots of f where f changes sign from - to +.          */
/* ========================================================================== */
static double steer_J(double a, double b, double c, double t) {
  return t + (4.0 * a) / t - (12.0 * b) / (t * t) + (12.0 * c) / (t * t * t);
}
static double steer_f(double a, double b, double c, double t) {
  return t * t * t * t - 4.0 * a * t * t + 24.0 * b * t - 36.0 * c;
}
static double steer_fp(double a, double b, double c, double t) {
  (void)c;
  return 4.0 * t * t * t - 8.0 * a * t + 24.0 * b;
}
typedef double (*orc_fn)(double, double, double, double);

/* Bisection on [lo, hi] for a function monotone there with a sign change.   */
/* Runs until the interval cannot shrink in double precision.                */
static double bisect(orc_fn g, double a, double b, double c, double lo, double hi, int increasing) {
  for (int it = 0; it < 4096; ++it) {
    double mid = lo + 0.5 * (hi - lo);
    if (!(mid > lo && mid < hi)) break;
    double v = g(a, b, c, mid);
    int root_right = increasing ? (v < 0.0) : (v > 0.0);
    if (root_right) lo = mid; else hi = mid;
  }
  return fabs(g(a, b, c, lo)) <= fabs(g(a, b, c, hi)) ? lo : hi;
}

static double grow_until_positive(orc_fn g, double a, double b, double c, double lo) {
  double hi = lo > 0.5 ? 2.0 * lo : 1.0;
  while (g(a, b, c, hi) <= 0.0 && hi < 1e300) hi *= 2.0;
  return hi;
}

/* Returns 0 and (tau*, J*) in double, or -1 for identical states (no edge). */
int orc_steer(const double* x0, const double* x1, double* tau_out, double* cost_out) {
  double a = 0.0, b = 0.0, c = 0.0;
  for (int j = 0; j < 3; ++j) {
    double dp = x1[j] - x0[j], v0 = x0[3 + j], v1 = x1[3 + j];
    a += v0 * v0 + v0 * v1 + v1 * v1;
    b += dp * (v0 + v1);
    c += dp * dp;
  }
  if (c == 0.0 && a == 0.0) return -1;
  /* f' is decreasing on [0, tc] and increasing on [tc, inf), tc = sqrt(2a/3). */
  double tc = sqrt(2.0 * a / 3.0);
  double inc_lo[2], inc_hi[2];   /* pieces of (0, inf) on which f increases; hi < 0 means inf */
  int n_inc = 0;
  if (steer_fp(a, b, c, tc) >= 0.0) {
    inc_lo[n_inc] = 0.0; inc_hi[n_inc++] = -1.0;
  } else {
    double up = grow_until_positive(steer_fp, a, b, c, tc);
    double tb = bisect(steer_fp, a, b, c, tc, up, 1);
    if (b > 0.0) {
      double ta = bisect(steer_fp, a, b, c, 0.0, tc, 0);
      inc_lo[n_inc] = 0.0; inc_hi[n_inc++] = ta;
    }
    inc_lo[n_inc] = tb; inc_hi[n_inc++] = -1.0;
  }
  double best_t = -1.0, best_J = INFINITY;
  for (int s = 0; s < n_inc; ++s) {
    double lo = inc_lo[s];
    double hi = inc_hi[s] < 0.0 ? grow_until_positive(steer_f, a, b, c, lo) : inc_hi[s];
    if (!(steer_f(a, b, c, lo) < 0.0 && steer_f(a, b, c, hi) > 0.0)) continue;
    double t = bisect(steer_f, a, b, c, lo, hi, 1);
    double J = steer_J(a, b, c, t);
    if (J < best_J || (J == best_J && t < best_t)) { best_J = J; best_t = t; }
  }
  if (best_t <= 0.0) return -1;
  *tau_out = best_t;
  *cost_out = best_J;
  return 0;
}

/* Velocity of the optimal connection at time t (derivative of the cubic below). */
static double nominal_vel(const double* x0, const double* x1, double tau, int j, double t) {
  double p0 = x0[j], v0 = x0[3 + j], p1 = x1[j], v1 = x1[3 + j];
  double dp = p1 - p0 - v0 * tau, dv = v1 - v0;
  double c2 = (3.0 * dp - dv * tau) / (tau * tau);
  double c3 = (dv * tau - 2.0 * dp) / (tau * tau * tau);
  return v0 + 2.0 * c2 * t + 3.0 * c3 * t * t;
}

/* Position of the optimal connection at time t (per axis cubic), duration tau. */
static double nominal_pos(const double* x0, const double* x1, double tau, int j, double t) {
  double p0 = x0[j], v0 = x0[3 + j], p1 = x1[j], v1 = x1[3 + j];
  double dp = p1 - p0 - v0 * tau, dv = v1 - v0;
  double c2 = (3.0 * dp - dv * tau) / (tau * tau);
  double c3 = (dv * tau - 2.0 * dp) / (tau * tau * tau);
  return p0 + v0 * t + c2 * t * t + c3 * t * t * t;
}

/* ========================================================================== */
/* O3  Tracking model (Eq. (1), Eq. (2)).  Per axis the state deviation is    */
/* (position, velocity); full-state LQR with Q = I, R = 1 gives the gain      */
/* K = [1, sqrt(3)] (our reading: the paper's LQG weights are not printed and */
/* the noise model has no measurement term).  The closed loop                  */
/*   A = [[0, 1], [-1, -sqrt(3)]]                                              */
/* is discretised exactly over a step h: Phi(h) = e^{A h}, and with process    */
/* noise V_c = sigma^2 I the step noise covariance is                          */
/*   Q(h) = integral_0^h e^{As} V_c e^{A^T s} ds = S - Phi S Phi^T,            */
/* S the stationary solution of A S + S A^T + V_c = 0.                         */
/* ========================================================================== */
static const double ORC_K1 = 1.0;
#define ORC_K2 1.7320508075688772 /* sqrt(3) */

static void mat2_mul(const double* X, const double* Y, double* Z) {
  double z0 = X[0] * Y[0] + X[1] * Y[2], z1 = X[0] * Y[1] + X[1] * Y[3];
  double z2 = X[2] * Y[0] + X[3] * Y[2], z3 = X[2] * Y[1] + X[3] * Y[3];
  Z[0] = z0; Z[1] = z1; Z[2] = z2; Z[3] = z3;
}

/* e^{A h} by the Taylor series of the exponential on A h / 2^s, then s squarings. */
static void closed_loop_expm(double h, double* Phi) {
  const double A[4] = {0.0, 1.0, -ORC_K1, -ORC_K2};
  double norm = (fabs(A[0]) + fabs(A[1]) > fabs(A[2]) + fabs(A[3]) ? fabs(A[0]) + fabs(A[1])
                                                                     : fabs(A[2]) + fabs(A[3])) * fabs(h);
  int s = 0;
  while (norm > 0.25) { norm *= 0.5; ++s; }
  double scale = h / ldexp(1.0, s);
  double M[4] = {A[0] * scale, A[1] * scale, A[2] * scale, A[3] * scale};
  double E[4] = {1.0, 0.0, 0.0, 1.0}, T[4] = {1.0, 0.0, 0.0, 1.0};
  for (int k = 1; k < 40; ++k) {
    mat2_mul(T, M, T);
    for (int q = 0; q < 4; ++q) T[q] /= (double)k;
    for (int q = 0; q < 4; ++q) E[q] += T[q];
  }
  for (int q = 0; q < s; ++q) mat2_mul(E, E, E);
  memcpy(Phi, E, sizeof(E));
}

/* Stationary covariance: solve the 3 Lyapunov equations for (S11, S12, S22). */
static void stationary_cov(double sigma, double* S /* S11, S12, S22 */) {
  const double A[2][2] = {{0.0, 1.0}, {-ORC_K1, -ORC_K2}};
  const double V[2][2] = {{sigma * sigma, 0.0}, {0.0, sigma * sigma}};
  /* unknown u = (S11, S12, S22); Sigma[k][l] = u[idx[k][l]] */
  const int idx[2][2] = {{0, 1}, {1, 2}};
  const int eqs[3][2] = {{0, 0}, {0, 1}, {1, 1}};
  double Mx[3][4];
  for (int r = 0; r < 3; ++r) {
    int i = eqs[r][0], j = eqs[r][1];
    for (int q = 0; q < 4; ++q) Mx[r][q] = 0.0;
    for (int k = 0; k < 2; ++k) {
      Mx[r][idx[k][j]] += A[i][k];   /* (A Sigma)_{ij}   */
      Mx[r][idx[i][k]] += A[j][k];   /* (Sigma A^T)_{ij} */
    }
    Mx[r][3] = -V[i][j];
  }
  /* Gaussian elimination with partial pivoting */
  for (int col = 0; col < 3; ++col) {
    int piv = col;
    for (int r = col + 1; r < 3; ++r) if (fabs(Mx[r][col]) > fabs(Mx[piv][col])) piv = r;
    if (piv != col) for (int q = 0; q < 4; ++q) { double t = Mx[col][q]; Mx[col][q] = Mx[piv][q]; Mx[piv][q] = t; }
    for (int r = col + 1; r < 3; ++r) {
      double f = Mx[r][col] / Mx[col][col];
      for (int q = col; q < 4; ++q) Mx[r][q] -= f * Mx[col][q];
    }
  }
  for (int r = 2; r >= 0; --r) {
    double v = Mx[r][3];
    for (int q = r + 1; q < 3; ++q) v -= Mx[r][q] * S[q];
    S[r] = v / Mx[r][r];
  }
}

/* Lower Cholesky factor (L00, L10, L11) of a symmetric 2x2 (q11, q12, q22);    */
/* a non-positive pivot (sigma = 0) gives a zero column.                        */
static void chol2(const double* q, double* L) {
  double l00 = q[0] > 0.0 ? sqrt(q[0]) : 0.0;
  double l10 = l00 > 0.0 ? q[1] / l00 : 0.0;
  double r = q[2] - l10 * l10;
  L[0] = l00; L[1] = l10; L[2] = r > 0.0 ? sqrt(r) : 0.0;
}

/* Double-precision model for step h: Phi (4), Q(h) (q11, q12, q22), L (3),    */
/* stationary S (3) and its factor Linf (3).                                     */
void orc_model(double sigma, double h, double* Phi, double* Q, double* L, double* S, double* Linf) {
  closed_loop_expm(h, Phi);
  stationary_cov(sigma, S);
  double Sm[4] = {S[0], S[1], S[1], S[2]}, T[4], PT[4] = {Phi[0], Phi[2], Phi[1], Phi[3]}, R[4];
  mat2_mul(Phi, Sm, T);
  mat2_mul(T, PT, R);
  Q[0] = S[0] - R[0]; Q[1] = S[1] - R[1]; Q[2] = S[2] - R[3];
  chol2(Q, L);
  chol2(S, Linf);
}

/* Float model for step h as handed to the particle recurrence. */
static void model_f32(double sigma, float h, float* Phi32, float* L32, float* Linf32) {
  double Phi[4], Q[3], L[3], S[3], Linf[3];
  orc_model(sigma, (double)h, Phi, Q, L, S, Linf);
  for (int q = 0; q < 4; ++q) Phi32[q] = (float)Phi[q];
  for (int q = 0; q < 3; ++q) { L32[q] = (float)L[q]; Linf32[q] = (float)Linf[q]; }
}

/* One step of the particle deviation recurrence for one axis, in float with  */
/* this fixed order of fused multiply-adds (the particle definition):          */
/*   n0 = L00 xi0;  n1 = L10 xi0 + L11 xi1;                                    */
/*   d0' = Phi00 d0 + (Phi01 d1 + n0);  d1' = Phi10 d0 + (Phi11 d1 + n1).      */
static void dev_step(const float* Phi, const float* L, float xi0, float xi1, float* d0, float* d1) {
  float n0 = L[0] * xi0;
  float n1 = fmaf(L[1], xi0, L[2] * xi1);
  float e0 = fmaf(Phi[0], *d0, fmaf(Phi[1], *d1, n0));
  float e1 = fmaf(Phi[2], *d0, fmaf(Phi[3], *d1, n1));
  *d0 = e0; *d1 = e1;
}
static void dev_init(const float* Linf, float xi0, float xi1, float* d0, float* d1) {
  *d0 = Linf[0] * xi0;
  *d1 = fmaf(Linf[1], xi0, Linf[2] * xi1);
}

static int in_box(const float* p, const float* box) {
  return box[0] <= p[0] && p[0] <= box[3] && box[1] <= p[1] && p[1] <= box[4] &&
         box[2] <= p[2] && p[2] <= box[5];
}
static int in_any_box(const float* p, const float* boxes, int n_boxes) {
  for (int o = 0; o < n_boxes; ++o)
    if (in_box(p, boxes + 6 * o)) return 1;
  return 0;
}

/* ========================================================================== */
/* O2  BuildGraph (Algorithm 3).                                                 */
/* SampleFree: a node is valid iff its position is outside every closed box.    */
/* Near: u in N(v) iff u != v, both valid, and float(Cost(v,u)) < r (strict).  */
/* Collision(v,u): the nominal connection is sampled at 4W uniform times in     */
/* (0, tau] (position rounded to float) and the edge is dropped if any sample   */
/* lies in a box.  Edge values handed on: cost and duration rounded to float,   */
/* waypoint step h = float(tau) / W in float, Phi(h) and L(h) rounded to float, */
/* and the W nominal waypoints at t_k = k h (double evaluation, float result).  */
/* Pruning shortcuts, both exact: with vbar = (v0 + v1)/2 the same cost reads   */
/*   J(tau) = tau + |dv|^2/tau + 12 |dp - vbar tau|^2 / tau^3.                  */
/* (i) J >= tau + |dv|^2/tau >= 2|dv|, so 2|dv| >= r rules the pair out.        */
/* (ii) J < r needs some tau < r with 12|dp - vbar tau|^2 < (r - tau) tau^3     */
/* <= 27 r^4 / 256, i.e. |dp| < |vbar| r + (3/32) r^2.                          */
/* Both are applied with a relative margin of 1e-9; `exhaustive` turns them off.*/
/* ========================================================================== */
typedef struct {
  int n, n_edges, W;
  double sigma;
  uint8_t* valid;
  int32_t* row_ptr;
  int32_t* col;
  float* ecost;
  float* tau;
  float* h;
  float* phi;   /* E x 4 */
  float* L;     /* E x 3 */
  float* nom;   /* E x W x 3 */
  float* nvel;  /* E x W x 3: nominal velocity at the waypoints */
  float linf[3];
  int64_t n_pairs_costed, n_near, n_collide_removed;
} orc_graph;

void orc_graph_free(orc_graph* g) {
  if (!g) return;
  free(g->valid); free(g->row_ptr); free(g->col); free(g->ecost); free(g->tau); free(g->h);
  free(g->phi); free(g->L); free(g->nom); free(g->nvel); free(g);
}

/* sigma is the problem's float noise level (as at the library boundary); it is widened to double. */
orc_graph* orc_graph_build(const float* states, int n, const float* boxes, int n_boxes, float r,
                           int W, float sigma, int exhaustive) {
  if (n <= 0 || W <= 0 || !(r > 0.0f)) return NULL;
  orc_graph* g = (orc_graph*)calloc(1, sizeof(orc_graph));
  if (!g) return NULL;
  g->n = n; g->W = W; g->sigma = (double)sigma;
  g->valid = (uint8_t*)malloc((size_t)n);
  g->row_ptr = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n + 1));
  size_t cap = 1024, E = 0;
  int32_t* col = (int32_t*)malloc(sizeof(int32_t) * cap);
  float* ecost = (float*)malloc(sizeof(float) * cap);
  float* tau = (float*)malloc(sizeof(float) * cap);
  if (!g->valid || !g->row_ptr || !col || !ecost || !tau) goto oom;
  for (int v = 0; v < n; ++v) g->valid[v] = !in_any_box(states + 6 * v, boxes, n_boxes);
  for (int v = 0; v < n; ++v) {
    g->row_ptr[v] = (int32_t)E;
    if (!g->valid[v]) continue;
    double xv[6];
    for (int q = 0; q < 6; ++q) xv[q] = (double)states[6 * v + q];
    for (int u = 0; u < n; ++u) {
      if (u == v || !g->valid[u]) continue;
      double xu[6];
      for (int q = 0; q < 6; ++q) xu[q] = (double)states[6 * u + q];
      if (!exhaustive) {
        double dv2 = 0.0, dp2 = 0.0, vb2 = 0.0, rd = (double)r;
        for (int j = 0; j < 3; ++j) {
          double dv = xu[3 + j] - xv[3 + j], dp = xu[j] - xv[j], vb = 0.5 * (xu[3 + j] + xv[3 + j]);
          dv2 += dv * dv; dp2 += dp * dp; vb2 += vb * vb;
        }
        if (2.0 * sqrt(dv2) >= rd * (1.0 + 1e-9)) continue;
        if (sqrt(dp2) >= (sqrt(vb2) * rd + 0.09375 * rd * rd) * (1.0 + 1e-9)) continue;
      }
      double t, J;
      g->n_pairs_costed++;
      if (orc_steer(xv, xu, &t, &J) != 0) continue;
      float J32 = (float)J;
      if (!(J32 < r)) continue;
      g->n_near++;
      float t32 = (float)t;
      /* Collision(v, u) on the nominal connection of duration float(tau) */
      double td = (double)t32;
      int hit = 0;
      for (int m = 1; m <= 4 * W && !hit; ++m) {
        double tm = td * ((double)m / (double)(4 * W));
        float p[3];
        for (int j = 0; j < 3; ++j) p[j] = (float)nominal_pos(xv, xu, td, j, tm);
        hit = in_any_box(p, boxes, n_boxes);
      }
      if (hit) { g->n_collide_removed++; continue; }
      if (E == cap) {
        cap *= 2;
        int32_t* c2 = (int32_t*)realloc(col, sizeof(int32_t) * cap);
        if (!c2) goto oom;
        col = c2;
        float* e2 = (float*)realloc(ecost, sizeof(float) * cap);
        if (!e2) goto oom;
        ecost = e2;
        float* t2 = (float*)realloc(tau, sizeof(float) * cap);
        if (!t2) goto oom;
        tau = t2;
      }
      col[E] = u; ecost[E] = J32; tau[E] = t32; ++E;
    }
  }
  g->row_ptr[n] = (int32_t)E;
  g->n_edges = (int)E;
  g->col = col; g->ecost = ecost; g->tau = tau;
  col = NULL; ecost = NULL; tau = NULL;
  g->h = (float*)malloc(sizeof(float) * (E ? E : 1));
  g->phi = (float*)malloc(sizeof(float) * 4 * (E ? E : 1));
  g->L = (float*)malloc(sizeof(float) * 3 * (E ? E : 1));
  g->nom = (float*)malloc(sizeof(float) * 3 * (size_t)W * (E ? E : 1));
  g->nvel = (float*)malloc(sizeof(float) * 3 * (size_t)W * (E ? E : 1));
  if (!g->h || !g->phi || !g->L || !g->nom || !g->nvel) goto oom;
  {
    float phi_dummy[4], l_dummy[3];
    model_f32(g->sigma, 1.0f, phi_dummy, l_dummy, g->linf);
  }
  for (int v = 0; v < n; ++v) {
    double xv[6];
    for (int q = 0; q < 6; ++q) xv[q] = (double)states[6 * v + q];
    for (int e = g->row_ptr[v]; e < g->row_ptr[v + 1]; ++e) {
      double xu[6];
      for (int q = 0; q < 6; ++q) xu[q] = (double)states[6 * g->col[e] + q];
      float h = g->tau[e] / (float)W;
      float lin[3];
      g->h[e] = h;
      model_f32(g->sigma, h, g->phi + 4 * (size_t)e, g->L + 3 * (size_t)e, lin);
      double td = (double)g->tau[e];
      for (int k = 1; k <= W; ++k) {
        double tk = (double)k * (double)h;
        for (int j = 0; j < 3; ++j) {
          g->nom[((size_t)e * W + (k - 1)) * 3 + j] = (float)nominal_pos(xv, xu, td, j, tk);
          g->nvel[((size_t)e * W + (k - 1)) * 3 + j] = (float)nominal_vel(xv, xu, td, j, tk);
        }
      }
    }
  }
  return g;
oom:
  free(col); free(ecost); free(tau);
  orc_graph_free(g);
  return NULL;
}

void orc_graph_counts(const orc_graph* g, int64_t* out /* n, E, pairs_costed, near, collide_removed */) {
  out[0] = g->n; out[1] = g->n_edges; out[2] = g->n_pairs_costed; out[3] = g->n_near;
  out[4] = g->n_collide_removed;
}

void orc_graph_nvel(const orc_graph* g, float* nvel) {
  if (nvel) memcpy(nvel, g->nvel, sizeof(float) * 3 * (size_t)g->W * (size_t)g->n_edges);
}

void orc_graph_export(const orc_graph* g, uint8_t* valid, int32_t* row_ptr, int32_t* col, float* ecost,
                      float* tau, float* h, float* phi, float* L, float* nom, float* linf) {
  size_t E = (size_t)g->n_edges;
  if (valid) memcpy(valid, g->valid, (size_t)g->n);
  if (row_ptr) memcpy(row_ptr, g->row_ptr, sizeof(int32_t) * (size_t)(g->n + 1));
  if (col) memcpy(col, g->col, sizeof(int32_t) * E);
  if (ecost) memcpy(ecost, g->ecost, sizeof(float) * E);
  if (tau) memcpy(tau, g->tau, sizeof(float) * E);
  if (h) memcpy(h, g->h, sizeof(float) * E);
  if (phi) memcpy(phi, g->phi, sizeof(float) * 4 * E);
  if (L) memcpy(L, g->L, sizeof(float) * 3 * E);
  if (nom) memcpy(nom, g->nom, sizeof(float) * 3 * (size_t)g->W * E);
  if (linf) memcpy(linf, g->linf, sizeof(float) * 3);
}

/* ========================================================================== */
/* O4  Edge particle collision masks (Section III-B, with the box test in     */
/* place of the half-space test).  Particle i of edge e: deviation starts at   */
/* Linf xi[i][0] and takes W steps with the edge's (Phi, L) and xi[i][k]; its  */
/* position at waypoint k is nominal_k + d0.  The particle collides iff any    */
/* waypoint position lies in any closed box; bit i of the mask is that event.  */
/* xi is laid out [N][W+1][3][2].  Masks are w = N/32 words per edge, particle */
/* i in word i/32, bit i%32.                                                     */
/* ========================================================================== */
static void edge_masks_range(int e0, int e1, int W, int N, const float* phi, const float* L, const float* nom,
                             const float* linf, const float* xi, const float* boxes, int n_boxes, uint32_t* mask) {
  int w = N / 32;
  for (int e = e0; e < e1; ++e) {
    for (int q = 0; q < w; ++q) mask[(size_t)e * w + q] = 0u;
    for (int i = 0; i < N; ++i) {
      int collisions = 0;
      float d0[3], d1[3];
      for (int j = 0; j < 3; ++j) {
        const float* x = xi + (((size_t)i * (W + 1) + 0) * 3 + j) * 2;
        dev_init(linf, x[0], x[1], &d0[j], &d1[j]);
      }
      for (int k = 1; k <= W; ++k) {
        float p[3];
        for (int j = 0; j < 3; ++j) {
          const float* x = xi + (((size_t)i * (W + 1) + k) * 3 + j) * 2;
          dev_step(phi + 4 * (size_t)e, L + 3 * (size_t)e, x[0], x[1], &d0[j], &d1[j]);
          p[j] = nom[((size_t)e * W + (k - 1)) * 3 + j] + d0[j];
        }
        for (int o = 0; o < n_boxes; ++o)
          if (in_box(p, boxes + 6 * o)) ++collisions;
      }
      if (collisions > 0) mask[(size_t)e * w + i / 32] |= 1u << (i % 32);
    }
  }
}

void orc_edge_masks(int n_edges, int W, int N, const float* phi, const float* L, const float* nom,
                    const float* linf, const float* xi, const float* boxes, int n_boxes, uint32_t* mask) {
  edge_masks_range(0, n_edges, W, N, phi, L, nom, linf, xi, boxes, n_boxes, mask);
}

/* All host cores: edges are independent, so threads take blocks of 64 edges from a shared     */
/* counter; every mask word is the single-thread word.                                          */
typedef struct {
  atomic_int* next;
  int n_edges, W, N, n_boxes;
  const float *phi, *L, *nom, *linf, *xi, *boxes;
  uint32_t* mask;
} masks_job;

static void* masks_worker(void* arg) {
  masks_job* j = (masks_job*)arg;
  for (;;) {
    int e0 = atomic_fetch_add(j->next, 64);
    if (e0 >= j->n_edges) break;
    int e1 = e0 + 64 < j->n_edges ? e0 + 64 : j->n_edges;
    edge_masks_range(e0, e1, j->W, j->N, j->phi, j->L, j->nom, j->linf, j->xi, j->boxes, j->n_boxes, j->mask);
  }
  return NULL;
}

void orc_edge_masks_mt(int n_edges, int W, int N, const float* phi, const float* L, const float* nom,
                       const float* linf, const float* xi, const float* boxes, int n_boxes, uint32_t* mask,
                       int n_threads) {
  if (n_threads < 2) {
    orc_edge_masks(n_edges, W, N, phi, L, nom, linf, xi, boxes, n_boxes, mask);
    return;
  }
  atomic_int next = 0;
  masks_job j = {&next, n_edges, W, N, n_boxes, phi, L, nom, linf, xi, boxes, mask};
  pthread_t* t = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)n_threads);
  int started = 0;
  for (int k = 0; k < n_threads; ++k)
    if (pthread_create(&t[started], NULL, masks_worker, &j) == 0) ++started;
  if (started == 0) masks_worker(&j);
  for (int k = 0; k < started; ++k) pthread_join(t[k], NULL);
  free(t);
}

/* ========================================================================== */
/* O4h  HSMC edge masks (Section III-B, Half-Space Monte Carlo; Eq. (eq:hs)).   */
/* Local convex region around a waypoint y (nominal position, float) with       */
/* nominal velocity v: repeatedly take the remaining box closest to y (least    */
/* squared distance from y to its closest point c, ties to the lower index),   */
/* d = c - y; record the half-space and prune every remaining box lying in     */
/* {z : d.(z - y) >= d.d} (the closest box always).  At most hmax half-spaces   */
/* per waypoint.  Each half-space is turned away from the direction of travel: */
/* a = d - ((d.v) / (v.v)) v (a = d if v = 0), b = a.a, and a particle with    */
/* position deviation dy fires it iff a.dy > b.  Our reading fixes the          */
/* arithmetic: float, every operation rounded as written (left to right), the  */
/* test dot product as fma(a2, dy2, fma(a1, dy1, a0 * dy0)).  A waypoint on or  */
/* inside a box (d = 0) ends its region.  The particle mask bit is the OR over  */
/* waypoints 1..W and half-spaces.                                               */
/* ========================================================================== */
int orc_halfspaces(const float* y, const float* v, const float* boxes, int n_boxes, int hmax, float* a_out,
                   float* b_out) {
  unsigned char* alive = (unsigned char*)malloc((size_t)(n_boxes > 0 ? n_boxes : 1));
  if (!alive) return -1;
  for (int o = 0; o < n_boxes; ++o) alive[o] = 1;
  int count = 0;
  const float vv = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
  while (count < hmax) {
    int best = -1;
    float bestd = INFINITY, d[3] = {0.f, 0.f, 0.f};
    for (int o = 0; o < n_boxes; ++o) {
      if (!alive[o]) continue;
      const float* b = boxes + 6 * o;
      float e[3];
      for (int j = 0; j < 3; ++j) e[j] = fminf(fmaxf(y[j], b[j]), b[3 + j]) - y[j];
      const float d2 = e[0] * e[0] + e[1] * e[1] + e[2] * e[2];
      if (d2 < bestd) {
        best = o; bestd = d2;
        d[0] = e[0]; d[1] = e[1]; d[2] = e[2];
      }
    }
    if (best < 0 || !(bestd > 0.f)) break;
    float a[3];
    if (vv > 0.f) {
      const float f = (d[0] * v[0] + d[1] * v[1] + d[2] * v[2]) / vv;
      for (int j = 0; j < 3; ++j) a[j] = d[j] - f * v[j];
    } else {
      for (int j = 0; j < 3; ++j) a[j] = d[j];
    }
    for (int j = 0; j < 3; ++j) a_out[3 * count + j] = a[j];
    b_out[count] = a[0] * a[0] + a[1] * a[1] + a[2] * a[2];
    ++count;
    alive[best] = 0;
    for (int o = 0; o < n_boxes; ++o) {
      if (!alive[o]) continue;
      const float* b = boxes + 6 * o;
      float m = 0.f;
      for (int j = 0; j < 3; ++j) m = m + fminf(d[j] * (b[j] - y[j]), d[j] * (b[3 + j] - y[j]));
      if (m >= bestd) alive[o] = 0;
    }
  }
  free(alive);
  return count;
}

static int hs_fires(const float* a, float b, const float* dy) {
  return fmaf(a[2], dy[2], fmaf(a[1], dy[1], a[0] * dy[0])) > b;
}

int orc_edge_masks_hs(int n_edges, int W, int N, const float* phi, const float* L, const float* nom,
                      const float* nvel, const float* linf, const float* xi, const float* boxes, int n_boxes,
                      int hmax, uint32_t* mask) {
  int w = N / 32;
  float* ha = (float*)malloc(sizeof(float) * 3 * (size_t)W * (size_t)(hmax > 0 ? hmax : 1));
  float* hb = (float*)malloc(sizeof(float) * (size_t)W * (size_t)(hmax > 0 ? hmax : 1));
  int* hc = (int*)malloc(sizeof(int) * (size_t)W);
  if (!ha || !hb || !hc) { free(ha); free(hb); free(hc); return -1; }
  for (int e = 0; e < n_edges; ++e) {
    for (int k = 1; k <= W; ++k) {
      const size_t q = (size_t)e * W + (k - 1);
      hc[k - 1] = orc_halfspaces(nom + 3 * q, nvel + 3 * q, boxes, n_boxes, hmax, ha + 3 * (size_t)(k - 1) * hmax,
                                 hb + (size_t)(k - 1) * hmax);
      if (hc[k - 1] < 0) { free(ha); free(hb); free(hc); return -1; }
    }
    for (int qw = 0; qw < w; ++qw) mask[(size_t)e * w + qw] = 0u;
    for (int i = 0; i < N; ++i) {
      int fired = 0;
      float d0[3], d1[3];
      for (int j = 0; j < 3; ++j) {
        const float* x = xi + (((size_t)i * (W + 1) + 0) * 3 + j) * 2;
        dev_init(linf, x[0], x[1], &d0[j], &d1[j]);
      }
      for (int k = 1; k <= W; ++k) {
        for (int j = 0; j < 3; ++j) {
          const float* x = xi + (((size_t)i * (W + 1) + k) * 3 + j) * 2;
          dev_step(phi + 4 * (size_t)e, L + 3 * (size_t)e, x[0], x[1], &d0[j], &d1[j]);
        }
        for (int h = 0; h < hc[k - 1]; ++h)
          if (hs_fires(ha + 3 * ((size_t)(k - 1) * hmax + h), hb[(size_t)(k - 1) * hmax + h], d0)) ++fired;
      }
      if (fired > 0) mask[(size_t)e * w + i / 32] |= 1u << (i % 32);
    }
  }
  free(ha); free(hb); free(hc);
  return 0;
}

/* ========================================================================== */
/* O5  Explore (Algorithm 4).                                                   */
/* Plans carry head, parent (path by parent links), float cost and the OR of   */
/* their edges' particle masks; the approximate CP is popcount(mask) / N.      */
/* Thresholds (Algorithm 2): alpha_max = eta alpha, alpha_min = alpha / eta,   */
/* applied as integers K_max = #{k >= 0 : k < alpha_max N} and K_min likewise: */
/* a candidate is kept iff popc < K_max, a goal plan stops the search iff      */
/* popc < K_min.  Group i = open plans with cost <= thr_i,                      */
/* thr_i = float(i * (lambda * r)) evaluated in double.                        */
/* Candidate order: group plans by ascending id, then adjacency order.  The     */
/* cost of a candidate is the float sum parent.cost + edge cost.               */
/* RemoveDominated follows Section IV: every OPEN plan p (including current    */
/* group members and the new candidates) is removed from P and P_open if some  */
/* plan d in P with the same head has d.cost < p.cost and d.popc <= p.popc.     */
/* Closed plans are never removed but still dominate.  New candidates that     */
/* survive get consecutive ids in candidate order.  Each plan records t, the   */
/* group index of the iteration that created it, and e, the group index at     */
/* which it was expanded (-1 if never).                                          */
/* ========================================================================== */
typedef struct {
  int status;
  int n_plans, n_words;
  int32_t* head;
  int32_t* parent;
  float* cost;
  uint32_t* mask;
  int32_t* popc;
  int32_t* t_created;
  int32_t* e_expanded;
  uint8_t* removed;
  int64_t n_candidates;
  int64_t n_kept;
  int32_t n_iterations;
  int32_t n_groups_expanded;
  int32_t n_goal;
  int32_t* goal_plans;
} orc_explore_result;

void orc_explore_free(orc_explore_result* R) {
  if (!R) return;
  free(R->head); free(R->parent); free(R->cost); free(R->mask); free(R->popc);
  free(R->t_created); free(R->e_expanded); free(R->removed); free(R->goal_plans); free(R);
}

typedef struct { int32_t* v; int n, cap; } ivec;
static int ivec_push(ivec* a, int32_t x) {
  if (a->n == a->cap) {
    int nc = a->cap ? 2 * a->cap : 8;
    int32_t* p = (int32_t*)realloc(a->v, sizeof(int32_t) * (size_t)nc);
    if (!p) return -1;
    a->v = p; a->cap = nc;
  }
  a->v[a->n++] = x;
  return 0;
}

static int popcount32(uint32_t x) {
  int c = 0;
  while (x) { c += (int)(x & 1u); x >>= 1; }
  return c;
}

static float group_threshold(int i, float lambda, float r) {
  return (float)((double)i * ((double)lambda * (double)r));
}

/* Candidate buffer of one expansion: records in candidate order. */
typedef struct {
  int64_t n, cap;
  int w;
  int32_t* head;
  int32_t* parent;
  float* cost;
  uint32_t* mask;
  int32_t* popc;
  uint8_t* dom;
  int64_t evaluated; /* pairs evaluated (partial plans), kept or not */
} cand_buf;

static int cand_reserve(cand_buf* c, int64_t need) {
  if (need <= c->cap) return 0;
  int64_t cap = c->cap ? c->cap : 1024;
  while (cap < need) cap *= 2;
  c->head = (int32_t*)realloc(c->head, sizeof(int32_t) * cap);
  c->parent = (int32_t*)realloc(c->parent, sizeof(int32_t) * cap);
  c->cost = (float*)realloc(c->cost, sizeof(float) * cap);
  c->mask = (uint32_t*)realloc(c->mask, sizeof(uint32_t) * cap * c->w);
  c->popc = (int32_t*)realloc(c->popc, sizeof(int32_t) * cap);
  c->dom = (uint8_t*)realloc(c->dom, cap);
  if (!c->head || !c->parent || !c->cost || !c->mask || !c->popc || !c->dom) return -1;
  c->cap = cap;
  return 0;
}

static void cand_free(cand_buf* c) {
  free(c->head); free(c->parent); free(c->cost); free(c->mask); free(c->popc); free(c->dom);
}

/* Expansion of group members group[g0 .. g1): for p in the group (in order), for x in          */
/* N(p.head) (in CSR order): q = (x, cost + Cost(head, x), mask OR edge mask); q is kept iff its */
/* CP-hat passes the alpha_max cutoff (popc < K_max).                                          */
typedef struct {
  const orc_explore_result* R;
  const int32_t* group;
  int g0, g1;
  const int32_t* row_ptr;
  const int32_t* col;
  const float* ecost;
  const uint32_t* emask;
  int K_max;
  cand_buf* out;
} expand_job;

static void* expand_members(void* arg) {
  expand_job* j = (expand_job*)arg;
  const orc_explore_result* R = j->R;
  cand_buf* c = j->out;
  int w = c->w;
  for (int gi = j->g0; gi < j->g1; ++gi) {
    int p = j->group[gi];
    int v = R->head[p];
    for (int e = j->row_ptr[v]; e < j->row_ptr[v + 1]; ++e) {
      c->evaluated++;
      uint32_t m[64];
      int pc = 0;
      for (int q = 0; q < w; ++q) {
        m[q] = R->mask[(size_t)p * w + q] | j->emask[(size_t)e * w + q];
        pc += popcount32(m[q]);
      }
      if (!(pc < j->K_max)) continue; /* CP cutoff */
      if (cand_reserve(c, c->n + 1)) return (void*)1;
      int64_t k = c->n++;
      c->head[k] = j->col[e];
      c->parent[k] = p;
      float pc_cost = R->cost[p];
      float ec = j->ecost[e];
      c->cost[k] = pc_cost + ec;
      for (int q = 0; q < w; ++q) c->mask[(size_t)k * w + q] = m[q];
      c->popc[k] = pc;
      c->dom[k] = 0;
    }
  }
  return NULL;
}

/* RemoveDominated at nodes touched[t0 .. t1).  S_x = P(x) plus the new candidates at x;        */
/* dominance is decided against the whole of S_x before anything is removed.  Removes the        */
/* dominated open plans of P(x) (from P(x), P_open and the arena's live set) and flags the        */
/* dominated candidates.  Each node's plans and candidates belong to that node alone.            */
typedef struct {
  orc_explore_result* R;
  uint8_t* open_;
  ivec* P;
  ivec* NEWAT;
  const int32_t* touched;
  int t0, t1;
  cand_buf* c;
  int64_t removed_open; /* open plans removed */
} dominate_job;

static void* dominate_nodes(void* arg) {
  dominate_job* j = (dominate_job*)arg;
  orc_explore_result* R = j->R;
  cand_buf* c = j->c;
  for (int ti = j->t0; ti < j->t1; ++ti) {
    int x = j->touched[ti];
    ivec* old = &j->P[x];
    ivec* nw = &j->NEWAT[x];
    uint8_t* old_dom = (uint8_t*)calloc((size_t)(old->n ? old->n : 1), 1);
    /* existing open plans */
    for (int a = 0; a < old->n; ++a) {
      int p = old->v[a];
      if (!j->open_[p]) continue;
      int dom = 0;
      for (int b2 = 0; b2 < old->n && !dom; ++b2) {
        int d = old->v[b2];
        if (R->cost[d] < R->cost[p] && R->popc[d] <= R->popc[p]) dom = 1;
      }
      for (int b2 = 0; b2 < nw->n && !dom; ++b2) {
        int d = nw->v[b2];
        if (c->cost[d] < R->cost[p] && c->popc[d] <= R->popc[p]) dom = 1;
      }
      old_dom[a] = (uint8_t)dom;
    }
    /* new candidates (all open) */
    for (int a = 0; a < nw->n; ++a) {
      int q = nw->v[a];
      int dom = 0;
      for (int b2 = 0; b2 < old->n && !dom; ++b2) {
        int d = old->v[b2];
        if (R->cost[d] < c->cost[q] && R->popc[d] <= c->popc[q]) dom = 1;
      }
      for (int b2 = 0; b2 < nw->n && !dom; ++b2) {
        int d = nw->v[b2];
        if (c->cost[d] < c->cost[q] && c->popc[d] <= c->popc[q]) dom = 1;
      }
      c->dom[q] = (uint8_t)dom;
    }
    /* apply removals of existing plans */
    int keep = 0;
    for (int a = 0; a < old->n; ++a) {
      int p = old->v[a];
      if (old_dom[a]) { R->removed[p] = 1; j->open_[p] = 0; j->removed_open++; }
      else old->v[keep++] = p;
    }
    old->n = keep;
    free(old_dom);
  }
  return NULL;
}

/* Runs fn over jobs[0 .. n): on the calling thread when n == 1, else one thread per job.       */
static int run_jobs(void* (*fn)(void*), void* jobs, size_t job_size, int n) {
  int rc = 0;
  if (n == 1) return fn(jobs) != NULL;
  pthread_t* t = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)n);
  int* live = (int*)calloc((size_t)n, sizeof(int));
  for (int k = 0; k < n; ++k) {
    void* jk = (char*)jobs + job_size * (size_t)k;
    if (pthread_create(&t[k], NULL, fn, jk) == 0) live[k] = 1;
    else if (fn(jk) != NULL) rc = 1;
  }
  for (int k = 0; k < n; ++k) {
    void* r = NULL;
    if (live[k]) {
      pthread_join(t[k], &r);
      if (r != NULL) rc = 1;
    }
  }
  free(t); free(live);
  return rc;
}

static orc_explore_result* explore_impl(int n, const int32_t* row_ptr, const int32_t* col, const float* ecost,
                                        const uint32_t* emask, int n_words, int start, const uint8_t* is_goal,
                                        int K_min, int K_max, float lambda, float r, int64_t max_plans,
                                        int flags, int max_iterations, int n_threads) {
  orc_explore_result* R = (orc_explore_result*)calloc(1, sizeof(orc_explore_result));
  if (!R) return NULL;
  R->n_words = n_words;
  if (n <= 0 || start < 0 || start >= n || n_words <= 0 || n_words > 64 || max_plans < 1) {
    R->status = ORC_ERR_INVALID_ARG;
    return R;
  }
  if (n_threads < 1) n_threads = 1;
  int w = n_words;
  int64_t cap = 1024;
#define GROW_PLANS(NEED)                                                                       \
  while ((NEED) > cap) {                                                                       \
    cap *= 2;                                                                                  \
    R->head = (int32_t*)realloc(R->head, sizeof(int32_t) * cap);                              \
    R->parent = (int32_t*)realloc(R->parent, sizeof(int32_t) * cap);                          \
    R->cost = (float*)realloc(R->cost, sizeof(float) * cap);                                  \
    R->mask = (uint32_t*)realloc(R->mask, sizeof(uint32_t) * cap * w);                        \
    R->popc = (int32_t*)realloc(R->popc, sizeof(int32_t) * cap);                              \
    R->t_created = (int32_t*)realloc(R->t_created, sizeof(int32_t) * cap);                    \
    R->e_expanded = (int32_t*)realloc(R->e_expanded, sizeof(int32_t) * cap);                  \
    R->removed = (uint8_t*)realloc(R->removed, cap);                                          \
    open_ = (uint8_t*)realloc(open_, cap);                                                     \
  }
  uint8_t* open_ = NULL;
  R->head = (int32_t*)malloc(sizeof(int32_t) * cap);
  R->parent = (int32_t*)malloc(sizeof(int32_t) * cap);
  R->cost = (float*)malloc(sizeof(float) * cap);
  R->mask = (uint32_t*)malloc(sizeof(uint32_t) * cap * w);
  R->popc = (int32_t*)malloc(sizeof(int32_t) * cap);
  R->t_created = (int32_t*)malloc(sizeof(int32_t) * cap);
  R->e_expanded = (int32_t*)malloc(sizeof(int32_t) * cap);
  R->removed = (uint8_t*)malloc(cap);
  open_ = (uint8_t*)malloc(cap);
  ivec* P = (ivec*)calloc((size_t)n, sizeof(ivec));      /* P(x): live plans with head x */
  ivec* NEWAT = (ivec*)calloc((size_t)n, sizeof(ivec));  /* new candidates per node, one iteration */
  ivec group = {0}, touched = {0}, next_group = {0};
  cand_buf cb = {0};                                     /* candidates of one iteration */
  cb.w = w;
  cand_buf* part = (cand_buf*)calloc((size_t)n_threads, sizeof(cand_buf)); /* per-thread parts */
  expand_job* ej = (expand_job*)calloc((size_t)n_threads, sizeof(expand_job));
  dominate_job* dj = (dominate_job*)calloc((size_t)n_threads, sizeof(dominate_job));
  for (int k = 0; k < n_threads; ++k) part[k].w = w;

  /* root plan (x_init, {}, 0, 0) */
  R->head[0] = start; R->parent[0] = -1; R->cost[0] = 0.0f;
  for (int q = 0; q < w; ++q) R->mask[q] = 0u;
  R->popc[0] = 0; R->t_created[0] = -1; R->e_expanded[0] = -1; R->removed[0] = 0; open_[0] = 1;
  R->n_plans = 1;
  int64_t n_open = 1;
  ivec_push(&P[start], 0);
  ivec_push(&group, 0);
  int i = 0;
  R->status = ORC_OK;
  for (;;) {
    if (n_open == 0) break;
    if (!(flags & ORC_NO_EARLY_STOP)) {
      int stop = 0;
      for (int gi = 0; gi < group.n; ++gi) {
        int p = group.v[gi];
        if (is_goal[R->head[p]] && R->popc[p] < K_min) { stop = 1; break; }
      }
      if (stop) break;
    }
    if (i >= max_iterations) { R->status = ORC_ERR_TIMEOUT; break; }
    /* expansion: candidates q = (x, path + head, cost + Cost(head, x), CP-hat), group members */
    /* in order, each member's out-edges in CSR order (members split into contiguous chunks   */
    /* across threads, the chunks' candidates concatenated in order)                          */
    int T = n_threads < group.n ? n_threads : (group.n > 0 ? group.n : 1);
    cb.n = 0;
    cb.evaluated = 0;
    for (int k = 0; k < T; ++k) {
      cand_buf* out = T == 1 ? &cb : &part[k];
      out->n = 0;
      out->evaluated = 0;
      expand_job J = {R, group.v, (int)((int64_t)group.n * k / T), (int)((int64_t)group.n * (k + 1) / T),
                      row_ptr, col, ecost, emask, K_max, out};
      ej[k] = J;
    }
    if (run_jobs(expand_members, ej, sizeof(expand_job), T)) { R->status = ORC_ERR_OOM; break; }
    if (T > 1) {
      for (int k = 0; k < T; ++k) {
        if (cand_reserve(&cb, cb.n + part[k].n)) { R->status = ORC_ERR_OOM; break; }
        int64_t m = part[k].n;
        memcpy(cb.head + cb.n, part[k].head, sizeof(int32_t) * m);
        memcpy(cb.parent + cb.n, part[k].parent, sizeof(int32_t) * m);
        memcpy(cb.cost + cb.n, part[k].cost, sizeof(float) * m);
        memcpy(cb.mask + cb.n * w, part[k].mask, sizeof(uint32_t) * m * w);
        memcpy(cb.popc + cb.n, part[k].popc, sizeof(int32_t) * m);
        memcpy(cb.dom + cb.n, part[k].dom, m);
        cb.n += m;
        cb.evaluated += part[k].evaluated;
      }
      if (R->status != ORC_OK) break;
    }
    R->n_candidates += cb.evaluated;
    int64_t nc = cb.n;
    for (int64_t q = 0; q < nc; ++q) {
      int x = cb.head[q];
      if (NEWAT[x].n == 0) ivec_push(&touched, x);
      ivec_push(&NEWAT[x], (int32_t)q);
    }
    R->n_kept += nc;
    /* RemoveDominated on every node that received candidates (nodes split across threads) */
    int TD = n_threads < touched.n ? n_threads : (touched.n > 0 ? touched.n : 1);
    for (int k = 0; k < TD; ++k) {
      dominate_job J = {R, open_, P, NEWAT, touched.v, (int)((int64_t)touched.n * k / TD),
                        (int)((int64_t)touched.n * (k + 1) / TD), &cb, 0};
      dj[k] = J;
    }
    run_jobs(dominate_nodes, dj, sizeof(dominate_job), TD);
    for (int k = 0; k < TD; ++k) n_open -= dj[k].removed_open;
    /* survivors get ids in candidate order */
    for (int64_t q = 0; q < nc; ++q) {
      if (cb.dom[q]) continue;
      if ((int64_t)R->n_plans + 1 > max_plans) { R->status = ORC_ERR_CAPACITY; break; }
      int64_t id = R->n_plans;
      GROW_PLANS(id + 1);
      R->head[id] = cb.head[q]; R->parent[id] = cb.parent[q]; R->cost[id] = cb.cost[q];
      for (int k = 0; k < w; ++k) R->mask[(size_t)id * w + k] = cb.mask[(size_t)q * w + k];
      R->popc[id] = cb.popc[q]; R->t_created[id] = i; R->e_expanded[id] = -1; R->removed[id] = 0;
      open_[id] = 1; ++n_open;
      ivec_push(&P[cb.head[q]], (int32_t)id);
      R->n_plans++;
    }
    for (int ti = 0; ti < touched.n; ++ti) NEWAT[touched.v[ti]].n = 0;
    touched.n = 0;
    if (R->status != ORC_OK) break;
    /* P_open <- P_open \ G */
    for (int gi = 0; gi < group.n; ++gi) {
      int p = group.v[gi];
      R->e_expanded[p] = i;
      if (open_[p]) { open_[p] = 0; --n_open; }
    }
    if (group.n) R->n_groups_expanded++;
    /* i <- i + 1; G <- {p in P_open : p.cost <= i lambda r} */
    ++i;
    float thr = group_threshold(i, lambda, r);
    next_group.n = 0;
    for (int p = 0; p < R->n_plans; ++p)
      if (open_[p] && R->cost[p] <= thr) ivec_push(&next_group, p);
    ivec tmp = group; group = next_group; next_group = tmp;
  }
  R->n_iterations = i;
  /* P_goal: plans in P(v) for v in X_goal */
  int64_t ng = 0;
  for (int p = 0; p < R->n_plans; ++p)
    if (is_goal[R->head[p]] && !R->removed[p]) ++ng;
  R->goal_plans = (int32_t*)malloc(sizeof(int32_t) * (size_t)(ng ? ng : 1));
  R->n_goal = 0;
  for (int p = 0; p < R->n_plans; ++p)
    if (is_goal[R->head[p]] && !R->removed[p]) R->goal_plans[R->n_goal++] = p;
  for (int v = 0; v < n; ++v) { free(P[v].v); free(NEWAT[v].v); }
  free(P); free(NEWAT); free(group.v); free(next_group.v); free(touched.v); free(open_);
  cand_free(&cb);
  for (int k = 0; k < n_threads; ++k) cand_free(&part[k]);
  free(part); free(ej); free(dj);
#undef GROW_PLANS
  return R;
}

orc_explore_result* orc_explore(int n, const int32_t* row_ptr, const int32_t* col, const float* ecost,
                                const uint32_t* emask, int n_words, int start, const uint8_t* is_goal,
                                int K_min, int K_max, float lambda, float r, int64_t max_plans,
                                int flags, int max_iterations) {
  return explore_impl(n, row_ptr, col, ecost, emask, n_words, start, is_goal, K_min, K_max, lambda, r, max_plans,
                      flags, max_iterations, 1);
}

/* Explore on all host cores (timing): the same run with the expansion split over group members */
/* and RemoveDominated over target nodes; every result equals orc_explore's.                    */
orc_explore_result* orc_explore_mt(int n, const int32_t* row_ptr, const int32_t* col, const float* ecost,
                                   const uint32_t* emask, int n_words, int start, const uint8_t* is_goal,
                                   int K_min, int K_max, float lambda, float r, int64_t max_plans,
                                   int flags, int max_iterations, int n_threads) {
  return explore_impl(n, row_ptr, col, ecost, emask, n_words, start, is_goal, K_min, K_max, lambda, r, max_plans,
                      flags, max_iterations, n_threads);
}

void orc_explore_summary(const orc_explore_result* R, int64_t* out /* status, n_plans, n_cand, n_kept, n_iter, n_groups, n_goal */) {
  out[0] = R->status; out[1] = R->n_plans; out[2] = R->n_candidates; out[3] = R->n_kept;
  out[4] = R->n_iterations; out[5] = R->n_groups_expanded; out[6] = R->n_goal;
}

void orc_explore_export(const orc_explore_result* R, int32_t* head, int32_t* parent, float* cost,
                        uint32_t* mask, int32_t* popc, int32_t* t_created, int32_t* e_expanded,
                        uint8_t* removed, int32_t* goal_plans) {
  size_t P = (size_t)R->n_plans;
  if (head) memcpy(head, R->head, sizeof(int32_t) * P);
  if (parent) memcpy(parent, R->parent, sizeof(int32_t) * P);
  if (cost) memcpy(cost, R->cost, sizeof(float) * P);
  if (mask) memcpy(mask, R->mask, sizeof(uint32_t) * P * (size_t)R->n_words);
  if (popc) memcpy(popc, R->popc, sizeof(int32_t) * P);
  if (t_created) memcpy(t_created, R->t_created, sizeof(int32_t) * P);
  if (e_expanded) memcpy(e_expanded, R->e_expanded, sizeof(int32_t) * P);
  if (removed) memcpy(removed, R->removed, P);
  if (goal_plans) memcpy(goal_plans, R->goal_plans, sizeof(int32_t) * (size_t)R->n_goal);
}

/* ========================================================================== */
/* Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of            */
/* (c0, c1, c2, c3) -> (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1,    */
/* lo(M0 c0)), the key advanced by the Weyl constants between rounds.           */
/* ========================================================================== */
static void mul64(uint64_t a, uint64_t b, uint64_t* hi, uint64_t* lo) {
  uint64_t a0 = a & 0xffffffffu, a1 = a >> 32, b0 = b & 0xffffffffu, b1 = b >> 32;
  uint64_t p00 = a0 * b0, p01 = a0 * b1, p10 = a1 * b0, p11 = a1 * b1;
  uint64_t mid = (p00 >> 32) + (p01 & 0xffffffffu) + (p10 & 0xffffffffu);
  *lo = (p00 & 0xffffffffu) | (mid << 32);
  *hi = p11 + (p01 >> 32) + (p10 >> 32) + (mid >> 32);
}

void orc_philox4x64(const uint64_t* ctr_in, const uint64_t* key_in, uint64_t* out) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
  uint64_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
  uint64_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) { k0 += W0; k1 += W1; }
    uint64_t hi0, lo0, hi1, lo1;
    mul64(M0, c[0], &hi0, &lo0);
    mul64(M1, c[2], &hi1, &lo1);
    uint64_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
  }
  for (int q = 0; q < 4; ++q) out[q] = c[q];
}

/* Philox4x32-10 (same paper): the 32-bit form, multipliers 0xD2511F53 and     */
/* 0xCD9E8D57, Weyl constants 0x9E3779B9 and 0xBB67AE85, the same round.         */
void orc_philox4x32(const uint32_t* ctr_in, const uint32_t* key_in, uint32_t* out) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) { k0 += W0; k1 += W1; }
    const uint64_t p0 = (uint64_t)M0 * c[0], p1 = (uint64_t)M1 * c[2];
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0, hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
  }
  for (int q = 0; q < 4; ++q) out[q] = c[q];
}

/* Standard normal pair from two nbits-bit integers (Box and Muller, 1958):    */
/* u = (bits + 1/2) 2^-nbits in (0, 1), z0 = sqrt(-2 ln u1) cos(2 pi u2),       */
/* z1 = sqrt(-2 ln u1) sin(2 pi u2), evaluated in double and rounded to float.  */
static void box_muller(uint64_t b1, uint64_t b2, int nbits, float* z0, float* z1) {
  const double scale = ldexp(1.0, -nbits);
  double u1 = ((double)b1 + 0.5) * scale;
  double u2 = ((double)b2 + 0.5) * scale;
  double rad = sqrt(-2.0 * log(u1));
  double ang = 6.283185307179586476925286766559 * u2;
  *z0 = (float)(rad * cos(ang));
  *z1 = (float)(rad * sin(ang));
}

/* Normals (xi0, xi1) of rollout m, step s, for the three axes: one            */
/* Philox4x32-10 call, counter (m, s lo, 0, s hi), key (seed lo, seed hi),      */
/* words w0..w3 cut into six 21-bit fields: b_j = top 21 bits of w_j (j < 4),   */
/* b4 = low 11 bits of w0 then bits 10..1 of w1, b5 the same from w2 and w3;    */
/* axis j takes u1 from b(2j) and u2 from b(2j+1), u = (b + 1/2) 2^-21.          */
void orc_mc_normals(uint64_t seed, uint64_t m, uint64_t s, float* xi /* 3 x 2 */) {
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  const uint32_t c[4] = {(uint32_t)m, (uint32_t)s, 0u, (uint32_t)(s >> 32)};
  uint32_t w[4];
  orc_philox4x32(c, key, w);
  const uint32_t b[6] = {w[0] >> 11, w[1] >> 11, w[2] >> 11, w[3] >> 11,
                         ((w[0] & 0x7FFu) << 10) | ((w[1] & 0x7FFu) >> 1),
                         ((w[2] & 0x7FFu) << 10) | ((w[3] & 0x7FFu) >> 1)};
  for (int j = 0; j < 3; ++j) box_muller(b[2 * j], b[2 * j + 1], 21, &xi[2 * j], &xi[2 * j + 1]);
}

/* ========================================================================== */
/* O6  MC(p): Monte Carlo collision probability of a plan (Section III-A; the  */
/* paper cites Janson et al. for the estimator).  Our reading: plain MC with   */
/* n_mc rollouts of the closed loop tracking the plan's nominal connections.   */
/* The deviation starts at Linf xi (stationary) and is carried across edges;   */
/* each waypoint interval of an edge is split into `substeps` steps of          */
/* hs = h / substeps (float), with Phi(hs), L(hs) rounded to float and the same */
/* recurrence as the particles.  The nominal position at the end of sub-step s  */
/* of interval k is the connection at t = ((k-1) substeps + s) hs (double      */
/* evaluation, float result).  A rollout collides iff any sub-step position     */
/* lies in a closed box.  Normals come from orc_mc_normals with the global     */
/* step counter (0 for the initial deviation).                                   */
/* path: node ids x_init .. head (len >= 1); edge_tau: float duration of each   */
/* connection (len - 1 values).                                                  */
/* ========================================================================== */
int64_t orc_mc_certify(const float* states, const int32_t* path, int len, const float* edge_tau, int W,
                       float sigma_f, const float* boxes, int n_boxes, int64_t n_mc, int substeps,
                       uint64_t seed) {
  const double sigma = (double)sigma_f;
  if (len < 1 || W < 1 || substeps < 1 || n_mc < 0) return -1;
  int n_edges = len - 1;
  float lin[3], phi_d[4], l_d[3];
  model_f32(sigma, 1.0f, phi_d, l_d, lin);
  int64_t collided = 0;
  for (int64_t m = 0; m < n_mc; ++m) {
    float d0[3], d1[3], xi[6];
    uint64_t step = 0;
    orc_mc_normals(seed, (uint64_t)m, step, xi);
    for (int j = 0; j < 3; ++j) dev_init(lin, xi[2 * j], xi[2 * j + 1], &d0[j], &d1[j]);
    int hit = 0;
    for (int ei = 0; ei < n_edges && !hit; ++ei) {
      double xv[6], xu[6];
      for (int q = 0; q < 6; ++q) { xv[q] = states[6 * path[ei] + q]; xu[q] = states[6 * path[ei + 1] + q]; }
      float t32 = edge_tau[ei];
      float h = t32 / (float)W;
      float hs = h / (float)substeps;
      float phi[4], L[3], lin_unused[3];
      model_f32(sigma, hs, phi, L, lin_unused);
      double td = (double)t32;
      for (int k = 1; k <= W && !hit; ++k) {
        for (int s = 1; s <= substeps && !hit; ++s) {
          ++step;
          orc_mc_normals(seed, (uint64_t)m, step, xi);
          double t = (double)((k - 1) * substeps + s) * (double)hs;
          float p[3];
          for (int j = 0; j < 3; ++j) {
            dev_step(phi, L, xi[2 * j], xi[2 * j + 1], &d0[j], &d1[j]);
            p[j] = (float)nominal_pos(xv, xu, td, j, t) + d0[j];
          }
          hit = in_any_box(p, boxes, n_boxes);
        }
      }
    }
    collided += hit;
  }
  return collided;
}

/* All ordered pair costs float(Cost(v,u)) (row v, column u), +inf on the       */
/* diagonal and for identical states; used to calibrate the connection radius. */
void orc_pair_costs(const float* states, int n, float* out) {
  for (int v = 0; v < n; ++v) {
    double xv[6];
    for (int q = 0; q < 6; ++q) xv[q] = (double)states[6 * v + q];
    for (int u = 0; u < n; ++u) {
      double xu[6], t, J;
      for (int q = 0; q < 6; ++q) xu[q] = (double)states[6 * u + q];
      out[(size_t)v * n + u] = (u != v && orc_steer(xv, xu, &t, &J) == 0) ? (float)J : INFINITY;
    }
  }
}

/* ========================================================================== */
/* O7  Draws of the learned sampling proposal (not part of the paper, which   */
/* has no learning).  Row r of draw set (t, stream) takes one Philox4x64-10    */
/* call with counter (t, r, stream, 0) and key (seed, 1); its four words give   */
/* eight standard normals through box_muller (word j: bits 63..40 -> u1, bits   */
/* 39..16 -> u2; z[2j], z[2j+1]).  With n_env > 0 the call with counter         */
/* (t, r, stream + 1, 0) picks the row's environment from its word 0:           */
/* env = floor((word0 >> 32) * n_env / 2^32).                                   */
/* ========================================================================== */
void orc_mlp_draws(uint64_t seed, uint64_t t, uint64_t stream, int64_t rows, int32_t n_env, float* z,
                   int32_t* env) {
  const uint64_t key[2] = {seed, 1};
  for (int64_t r = 0; r < rows; ++r) {
    uint64_t c[4] = {t, (uint64_t)r, stream, 0}, o[4];
    orc_philox4x64(c, key, o);
    for (int j = 0; j < 4; ++j)
      box_muller(o[j] >> 40, (o[j] >> 16) & 0xFFFFFFull, 24, &z[8 * r + 2 * j], &z[8 * r + 2 * j + 1]);
    if (n_env > 0 && env) {
      uint64_t c2[4] = {t, (uint64_t)r, stream + 1, 0};
      orc_philox4x64(c2, key, o);
      env[r] = (int32_t)(((o[0] >> 32) * (uint64_t)n_env) >> 32);
    }
  }
}
