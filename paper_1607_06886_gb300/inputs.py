"""Seeded synthetic inputs for PUMP workloads.

This module is the only code shared by the CUDA path and the CPU oracle.  It
holds no arithmetic of the planning method itself: it draws samples, obstacle
boxes, the particle normals and random explore graphs from numpy's PCG64, and
it states the problem (start, goal region, tuning parameters).  Everything the
method computes from these inputs (steering costs, neighbour sets, particle
positions, masks, dominance, plan selection) lives on either side separately.

Workload shapes follow the paper's experiments (Section V-A and Table I): a
6D double integrator in a unit-scale 3D workspace, unions of axis-aligned boxes
as obstacles (Section V-C), thousands of samples, N = 128 particles.  The
paper's own environments (Fig. 1) are not published, so the scenes below are
synthetic stand-ins with the same shape: a few random boxes ("3 obstacles")
and an indoor-like scene of walls with doors, a floor slab and clutter.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

START_STATE = (0.1, 0.1, 0.1, 0.0, 0.0, 0.0)
GOAL_STATE = (0.9, 0.9, 0.9, 0.0, 0.0, 0.0)
GOAL_RADIUS = 0.05          # goal region: position within this distance of the goal
VEL_MAX = 0.1               # sampled velocities U[-VEL_MAX, VEL_MAX]^3
START_GOAL_CLEARANCE = 0.05  # obstacles keep this margin around start and goal


@dataclasses.dataclass
class Workload:
    """One planning query: states, obstacles, particle normals and parameters."""
    name: str
    seed: int
    states: np.ndarray        # (n, 6) float32: rows 0 = start, 1 = goal, rest = samples
    boxes: np.ndarray         # (O, 6) float32: lo_x, lo_y, lo_z, hi_x, hi_y, hi_z (closed)
    goal_idx: np.ndarray      # (G,) int32 members of X_goal (node 1 plus samples near it)
    xi: np.ndarray            # (N, W+1, 3, 2) float32 standard normals for the particles
    radius: float             # r_n: edge v->u iff Cost(v,u) < r_n
    n_particles: int          # N
    n_waypoints: int          # W
    sigma: float              # process-noise standard deviation
    alpha: float              # CP target
    eta: float                # CP approximation factor (Algorithm 2)
    lam: float                # group cost factor lambda (Algorithm 2)
    n_mc: int = 10000         # Monte Carlo rollouts for certification
    mc_substeps: int = 4      # rollout sub-steps per waypoint interval
    mc_seed: int = 0

    @property
    def n(self) -> int:
        return int(self.states.shape[0])

    @property
    def start_idx(self) -> int:
        return 0


# ---------------------------------------------------------------------------
# Radius table.  r_n is a tuning parameter of the method (Section IV); these
# values give an obstacle-free mean out-degree of about 40 ln(n) / ln(4000)
# for the uniform sample distribution below (33 at n = 1002, 40 at n = 4002).
# They were calibrated once with the CPU oracle's steering cost
# (oracle/calibrate_radius.py) and are plain inputs from here on.
RADIUS_TABLE = {1002: 1.5507, 4002: 1.2519}


def radius_for(n_total: int) -> float:
    """Connection radius for a sample count: table value, else a power-law fit.

    The fit interpolates log r against log n through the table points; it is
    only used for sample counts outside the table (batched/served mixes)."""
    if n_total in RADIUS_TABLE:
        return RADIUS_TABLE[n_total]
    (n1, r1), (n2, r2) = sorted(RADIUS_TABLE.items())
    slope = math.log(r2 / r1) / math.log(n2 / n1)
    return float(r1 * (n_total / n1) ** slope)


# ---------------------------------------------------------------------------
def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([int(seed), int(stream)]))


def sample_states(n_samples: int, seed: int) -> np.ndarray:
    """Start, goal and n_samples uniform states: position U[0,1]^3, velocity U[-0.1,0.1]^3.

    The velocity range sets how many connections a plan needs: with it the searches
    at 1k-4k samples take 6-10 connections and evaluate 3e4-1.4e5 partial plans, the
    scale Table I reports for 4k samples."""
    g = _rng(seed, 1)
    pos = g.uniform(0.0, 1.0, size=(n_samples, 3))
    vel = g.uniform(-VEL_MAX, VEL_MAX, size=(n_samples, 3))
    st = np.empty((n_samples + 2, 6), dtype=np.float32)
    st[0] = START_STATE
    st[1] = GOAL_STATE
    st[2:, :3] = pos
    st[2:, 3:] = vel
    return st


def goal_members(states: np.ndarray) -> np.ndarray:
    """X_goal: node 1 and every sample whose position lies within GOAL_RADIUS of it."""
    p = states[:, :3].astype(np.float64)
    d = np.sqrt(((p - np.asarray(GOAL_STATE[:3])) ** 2).sum(axis=1))
    idx = [1] + [i for i in range(2, states.shape[0]) if d[i] <= GOAL_RADIUS]
    return np.asarray(idx, dtype=np.int32)


def _overlaps(lo, hi, c, m):
    return bool(np.all(lo <= np.asarray(c) + m) and np.all(hi >= np.asarray(c) - m))


def _clear_of_start_goal(lo, hi) -> bool:
    return not (_overlaps(lo, hi, START_STATE[:3], START_GOAL_CLEARANCE)
                or _overlaps(lo, hi, GOAL_STATE[:3], START_GOAL_CLEARANCE))


def random_boxes(count: int, seed: int, ext_lo: float, ext_hi: float,
                 centre_lo: float = 0.2, centre_hi: float = 0.8, stream: int = 2) -> List[np.ndarray]:
    """Random boxes: per-axis extents U[ext_lo, ext_hi], centres U[centre_lo, centre_hi]^3,
    clipped to the unit cube, redrawn while they touch the start or goal clearance."""
    g = _rng(seed, stream)
    out = []
    while len(out) < count:
        ext = g.uniform(ext_lo, ext_hi, size=3)
        c = g.uniform(centre_lo, centre_hi, size=3)
        lo = np.clip(c - ext / 2, 0.0, 1.0)
        hi = np.clip(c + ext / 2, 0.0, 1.0)
        if _clear_of_start_goal(lo, hi):
            out.append(np.concatenate([lo, hi]))
    return out


def indoor_boxes(seed: int, n_clutter: int = 15) -> List[np.ndarray]:
    """Indoor-like scene: two walls across x with a full-height door each (two boxes
    per wall), a floor slab, and n_clutter boxes with extents U[0.05, 0.2]."""
    g = _rng(seed, 3)
    out = []
    for x_lo, x_hi in ((0.3, 0.4), (0.6, 0.7)):
        x0 = g.uniform(x_lo, x_hi)
        t = g.uniform(0.02, 0.05)
        gw = g.uniform(0.15, 0.25)
        g0 = g.uniform(0.05, 0.95 - gw)
        out.append(np.array([x0, 0.0, 0.0, x0 + t, g0, 1.0]))
        out.append(np.array([x0, g0 + gw, 0.0, x0 + t, 1.0, 1.0]))
    out.append(np.array([0.0, 0.0, 0.0, 1.0, 1.0, 0.03]))
    out += random_boxes(n_clutter, seed, 0.05, 0.2, 0.0, 1.0, stream=4)
    return out


def particle_normals(n_particles: int, n_waypoints: int, seed: int) -> np.ndarray:
    """Standard normals xi[i][k][axis][component] shared by every edge (common random
    numbers): k = 0 seeds the initial deviation, k = 1..W drive the W steps."""
    g = _rng(seed, 5)
    return g.standard_normal((n_particles, n_waypoints + 1, 3, 2)).astype(np.float32)


def make_workload(name: str, seed: int = 0, n_samples: Optional[int] = None) -> Workload:
    """Named workloads.

    three_box_1k  : 3 random boxes (extents U[0.1, 0.3]), 1000 samples, N = 32, W = 8,
                    sigma = 0.01, CP target 5 %, eta = 2, lambda = 0.5.
    indoor_4k     : indoor-like scene (20 boxes), 4000 samples, N = 128, W = 10,
                    sigma = 0.01, CP target 1 %, eta = 2, lambda = 0.5.
    Either accepts a smaller n_samples for tests (radius from radius_for)."""
    if name == "three_box_1k":
        ns = 1000 if n_samples is None else n_samples
        boxes = random_boxes(3, seed, 0.1, 0.3)
        N, W, alpha = 32, 8, 0.05
    elif name == "indoor_4k":
        ns = 4000 if n_samples is None else n_samples
        boxes = indoor_boxes(seed)
        N, W, alpha = 128, 10, 0.01
    else:
        raise ValueError(f"unknown workload {name!r}")
    states = sample_states(ns, seed)
    return Workload(
        name=name, seed=seed, states=states,
        boxes=np.asarray(boxes, dtype=np.float32).reshape(-1, 6),
        goal_idx=goal_members(states),
        xi=particle_normals(N, W, seed),
        radius=radius_for(ns + 2), n_particles=N, n_waypoints=W,
        sigma=0.01, alpha=alpha, eta=2.0, lam=0.5, mc_seed=seed)


def batch_workloads(n_queries: int, seed: int = 0, n_range=(1000, 8000), o_range=(5, 50),
                    particles=(64, 128, 256)) -> List[Workload]:
    """Independent queries of uneven size for the batched form: query j (seed + j) draws its
    sample count U{n_range}, its box count U{o_range} (indoor walls and floor, 5 boxes, plus
    clutter) and N from `particles`; W = 10, sigma = 0.01, CP target 1 %, eta = 2, lambda = 0.5."""
    out = []
    for j in range(n_queries):
        qs = seed + j
        g = _rng(qs, 7)
        ns = int(g.integers(n_range[0], n_range[1] + 1))
        n_obs = int(g.integers(o_range[0], o_range[1] + 1))
        N = int(particles[int(g.integers(0, len(particles)))])
        boxes = indoor_boxes(qs, n_clutter=max(n_obs - 5, 0))
        states = sample_states(ns, qs)
        out.append(Workload(
            name="batch", seed=qs, states=states,
            boxes=np.asarray(boxes, dtype=np.float32).reshape(-1, 6),
            goal_idx=goal_members(states),
            xi=particle_normals(N, 10, qs),
            radius=radius_for(ns + 2), n_particles=N, n_waypoints=10,
            sigma=0.01, alpha=0.01, eta=2.0, lam=0.5, mc_seed=qs))
    return out


# ---------------------------------------------------------------------------
# Random explore graphs: CSR adjacency, edge costs and edge masks drawn directly,
# with the degree, cost and mask-density structure of the dynamics-built graphs.
@dataclasses.dataclass
class ExploreGraph:
    n: int
    row_ptr: np.ndarray   # (n+1,) int32
    col: np.ndarray       # (E,) int32, ascending within each row, no self loops
    ecost: np.ndarray     # (E,) float32, in [cost_lo, radius)
    emask: np.ndarray     # (E, w) uint32
    radius: float
    n_words: int


def random_explore_graph(n: int, mean_degree: float, n_particles: int, seed: int,
                         radius: float = 2.4, bit_prob: float = 0.004,
                         hot_edge_frac: float = 0.05, hot_bit_prob: float = 0.2) -> ExploreGraph:
    """Random directed graph for Explore tests.  Out-degrees ~ Poisson(mean_degree)
    capped at n-1; targets uniform without replacement; costs U[0.2 r, r); mask bits
    are rare except on a small fraction of 'hot' edges that pass near obstacles."""
    g = _rng(seed, 7)
    w = n_particles // 32
    deg = np.minimum(g.poisson(mean_degree, size=n), n - 1) if n > 1 else np.zeros(n, np.int64)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    row_ptr[1:] = np.cumsum(deg)
    E = int(row_ptr[-1])
    col = np.empty(E, dtype=np.int32)
    for v in range(n):
        if deg[v]:
            others = np.delete(np.arange(n), v)
            col[row_ptr[v]:row_ptr[v + 1]] = np.sort(g.choice(others, size=deg[v], replace=False))
    ecost = g.uniform(0.2 * radius, radius, size=E).astype(np.float32)
    ecost = np.minimum(ecost, np.nextafter(np.float32(radius), np.float32(0)))
    hot = g.random(E) < hot_edge_frac
    p = np.where(hot, hot_bit_prob, bit_prob)[:, None]
    bits = g.random((E, n_particles)) < p
    emask = np.zeros((E, w), dtype=np.uint32)
    for j in range(w):
        blk = bits[:, 32 * j:32 * (j + 1)].astype(np.uint64)
        emask[:, j] = (blk << np.arange(32, dtype=np.uint64)).sum(axis=1).astype(np.uint32)
    return ExploreGraph(n=n, row_ptr=row_ptr.astype(np.int32), col=col, ecost=ecost,
                        emask=emask, radius=float(radius), n_words=w)


# ---------------------------------------------------------------------------
# Environments of the learned sampling proposal (an extension; the paper draws samples
# uniformly).  Indoor-like scenes whose box count is drawn per seed so that every scene fits the
# proposal's 32 box slots.
PROPOSAL_BOX_RANGE = (10, 32)


def proposal_workload(seed: int, n_samples: int = 4000) -> Workload:
    """Environment `seed` of the learned-proposal workloads: indoor walls and floor (5 boxes) plus
    U{5..27} clutter boxes (U{10..32} in all), n_samples uniform samples, N = 128, W = 10,
    sigma = 0.01, CP target 1 %, eta = 2, lambda = 0.5."""
    g = _rng(seed, 8)
    n_obs = int(g.integers(PROPOSAL_BOX_RANGE[0], PROPOSAL_BOX_RANGE[1] + 1))
    boxes = indoor_boxes(seed, n_clutter=n_obs - 5)
    states = sample_states(n_samples, seed)
    return Workload(
        name="proposal", seed=seed, states=states,
        boxes=np.asarray(boxes, dtype=np.float32).reshape(-1, 6),
        goal_idx=goal_members(states),
        xi=particle_normals(128, 10, seed),
        radius=radius_for(n_samples + 2), n_particles=128, n_waypoints=10,
        sigma=0.01, alpha=0.01, eta=2.0, lam=0.5, mc_seed=seed)


def with_samples(wl: Workload, samples: np.ndarray) -> Workload:
    """The same query with its samples replaced (start and goal kept): goal region and radius
    follow the new sample set."""
    states = np.concatenate([wl.states[:2], np.asarray(samples, np.float32).reshape(-1, 6)]).astype(np.float32)
    return dataclasses.replace(wl, states=states, goal_idx=goal_members(states), radius=radius_for(states.shape[0]))
