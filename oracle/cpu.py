"""ctypes front end of the CPU oracle (pump_oracle.c).

TEST INFRASTRUCTURE: only the tests, the smoke check and the benchmark's CPU
baseline use this module.  It builds pump_oracle.c with gcc (no fused
multiply-add contraction) and exposes its functions on numpy arrays.  The
Python here marshals arguments; three small pieces of the method are restated
in it directly: the integer CP thresholds of Algorithm 2, plan backtracking by
parent links, and the ordering and bisection of PlanSelection (Algorithm 5).
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading
from typing import Dict, Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "pump_oracle.c")
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "liboracle.so")

OK, ERR_INVALID_ARG, ERR_OOM, ERR_CAPACITY, ERR_TIMEOUT, ERR_INFEASIBLE = 0, 1, 2, 4, 5, 6
NO_EARLY_STOP = 1

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so (plain C11, -O2, no FP contraction)."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    if not force and os.path.exists(LIB_PATH) and os.path.getmtime(LIB_PATH) >= os.path.getmtime(SRC):
        return LIB_PATH
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
           "-Wall", "-pthread", "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = C.CDLL(path)
            P = C.c_void_p
            L.orc_steer.argtypes = [P, P, P, P]
            L.orc_steer.restype = C.c_int
            L.orc_model.argtypes = [C.c_double, C.c_double, P, P, P, P, P]
            L.orc_model.restype = None
            L.orc_graph_build.argtypes = [P, C.c_int, P, C.c_int, C.c_float, C.c_int, C.c_float, C.c_int]
            L.orc_graph_build.restype = P
            L.orc_graph_counts.argtypes = [P, P]
            L.orc_graph_export.argtypes = [P] * 11
            L.orc_graph_free.argtypes = [P]
            L.orc_edge_masks.argtypes = [C.c_int, C.c_int, C.c_int, P, P, P, P, P, P, C.c_int, P]
            L.orc_edge_masks_mt.argtypes = [C.c_int, C.c_int, C.c_int, P, P, P, P, P, P, C.c_int, P, C.c_int]
            L.orc_graph_nvel.argtypes = [P, P]
            L.orc_halfspaces.argtypes = [P, P, P, C.c_int, C.c_int, P, P]
            L.orc_halfspaces.restype = C.c_int
            L.orc_edge_masks_hs.argtypes = [C.c_int, C.c_int, C.c_int, P, P, P, P, P, P, P, C.c_int, C.c_int, P]
            L.orc_edge_masks_hs.restype = C.c_int
            L.orc_explore.argtypes = [C.c_int, P, P, P, P, C.c_int, C.c_int, P, C.c_int, C.c_int,
                                      C.c_float, C.c_float, C.c_int64, C.c_int, C.c_int]
            L.orc_explore.restype = P
            L.orc_explore_mt.argtypes = L.orc_explore.argtypes + [C.c_int]
            L.orc_explore_mt.restype = P
            L.orc_explore_summary.argtypes = [P, P]
            L.orc_explore_export.argtypes = [P] * 10
            L.orc_explore_free.argtypes = [P]
            L.orc_pair_costs.argtypes = [P, C.c_int, P]
            L.orc_philox4x64.argtypes = [P, P, P]
            L.orc_philox4x32.argtypes = [P, P, P]
            L.orc_mc_normals.argtypes = [C.c_uint64, C.c_uint64, C.c_uint64, P]
            L.orc_mlp_draws.argtypes = [C.c_uint64, C.c_uint64, C.c_uint64, C.c_int64, C.c_int32, P, P]
            L.orc_mc_certify.argtypes = [P, P, C.c_int, P, C.c_int, C.c_float, P, C.c_int, C.c_int64,
                                         C.c_int, C.c_uint64]
            L.orc_mc_certify.restype = C.c_int64
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# ---------------------------------------------------------------------------
def steer(x0, x1):
    """Cost(u, v) of the optimal connection and its duration, in double; None for identical states."""
    a = _c(x0, np.float64)
    b = _c(x1, np.float64)
    t = np.zeros(1, np.float64)
    j = np.zeros(1, np.float64)
    rc = lib().orc_steer(_p(a), _p(b), _p(t), _p(j))
    return None if rc != 0 else (float(t[0]), float(j[0]))


def model(sigma: float, h: float) -> Dict[str, np.ndarray]:
    """Double-precision tracking model for a step h: Phi, Q(h), L(h), stationary S, Linf."""
    Phi = np.zeros(4); Q = np.zeros(3); L = np.zeros(3); S = np.zeros(3); Linf = np.zeros(3)
    lib().orc_model(float(sigma), float(h), _p(Phi), _p(Q), _p(L), _p(S), _p(Linf))
    return {"Phi": Phi.reshape(2, 2), "Q": np.array([[Q[0], Q[1]], [Q[1], Q[2]]]),
            "L": np.array([[L[0], 0.0], [L[1], L[2]]]), "S": np.array([[S[0], S[1]], [S[1], S[2]]]),
            "Linf": np.array([[Linf[0], 0.0], [Linf[1], Linf[2]]])}


def graph_build(states, boxes, radius: float, W: int, sigma: float, exhaustive: bool = False) -> Dict:
    """BuildGraph (Algorithm 3) with the edge values the search uses."""
    st = _c(states, np.float32)
    bx = _c(boxes, np.float32).reshape(-1, 6)
    n = st.shape[0]
    g = lib().orc_graph_build(_p(st), n, _p(bx), bx.shape[0], C.c_float(radius), int(W), C.c_float(sigma),
                              int(bool(exhaustive)))
    if not g:
        raise RuntimeError("oracle graph build failed")
    try:
        cnt = np.zeros(5, np.int64)
        lib().orc_graph_counts(g, _p(cnt))
        E = int(cnt[1])
        out = {"valid": np.zeros(n, np.uint8), "row_ptr": np.zeros(n + 1, np.int32),
               "col": np.zeros(E, np.int32), "ecost": np.zeros(E, np.float32),
               "tau": np.zeros(E, np.float32), "h": np.zeros(E, np.float32),
               "phi": np.zeros((E, 4), np.float32), "L": np.zeros((E, 3), np.float32),
               "nom": np.zeros((E, W, 3), np.float32), "linf": np.zeros(3, np.float32)}
        lib().orc_graph_export(g, *[_p(out[k]) for k in ("valid", "row_ptr", "col", "ecost", "tau", "h",
                                                          "phi", "L", "nom", "linf")])
        out["nvel"] = np.zeros((E, W, 3), np.float32)
        lib().orc_graph_nvel(g, _p(out["nvel"]))
        out.update(n=n, n_edges=E, W=W, pairs_costed=int(cnt[2]), n_near=int(cnt[3]),
                   n_collide_removed=int(cnt[4]))
        return out
    finally:
        lib().orc_graph_free(g)


def pair_costs(states) -> np.ndarray:
    """(n, n) float32 matrix of float(Cost(v, u)), +inf on the diagonal."""
    st = _c(states, np.float32)
    n = st.shape[0]
    out = np.empty((n, n), np.float32)
    lib().orc_pair_costs(_p(st), n, _p(out))
    return out


def edge_masks(graph: Dict, xi, boxes, n_particles: int, n_threads: int = 1) -> np.ndarray:
    """Per-edge particle collision masks, (E, N/32) uint32.  n_threads > 1 splits the edges over
    host threads (timing only; the masks are the single-thread masks)."""
    E, W = graph["n_edges"], graph["W"]
    w = n_particles // 32
    out = np.zeros((E, w), np.uint32)
    x = _c(xi, np.float32)
    bx = _c(boxes, np.float32).reshape(-1, 6)
    args = (E, W, n_particles, _p(graph["phi"]), _p(graph["L"]), _p(graph["nom"]), _p(graph["linf"]), _p(x), _p(bx),
            bx.shape[0], _p(out))
    if n_threads > 1:
        lib().orc_edge_masks_mt(*args, int(n_threads))
    else:
        lib().orc_edge_masks(*args)
    return out


def halfspaces(y, v, boxes, hmax: int = 8):
    """HSMC local convex region of one waypoint (section 'Half-Space Monte Carlo', Eq. (eq:hs)):
    (a (h, 3), b (h,)) in construction order."""
    yy = _c(y, np.float32); vv = _c(v, np.float32)
    bx = _c(boxes, np.float32).reshape(-1, 6)
    a = np.zeros((max(hmax, 1), 3), np.float32); b = np.zeros(max(hmax, 1), np.float32)
    k = lib().orc_halfspaces(_p(yy), _p(vv), _p(bx), bx.shape[0], int(hmax), _p(a), _p(b))
    if k < 0:
        raise MemoryError("oracle halfspaces failed")
    return a[:k].copy(), b[:k].copy()


def edge_masks_hs(graph: Dict, xi, boxes, n_particles: int, hmax: int = 8) -> np.ndarray:
    """HSMC particle masks per edge (E, N/32) uint32."""
    E, W = graph["n_edges"], graph["W"]
    w = n_particles // 32
    out = np.zeros((E, w), np.uint32)
    x = _c(xi, np.float32)
    bx = _c(boxes, np.float32).reshape(-1, 6)
    rc = lib().orc_edge_masks_hs(E, W, n_particles, _p(graph["phi"]), _p(graph["L"]), _p(graph["nom"]),
                                 _p(graph["nvel"]), _p(graph["linf"]), _p(x), _p(bx), bx.shape[0], int(hmax), _p(out))
    if rc:
        raise MemoryError("oracle HSMC masks failed")
    return out


def cp_thresholds(alpha: float, eta: float, n_particles: int):
    """(K_min, K_max): alpha_min = alpha/eta and alpha_max = eta*alpha (Algorithm 2) as popcount
    bounds.  CP-hat = popc/N < alpha_x  <=>  popc < K_x with K_x = #{k >= 0 : k < alpha_x N}.
    alpha and eta are taken as float32 (their type at the library boundary) and the products
    (eta*alpha)*N and (alpha/eta)*N are formed in double."""
    a = float(np.float32(alpha)); e = float(np.float32(eta)); N = float(n_particles)
    amax = (e * a) * N
    amin = (a / e) * N
    kmax = int(math.ceil(amax)) if amax > 0 else 0
    kmin = int(math.ceil(amin)) if amin > 0 else 0
    return kmin, kmax


def explore(n: int, row_ptr, col, ecost, emask, start: int, goal_idx, K_min: int, K_max: int,
            lam: float, radius: float, max_plans: int = 1 << 24, flags: int = 0,
            max_iterations: int = 1 << 20, n_threads: int = 1) -> Dict:
    """Explore (Algorithm 4) on a CSR graph with edge costs and edge masks.  n_threads > 1 splits
    the expansion over group members and RemoveDominated over target nodes (timing only; the
    result is the single-thread result)."""
    rp = _c(row_ptr, np.int32); cl = _c(col, np.int32); ec = _c(ecost, np.float32)
    em = _c(emask, np.uint32)
    w = em.shape[1] if em.ndim == 2 else 1
    is_goal = np.zeros(n, np.uint8)
    is_goal[np.asarray(goal_idx, dtype=np.int64)] = 1
    args = (n, _p(rp), _p(cl), _p(ec), _p(em), w, int(start), _p(is_goal), int(K_min), int(K_max), C.c_float(lam),
            C.c_float(radius), int(max_plans), int(flags), int(max_iterations))
    R = lib().orc_explore_mt(*args, int(n_threads)) if n_threads > 1 else lib().orc_explore(*args)
    if not R:
        raise MemoryError("oracle explore failed")
    try:
        s = np.zeros(7, np.int64)
        lib().orc_explore_summary(R, _p(s))
        P = int(s[1]); G = int(s[6])
        out = {"head": np.zeros(P, np.int32), "parent": np.zeros(P, np.int32),
               "cost": np.zeros(P, np.float32), "mask": np.zeros((P, w), np.uint32),
               "popc": np.zeros(P, np.int32), "t_created": np.zeros(P, np.int32),
               "e_expanded": np.zeros(P, np.int32), "removed": np.zeros(P, np.uint8),
               "goal_plans": np.zeros(G, np.int32)}
        lib().orc_explore_export(R, *[_p(out[k]) for k in ("head", "parent", "cost", "mask", "popc",
                                                            "t_created", "e_expanded", "removed",
                                                            "goal_plans")])
        out.update(status=int(s[0]), n_plans=P, n_candidates=int(s[2]), n_kept=int(s[3]),
                   n_iterations=int(s[4]), n_groups_expanded=int(s[5]), n_goal=G)
        return out
    finally:
        lib().orc_explore_free(R)


def philox4x64(counter, key) -> np.ndarray:
    c = _c(counter, np.uint64); k = _c(key, np.uint64); o = np.zeros(4, np.uint64)
    lib().orc_philox4x64(_p(c), _p(k), _p(o))
    return o


def philox4x32(counter, key) -> np.ndarray:
    c = _c(counter, np.uint32); k = _c(key, np.uint32); o = np.zeros(4, np.uint32)
    lib().orc_philox4x32(_p(c), _p(k), _p(o))
    return o


def mc_normals(seed: int, m: int, s: int) -> np.ndarray:
    o = np.zeros(6, np.float32)
    lib().orc_mc_normals(C.c_uint64(seed), C.c_uint64(m), C.c_uint64(s), _p(o))
    return o.reshape(3, 2)


def mlp_draws(seed: int, t: int, stream: int, rows: int, n_env: int = 0):
    """Latents (rows x 8 float32) and, with n_env > 0, environment indices of draw set (t, stream)."""
    z = np.zeros((rows, 8), np.float32)
    env = np.zeros(rows, np.int32)
    lib().orc_mlp_draws(C.c_uint64(seed), C.c_uint64(t), C.c_uint64(stream), C.c_int64(rows), C.c_int32(n_env),
                        _p(z), _p(env))
    return z, (env if n_env > 0 else None)


def backtrack(parent, head, p: int) -> np.ndarray:
    path = []
    while p >= 0:
        path.append(int(head[p]))
        p = int(parent[p])
    return np.asarray(path[::-1], dtype=np.int32)


def edge_of(graph: Dict, v: int, u: int) -> int:
    rp, col = graph["row_ptr"], graph["col"]
    seg = col[rp[v]:rp[v + 1]]
    k = np.nonzero(seg == u)[0]
    if len(k) == 0:
        raise KeyError((v, u))
    return int(rp[v] + k[0])


def mc_certify(states, path, edge_tau, W: int, sigma: float, boxes, n_mc: int, substeps: int,
               seed: int) -> int:
    st = _c(states, np.float32); pa = _c(path, np.int32); et = _c(edge_tau, np.float32)
    bx = _c(boxes, np.float32).reshape(-1, 6)
    if len(et) == 0:
        et = np.zeros(1, np.float32)
    return int(lib().orc_mc_certify(_p(st), _p(pa), len(pa), _p(et), int(W), C.c_float(sigma), _p(bx),
                                    bx.shape[0], int(n_mc), int(substeps), C.c_uint64(seed)))


def selection_order(goal_plans, popc, cost):
    """P_goal sorted for PlanSelection (Algorithm 5, "ascending CP-hat"): by popc ascending; ties
    (the paper gives no rule) by cost descending, then plan id ascending, so that among plans of
    equal CP-hat the cheaper one sits at the higher index, which the bisection prefers."""
    return sorted((int(p) for p in goal_plans), key=lambda p: (int(popc[p]), -float(cost[p]), p))


def bisect_select(order, mc_count, n_mc: int, alpha: float):
    """The bisection of PlanSelection (Algorithm 5) over `order` with 1-based indices as printed:
    l = 1, u = |P|, m = ceil((l + u) / 2); while l != u: u = m - 1 if MC(P_m) > alpha else l = m,
    then m = ceil((l + u) / 2); finally failure iff MC(P_m) > alpha.  MC(p) > alpha is
    mc_count(p) / n_mc > alpha in double, alpha taken as float32 (its type at the boundary).
    Returns (status, chosen plan or -1 when P_goal is empty, its count, probed indices)."""
    if len(order) == 0:
        return ERR_INFEASIBLE, -1, -1, []
    a = float(np.float32(alpha))
    over = lambda c: c / n_mc > a
    l, u = 1, len(order)
    m = (l + u + 1) // 2
    probed = []
    while l != u:
        probed.append(m)
        if over(mc_count(order[m - 1])):
            u = m - 1
        else:
            l = m
        m = (l + u + 1) // 2
    c = mc_count(order[m - 1])
    return (ERR_INFEASIBLE if over(c) else OK), order[m - 1], c, probed


def plan_select(graph: Dict, ex: Dict, alpha: float, states, boxes, sigma: float, n_mc: int,
                substeps: int, seed: int, mc_count=None) -> Dict:
    """PlanSelection (Algorithm 5) on an Explore result of the oracle: selection_order, then
    bisect_select with MC(p) from mc_certify on p's backtracked path (or `mc_count(p)` when given,
    for tests that script the Monte Carlo outcomes).  Smoothing is not applied: it follows a cited
    method."""
    st = _c(states, np.float32); bx = _c(boxes, np.float32).reshape(-1, 6)
    if ex["n_goal"] == 0:
        return {"status": ERR_INFEASIBLE, "chosen": -1, "collisions": -1, "sorted_goal": np.zeros(0, np.int32),
                "n_probes": 0}
    order = selection_order(ex["goal_plans"].tolist(), ex["popc"], ex["cost"])
    cache = {}

    def mc(p):
        if p not in cache:
            if mc_count is not None:
                cache[p] = int(mc_count(p))
            else:
                path = backtrack(ex["parent"], ex["head"], p)
                taus = [graph["tau"][edge_of(graph, int(path[k]), int(path[k + 1]))] for k in range(len(path) - 1)]
                cache[p] = mc_certify(st, path, np.asarray(taus, np.float32), graph["W"], sigma, bx, n_mc,
                                      substeps, seed)
        return cache[p]

    status, chosen, c, probed = bisect_select(order, mc, n_mc, alpha)
    return {"status": status, "chosen": chosen, "collisions": c, "sorted_goal": np.asarray(order, np.int32),
            "n_probes": len(probed)}


def plan(wl, exhaustive: bool = False, flags: int = 0, max_plans: int = 1 << 24) -> Dict:
    """Algorithm 2 end to end on a Workload: BuildGraph, masks, Explore, PlanSelection."""
    g = graph_build(wl.states, wl.boxes, wl.radius, wl.n_waypoints, wl.sigma, exhaustive=exhaustive)
    masks = edge_masks(g, wl.xi, wl.boxes, wl.n_particles)
    kmin, kmax = cp_thresholds(wl.alpha, wl.eta, wl.n_particles)
    ex = explore(g["n"], g["row_ptr"], g["col"], g["ecost"], masks, wl.start_idx, wl.goal_idx, kmin, kmax,
                 wl.lam, wl.radius, max_plans=max_plans, flags=flags)
    sel = plan_select(g, ex, wl.alpha, wl.states, wl.boxes, wl.sigma, wl.n_mc, wl.mc_substeps, wl.mc_seed)
    return {"graph": g, "masks": masks, "explore": ex, "select": sel, "K_min": kmin, "K_max": kmax}
