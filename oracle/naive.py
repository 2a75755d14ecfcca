"""Second, deliberately naive restatement of Explore (Algorithm 4).

TEST INFRASTRUCTURE, small graphs only.  It keeps P, P_open and the group as
plain Python sets and lists, re-scans every plan of P in RemoveDominated and
every open plan when forming the next group, and represents masks as Python
integers.  It shares no code with pump_oracle.c; the two must agree exactly,
which pins the C oracle's per-node bookkeeping and its restriction of
RemoveDominated to the nodes that received candidates.

Conventions (the same readings as the C oracle): candidates in ascending group
id, then adjacency order; cost = float32(parent.cost + edge cost); CP cutoff
popc < K_max; a goal plan in the group with popc < K_min stops the search;
group i holds open plans with cost <= float32(i * (lambda * r)) computed in
double; surviving candidates get consecutive ids in candidate order.
"""
from __future__ import annotations

from typing import Dict, List, Sequence

import numpy as np


def _thr(i: int, lam: float, r: float) -> np.float32:
    return np.float32(float(i) * (float(np.float32(lam)) * float(np.float32(r))))


def explore_naive(n: int, row_ptr, col, ecost, emask_words, start: int, goal_idx: Sequence[int],
                  K_min: int, K_max: int, lam: float, r: float, no_early_stop: bool = False,
                  max_iterations: int = 100000) -> Dict:
    w = emask_words.shape[1]
    emask = [sum(int(emask_words[e, j]) << (32 * j) for j in range(w)) for e in range(len(col))]
    goal = set(int(g) for g in goal_idx)
    # plan records
    head: List[int] = [start]
    parent: List[int] = [-1]
    cost: List[np.float32] = [np.float32(0.0)]
    mask: List[int] = [0]
    t_created: List[int] = [-1]
    e_expanded: List[int] = [-1]
    P = {0}          # live plans
    P_open = {0}
    removed = set()
    group = [0]
    i = 0
    n_cand = 0
    while P_open and (no_early_stop or not any(head[g] in goal and bin(mask[g]).count("1") < K_min
                                                for g in group)):
        if i >= max_iterations:
            raise RuntimeError("iteration cap")
        cands = []
        for p in sorted(group):
            v = head[p]
            for e in range(int(row_ptr[v]), int(row_ptr[v + 1])):
                n_cand += 1
                m = mask[p] | emask[e]
                if bin(m).count("1") < K_max:
                    cands.append((int(col[e]), p, np.float32(cost[p] + np.float32(ecost[e])), m))
        # P <- P u {q}, P_open <- P_open u {q}: provisional keys ('c', k)
        cand_keys = [("c", k) for k in range(len(cands))]

        def rec(key):
            if isinstance(key, tuple):
                x, _, c, m = cands[key[1]]
                return x, c, bin(m).count("1")
            return head[key], cost[key], bin(mask[key]).count("1")

        allP = list(P) + cand_keys
        openP = set(P_open) | set(cand_keys)
        # RemoveDominated(P, P_open): decided against the whole of P before removing
        doomed = set()
        for p in openP:
            xp, cp, kp = rec(p)
            for d in allP:
                xd, cd, kd = rec(d)
                if xd == xp and cd < cp and kd <= kp:
                    doomed.add(p)
                    break
        for p in doomed:
            if isinstance(p, tuple):
                continue
            P.discard(p); P_open.discard(p); removed.add(p)
        for k, (x, par, c, m) in enumerate(cands):
            if ("c", k) in doomed:
                continue
            pid = len(head)
            head.append(x); parent.append(par); cost.append(c); mask.append(m)
            t_created.append(i); e_expanded.append(-1)
            P.add(pid); P_open.add(pid)
        for p in group:
            e_expanded[p] = i
            P_open.discard(p)
        i += 1
        thr = _thr(i, lam, r)
        group = sorted(p for p in P_open if cost[p] <= thr)
    goal_plans = sorted(p for p in P if head[p] in goal)
    return {"head": np.asarray(head, np.int32), "parent": np.asarray(parent, np.int32),
            "cost": np.asarray(cost, np.float32), "mask_int": mask,
            "popc": np.asarray([bin(m).count("1") for m in mask], np.int32),
            "t_created": np.asarray(t_created, np.int32), "e_expanded": np.asarray(e_expanded, np.int32),
            "removed": np.asarray([1 if p in removed else 0 for p in range(len(head))], np.uint8),
            "goal_plans": np.asarray(goal_plans, np.int32), "n_candidates": n_cand, "n_iterations": i,
            "n_plans": len(head)}
