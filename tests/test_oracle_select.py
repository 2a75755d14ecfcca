"""Pins of the oracle's PlanSelection (Algorithm 5) with scripted Monte Carlo outcomes.

The ordering (ascending CP-hat, ties by descending cost then ascending id) and the printed 1-based
bisection are checked against what they must compute, independently of the GPU:
  * hand-traced probe sequences and results (tests/golden/plan_select_bisection.txt);
  * for every list length and every monotone outcome (the first k plans certify, the rest do not),
    the bisection returns the k-th plan, or failure when k = 0: the last index of a monotone
    predicate, found here by brute force, with at most ceil(log2 |P|) probes;
  * the order of a hand-built P_goal with ties in CP-hat and in cost, written out by hand;
  * MC(p) > alpha is strict, with alpha taken as float32;
  * the whole plan_select on an oracle Explore result with scripted counts.
"""
import math
import os

import numpy as np
import pytest

from oracle import cpu
from paper_1607_06886_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
N_MC = 10000


def scripted(order, k):
    """MC counts: the first k plans of `order` pass (0 collisions), the others fail (all collide)."""
    ok = set(order[:k])
    return lambda p: 0 if p in ok else N_MC


def test_bisection_matches_hand_traces():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "plan_select_bisection.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) >= 8
    for G, k, probes, res in rows:
        G, k = int(G), int(k)
        order = list(range(100, 100 + G))  # plan ids, already in selection order
        st, chosen, _, probed = cpu.bisect_select(order, scripted(order, k), N_MC, 0.05)
        assert probed == ([] if probes == "-" else [int(x) for x in probes.split(",")]), (G, k, probed)
        if res == "F":
            assert st == cpu.ERR_INFEASIBLE
        else:
            assert st == cpu.OK and chosen == order[int(res) - 1]


@pytest.mark.parametrize("G", list(range(1, 40)))
def test_bisection_finds_last_certified_plan_of_monotone_outcomes(G):
    order = list(range(G))
    for k in range(G + 1):
        st, chosen, _, probed = cpu.bisect_select(order, scripted(order, k), N_MC, 0.01)
        passing = [i for i in range(1, G + 1) if i <= k]   # brute force: 1-based indices that certify
        if passing:
            assert st == cpu.OK and chosen == order[max(passing) - 1]
        else:
            assert st == cpu.ERR_INFEASIBLE
        assert len(probed) <= math.ceil(math.log2(G)) if G > 1 else probed == []
        assert all(1 <= m <= G for m in probed)


def test_bisection_empty_goal_set_is_infeasible():
    st, chosen, _, probed = cpu.bisect_select([], lambda p: 0, N_MC, 0.01)
    assert st == cpu.ERR_INFEASIBLE and chosen == -1 and probed == []


def test_bisection_threshold_is_strict_with_float_alpha():
    # alpha = 0.5 is exact in float: 5000 / 10000 is not above it, 5001 / 10000 is
    assert cpu.bisect_select([7], lambda p: 5000, N_MC, 0.5)[0] == cpu.OK
    assert cpu.bisect_select([7], lambda p: 5001, N_MC, 0.5)[0] == cpu.ERR_INFEASIBLE
    # alpha = 0.01 as float32 is 0.00999999977...: 99 / 10000 passes, 100 / 10000 is above it
    assert cpu.bisect_select([7], lambda p: 99, N_MC, 0.01)[0] == cpu.OK
    assert cpu.bisect_select([7], lambda p: 100, N_MC, 0.01)[0] == cpu.ERR_INFEASIBLE


def test_selection_order_ties_by_hand():
    # (id, popc, cost); expected order written by hand from the rule: popc ascending, then cost
    # descending, then id ascending
    plans = [(10, 1, 2.0), (3, 0, 5.0), (7, 0, 5.0), (4, 0, 6.0), (9, 1, 2.5), (2, 2, 1.0), (5, 1, 2.0)]
    popc = np.zeros(16, np.int32)
    cost = np.zeros(16, np.float32)
    for i, pc, c in plans:
        popc[i], cost[i] = pc, c
    order = cpu.selection_order([p[0] for p in plans], popc, cost)
    assert order == [4, 3, 7, 9, 5, 10, 2]
    # every plan certifies: the bisection ends at the last (cheapest, riskiest) plan
    assert cpu.bisect_select(order, lambda p: 0, N_MC, 0.01)[1] == 2
    # only the popc-0 plans certify: among the equal-cost pair the higher id is chosen
    assert cpu.bisect_select(order, lambda p: 0 if popc[p] == 0 else N_MC, N_MC, 0.01)[1] == 7
    # the popc-0 and popc-1 plans certify: the cheaper of the equal-cost popc-1 pair, higher id
    assert cpu.bisect_select(order, lambda p: 0 if popc[p] <= 1 else N_MC, N_MC, 0.01)[1] == 10


def test_plan_select_on_explore_result_with_scripted_counts():
    """plan_select on a real Explore result: with MC scripted to pass exactly the plans whose CP-hat
    is below a threshold (monotone along the order), the chosen plan is the last such plan of the
    order, i.e. the cheapest plan among those of the highest passing CP-hat."""
    wl = inputs.make_workload("indoor_4k", seed=2, n_samples=400)
    g = cpu.graph_build(wl.states, wl.boxes, wl.radius, wl.n_waypoints, wl.sigma)
    masks = cpu.edge_masks(g, wl.xi, wl.boxes, wl.n_particles)
    kmin, kmax = cpu.cp_thresholds(wl.alpha, wl.eta, wl.n_particles)
    ex = cpu.explore(g["n"], g["row_ptr"], g["col"], g["ecost"], masks, wl.start_idx, wl.goal_idx, kmin, kmax,
                     wl.lam, wl.radius, flags=cpu.NO_EARLY_STOP)
    assert ex["n_goal"] >= 3
    popc, cost = ex["popc"], ex["cost"]
    for thr in sorted(set(popc[ex["goal_plans"]].tolist())):
        sel = cpu.plan_select(g, ex, wl.alpha, wl.states, wl.boxes, wl.sigma, N_MC, 4, 0,
                              mc_count=lambda p: 0 if popc[p] <= thr else N_MC)
        order = sel["sorted_goal"].tolist()
        assert sorted(order) == sorted(ex["goal_plans"].tolist())
        keys = [(int(popc[p]), -float(cost[p]), p) for p in order]
        assert keys == sorted(keys)
        expect = max(i for i, p in enumerate(order) if popc[p] <= thr)
        assert sel["status"] == cpu.OK and sel["chosen"] == order[expect]
        assert float(cost[sel["chosen"]]) == min(float(cost[p]) for p in order if popc[p] == popc[order[expect]])
