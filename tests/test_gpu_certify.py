"""MC(p) certification on the GPU vs the CPU oracle.

Both sides draw the same Philox4x32-10 words for every rollout, step and axis and map them to the
same uniforms; Box-Muller differs (the GPU's hardware log and sine/cosine approximations, absolute
error ~2^-21 per normal, against double rounded to float in the oracle), and the GPU's warp-scan
form (one or two plans) composes the deviation recurrence across lanes (float rounding ~1e-7
relative).  Deviations therefore differ by ~1e-8 and a rollout's outcome can only flip when its
path grazes a box face at that scale.  Tolerance: |count_gpu - count_oracle| <= 3 + 0.002 count.
With independent seeds the two estimates agree within their binomial spread."""
import math

import numpy as np
import pytest

from oracle import cpu
from paper_1607_06886_gb300 import inputs, pump

from _util import export_arena, gpu_graph, plan_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    pump.load()
    pump.use_torch_allocator()
    yield


@pytest.fixture(scope="module")
def planned():
    wl = inputs.make_workload("indoor_4k", 0, 700)
    G = gpu_graph(wl)
    res = G.plan(plan_params(wl, n_mc=2000))
    og = cpu.graph_build(wl.states, wl.boxes, wl.radius, wl.n_waypoints, wl.sigma)
    return wl, G, res, og


def _oracle_count(wl, og, path, n_mc, substeps, seed):
    taus = [og["tau"][cpu.edge_of(og, int(path[k]), int(path[k + 1]))] for k in range(len(path) - 1)]
    return cpu.mc_certify(wl.states, path, np.asarray(taus, np.float32), wl.n_waypoints, wl.sigma, wl.boxes, n_mc,
                          substeps, seed)


@pytest.mark.parametrize("seed,substeps,n_mc", [(0, 4, 3000), (7, 1, 2000), (123, 3, 1500)])
def test_certify_matches_oracle_same_stream(planned, seed, substeps, n_mc):
    wl, G, res, og = planned
    a = export_arena(G)
    # certify several goal plans and the chosen one
    plans = list(a["goal_plans"][:4]) + ([res["chosen_plan"]] if res["chosen_plan"] >= 0 else [])
    assert plans
    for p in plans:
        path = cpu.backtrack(a["plan_parent"], a["plan_head"], int(p))
        c_gpu, cp = G.certify(path, n_mc, substeps, seed)
        c_orc = _oracle_count(wl, og, path, n_mc, substeps, seed)
        assert abs(c_gpu - c_orc) <= 3 + int(0.002 * c_orc), (p, c_gpu, c_orc)
        assert cp == pytest.approx(c_gpu / n_mc)


def test_certify_independent_streams_agree_statistically(planned):
    wl, G, res, og = planned
    a = export_arena(G)
    path = cpu.backtrack(a["plan_parent"], a["plan_head"], int(a["goal_plans"][-1]))
    M = 20000
    c1, _ = G.certify(path, M, 4, 1)
    c2 = _oracle_count(wl, og, path, M, 4, 2)
    p = (c1 + c2) / (2 * M)
    assert abs(c1 - c2) / M <= 4 * math.sqrt(max(p * (1 - p), 1e-9) * 2 / M) + 1.0 / M


def test_certify_single_node_path_and_zero_rollouts(planned):
    wl, G, res, og = planned
    assert G.certify([0], 100, 4, 0) == (0, 0.0)
    assert G.certify([0, int(G.export("col")[0])] if G.export("row_ptr")[1] > 0 else [0], 0, 4, 0)[0] == 0


def test_certify_rejects_paths_off_the_graph(planned):
    wl, G, res, og = planned
    rp, col = G.export("row_ptr"), G.export("col")
    nbrs = set(col[rp[0]:rp[1]].tolist())
    u = next(v for v in range(1, wl.n) if v not in nbrs)
    with pytest.raises(pump.PumpError) as e:
        G.certify([0, u], 10, 4, 0)
    assert e.value.status == pump.ERR_INVALID_ARG
    with pytest.raises(pump.PumpError):
        G.certify([0, wl.n + 5], 10, 4, 0)


@pytest.mark.parametrize("seed,lo,hi", [(2, 1, 2), (0, 3, 6), (1, 7, 32)])
def test_plan_certification_forms_match_oracle(seed, lo, hi):
    """PlanSelection certifies its first batch of goal plans with the form that suits their count:
    the warp scan for one or two plans, two lanes per rollout up to six, one lane beyond.  Full
    indoor queries whose P_goal sizes fall in each range; the chosen plan's count is checked
    against the oracle's MC of the same path and stream."""
    wl = inputs.make_workload("indoor_4k", seed)
    G = gpu_graph(wl)
    n_mc = 4000
    res = G.plan(plan_params(wl, n_mc=n_mc))
    assert lo <= res["n_goal"] <= hi, res["n_goal"]
    assert res["chosen_plan"] >= 0
    og = cpu.graph_build(wl.states, wl.boxes, wl.radius, wl.n_waypoints, wl.sigma)
    c_orc = _oracle_count(wl, og, res["path"], n_mc, wl.mc_substeps, wl.mc_seed)
    assert abs(res["mc_collisions"] - c_orc) <= 3 + int(0.002 * c_orc), (res["mc_collisions"], c_orc)
    G.close()
