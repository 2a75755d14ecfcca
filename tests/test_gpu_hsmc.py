"""Half-Space Monte Carlo masks on the GPU (graph built with GRAPH_HSMC) vs the CPU oracle: masks
bit for bit on every edge whose float descriptors, nominal waypoints and nominal velocities agree
bit for bit (the half-space construction and the particle test are float arithmetic with a fixed
order on both sides), then Explore on those masks record by record, and PlanSelection on top."""
import numpy as np
import pytest

from oracle import cpu
from paper_1607_06886_gb300 import inputs, pump

from _util import assert_arena_equal, compare_graphs, export_arena, export_graph, plan_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    pump.load()
    pump.use_torch_allocator()
    yield


def hsmc_graph(wl):
    return pump.Graph.build(wl.states, wl.goal_idx, wl.boxes, wl.xi, wl.radius, wl.n_particles, wl.n_waypoints,
                            wl.sigma, flags=pump.GRAPH_HSMC)


def same_edges(G, og, diff):
    nv = G.export("nominal_vel")
    return ~diff & np.all(nv.view(np.uint32).reshape(len(diff), -1) == og["nvel"].view(np.uint32).reshape(len(diff), -1),
                          axis=1)


@pytest.mark.parametrize("name,seed,ns", [("three_box_1k", 0, 300), ("three_box_1k", 2, 500), ("indoor_4k", 1, 400),
                                          ("indoor_4k", 3, 700)])
def test_hsmc_masks_match_oracle(name, seed, ns):
    wl = inputs.make_workload(name, seed, ns)
    G = hsmc_graph(wl)
    og = cpu.graph_build(wl.states, wl.boxes, wl.radius, wl.n_waypoints, wl.sigma)
    ndiff, diff = compare_graphs(export_graph(G), og, wl.radius)
    same = same_edges(G, og, diff)
    assert same.sum() >= len(same) - max(2, int(1e-4 * len(same)))
    G.edge_masks()
    gm = G.export("masks")
    om = cpu.edge_masks_hs(og, wl.xi, wl.boxes, wl.n_particles)
    np.testing.assert_array_equal(gm[same], om[same])
    assert (om != 0).any() and (om == 0).any()


def test_hsmc_plan_matches_oracle_explore():
    wl = inputs.make_workload("indoor_4k", 0, 600)
    G = hsmc_graph(wl)
    og = cpu.graph_build(wl.states, wl.boxes, wl.radius, wl.n_waypoints, wl.sigma)
    res = G.plan(plan_params(wl, n_mc=2000))
    om = cpu.edge_masks_hs(og, wl.xi, wl.boxes, wl.n_particles)
    np.testing.assert_array_equal(G.export("masks"), om)   # this seed has no boundary edge
    kmin, kmax = cpu.cp_thresholds(wl.alpha, wl.eta, wl.n_particles)
    ex = cpu.explore(og["n"], og["row_ptr"], og["col"], og["ecost"], om, 0, wl.goal_idx, kmin, kmax, wl.lam,
                     wl.radius)
    assert res["n_candidates"] == ex["n_candidates"] and res["n_plans"] == ex["n_plans"]
    assert_arena_equal(export_arena(G), ex, wl.n_particles // 32)
    assert res["rc"] in (pump.OK, pump.ERR_INFEASIBLE)


def test_hsmc_and_box_masks_differ_but_both_see_the_obstacles():
    wl = inputs.make_workload("indoor_4k", 4, 500)
    Gb = pump.Graph.build(wl.states, wl.goal_idx, wl.boxes, wl.xi, wl.radius, wl.n_particles, wl.n_waypoints,
                          wl.sigma)
    Gh = hsmc_graph(wl)
    Gb.edge_masks()
    Gh.edge_masks()
    mb, mh = Gb.export("masks"), Gh.export("masks")
    assert mb.shape == mh.shape and (mb != 0).any() and (mh != 0).any()
    assert not np.array_equal(mb, mh)
