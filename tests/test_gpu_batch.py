"""pump_plan_batch: the box masks of many queries in one persistent launch, their Explore runs in
another.  Each query's result must equal the single-query result (pump_plan on the same graph) bit
for bit: counters, the whole plan arena, P_goal, the selected plan and its Monte Carlo count.  One
batch is also checked against the CPU oracle directly.  Covers the launch forms (cluster sizes 16,
8, 4; dominance table on chip and in global memory; fewer clusters than queries; mask passes of
one or two word pairs, 1 to 64 edges per warp take and 32 to 4096 edges per block item; graphs of
different particle and box counts in one mask launch; an HSMC graph beside box graphs),
explore-only queries mixed with full ones, and the argument checks."""
import numpy as np
import pytest

from oracle import cpu
from paper_1607_06886_gb300 import inputs, pump

from _util import assert_arena_equal, compare_graphs, export_arena, export_graph, gpu_graph, plan_params

pytestmark = pytest.mark.gpu

RESULT_KEYS = ("status", "chosen_plan", "cost", "popc", "cp_hat", "cp_mc", "mc_collisions", "n_candidates", "n_kept",
               "n_plans", "n_iterations", "n_groups", "n_goal", "n_certified", "path_len", "path_truncated")

QUERIES = [("three_box_1k", 0, 250), ("indoor_4k", 1, 400), ("three_box_1k", 2, 400), ("indoor_4k", 3, 600),
           ("three_box_1k", 4, 150), ("indoor_4k", 5, 300), ("three_box_1k", 6, 300), ("indoor_4k", 7, 500),
           ("three_box_1k", 8, 200), ("indoor_4k", 9, 350), ("three_box_1k", 10, 350)]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    pump.load()
    pump.use_torch_allocator()
    yield


@pytest.fixture(scope="module")
def queries():
    """Graphs, params and single-query reference results (results, arenas)."""
    out = []
    for name, seed, ns in QUERIES:
        wl = inputs.make_workload(name, seed, ns)
        G = gpu_graph(wl)
        prm = plan_params(wl, n_mc=2000)
        ref = G.plan(prm)
        out.append((wl, G, prm, ref, export_arena(G)))
    return out


def check_same(ref, ref_arena, res, G):
    for k in RESULT_KEYS:
        assert res[k] == ref[k], (k, res[k], ref[k])
    arena = export_arena(G)
    for k, v in ref_arena.items():
        np.testing.assert_array_equal(arena[k], v, err_msg=k)


@pytest.mark.parametrize("cfg", [None, (16, 0, 0, 0, 0), (8, 0, 0, 1, 1, 32), (4, 0, 2, 2, 16, 4096),
                                 (16, 1, 0, 1, 64, 96), (8, 1, 3, 2, 3, 256)])
def test_batch_equals_single_queries(queries, cfg):
    """Every launch form (Explore: CTAs per query, table placement, clusters in flight; masks: word
    pairs per warp pass, edges per warp take, edges per block item) gives the single-query
    results."""
    config = None if cfg is None else pump.BatchConfig(*cfg)
    rc, res = pump.plan_batch([q[1] for q in queries], [q[2] for q in queries], config)
    assert rc in (pump.OK, pump.ERR_INFEASIBLE)
    for (wl, G, prm, ref, ref_arena), r in zip(queries, res):
        check_same(ref, ref_arena, r, G)


def test_batch_mixed_explore_only(queries):
    prms = []
    for j, q in enumerate(queries):
        p = plan_params(q[0], n_mc=2000, flags=pump.EXPLORE_ONLY if j % 2 else 0)
        prms.append(p)
    rc, res = pump.plan_batch([q[1] for q in queries], prms)
    for j, ((wl, G, prm, ref, ref_arena), r) in enumerate(zip(queries, res)):
        if j % 2:
            assert r["status"] == pump.OK and r["chosen_plan"] == -1
            for k in ("n_candidates", "n_kept", "n_plans", "n_iterations", "n_groups", "n_goal"):
                assert r[k] == ref[k], k
            arena = export_arena(G)
            for k, v in ref_arena.items():
                np.testing.assert_array_equal(arena[k], v, err_msg=k)
        else:
            check_same(ref, ref_arena, r, G)


def test_batch_matches_oracle():
    """A batch of three queries against the CPU oracle (graph tier, masks, Explore bit for bit)."""
    wls = [inputs.make_workload("three_box_1k", s, 250) for s in (11, 12, 13)]
    Gs = [gpu_graph(wl) for wl in wls]
    rc, res = pump.plan_batch(Gs, [plan_params(wl, n_mc=2000) for wl in wls])
    for wl, G, r in zip(wls, Gs, res):
        o = cpu.plan(wl)
        og, ex = o["graph"], o["explore"]
        ndiff, _ = compare_graphs(export_graph(G), og, wl.radius)
        assert ndiff <= 2
        np.testing.assert_array_equal(G.export("col"), og["col"])
        np.testing.assert_array_equal(G.export("ecost").view(np.uint32), og["ecost"].view(np.uint32))
        np.testing.assert_array_equal(G.export("masks"), o["masks"])
        assert r["n_candidates"] == ex["n_candidates"] and r["n_plans"] == ex["n_plans"]
        assert_arena_equal(export_arena(G), ex, wl.n_particles // 32)


def test_batch_single_query_and_many_clusters(queries):
    wl, G, prm, ref, ref_arena = queries[1]
    rc, res = pump.plan_batch([G], [prm], pump.BatchConfig(0, 0, 64, 0, 0))
    check_same(ref, ref_arena, res[0], G)


def test_batch_rejects_bad_arguments(queries):
    G0, G1 = queries[0][1], queries[1][1]
    p0 = queries[0][2]
    rc, _ = pump.plan_batch([G0, G0], [p0, p0])
    assert rc == pump.ERR_INVALID_ARG
    for bad in [(3, 0, 0, 0, 0), (32, 0, 0, 0, 0), (0, 2, 0, 0, 0), (0, 0, -1, 0, 0), (0, 0, 0, 3, 0),
                (0, 0, 0, -1, 0), (0, 0, 0, 0, 65), (0, 0, 0, 0, -2), (0, 0, 0, 0, 0, -32), (0, 0, 0, 0, 0, 48),
                (0, 0, 0, 0, 0, 65568)]:
        rc, _ = pump.plan_batch([G0, G1], [p0, queries[1][2]], pump.BatchConfig(*bad))
        assert rc == pump.ERR_INVALID_ARG, bad
    g = inputs.random_explore_graph(20, 3, 32, 0)
    imported = pump.Graph.from_csr(g.n, g.row_ptr, g.col, g.ecost, g.emask, 32, 0, [1])
    rc, _ = pump.plan_batch([G0, imported], [p0, p0])
    assert rc == pump.ERR_INVALID_ARG
    bad_p = pump.default_plan_params(alpha=0.01, lam=2.0)
    rc, _ = pump.plan_batch([G0], [bad_p])
    assert rc == pump.ERR_INVALID_ARG


def test_batch_with_an_hsmc_graph(queries):
    """An HSMC graph takes its own mask pass beside the box graphs' shared launch; every result
    equals its single query."""
    wl = inputs.make_workload("indoor_4k", 21, 300)
    Gh = pump.Graph.build(wl.states, wl.goal_idx, wl.boxes, wl.xi, wl.radius, wl.n_particles, wl.n_waypoints,
                          wl.sigma, flags=pump.GRAPH_HSMC)
    ph = plan_params(wl, n_mc=2000)
    refh = Gh.plan(ph)
    arh = export_arena(Gh)
    sel = [queries[0], queries[1], queries[3]]
    rc, res = pump.plan_batch([sel[0][1], Gh, sel[1][1], sel[2][1]], [sel[0][2], ph, sel[1][2], sel[2][2]])
    assert rc in (pump.OK, pump.ERR_INFEASIBLE)
    check_same(refh, arh, res[1], Gh)
    for (wl_, G, prm, ref, ref_arena), r in zip(sel, [res[0], res[2], res[3]]):
        check_same(ref, ref_arena, r, G)
