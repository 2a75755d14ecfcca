"""The fused launch: a query's edge masks computed by worker clusters inside the Explore launch
(rows taken in order of shortest-path cost from the start, Explore waiting per row for its masks).

Results must equal the separate launches (masks kernel, then Explore) bit for bit, and through
them the oracle (test_gpu_plan.py compares pump_plan, which takes the fused form by default, with
the oracle).  The edge order must be a valid order of every edge, rows in cost order.  A row
whose count never completes (a test hook) must end the run with a timeout status, and the next
run on the same graph must be correct."""
import contextlib
import heapq
import os

import numpy as np
import pytest

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


@contextlib.contextmanager
def env(**kv):
    old = {k: os.environ.get(k) for k in kv}
    os.environ.update({k: str(v) for k, v in kv.items()})
    try:
        yield
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def workload(name, seed, ns, n_particles=None):
    wl = inputs.make_workload(name, seed, ns)
    if n_particles is not None:
        wl.n_particles = n_particles
        wl.xi = inputs.particle_normals(n_particles, wl.n_waypoints, seed)
    return wl


def run(wl, fused, flags=0):
    with env(PUMP_FUSED_MASKS=1 if fused else 0):
        G = gpu_graph(wl)
        r = G.plan(plan_params(wl, flags=flags))
        return r, G.export("masks"), export_arena(G), G


CASES = [("indoor_4k", 0, None, None), ("indoor_4k", 5, 1500, 64), ("indoor_4k", 6, 1200, 256),
         ("three_box_1k", 2, 600, None), ("three_box_1k", 3, 200, 96)]


@pytest.mark.parametrize("name,seed,ns,N", CASES)
def test_fused_equals_separate_launches(name, seed, ns, N):
    wl = workload(name, seed, ns, N)
    r1, m1, a1, _ = run(wl, True)
    r0, m0, a0, _ = run(wl, False)
    assert r1["fused"] == 1 and r0["fused"] == 0
    np.testing.assert_array_equal(m1, m0)
    for k in a0:
        np.testing.assert_array_equal(a1[k], a0[k])
    for k in ("rc", "status", "chosen_plan", "mc_collisions", "n_candidates", "n_kept", "n_plans", "n_iterations",
              "n_groups", "n_goal", "cost", "popc"):
        assert r1[k] == r0[k], k
    np.testing.assert_array_equal(r1["path"], r0["path"])


def test_fused_form_is_taken():
    """The graph build lays out the edge order (beside its own last kernels) and every query runs
    the fused launch: one kernel for an explore-only query (initialisation, masks, Explore and the
    P_goal order), against four separately (masks, initialisation, Explore, P_goal order);
    PUMP_FUSED_MASKS=0 keeps them separate, and a graph built under it gets its order from its
    first fused query."""
    wl = workload("indoor_4k", 1, 1500)
    p = plan_params(wl, flags=pump.EXPLORE_ONLY)
    with env(PUMP_FUSED_MASKS=""):
        os.environ.pop("PUMP_FUSED_MASKS")
        G = gpu_graph(wl)
        G.export("edge_order")
        r = G.plan(p)
        assert r["rc"] == pump.OK and r["fused"] == 1
        n0 = pump.kernel_launches()
        r = G.plan(p)
        assert r["rc"] == pump.OK and r["fused"] == 1
        n1 = pump.kernel_launches()
    with env(PUMP_FUSED_MASKS=0):
        r = G.plan(p)
        assert r["rc"] == pump.OK and r["fused"] == 0
        n2 = pump.kernel_launches()
        G2 = gpu_graph(wl)
    assert n1 - n0 == 1 and n2 - n1 == 4
    with pytest.raises(pump.PumpError):
        G2.export("edge_order")
    with env(PUMP_FUSED_MASKS=1):
        r2 = G2.plan(p)
    assert r2["fused"] == 1 and r2["n_candidates"] == r["n_candidates"]
    # the lazily laid out order is an order of the same edges (rows within a cost level may differ)
    np.testing.assert_array_equal(np.sort(G2.export("edge_order")[:, 0]), np.sort(G.export("edge_order")[:, 0]))


def shortest_costs(row_ptr, col, ecost, start):
    n = len(row_ptr) - 1
    d = np.full(n, np.inf)
    d[start] = 0.0
    pq = [(0.0, start)]
    while pq:
        c, x = heapq.heappop(pq)
        if c > d[x]:
            continue
        for e in range(row_ptr[x], row_ptr[x + 1]):
            y, nc = int(col[e]), c + float(ecost[e])
            if nc < d[y]:
                d[y] = nc
                heapq.heappush(pq, (nc, y))
    return d


@pytest.mark.parametrize("name,seed,ns", [("indoor_4k", 0, None), ("three_box_1k", 4, 500)])
def test_edge_order_is_a_row_order_by_cost(name, seed, ns):
    wl = workload(name, seed, ns)
    G = gpu_graph(wl)
    with env(PUMP_FUSED_MASKS=1):
        assert G.plan(plan_params(wl, flags=pump.EXPLORE_ONLY))["fused"] == 1
    eo = G.export("edge_order")
    rp, col, ec = G.export("row_ptr"), G.export("col"), G.export("ecost")
    n, E = len(rp) - 1, len(col)
    # every edge once, with its source row
    np.testing.assert_array_equal(np.sort(eo[:, 0]), np.arange(E))
    src = np.repeat(np.arange(n), np.diff(rp))
    np.testing.assert_array_equal(eo[:, 1], src[eo[:, 0]])
    # a row's edges contiguous and ascending
    starts = np.flatnonzero(np.r_[True, eo[1:, 1] != eo[:-1, 1]])
    rows = eo[starts, 1]
    assert len(np.unique(rows)) == len(rows)
    for a, b in zip(starts, np.r_[starts[1:], E]):
        x = eo[a, 1]
        np.testing.assert_array_equal(eo[a:b, 0], np.arange(rp[x], rp[x + 1]))
    # the start's row first (the fused launch's prologue computes exactly its edges)
    assert rows[0] == wl.start_idx
    # rows by cost from the start: nondecreasing up to the quantisation (4093 levels over the
    # largest finite cost) and the float sums the device adds in another order; unreachable last
    d = shortest_costs(rp, col, ec, wl.start_idx)
    dr = d[rows]
    fin = np.isfinite(dr)
    if (~fin).any():
        assert not fin[np.argmax(~fin):].any()
    q = dr[fin].max() / 4094.0
    run_max = np.maximum.accumulate(dr[fin])
    assert np.all(dr[fin] >= run_max - 2 * q - 1e-4 * run_max)


def test_row_wait_runs_out_then_recovers():
    """The start row's count is never completed (test hook): Explore's first wait runs out after
    the shortened limit and the run ends with ERR_TIMEOUT; the next run on the graph is exact."""
    wl = workload("three_box_1k", 7, 400)
    G = gpu_graph(wl)
    p = plan_params(wl, flags=pump.EXPLORE_ONLY)
    with env(PUMP_FUSED_MASKS=1, PUMP_TEST_FUSED_HOLD_ROW=wl.start_idx, PUMP_TEST_SPIN_LIMIT=2000):
        r = G.plan(p)
    assert r["rc"] == pump.ERR_TIMEOUT
    with env(PUMP_FUSED_MASKS=1):
        r1 = G.plan(plan_params(wl))
    assert r1["fused"] == 1
    r0, m0, a0, _ = run(wl, False)
    np.testing.assert_array_equal(G.export("masks"), m0)
    for k in ("rc", "chosen_plan", "mc_collisions", "n_candidates", "n_plans", "cost"):
        assert r1[k] == r0[k], k
    a1 = export_arena(G)
    for k in a0:
        np.testing.assert_array_equal(a1[k], a0[k])


def test_repeated_fused_runs_are_identical():
    """Row counts accumulate over runs (run e expects e x degree); five fused runs in a row, and a
    separate run between them, give the same arena and result."""
    wl = workload("indoor_4k", 8, 1500)
    G = gpu_graph(wl)
    outs = []
    for k in range(6):
        with env(PUMP_FUSED_MASKS=0 if k == 3 else 1):
            r = G.plan(plan_params(wl))
        assert r["fused"] == (0 if k == 3 else 1)
        outs.append((r, G.export("masks"), export_arena(G)))
    r0, m0, a0 = outs[0]
    for r, m, a in outs[1:]:
        np.testing.assert_array_equal(m, m0)
        for k in a0:
            np.testing.assert_array_equal(a[k], a0[k])
        for k in ("rc", "chosen_plan", "mc_collisions", "n_candidates", "n_plans", "cost"):
            assert r[k] == r0[k], k


def test_separate_masks_flag():
    """PUMP_GRAPH_SEPARATE_MASKS (the request server's graphs): no edge order is laid out, every
    query keeps the masks in their own launch, and the results equal a default graph's."""
    wl = workload("indoor_4k", 9, 900)
    Gs = pump.Graph.build(wl.states, wl.goal_idx, wl.boxes, wl.xi, wl.radius, wl.n_particles, wl.n_waypoints,
                          wl.sigma, flags=pump.GRAPH_SEPARATE_MASKS)
    with pytest.raises(pump.PumpError):
        Gs.export("edge_order")
    rs = Gs.plan(plan_params(wl))
    assert rs["fused"] == 0
    r1, m1, a1, _ = run(wl, True)
    assert r1["fused"] == 1
    np.testing.assert_array_equal(Gs.export("masks"), m1)
    for k in ("rc", "chosen_plan", "mc_collisions", "n_candidates", "n_plans", "cost"):
        assert rs[k] == r1[k], k
    a = export_arena(Gs)
    for k in a1:
        np.testing.assert_array_equal(a[k], a1[k])


def test_queries_enqueued_without_waiting_equal_a_synchronous_query():
    """PUMP_NO_WAIT: explore-only queries enqueued back to back on one graph (fused and separate,
    with an L2-sized buffer write between them on the same stream) leave the arena and counters of
    a synchronous query; pump_plan_collect reads them."""
    import torch
    wl = workload("indoor_4k", 4, 2000)
    G = gpu_graph(wl)
    ref = G.plan(plan_params(wl, flags=pump.EXPLORE_ONLY))
    a_ref = export_arena(G)
    junk = torch.empty(1 << 26, dtype=torch.float32, device="cuda")
    for fused in (1, 0):
        with env(PUMP_FUSED_MASKS=fused):
            for _ in range(5):
                r = G.plan(plan_params(wl, flags=pump.EXPLORE_ONLY | pump.NO_WAIT))
                assert r["rc"] == pump.OK and r["n_candidates"] == 0 and r["fused"] == fused
                junk.zero_()
        c = G.collect()
        assert c["rc"] == pump.OK
        for k in ("n_candidates", "n_plans", "n_kept", "n_iterations", "n_groups", "n_goal"):
            assert c[k] == ref[k], k
        a = export_arena(G)
        for k in a_ref:
            np.testing.assert_array_equal(a[k], a_ref[k])
    bad = G.plan(plan_params(wl, flags=pump.NO_WAIT))  # no-wait needs explore-only
    assert bad["rc"] == pump.ERR_INVALID_ARG
    G.close()
