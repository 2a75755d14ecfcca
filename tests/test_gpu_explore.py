"""Explore (Algorithm 4) on the GPU vs the CPU oracle, bit for bit, on imported graphs.

Both sides receive the same seeded random graph (CSR, edge costs, edge masks) and must produce
the same arena: plan ids, heads, parents, cost bits, masks, creation and expansion group indices,
the same P_goal in PlanSelection order, and the same counters.  Covers the thread-block cluster
kernel (cluster sizes 16, 8 and 4; dominance table on chip and in global memory; groups larger than
the on-chip candidate cache; next group indices beyond the counted window), the grid-wide
cooperative kernel and the stepwise launches, several particle counts, CP cutoffs, early stop on
and off, and the degenerate cases."""
import numpy as np
import pytest

from oracle import cpu
from paper_1607_06886_gb300 import inputs, pump

from _util import assert_arena_equal

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    pump.load()
    pump.use_torch_allocator()
    yield


def run_both(g, start, goal, alpha, eta, lam, flags=0, max_plans=1 << 22, max_iter=1 << 20, N=None):
    N = N or g.n_words * 32
    kmin, kmax = cpu.cp_thresholds(alpha, eta, N)
    ex = cpu.explore(g.n, g.row_ptr, g.col, g.ecost, g.emask, start, goal, kmin, kmax, lam, g.radius,
                     max_plans=max_plans, flags=1 if flags & pump.NO_EARLY_STOP else 0, max_iterations=max_iter)
    G = pump.Graph.from_csr(g.n, g.row_ptr, g.col, g.ecost, g.emask, N, start, goal)
    prm = pump.default_plan_params(alpha=alpha, eta=eta, lam=lam, max_plans=max_plans, max_iterations=max_iter,
                                   flags=flags)
    st = G.explore(prm, radius=g.radius)
    return G, st, ex


CASES = [
    # n, degree, N, alpha, eta, lam, flags, seed
    (60, 6, 32, 0.05, 2.0, 0.5, 0, 0),
    (300, 12, 32, 0.05, 2.0, 0.5, 0, 1),
    (300, 12, 64, 0.02, 2.0, 0.5, pump.NO_EARLY_STOP, 2),
    (500, 20, 128, 0.01, 2.0, 0.5, 0, 3),
    (500, 20, 128, 0.01, 2.0, 0.5, pump.NO_EARLY_STOP, 4),
    (400, 16, 256, 0.01, 2.0, 0.25, 0, 5),
    (250, 10, 1024, 0.02, 2.0, 1.0, pump.NO_EARLY_STOP, 6),
    (800, 30, 128, 0.05, 2.0, 0.5, pump.NO_EARLY_STOP, 7),
    (300, 12, 32, 0.5, 2.0, 0.5, pump.NO_EARLY_STOP, 8),
    (300, 12, 32, 0.05, 2.0, 0.004, pump.NO_EARLY_STOP, 12),
]

MODES = {"cluster": 0, "grid": pump.EXPLORE_GRID, "stepwise": pump.STEPWISE}


def check_explore(n, deg, N, alpha, eta, lam, flags, seed):
    g = inputs.random_explore_graph(n, deg, N, seed, radius=1.3, bit_prob=0.01, hot_edge_frac=0.08,
                                    hot_bit_prob=0.15)
    goal = [n - 1, n - 2, n // 2]
    G, st, ex = run_both(g, 0, goal, alpha, eta, lam, flags=flags)
    assert st["rc"] == pump.OK and ex["status"] == cpu.OK
    assert ex["n_plans"] > 1
    assert st["n_plans"] == ex["n_plans"]
    assert st["n_candidates"] == ex["n_candidates"]
    assert st["n_kept"] == ex["n_kept"]
    assert st["n_iterations"] == ex["n_iterations"]
    assert st["n_groups"] == ex["n_groups_expanded"]
    assert st["n_goal"] == ex["n_goal"]
    assert_arena_equal({k: G.export(k) for k in ("plan_head", "plan_parent", "plan_cost", "plan_mask", "plan_popc",
                                                 "plan_created", "plan_expanded", "goal_plans")}, ex, g.n_words)


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("n,deg,N,alpha,eta,lam,flags,seed", CASES)
def test_explore_bit_exact(n, deg, N, alpha, eta, lam, flags, seed, mode):
    check_explore(n, deg, N, alpha, eta, lam, flags | MODES[mode], seed)


@pytest.mark.parametrize("cluster,mbest_global", [(8, False), (4, False), (16, True), (4, True)])
@pytest.mark.parametrize("case", [1, 4, 6, 7, 9])
def test_explore_cluster_forms(monkeypatch, cluster, mbest_global, case):
    """The cluster kernel at other cluster sizes and with the dominance table in global memory."""
    monkeypatch.setenv("PUMP_EXPLORE_CLUSTER", str(cluster))
    monkeypatch.setenv("PUMP_EXPLORE_MBEST_GLOBAL", "1" if mbest_global else "0")
    check_explore(*CASES[case])


def test_explore_cluster_large_groups(monkeypatch):
    """Groups with more candidates than four CTAs cache on chip: candidates are recomputed from the
    group list and members read back from the arena after an extra barrier."""
    monkeypatch.setenv("PUMP_EXPLORE_CLUSTER", "4")
    g = inputs.random_explore_graph(4002, 33, 128, 11, radius=1.25, bit_prob=0.003, hot_edge_frac=0.05,
                                    hot_bit_prob=0.1)
    G, st, ex = run_both(g, 0, [1, 2, 3], 0.01, 2.0, 0.5, flags=pump.NO_EARLY_STOP)
    assert st["rc"] == pump.OK and st["n_candidates"] == ex["n_candidates"]
    cre, exp_ = ex["t_created"], ex["e_expanded"]
    deg = np.diff(g.row_ptr)
    per_group = np.bincount(exp_[exp_ >= 0], weights=deg[ex["head"][exp_ >= 0]])
    assert per_group.max() > 4 * 2048
    assert_arena_equal({k: G.export(k) for k in ("plan_head", "plan_parent", "plan_cost", "plan_mask", "plan_popc",
                                                 "plan_created", "plan_expanded", "goal_plans")}, ex, g.n_words)


def test_explore_paper_scale_graph():
    """A random graph with the size of the indoor 4000-sample workload (4002 nodes, mean degree 33,
    N = 128, CP target 1 %), run to exhaustion."""
    g = inputs.random_explore_graph(4002, 33, 128, 11, radius=1.25, bit_prob=0.003, hot_edge_frac=0.05,
                                    hot_bit_prob=0.1)
    G, st, ex = run_both(g, 0, [1, 2, 3], 0.01, 2.0, 0.5, flags=pump.NO_EARLY_STOP)
    assert st["rc"] == pump.OK and st["n_candidates"] == ex["n_candidates"] > 100000
    assert_arena_equal({k: G.export(k) for k in ("plan_head", "plan_parent", "plan_cost", "plan_mask", "plan_popc",
                                                 "plan_created", "plan_expanded", "goal_plans")}, ex, g.n_words)


def test_explore_repeatable():
    g = inputs.random_explore_graph(700, 20, 128, 21, radius=1.3, bit_prob=0.01)
    G = pump.Graph.from_csr(g.n, g.row_ptr, g.col, g.ecost, g.emask, 128, 0, [5])
    prm = pump.default_plan_params(alpha=0.02, flags=pump.NO_EARLY_STOP)
    G.explore(prm, radius=g.radius)
    a = {k: G.export(k) for k in ("plan_head", "plan_parent", "plan_cost", "plan_mask", "plan_expanded")}
    G.explore(prm, radius=g.radius)
    b = {k: G.export(k) for k in ("plan_head", "plan_parent", "plan_cost", "plan_mask", "plan_expanded")}
    for k in a:
        np.testing.assert_array_equal(a[k], b[k])


def test_explore_start_is_goal():
    g = inputs.random_explore_graph(50, 5, 32, 3, radius=1.0)
    G, st, ex = run_both(g, 7, [7], 0.05, 2.0, 0.5)
    assert st["rc"] == pump.OK and st["n_plans"] == 1 and st["n_candidates"] == 0 and st["n_iterations"] == 0
    assert G.export("goal_plans").tolist() == [0]


def test_explore_start_without_edges():
    n = 10
    row_ptr = np.zeros(n + 1, np.int32)
    row_ptr[2:] = 1
    col = np.array([3], np.int32)
    G = pump.Graph.from_csr(n, row_ptr, col, np.array([0.5], np.float32), np.zeros((1, 1), np.uint32), 32, 0, [3])
    st = G.explore(pump.default_plan_params(alpha=0.05), radius=1.0)
    ex = cpu.explore(n, row_ptr, col, np.array([0.5], np.float32), np.zeros((1, 1), np.uint32), 0, [3], 1, 4, 0.5, 1.0)
    assert st["rc"] == pump.OK and st["n_plans"] == 1 == ex["n_plans"] and st["n_goal"] == 0
    assert st["n_iterations"] == ex["n_iterations"] == 1


def test_explore_empty_graph():
    n = 5
    G = pump.Graph.from_csr(n, np.zeros(n + 1, np.int32), np.zeros(0, np.int32), np.zeros(0, np.float32),
                            np.zeros((0, 2), np.uint32), 64, 0, [4])
    st = G.explore(pump.default_plan_params(alpha=0.05), radius=1.0)
    assert st["rc"] == pump.OK and st["n_plans"] == 1 and st["n_candidates"] == 0


def test_explore_zero_alpha_keeps_nothing():
    g = inputs.random_explore_graph(100, 8, 32, 4, radius=1.0)
    G, st, ex = run_both(g, 0, [1], 0.0, 2.0, 0.5)
    assert st["rc"] == pump.OK and st["n_plans"] == ex["n_plans"] == 1
    assert st["n_candidates"] == ex["n_candidates"] > 0 and st["n_kept"] == 0


def test_explore_capacity_error_matches_oracle():
    g = inputs.random_explore_graph(300, 12, 32, 9, radius=1.3)
    G, st, ex = run_both(g, 0, [1], 0.05, 2.0, 0.5, flags=pump.NO_EARLY_STOP, max_plans=40)
    assert ex["status"] == cpu.ERR_CAPACITY
    assert st["rc"] == pump.ERR_CAPACITY


def test_explore_iteration_cap_matches_oracle():
    g = inputs.random_explore_graph(300, 12, 32, 10, radius=1.3)
    G, st, ex = run_both(g, 0, [1], 0.05, 2.0, 0.5, flags=pump.NO_EARLY_STOP, max_iter=3)
    assert ex["status"] == cpu.ERR_TIMEOUT
    assert st["rc"] == pump.ERR_TIMEOUT


def test_imported_graph_rejects_geometry_calls():
    g = inputs.random_explore_graph(20, 3, 32, 0)
    G = pump.Graph.from_csr(g.n, g.row_ptr, g.col, g.ecost, g.emask, 32, 0, [1])
    with pytest.raises(pump.PumpError):
        G.edge_masks()
    with pytest.raises(pump.PumpError):
        G.certify([0], 10, 4, 0)


def test_from_csr_rejects_bad_graphs():
    with pytest.raises(pump.PumpError):   # self loop
        pump.Graph.from_csr(3, [0, 1, 1, 1], [0], [0.5], np.zeros((1, 1), np.uint32), 32, 0, [1])
    with pytest.raises(pump.PumpError):   # unsorted row
        pump.Graph.from_csr(3, [0, 2, 2, 2], [2, 1], [0.5, 0.5], np.zeros((2, 1), np.uint32), 32, 0, [1])
    with pytest.raises(pump.PumpError):   # negative cost
        pump.Graph.from_csr(3, [0, 1, 1, 1], [1], [-0.5], np.zeros((1, 1), np.uint32), 32, 0, [1])
    with pytest.raises(pump.PumpError):   # N not a multiple of 32
        pump.Graph.from_csr(3, [0, 1, 1, 1], [1], [0.5], np.zeros((1, 1), np.uint32), 48, 0, [1])
