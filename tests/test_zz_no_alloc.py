"""pump_explore_noalloc: Explore for callers that cannot allocate device memory while they plan.

Such callers (a robot's real-time control loop that reserves its device memory at start-up, an
embedded runtime with a fixed memory budget, a process whose allocator belongs to a host
framework) hand the library every input and output buffer; the entry point keeps its own scratch
in a fixed device array and calls no allocator.  These tests call it through the C ABI on
caller-owned torch buffers, twice in a row on different graphs and once more on the first, in each
Explore form (thread-block cluster, grid-wide kernel, stepwise launches), and check each result
bit for bit against the allocating entry point (pump_graph_from_csr + pump_explore + pump_export);
one graph is also checked record by record against the oracle's Explore.  The file sorts last so
that a run stopping at the first failure has run every other test first."""
import numpy as np
import pytest

from oracle import cpu
from paper_1607_06886_gb300 import inputs, pump

from _util import assert_arena_equal

pytestmark = pytest.mark.gpu

FIELDS = ("plan_head", "plan_parent", "plan_cost", "plan_mask", "plan_popc", "plan_created", "plan_expanded")
MODES = {"cluster": 0, "grid": pump.EXPLORE_GRID, "stepwise": pump.STEPWISE}
CAP = 1 << 18


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    pump.load()
    pump.use_torch_allocator()
    yield


def reference(g, goal, prm):
    G = pump.Graph.from_csr(g.n, g.row_ptr, g.col, g.ecost, g.emask, g.n_words * 32, 0, goal)
    st = G.explore(prm, radius=g.radius)
    assert st["rc"] == pump.OK
    out = {k: G.export(k) for k in FIELDS + ("goal_plans",)}
    G.close()
    return st, out


def no_alloc(g, goal, prm, capacity):
    import torch
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    is_goal = np.zeros(g.n, np.uint8)
    is_goal[goal] = 1
    w = g.n_words
    out = {"plan_head": torch.full((capacity,), -7, dtype=torch.int32, device="cuda"),
           "plan_parent": torch.full((capacity,), -7, dtype=torch.int32, device="cuda"),
           "plan_cost": torch.full((capacity,), -1.0, dtype=torch.float32, device="cuda"),
           "plan_mask": torch.zeros((capacity, w), dtype=torch.int32, device="cuda"),
           "plan_popc": torch.zeros((capacity,), dtype=torch.int32, device="cuda"),
           "plan_created": torch.zeros((capacity,), dtype=torch.int32, device="cuda"),
           "plan_expanded": torch.zeros((capacity,), dtype=torch.int32, device="cuda"),
           "goal_plans": torch.full((capacity,), -7, dtype=torch.int32, device="cuda")}
    ins = [dev(g.row_ptr), dev(g.col), dev(g.ecost), dev(g.emask.view(np.int32)), dev(is_goal)]
    st = pump.explore_noalloc(g.n, ins[0], ins[1], ins[2], ins[3], w * 32, 0, ins[4], g.radius, prm, capacity, out)
    torch.cuda.synchronize()
    P = st["n_plans"]
    assert 1 <= P < capacity, (P, capacity)  # the run stayed inside the caller's arena
    res = {k: out[k][:P].cpu().numpy() for k in FIELDS}
    res["plan_mask"] = res["plan_mask"].view(np.uint32)
    res["goal_plans"] = out["goal_plans"][:st["n_goal"]].cpu().numpy()
    return st, res


def check_same(st_a, out_a, st_b, out_b):
    assert st_b["rc"] == pump.OK
    for k in ("n_plans", "n_candidates", "n_kept", "n_iterations", "n_groups", "n_goal"):
        assert st_a[k] == st_b[k], k
    for k in FIELDS:
        a, b = out_a[k], out_b[k]
        if a.dtype == np.float32:
            a, b = a.view(np.uint32), b.view(np.uint32)
        np.testing.assert_array_equal(a.reshape(b.shape), b, err_msg=k)
    np.testing.assert_array_equal(out_a["goal_plans"], out_b["goal_plans"])


def graphs():
    g1 = inputs.random_explore_graph(1500, 24, 128, 31, radius=1.3, bit_prob=0.005, hot_edge_frac=0.06,
                                     hot_bit_prob=0.12)
    g2 = inputs.random_explore_graph(900, 18, 64, 32, radius=1.2, bit_prob=0.01, hot_edge_frac=0.08,
                                     hot_bit_prob=0.2)
    return (g1, [1, 2, 700]), (g2, [5, 400])


@pytest.mark.parametrize("mode", list(MODES))
def test_no_alloc_explore_matches_allocating_entry_point(mode):
    (g1, goal1), (g2, goal2) = graphs()
    prm1 = pump.default_plan_params(alpha=0.01, flags=pump.NO_EARLY_STOP | MODES[mode])
    prm2 = pump.default_plan_params(alpha=0.03, flags=MODES[mode])
    ref1, ref2 = reference(g1, goal1, prm1), reference(g2, goal2, prm2)
    check_same(*ref1, *no_alloc(g1, goal1, prm1, CAP))   # first call
    check_same(*ref2, *no_alloc(g2, goal2, prm2, CAP))   # second call in a row, other graph
    check_same(*ref1, *no_alloc(g1, goal1, prm1, CAP))   # scratch left by the second call is not read


def test_no_alloc_explore_matches_oracle():
    """The same run against the oracle's Explore (Algorithm 4), record by record."""
    (g, goal), _ = graphs()
    N = g.n_words * 32
    alpha, eta, lam = 0.01, 2.0, 0.5
    kmin, kmax = cpu.cp_thresholds(alpha, eta, N)
    ex = cpu.explore(g.n, g.row_ptr, g.col, g.ecost, g.emask, 0, goal, kmin, kmax, lam, g.radius, flags=1)
    prm = pump.default_plan_params(alpha=alpha, eta=eta, lam=lam, flags=pump.NO_EARLY_STOP)
    for _ in range(2):
        st, out = no_alloc(g, goal, prm, CAP)
        assert st["rc"] == pump.OK and ex["status"] == cpu.OK
        assert st["n_plans"] == ex["n_plans"] and st["n_candidates"] == ex["n_candidates"]
        assert st["n_iterations"] == ex["n_iterations"] and st["n_goal"] == ex["n_goal"]
        assert_arena_equal(out, ex, g.n_words)


def test_no_alloc_rejects_host_pointers_and_oversized_problems():
    import torch
    g = inputs.random_explore_graph(50, 5, 32, 3)
    prm = pump.default_plan_params(alpha=0.05)
    out = {k: torch.zeros(64, dtype=torch.int32, device="cuda") for k in FIELDS + ("goal_plans",)}
    out["plan_cost"] = torch.zeros(64, dtype=torch.float32, device="cuda")
    is_goal = np.zeros(g.n, np.uint8)
    st = pump.explore_noalloc(g.n, g.row_ptr, g.col, g.ecost, g.emask, 32, 0, is_goal, g.radius, prm, 64, out)
    assert st["rc"] == pump.ERR_INVALID_ARG          # host inputs
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    big = pump.default_plan_params(alpha=0.05, max_plans=1 << 30)
    st = pump.explore_noalloc(g.n, dev(g.row_ptr), dev(g.col), dev(g.ecost), dev(g.emask.view(np.int32)), 32, 0,
                              dev(is_goal), g.radius, big, 1 << 30, out)
    assert st["rc"] == pump.ERR_INVALID_ARG          # scratch for 2^30 plans exceeds the fixed array
    # a large caller capacity with a small max_plans sizes the scratch by max_plans: accepted
    small = pump.default_plan_params(alpha=0.05, max_plans=60)
    st = pump.explore_noalloc(g.n, dev(g.row_ptr), dev(g.col), dev(g.ecost), dev(g.emask.view(np.int32)), 32, 0,
                              dev(is_goal), g.radius, small, 1 << 30, out)
    assert st["rc"] in (pump.OK, pump.ERR_CAPACITY)
