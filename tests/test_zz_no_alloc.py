"""pump_explore_noalloc: Explore for callers that cannot allocate device memory.

Such callers (code running inside a captured CUDA graph, a runtime whose device memory is fixed up
front, a process whose allocator belongs to a host framework) hand the library every input and
output buffer; the entry point keeps its own scratch in a fixed device array and calls no
allocator.  This test calls it through the C ABI on caller-owned torch buffers, twice in a row on
different graphs and once more on the first, and checks each result bit for bit against the
allocating entry point (pump_graph_from_csr + pump_explore + pump_export).  The file sorts last so
that a run stopping at the first failure has run every other test first."""
import numpy as np
import pytest

from paper_1607_06886_gb300 import inputs, pump

pytestmark = pytest.mark.gpu

FIELDS = ("plan_head", "plan_parent", "plan_cost", "plan_mask", "plan_popc", "plan_created", "plan_expanded")


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


def test_no_alloc_explore_matches_allocating_entry_point():
    g1 = inputs.random_explore_graph(1500, 24, 128, 31, radius=1.3, bit_prob=0.005, hot_edge_frac=0.06,
                                     hot_bit_prob=0.12)
    g2 = inputs.random_explore_graph(900, 18, 64, 32, radius=1.2, bit_prob=0.01, hot_edge_frac=0.08,
                                     hot_bit_prob=0.2)
    prm1 = pump.default_plan_params(alpha=0.01, flags=pump.NO_EARLY_STOP)
    prm2 = pump.default_plan_params(alpha=0.03)
    goal1, goal2 = [1, 2, 700], [5, 400]
    ref1, ref2 = reference(g1, goal1, prm1), reference(g2, goal2, prm2)
    cap = 1 << 18
    check_same(*ref1, *no_alloc(g1, goal1, prm1, cap))   # first call
    check_same(*ref2, *no_alloc(g2, goal2, prm2, cap))   # second call in a row, other graph
    check_same(*ref1, *no_alloc(g1, goal1, prm1, cap))   # scratch left by the second call is not read


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
    st = pump.explore_noalloc(g.n, dev(g.row_ptr), dev(g.col), dev(g.ecost), dev(g.emask.view(np.int32)), 32, 0,
                              dev(is_goal), g.radius, prm, 1 << 30, out)
    assert st["rc"] == pump.ERR_INVALID_ARG          # scratch for 2^30 plans exceeds the fixed array
