"""Serving with continuous batching (pump_server): requests arriving while others run are admitted
as slots and device memory free up, and run concurrently on their own streams.  Each served result
must equal the result of the same request run alone (graph build + pump_plan): every result field,
the path and the Monte Carlo count, bit for bit.  Also checks memory-based admission, counters and
argument errors."""
import time

import numpy as np
import pytest

from paper_1607_06886_gb300 import inputs, pump

from _util import gpu_graph, plan_params

pytestmark = pytest.mark.gpu

KEYS = ("status", "chosen_plan", "cost", "popc", "cp_hat", "cp_mc", "mc_collisions", "n_candidates", "n_kept",
        "n_plans", "n_iterations", "n_groups", "n_goal", "n_certified", "path_len", "path_truncated")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    pump.load()
    pump.use_torch_allocator()
    yield


def requests():
    wls = [inputs.make_workload("three_box_1k", s, 200 + 40 * s) for s in range(4)]
    wls += [inputs.make_workload("indoor_4k", s, 300 + 60 * s) for s in range(4)]
    wls += inputs.batch_workloads(4, seed=500, n_range=(500, 1500))
    return wls


@pytest.fixture(scope="module")
def alone():
    out = []
    for wl in requests():
        G = gpu_graph(wl)
        r = G.plan(plan_params(wl, n_mc=2000), path_cap=4097)
        G.close()
        out.append((wl, r))
    return out


def submit(srv, wl):
    return srv.submit(wl.states, wl.goal_idx, wl.boxes, wl.xi, wl.radius, wl.n_particles, wl.n_waypoints, wl.sigma,
                      plan_params(wl, n_mc=2000))


def check(ref, got):
    for k in KEYS:
        assert got[k] == ref[k], (k, got[k], ref[k])
    np.testing.assert_array_equal(got["path"], ref["path"])
    assert got["latency_ms"] > 0


@pytest.mark.parametrize("slots", [1, 4, 8])
def test_served_results_equal_alone(alone, slots):
    srv = pump.Server(slots, 8 << 30)
    tickets = [submit(srv, wl) for wl, _ in alone]
    for (wl, ref), t in zip(alone, tickets):
        check(ref, srv.wait(t))
    st = srv.stats()
    assert st["submitted"] == st["completed"] == len(alone) and st["queued"] == 0 and st["running"] == 0
    assert st["peak_running"] <= slots
    srv.close()


def test_staggered_arrivals_are_admitted_while_others_run(alone):
    srv = pump.Server(4, 8 << 30)
    tickets = []
    for wl, _ in alone:
        tickets.append(submit(srv, wl))
        time.sleep(0.002)
    for (wl, ref), t in zip(alone, tickets):
        check(ref, srv.wait(t))
    assert srv.stats()["peak_running"] >= 2
    srv.close()


def test_memory_budget_serialises_admission(alone):
    """With a budget smaller than any request, each runs alone (admitted only when nothing runs)."""
    srv = pump.Server(8, 1)
    tickets = [submit(srv, wl) for wl, _ in alone[:5]]
    for (wl, ref), t in zip(alone[:5], tickets):
        check(ref, srv.wait(t))
    assert srv.stats()["peak_running"] == 1
    srv.close()


def test_wait_timeout_and_unknown_ticket(alone):
    srv = pump.Server(1, 8 << 30)
    wl = alone[7][0]
    t = submit(srv, wl)
    r = srv.wait(t, timeout=0.0)
    assert r["rc"] in (pump.ERR_TIMEOUT, pump.OK, pump.ERR_INFEASIBLE)
    if r["rc"] == pump.ERR_TIMEOUT:
        r = srv.wait(t)
    check(alone[7][1], r)
    assert srv.wait(t, timeout=0.0)["rc"] == pump.ERR_INVALID_ARG   # forgotten after completion
    assert srv.wait(12345, timeout=0.0)["rc"] == pump.ERR_INVALID_ARG
    srv.close()


def test_destroy_drops_queued_requests(alone):
    srv = pump.Server(1, 8 << 30)
    for wl, _ in alone:
        submit(srv, wl)
    srv.close()   # admitted one finishes, the rest are dropped; no hang


def test_bad_requests_are_rejected():
    srv = pump.Server(2, 1 << 30)
    wl = inputs.make_workload("three_box_1k", 0, 100)
    with pytest.raises(pump.PumpError):
        srv.submit(wl.states, wl.goal_idx, wl.boxes, wl.xi, wl.radius, 48, wl.n_waypoints, wl.sigma, plan_params(wl))
    with pytest.raises(pump.PumpError):
        srv.submit(wl.states[:1], wl.goal_idx, wl.boxes, wl.xi, wl.radius, 32, wl.n_waypoints, wl.sigma, plan_params(wl))
    srv.close()
    with pytest.raises(pump.PumpError):
        pump.Server(0, 1 << 30)
