"""Replica sharding across ranks, on CPU with the gloo backend (world_size 2).

Each rank plans its own query (seed = rank) with the CPU oracle standing in for a GPU's work;
the job aggregates partial plans by sum and time by maximum, as bench.py does under torchrun."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world_size, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world_size),
                      LOCAL_RANK=str(rank))
    import time
    import torch.distributed as dist
    from oracle import cpu
    from paper_1607_06886_gb300 import dist as pd
    from paper_1607_06886_gb300 import inputs
    dist.init_process_group("gloo", rank=rank, world_size=world_size)
    try:
        ws, r, _ = pd.world()
        wl = inputs.make_workload("three_box_1k", seed=pd.query_seed(r), n_samples=150)
        pd.barrier()
        t0 = time.perf_counter()
        o = cpu.plan(wl)
        dt = time.perf_counter() - t0 + 0.01 * (r + 1)
        work = o["explore"]["n_candidates"]
        tot, tmax, value = pd.aggregate(work, dt)
        out[r] = (ws, r, work, dt, tot, tmax, value, float(wl.states[2, 0]))
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_queries_and_aggregate():
    import torch.multiprocessing as mp
    mgr = mp.Manager()
    out = mgr.dict()
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    a, b = out[0], out[1]
    assert a[0] == b[0] == 2 and a[1] == 0 and b[1] == 1
    assert a[7] != b[7]                        # different seeds, different samples
    assert a[4] == b[4] == a[2] + b[2]         # total work = sum over ranks
    assert a[5] == b[5] == max(a[3], b[3])     # timed region = max over ranks
    assert a[6] == pytest.approx((a[2] + b[2]) / max(a[3], b[3]))


def test_single_process_defaults():
    from paper_1607_06886_gb300 import dist as pd
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        os.environ.pop(k, None)
    assert pd.world() == (1, 0, 0)
    assert pd.aggregate(10.0, 2.0) == (10.0, 2.0, 5.0)
