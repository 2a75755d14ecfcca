"""Autotuner host logic on CPU: batch keys, the choice of the fastest form, and the JSON cache
(the batched launch itself is replaced by a fake with known timings)."""
import json

import numpy as np

from paper_1607_06886_gb300 import autotune, pump


class FakeGraph:
    def __init__(self, n, N):
        self._c = np.array([n, 10 * n, 0, 0, N, 10, N // 32, n], np.int64)

    def counts(self):
        return self._c


def test_batch_key_buckets():
    gs = [FakeGraph(1002, 64), FakeGraph(7000, 256), FakeGraph(3000, 128)]
    assert autotune.batch_key(gs) == "q4-N64/128/256-n8192"
    assert autotune.batch_key(gs[:1]) == "q1-N64-n1024"


def test_tune_picks_fastest_and_caches(tmp_path, monkeypatch):
    monkeypatch.setenv("PUMP_TUNE_CACHE", str(tmp_path / "tune.json"))
    timing = {(16, 0): 5.0, (16, 1): 4.0, (8, 0): 3.0, (8, 1): 3.5, (4, 0): 6.0}
    calls = []

    mask_timing = {(2, 4, 1024): 7.0, (2, 1, 1024): 8.0, (2, 4, 512): 7.5, (2, 4, 2048): 6.0, (2, 16, 1024): 6.5,
                   (1, 4, 1024): 9.0}

    def fake_batch(graphs, params, cfg=None, stream=None):
        calls.append((cfg.cluster_size, cfg.mbest_global))
        assert all(p.flags & pump.EXPLORE_ONLY for p in params)
        mk = mask_timing.get((cfg.mask_pairs, cfg.mask_chunk, cfg.mask_span), 10.0)
        return pump.OK, [{"ms_explore": timing[(cfg.cluster_size, cfg.mbest_global)], "ms_masks": mk} for _ in graphs]

    monkeypatch.setattr(pump, "plan_batch", fake_batch)
    gs = [FakeGraph(2000, 128), FakeGraph(4000, 128)]
    prm = pump.default_plan_params(alpha=0.01)
    cfg, rec = autotune.tune_batch(gs, prm, reps=1)
    assert (cfg.cluster_size, cfg.mbest_global) == (8, 0)
    # the mask form, timed with the chosen Explore form
    assert (cfg.mask_pairs, cfg.mask_chunk, cfg.mask_span) == (2, 4, 2048)
    assert rec["mask_ms"]["1/4/1024"] == 9.0
    assert prm.flags & pump.EXPLORE_ONLY == 0          # caller's params untouched
    stored = json.loads((tmp_path / "tune.json").read_text())
    assert stored[autotune.batch_key(gs)]["cluster_size"] == 8
    n_calls = len(calls)
    cfg2, _ = autotune.tune_batch(gs, prm, reps=1)     # cached: no timing
    assert len(calls) == n_calls and cfg2.cluster_size == 8
    assert (cfg2.mask_pairs, cfg2.mask_chunk, cfg2.mask_span) == (2, 4, 2048)


def test_tune_skips_failing_forms(tmp_path, monkeypatch):
    monkeypatch.setenv("PUMP_TUNE_CACHE", str(tmp_path / "tune.json"))

    def fake_batch(graphs, params, cfg=None, stream=None):
        if cfg.cluster_size == 16:
            return pump.ERR_CUDA, []
        return pump.OK, [{"ms_explore": float(cfg.cluster_size + cfg.mbest_global), "ms_masks": 1.0} for _ in graphs]

    monkeypatch.setattr(pump, "plan_batch", fake_batch)
    cfg, rec = autotune.tune_batch([FakeGraph(1000, 32)], pump.default_plan_params(alpha=0.05), reps=1)
    assert (cfg.cluster_size, cfg.mbest_global) == (4, 0)
    assert "16/0" not in rec["explore_ms"]
