"""Launch-form autotuner for the batched form (pump_plan_batch).

For a batch it times, on the batch itself, the candidate forms of the Explore launch (the tile of
a query: CTAs per query, dominance table on chip or in global memory) and then those of the
edge-mask launch (the particle block: mask-word pairs a warp advances side by side; the edges a
warp takes at a time; the edges of one graph a block takes at a time), keeps the fastest of each, and remembers the choice in a JSON file
keyed by the batch's shape: query count, particle counts and sample-count bucket.  Later batches of
the same shape reuse it without timing.  Every form gives the same results; only the time
differs.

The cache lives at $PUMP_TUNE_CACHE, else ~/.cache/pump_gb300/tune.json.
"""
from __future__ import annotations

import json
import math
import os
from typing import Dict, List, Optional, Sequence, Tuple

from . import pump

CANDIDATES: Tuple[Tuple[int, int], ...] = ((16, 0), (16, 1), (8, 0), (8, 1), (4, 0))
# (word pairs, edges per warp take, edges per block item)
MASK_CANDIDATES: Tuple[Tuple[int, int, int], ...] = ((2, 4, 1024), (2, 1, 1024), (2, 4, 512), (2, 4, 2048),
                                                     (2, 16, 1024), (1, 4, 1024))


def cache_path() -> str:
    p = os.environ.get("PUMP_TUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "pump_gb300", "tune.json")


def _bucket(x: int) -> int:
    return int(2 ** round(math.log2(max(x, 1))))


def batch_key(graphs: Sequence["pump.Graph"]) -> str:
    """Shape of a batch: query count bucket, particle counts, largest sample-count and box-count buckets."""
    cnt = [g.counts() for g in graphs]
    Ns = sorted({int(c[4]) for c in cnt})
    n_max = max(int(c[0]) for c in cnt)
    return f"q{_bucket(len(graphs))}-N{'/'.join(map(str, Ns))}-n{_bucket(n_max)}"


def _load() -> Dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(d: Dict) -> None:
    p = cache_path()
    try:
        os.makedirs(os.path.dirname(p), exist_ok=True)
        tmp = p + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(d, f, indent=1, sort_keys=True)
        os.replace(tmp, p)
    except OSError:
        pass


def _timed(graphs, prm, cfg, reps: int, field: str) -> Optional[float]:
    ms = []
    for _ in range(reps + 1):
        rc, res = pump.plan_batch(graphs, prm, cfg)
        if rc not in (pump.OK, pump.ERR_INFEASIBLE):
            return None
        ms.append(res[0][field])
    return min(ms[1:])


def tune_batch(graphs: Sequence["pump.Graph"], params, reps: int = 2, force: bool = False,
               candidates: Sequence[Tuple[int, int]] = CANDIDATES,
               mask_candidates: Sequence[Tuple[int, int, int]] = MASK_CANDIDATES) -> Tuple["pump.BatchConfig", Dict]:
    """Best BatchConfig for this batch shape (timed now unless cached).  Returns (config, record)
    where the record holds the per-form Explore and mask times in ms."""
    key = batch_key(graphs)
    cache = _load()
    if not force and key in cache:
        rec = cache[key]
        return pump.BatchConfig(int(rec["cluster_size"]), int(rec["mbest_global"]), 0, int(rec.get("mask_pairs", 0)),
                                int(rec.get("mask_chunk", 0)), int(rec.get("mask_span", 0))), rec
    if isinstance(params, pump.PlanParams):
        params = [params] * len(graphs)
    prm = []
    for p in params:   # time Explore and the masks only
        q = pump.PlanParams.from_buffer_copy(p)
        q.flags |= pump.EXPLORE_ONLY
        prm.append(q)
    times: Dict[str, float] = {}
    best, best_ms = None, math.inf
    for cs, mg in candidates:
        t = _timed(graphs, prm, pump.BatchConfig(cs, mg, 0, 0, 0), reps, "ms_explore")
        if t is None:
            continue
        times[f"{cs}/{mg}"] = t
        if t < best_ms:
            best, best_ms = (cs, mg), t
    if best is None:
        best = (0, 0)
    mtimes: Dict[str, float] = {}
    mbest, mbest_ms = (0, 0, 0), math.inf
    for pairs, chunk, span in mask_candidates:
        t = _timed(graphs, prm, pump.BatchConfig(best[0], best[1], 0, pairs, chunk, span), reps, "ms_masks")
        if t is None:
            continue
        mtimes[f"{pairs}/{chunk}/{span}"] = t
        if t < mbest_ms:
            mbest, mbest_ms = (pairs, chunk, span), t
    rec = {"cluster_size": best[0], "mbest_global": best[1], "explore_ms": times, "mask_pairs": mbest[0],
           "mask_chunk": mbest[1], "mask_span": mbest[2], "mask_ms": mtimes}
    cache[key] = rec
    _store(cache)
    return pump.BatchConfig(best[0], best[1], 0, mbest[0], mbest[1], mbest[2]), rec
