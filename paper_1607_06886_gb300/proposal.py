"""Learned sampling proposal: data collection, training and paired evaluation.

The paper draws SampleFree uniformly (Algorithm 3).  This extension learns where certified plans
run and proposes part of the samples there:

1. collect  - plain PUMP (uniform samples, the full pipeline of graph build, Explore,
              PlanSelection and MC certification) on seeded training environments through the
              request server; every certified plan gives its intermediate states as targets.
2. train    - the BF16 network (pump_mlp_*) learns, for an environment's features and eight
              normals, a state near one of those targets (winner takes all), with the training
              loop on the device.
3. evaluate - on held-out environments, the same query planned twice: all samples uniform, and
              the same first uniform samples plus proposals kept clear of the boxes (LEARNED of
              4000 by default); success and certified cost are compared pair by pair.

Features of an environment (204 floats): its boxes (lo, hi) in scene order, zero rows up to 32
slots, then the start and goal states.  Network input: the features, the eight normals, zeros
up to 224.  Hidden widths 3 x 256, output 16 (the first six used).
"""
from __future__ import annotations

import dataclasses
import time
from typing import Dict, List, Optional, Sequence

import numpy as np

from . import inputs, pump

BOX_SLOTS = 32
FEAT = BOX_SLOTS * 6 + 12
DIMS = (224, 256, 256, 256, 16)
MAX_TARGETS = 16
# Proposal settings chosen on validation environments (seeds 2,000,000 on), not on the held-out
# evaluation set: proposals closer than CLEARANCE to a box are dropped (see mixed_workload), and
# LEARNED of a query's 4000 samples are proposals.
CLEARANCE = 0.10
LEARNED = 1000
VALIDATION_SEED0 = 2_000_000
HELDOUT_SEED0 = 1_000_000


def env_features(boxes, start, goal) -> np.ndarray:
    bx = np.asarray(boxes, np.float32).reshape(-1, 6)
    if bx.shape[0] > BOX_SLOTS:
        raise ValueError(f"at most {BOX_SLOTS} boxes")
    f = np.zeros(FEAT, np.float32)
    f[:bx.size] = bx.ravel()
    f[BOX_SLOTS * 6:BOX_SLOTS * 6 + 6] = start
    f[BOX_SLOTS * 6 + 6:] = goal
    return f


def workload_features(wl: inputs.Workload) -> np.ndarray:
    return env_features(wl.boxes, wl.states[wl.start_idx], wl.states[1])


def plan_params(wl: inputs.Workload) -> pump.PlanParams:
    return pump.default_plan_params(alpha=wl.alpha, eta=wl.eta, lam=wl.lam, n_mc=wl.n_mc, mc_substeps=wl.mc_substeps,
                                    mc_seed=wl.mc_seed)


def run_queries(wls: Sequence[inputs.Workload], slots: int = 8, device_bytes: int = 64 << 30) -> List[Dict]:
    """Plan every workload through the request server (continuous batching over `slots`)."""
    srv = pump.Server(slots, device_bytes)
    try:
        tickets = [srv.submit(w.states, w.goal_idx, w.boxes, w.xi, w.radius, w.n_particles, w.n_waypoints, w.sigma,
                              plan_params(w)) for w in wls]
        return [srv.wait(t) for t in tickets]
    finally:
        srv.close()


def certified(res: Dict) -> bool:
    return res["rc"] == pump.OK and res["status"] == pump.OK and len(res["path"]) >= 2


@dataclasses.dataclass
class Dataset:
    seeds: np.ndarray      # (n,) environment seeds
    feat: np.ndarray       # (n, 204) float32
    targets: np.ndarray    # (n, MAX_TARGETS, 6) float32
    n_targets: np.ndarray  # (n,) int32
    stats: Dict
    cp_mc: Optional[np.ndarray] = None  # (n,) Monte Carlo CP of each environment's certified plan

    def subset(self, keep: np.ndarray) -> "Dataset":
        keep = np.asarray(keep, bool)
        return Dataset(self.seeds[keep], self.feat[keep], self.targets[keep], self.n_targets[keep],
                       dict(self.stats, kept=int(keep.sum())),
                       None if self.cp_mc is None else self.cp_mc[keep])

    def safest(self, max_cp: float) -> "Dataset":
        """Only the environments whose certified plan has a Monte Carlo CP of at most max_cp."""
        return self.subset(self.cp_mc <= max_cp)


def collect(seeds: Sequence[int], n_samples: int = 4000, slots: int = 8, chunk: int = 512) -> Dataset:
    """Certified plain-PUMP plans on the environments `seeds`; environments without a certified
    plan, or whose plan has no intermediate state, are left out."""
    t0 = time.perf_counter()
    keep_seed, feats, tgs, nts, cps = [], [], [], [], []
    solved = 0
    for c0 in range(0, len(seeds), chunk):
        wls = [inputs.proposal_workload(int(s), n_samples) for s in seeds[c0:c0 + chunk]]
        for w, r in zip(wls, run_queries(wls, slots)):
            if not certified(r):
                continue
            solved += 1
            mid = w.states[r["path"][1:-1]][:MAX_TARGETS]
            if len(mid) == 0:
                continue
            t = np.zeros((MAX_TARGETS, 6), np.float32)
            t[:len(mid)] = mid
            keep_seed.append(w.seed)
            feats.append(workload_features(w))
            tgs.append(t)
            nts.append(len(mid))
            cps.append(float(r["cp_mc"]))
    n = len(keep_seed)
    return Dataset(seeds=np.asarray(keep_seed, np.int64), feat=np.asarray(feats, np.float32).reshape(n, FEAT),
                   targets=np.asarray(tgs, np.float32).reshape(n, MAX_TARGETS, 6),
                   n_targets=np.asarray(nts, np.int32),
                   stats={"environments": len(seeds), "certified": solved, "kept": n,
                          "mean_targets": float(np.mean(nts)) if nts else 0.0,
                          "seconds": time.perf_counter() - t0},
                   cp_mc=np.asarray(cps, np.float64))


WTA, PATH_INDEXED = 0, 1


def make_model(seed: int = 0, loss: int = PATH_INDEXED) -> pump.MLP:
    """The proposal network; `loss` WTA (winner takes all over the path's states) or
    PATH_INDEXED (the first latent picks the fraction along the path)."""
    m = pump.MLP(DIMS, seed)
    m.set_loss(loss, FEAT)
    return m


def train(model: pump.MLP, data: Dataset, steps: int, batch: int = 2048, lr: float = 1e-3, seed: int = 0,
          vmax: float = inputs.VEL_MAX) -> Dict:
    model.set_data(data.feat, data.targets, data.n_targets)
    t0 = time.perf_counter()
    trace = model.train(batch, steps, lr, vmax, seed)
    return {"steps": int(steps), "batch": int(batch), "lr": float(lr), "seconds": time.perf_counter() - t0,
            "loss_first": float(np.mean(trace[:max(1, min(50, len(trace)))])) if len(trace) else None,
            "loss_last": float(np.mean(trace[-max(1, min(50, len(trace))):])) if len(trace) else None,
            "trace": trace}


def box_distance(p: np.ndarray, boxes: np.ndarray) -> np.ndarray:
    """Euclidean distance from each position p (n x 3) to the nearest closed box (0 inside one)."""
    bx = np.asarray(boxes, np.float32).reshape(-1, 6)
    if bx.shape[0] == 0:
        return np.full(p.shape[0], np.inf)
    d = np.maximum(np.maximum(bx[None, :, :3] - p[:, None, :], 0.0), p[:, None, :] - bx[None, :, 3:])
    return np.sqrt((d * d).sum(axis=2)).min(axis=1)


def mixed_workload(model: pump.MLP, wl: inputs.Workload, n_learned: int, seed: Optional[int] = None,
                   vmax: float = inputs.VEL_MAX, spread: float = 0.0, clearance: float = CLEARANCE) -> inputs.Workload:
    """The query with its last n_learned samples replaced by proposals for its environment.

    clearance > 0: proposals whose position lies closer than `clearance` to a box are dropped (the
    learned part of SampleFree keeps a margin).  The network's errors otherwise put some proposals
    next to box faces, where edges through them have a true CP of a few percent that N = 128
    particles often estimate as 0; Explore then stops at such a plan (goal plan with CP-hat below
    alpha_min) and PlanSelection certifies none.  The uniform samples still reach every corner.
    spread > 0: each proposed position moves by a seeded normal offset of that standard deviation
    (clipped to the unit cube)."""
    sd = wl.seed if seed is None else seed
    if clearance > 0.0 and n_learned > 0:
        # proposals closer than `clearance` to a box are dropped; the network is asked for more
        # (later draws of the same seeded stream) until n_learned are kept or four rounds pass,
        # and the remainder stays uniform
        cand = model.propose(workload_features(wl), 4 * n_learned, sd, vmax)
        ok = box_distance(cand[:, :3], wl.boxes) >= clearance
        prop = cand[ok][:n_learned]
    else:
        prop = model.propose(workload_features(wl), n_learned, sd, vmax)
    if spread > 0.0 and len(prop) > 0:
        g = np.random.default_rng([int(sd) & 0xFFFFFFFF, 0x5EED])
        prop = prop.copy()
        prop[:, :3] = np.clip(prop[:, :3] + g.normal(0.0, spread, (len(prop), 3)), 0.0, 1.0).astype(np.float32)
    uni = wl.states[2:wl.states.shape[0] - len(prop)]
    return inputs.with_samples(wl, np.concatenate([uni, prop]))


def _errors(rs) -> Dict[str, int]:
    """Queries that ended in an error (neither a certified plan nor INFEASIBLE), by status."""
    out: Dict[str, int] = {}
    for r in rs:
        if r["rc"] not in (pump.OK, pump.ERR_INFEASIBLE):
            k = pump.status_str(r["rc"])
            out[k] = out.get(k, 0) + 1
    return out


def evaluate(model: pump.MLP, seeds: Sequence[int], n_samples: int = 4000, n_learned: int = LEARNED,
             slots: int = 8, raw: bool = False, spread: float = 0.0, uniform: Optional[List[Dict]] = None,
             clearance: float = CLEARANCE) -> Dict:
    """Paired comparison on held-out environments: uniform (n_samples) against uniform
    (n_samples - n_learned, the same ones) + n_learned proposals (with `spread`, see
    mixed_workload).  `uniform`: the uniform arm's results when already planned."""
    base = [inputs.proposal_workload(int(s), n_samples) for s in seeds]
    t0 = time.perf_counter()
    mixed = [mixed_workload(model, w, n_learned, spread=spread, clearance=clearance) for w in base]
    t_prop = time.perf_counter() - t0
    ru = uniform if uniform is not None else run_queries(base, slots)
    rm = run_queries(mixed, slots)
    ok_u = np.array([certified(r) for r in ru])
    ok_m = np.array([certified(r) for r in rm])
    cu = np.array([r["cost"] for r in ru], np.float64)
    cm = np.array([r["cost"] for r in rm], np.float64)
    both = ok_u & ok_m
    ratio = cm[both] / cu[both]
    return {"environments": len(seeds), "samples": n_samples, "learned": n_learned, "spread": spread,
            "clearance": clearance,
            "success_uniform": float(ok_u.mean()), "success_mixed": float(ok_m.mean()),
            "solved_only_uniform": int((ok_u & ~ok_m).sum()), "solved_only_mixed": int((ok_m & ~ok_u).sum()),
            "paired": int(both.sum()),
            "mean_cost_uniform": float(cu[both].mean()) if both.any() else None,
            "mean_cost_mixed": float(cm[both].mean()) if both.any() else None,
            "median_cost_ratio": float(np.median(ratio)) if both.any() else None,
            "mixed_cheaper": int((ratio < 1).sum()), "mixed_dearer": int((ratio > 1).sum()),
            "mean_candidates_uniform": float(np.mean([r["n_candidates"] for r in ru])),
            "mean_candidates_mixed": float(np.mean([r["n_candidates"] for r in rm])),
            "propose_ms_per_query": 1e3 * t_prop / max(len(seeds), 1),
            "errors_uniform": _errors(ru), "errors_mixed": _errors(rm),
            **({"raw_uniform": ru, "raw_mixed": rm} if raw else {})}


def _main(argv=None) -> int:
    """Training loop alone on a seeded synthetic training set (no planning), for timing and
    profiling the network kernels: python -m paper_1607_06886_gb300.proposal --steps 20."""
    import argparse
    import json
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--batch", type=int, default=2048)
    ap.add_argument("--envs", type=int, default=1000)
    args = ap.parse_args(argv)
    g = np.random.default_rng(0)
    feat = np.zeros((args.envs, FEAT), np.float32)
    feat[:, :BOX_SLOTS * 6] = g.uniform(0, 1, (args.envs, BOX_SLOTS * 6))
    tg = np.concatenate([g.uniform(0, 1, (args.envs, MAX_TARGETS, 3)),
                         g.uniform(-inputs.VEL_MAX, inputs.VEL_MAX, (args.envs, MAX_TARGETS, 3))], axis=2)
    nt = g.integers(1, MAX_TARGETS + 1, size=args.envs)
    data = Dataset(np.arange(args.envs), feat, tg.astype(np.float32), nt.astype(np.int32), {})
    m = make_model(0)
    tr = train(m, data, args.steps, args.batch)
    tr.pop("trace")
    print(json.dumps(tr))
    m.close()
    return 0


if __name__ == "__main__":
    raise SystemExit(_main())
