#!/usr/bin/env python3
"""Benchmark: partial plans evaluated per second by PUMP's exploration on one GB300.

A step is one pass of the exploration hot path on a device-resident graph, through the C ABI
(pump_plan with PUMP_EXPLORE_ONLY): the particle edge masks for the query's obstacles and Explore
(Algorithm 4).  `value` = partial plans evaluated (candidates of Algorithm 4) per second over the
timed steps, summed over ranks.  `full_query` times the whole query on the resident graph (with
PlanSelection and Monte Carlo certification, Algorithm 5), and `e2e` the whole query through the
public API from pinned host buffers: graph build from host arrays + plan + result readback.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload indoor_4k]

Under torchrun each rank plans its own query (seed = rank): weak scaling, no collective on the
data path; the timed region is bracketed by a barrier and the maximum over ranks is reported.
`--impl reference` times the CPU oracle (plain C restatement of the method) on the same workload
on every usable host core, rank 0 only.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L2_BYTES = 129 * 1024 * 1024
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        d["_source"] = "measured"
        return d
    d = dict(PEAKS_FALLBACK)
    d["_source"] = "fallback"
    return d


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        except Exception:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_setup():
    import torch
    from paper_1607_06886_gb300 import dist as pd
    ws, rank, local = pd.world()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    return ws, rank, local


def barrier(ws):
    from paper_1607_06886_gb300 import dist as pd
    pd.barrier()


def max_over_ranks(x, ws):
    from paper_1607_06886_gb300 import dist as pd
    return pd.reduce_max(x, device="cuda")


def sum_over_ranks(x, ws):
    from paper_1607_06886_gb300 import dist as pd
    return pd.reduce_sum(x, device="cuda")


def plan_params(pump, wl):
    return pump.default_plan_params(alpha=wl.alpha, eta=wl.eta, lam=wl.lam, n_mc=wl.n_mc, mc_substeps=wl.mc_substeps,
                                    mc_seed=wl.mc_seed)


def cpu_info():
    """Host cores this process may use, and the CPU model (lscpu), recorded beside oracle timings."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    try:
        usable = len(os.sched_getaffinity(0))
    except AttributeError:
        usable = os.cpu_count()
    return {"nproc": os.cpu_count(), "usable": usable, "model": model}


def oracle_step(g, wl, kmin, kmax, threads=1):
    """One oracle step of the same hot path on the oracle's own graph: every edge mask, then
    Explore, on `threads` host threads.  Returns (seconds, candidates)."""
    from oracle import cpu
    t0 = time.perf_counter()
    masks = cpu.edge_masks(g, wl.xi, wl.boxes, wl.n_particles, n_threads=threads)
    ex = cpu.explore(g["n"], g["row_ptr"], g["col"], g["ecost"], masks, 0, wl.goal_idx, kmin, kmax, wl.lam,
                     wl.radius, n_threads=threads)
    return time.perf_counter() - t0, ex["n_candidates"]


def time_cpu_oracle(wl):
    """cpu_baseline: full oracle steps of the same query (all edge masks + Explore; graph built
    untimed, as for the GPU step): one on a single thread, then the median of three on every
    usable host core."""
    from oracle import cpu
    info = cpu_info()
    g = cpu.graph_build(wl.states, wl.boxes, wl.radius, wl.n_waypoints, wl.sigma)
    kmin, kmax = cpu.cp_thresholds(wl.alpha, wl.eta, wl.n_particles)
    s1, c1 = oracle_step(g, wl, kmin, kmax, 1)
    T = max(1, int(info["usable"] or 1))
    oracle_step(g, wl, kmin, kmax, T)
    runs = [oracle_step(g, wl, kmin, kmax, T) for _ in range(3)]
    sT = float(np.median([r[0] for r in runs]))
    return {"value": runs[0][1] / sT, "unit": "partial_plans/s", "cores": T, "kind": "oracle",
            "sample": f"full steps of the same query (all edge masks + Explore, graph built untimed): median of 3 on "
                      f"{T} threads ({sT:.2f} s each); one single-thread step ({s1:.1f} s)",
            "single_core": {"value": c1 / s1, "cores": 1, "seconds": s1},
            "all_cores": {"value": runs[0][1] / sT, "cores": T, "seconds": sT},
            "host": info}


def run_reference(args):
    """--impl reference: the CPU oracle as it stands, on this arm's workload and metric.  Every
    step is a full oracle step (all edge masks + Explore) on every usable host core; the oracle
    graph is built once, untimed (the GPU step also runs on a resident graph)."""
    from paper_1607_06886_gb300 import inputs
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from oracle import cpu
    cpu.build()
    info = cpu_info()
    T = max(1, int(info["usable"] or 1))
    wl = inputs.make_workload(args.workload, seed=0)
    g = cpu.graph_build(wl.states, wl.boxes, wl.radius, wl.n_waypoints, wl.sigma)
    kmin, kmax = cpu.cp_thresholds(wl.alpha, wl.eta, wl.n_particles)
    for k in range(args.warmup):
        oracle_step(g, wl, kmin, kmax, T)
    tot, cands = 0.0, 0
    for k in range(args.steps):
        sec, c = oracle_step(g, wl, kmin, kmax, T)
        tot += sec
        cands += c
    value = cands / tot
    s1, c1 = oracle_step(g, wl, kmin, kmax, 1)
    line = {"impl": "reference", "metric": "partial plans evaluated per second", "value": value,
            "unit": "partial_plans/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "samples": wl.n - 2, "particles": wl.n_particles,
                       "waypoints": wl.n_waypoints, "boxes": int(wl.boxes.shape[0]), "cp_target": wl.alpha,
                       "seed": 0},
            "cpu_baseline": {"value": value, "unit": "partial_plans/s", "cores": T, "kind": "oracle",
                             "sample": f"every step a full oracle step of the workload (all edge masks + Explore) "
                                       f"on {T} host threads; graph built once untimed; after the timed steps one "
                                       f"single-thread step ({s1:.1f} s)",
                             "single_core": {"value": c1 / s1, "cores": 1, "seconds": s1}, "host": info},
            "e2e": {"value": value, "unit": "partial_plans/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="indoor_4k")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--hsmc-seeds", type=int, default=8,
                    help="queries of the HSMC leg (CP-hat vs Monte Carlo for box and half-space masks); 0 skips it")
    ap.add_argument("--serve-requests", type=int, default=2000,
                    help="requests of the served leg per arrival rate (Poisson arrivals, continuous batching); 0 "
                         "skips it")
    ap.add_argument("--serve-rate", default="50,100,200,500",
                    help="arrival rates of the served leg (requests/s, comma-separated)")
    ap.add_argument("--learned-envs", type=int, default=10000,
                    help="training environments of the learned-proposal leg (plain PUMP solutions, then training "
                         "and a paired held-out evaluation); 0 skips it")
    ap.add_argument("--learned-eval", type=int, default=200, help="held-out environments of the learned leg")
    ap.add_argument("--learned-steps", type=int, default=5000, help="training steps of the learned leg")
    ap.add_argument("--batch-queries", type=int, default=256,
                    help="queries of the batched leg (uneven sizes, one persistent Explore launch); 0 skips it")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_1607_06886_gb300 import inputs, pump

    ws, rank, local = dist_setup()
    pump.load()
    pump.use_torch_allocator()
    dev = torch.device("cuda", torch.cuda.current_device())
    from paper_1607_06886_gb300 import dist as pd
    wl = inputs.make_workload(args.workload, seed=pd.query_seed(rank))
    prm = plan_params(pump, wl)
    prm_step = plan_params(pump, wl)
    prm_step.flags = pump.EXPLORE_ONLY
    todev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    G = pump.Graph.build(todev(wl.states), todev(wl.goal_idx), todev(wl.boxes), todev(wl.xi), wl.radius,
                         wl.n_particles, wl.n_waypoints, wl.sigma)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    # warm-up (synchronous: gives the step's partial-plan count)
    for _ in range(max(args.warmup, 3)):
        res = G.plan(prm_step)
        assert res["rc"] == pump.OK, res
    torch.cuda.synchronize()
    step_cands = res["n_candidates"]

    # timed region: K steps enqueued back to back (PUMP_NO_WAIT: no host round trip per query),
    # device time of each by CUDA events on the launching stream; L2 flushed between steps
    prm_async = plan_params(pump, wl)
    prm_async.flags = pump.EXPLORE_ONLY | pump.NO_WAIT
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    launches0 = pump.kernel_launches()
    fused_steps = 0
    with ClockSampler(torch.cuda.current_device()) as clk:
        barrier(ws)
        torch.cuda.synchronize()
        for _ in range(4):  # device work ahead of the first step, so its launch is not waited for
            flush.zero_()
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            r = G.plan(prm_async)
            ev[k][1].record(stream)
            assert r["rc"] == pump.OK, r
            fused_steps += r["fused"]
        torch.cuda.synchronize()
        barrier(ws)
    launches = pump.kernel_launches() - launches0
    chk = G.collect()  # the last step's counters: the same query every step
    assert chk["rc"] == pump.OK and chk["n_candidates"] == step_cands, (chk, step_cands)
    cands = args.steps * step_cands
    step_times = [a.elapsed_time(b) for a, b in ev]
    ms = sum(step_times)
    ms_max = max_over_ranks(ms, ws)
    cands_all = sum_over_ranks(cands, ws)
    value = cands_all / (ms_max / 1000.0)
    ms_per_step = ms_max / args.steps

    # the same step as a synchronous call (host launch path, read-back and wait included)
    sync_t = []
    for _ in range(max(10, min(args.steps, 40))):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        rs = G.plan(prm_step)
        b.record(stream)
        sync_t.append((a, b))
    torch.cuda.synchronize()
    sync_ms = [a.elapsed_time(b) for a, b in sync_t]

    # the whole query on the resident graph (with PlanSelection and Monte Carlo certification)
    fq = []
    for _ in range(max(20, min(5 * args.steps, 100))):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        full = G.plan(prm)
        b.record(stream)
        fq.append((a, b, full))
    torch.cuda.synchronize()
    fq_all = [a.elapsed_time(b) for a, b, _ in fq]
    fq_ms = float(np.median(fq_all))
    full = fq[-1][2]
    assert full["rc"] in (pump.OK, pump.ERR_INFEASIBLE), full

    # dominant kernels timed alone with CUDA events on the launching stream; in the fused form a
    # step is the one Explore launch, so its mean device time is the launch's
    fused_ms = ms / args.steps if fused_steps == args.steps else None
    roof, kernel_detail = roofline_measure(pump, G, prm, wl, dev, flush, args.steps, fused_ms)

    # end to end through the public API from pinned host buffers
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    h_states, h_goal, h_boxes, h_xi = pin(wl.states), pin(wl.goal_idx), pin(wl.boxes), pin(wl.xi)
    h2d = sum(int(t.numel() * t.element_size()) for t in (h_states, h_goal, h_boxes, h_xi))
    e2e_steps = max(10, min(args.steps, 40))
    for _ in range(2):
        G2 = pump.Graph.build(h_states, h_goal, h_boxes, h_xi, wl.radius, wl.n_particles, wl.n_waypoints, wl.sigma)
        G2.plan(prm)
        G2.close()
    torch.cuda.synchronize()
    barrier(ws)
    e_cands = 0
    e_ev = []
    for _ in range(e2e_steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        G2 = pump.Graph.build(h_states, h_goal, h_boxes, h_xi, wl.radius, wl.n_particles, wl.n_waypoints, wl.sigma)
        r2 = G2.plan(prm)
        e_cands += r2["n_candidates"]
        G2.close()
        e1.record(stream)
        e_ev.append((e0, e1))
    torch.cuda.synchronize()
    e_all = [a.elapsed_time(b) for a, b in e_ev]
    e_ms = max_over_ranks(sum(e_all), ws)
    e_value = sum_over_ranks(e_cands, ws) / (e_ms / 1000.0)
    d2h = 4 * int(r2["path_len"]) + 128  # result record and path

    line = {
        "metric": "partial plans evaluated per second", "value": value, "unit": "partial_plans/s",
        "n_gpus": ws, "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "samples": wl.n - 2, "particles": wl.n_particles,
                   "waypoints": wl.n_waypoints, "boxes": int(wl.boxes.shape[0]), "cp_target": wl.alpha,
                   "edges": int(G.counts()[1]), "partial_plans_per_step": res["n_candidates"],
                   "plans_per_step": res["n_plans"], "groups": res["n_groups"], "seed_per_rank": "rank",
                   "l2": "flushed between steps (2x L2 buffer write)", "parallelism": f"replicas{ws}",
                   "steps_enqueued": "back to back without a host wait (PUMP_NO_WAIT); counts read once after"},
        "step": "edge masks + Explore (Algorithm 4), graph resident",
        "step_form": ("fused: masks computed by worker clusters inside the Explore launch"
                      if fused_steps == args.steps else "separate launches: masks kernel, then Explore"),
        "step_ms": {"enqueued_mean": ms / args.steps, "enqueued_min": min(step_times),
                    "enqueued_max": max(step_times), "synchronous_p50": float(np.percentile(sync_ms, 50)),
                    "synchronous_p99": float(np.percentile(sync_ms, 99)),
                    "synchronous": "one pump_plan call per step that waits for its counters (host launch path "
                                   "and read-back included)"},
        "full_query": {"ms": fq_ms, "value": full["n_candidates"] / (fq_ms / 1000.0), "unit": "partial_plans/s",
                       "ms_masks": full["ms_masks"], "ms_explore": full["ms_explore"], "ms_select": full["ms_select"],
                       "includes": "edge masks + Explore + PlanSelection with Monte Carlo certification"},
        "latency_ms": {"plan_p50": float(np.percentile(fq_all, 50)), "plan_p99": float(np.percentile(fq_all, 99)),
                       "plan_samples": len(fq_all), "e2e_p50": float(np.percentile(e_all, 50)),
                       "e2e_p99": float(np.percentile(e_all, 99)), "e2e_samples": len(e_all),
                       "plan": "one query on the resident graph (masks + Explore + PlanSelection with MC), L2 "
                               "flushed before each", "e2e": "graph build from pinned host arrays + plan + readback"},
        "result": {"cost": full["cost"], "cp_hat": full["cp_hat"], "cp_mc": full["cp_mc"], "status": full["status"],
                   "goal_plans": full["n_goal"], "certified": full["n_certified"]},
        "clocks": clk.summary(),
        "e2e": {"value": e_value, "unit": "partial_plans/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": e_ms / e2e_steps, "includes": "graph build from pinned host arrays + plan + readback"},
        "gpu_launches": int(launches),
        "roofline": roof,
        "kernels": kernel_detail,
    }
    if args.batch_queries > 0:
        line["batched"] = batched_measure(pump, args, dev, flush, rank, ws)
    if args.serve_requests > 0:
        rates = [float(x) for x in str(args.serve_rate).split(",") if x.strip()]
        line["served"] = [served_measure(pump, args, rank, ws, r) for r in rates]
    if args.hsmc_seeds > 0:
        line["hsmc"] = hsmc_measure(pump, args, dev, flush)
    if args.learned_envs > 0 and rank == 0:
        line["learned"] = learned_measure(pump, args)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        from oracle import cpu
        cpu.build()
        line["cpu_baseline"] = time_cpu_oracle(wl)
    if rank == 0:
        print(json.dumps(line))
    G.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def measured_traffic(kernel):
    """DRAM bytes (read + write) per launch of `kernel` from the committed ncu capture of the same
    workload, or None when the kernel's source has changed since that capture."""
    import hashlib
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))[kernel]
        names = rec["sources"] if "sources" in rec else [rec["source"]]
        src = b"".join(open(os.path.join(ROOT, f), "rb").read() for f in names)
    except (OSError, KeyError, ValueError):
        return None
    if hashlib.sha256(src).hexdigest() != rec["source_sha256"]:
        return None
    return float(rec["dram_bytes_per_launch"])


def mlp_flops_per_step(dims, B):
    """Tensor-core flops of one training step: forward products, the weight-gradient products of
    every layer and the input-gradient products of every layer but the first (2 flops a MAC)."""
    macs = sum(dims[l] * dims[l + 1] for l in range(len(dims) - 1))
    first = dims[0] * dims[1]
    return 2.0 * B * (3 * macs - first)


def learned_measure(pump, args):
    """The learned sampling proposal: plain PUMP on args.learned_envs seeded training environments
    (indoor scenes, U{10..32} boxes, 4000 uniform samples, N = 128, W = 10, CP 1 %) through the
    request server; the BF16 network trained on the certified plans' states with the device loop
    (batch 2048, Adam 1e-3, args.learned_steps steps) under both losses; then the paired held-out
    evaluation (seeds 1,000,000 on): 4000 uniform samples against the same first uniform samples
    plus proposals kept clear of the boxes, at the fraction chosen on validation environments (seeds
    2,000,000 on) and at the configuration's 50 %.  Also the training step's time and tensor
    throughput."""
    from paper_1607_06886_gb300 import inputs, proposal
    peak = float(load_peaks()["bf16_tflops"])
    data = proposal.collect(list(range(args.learned_envs)))
    held = list(range(proposal.HELDOUT_SEED0, proposal.HELDOUT_SEED0 + args.learned_eval))
    val = list(range(proposal.VALIDATION_SEED0, proposal.VALIDATION_SEED0 + args.learned_eval))
    ru = proposal.run_queries([inputs.proposal_workload(int(s), 4000) for s in held])
    ru_val = proposal.run_queries([inputs.proposal_workload(int(s), 4000) for s in val])
    out = {"workload": f"proposal_indoor_4k_{args.learned_envs}env", "collect": data.stats,
           "clearance": proposal.CLEARANCE, "learned": proposal.LEARNED,
           "selection": "clearance and learned fraction chosen on validation environments (seeds 2,000,000 on): "
                        "success at least uniform, then the lowest median cost ratio"}
    sig0 = [(r["rc"], r["cost"], r["n_candidates"]) for r in ru]
    for name, kind in (("path_indexed", proposal.PATH_INDEXED), ("wta", proposal.WTA)):
        m = proposal.make_model(0, kind)
        tr = proposal.train(m, data, args.learned_steps)
        tr.pop("trace")
        out[f"train_{name}"] = tr
        out[f"eval_{name}"] = proposal.evaluate(m, held, uniform=ru)
        out[f"validation_{name}"] = proposal.evaluate(m, val, uniform=ru_val)
        if kind == proposal.PATH_INDEXED:
            out["eval_path_indexed_half_learned"] = proposal.evaluate(m, held, n_learned=2000, uniform=ru)
            out["eval_path_indexed_no_clearance"] = proposal.evaluate(m, held, n_learned=2000, uniform=ru,
                                                                      clearance=0.0)
            perf = {}
            for B, steps in ((2048, 500), (32768, 50)):
                m.train(B, 3, 1e-3, 0.1, 1)
                t0 = time.perf_counter()
                m.train(B, steps, 1e-3, 0.1, 1)
                ms = 1e3 * (time.perf_counter() - t0) / steps
                tf = mlp_flops_per_step(proposal.DIMS, B) / (ms * 1e-3) / 1e12
                perf[f"b{B}"] = {"ms_per_step": ms, "tflops": tf, "frac_of_measured_peak": tf / peak}
            out["train_step"] = dict(perf, peak_tflops=peak, dims=list(proposal.DIMS),
                                     note="one training step = draws + forward + loss + backward + Adam, replayed as "
                                          "a CUDA graph; host-timed over the replays (one sync)")
        m.close()
    # the uniform arm planned again: the same results (each query is deterministic)
    ru2 = proposal.run_queries([inputs.proposal_workload(int(s), 4000) for s in held])
    sig1 = [(r["rc"], r["cost"], r["n_candidates"]) for r in ru2]
    out["uniform_arm_repeat_equal"] = sig0 == sig1
    if sig0 != sig1:
        bad = [i for i, (a, b) in enumerate(zip(sig0, sig1)) if a != b]
        out["uniform_arm_differs"] = {"queries": bad[:10], "first": [sig0[bad[0]], sig1[bad[0]]]}
    return out


def hsmc_measure(pump, args, dev, flush):
    """Half-Space Monte Carlo masks (the paper's CP approximation) beside the particle-in-box masks
    on the indoor workload: graph build and mask-pass times, and over args.hsmc_seeds queries the
    selected plan's CP-hat against its Monte Carlo CP for each mask kind."""
    import torch
    from paper_1607_06886_gb300 import inputs
    todev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    stream = torch.cuda.current_stream()

    def timed(fn, reps=5):
        fn()
        ts = []
        for _ in range(reps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            out = fn()
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return float(np.median(ts)), out

    wl = inputs.make_workload(args.workload, 0)
    build = lambda f: pump.Graph.build(todev(wl.states), todev(wl.goal_idx), todev(wl.boxes), todev(wl.xi), wl.radius,
                                       wl.n_particles, wl.n_waypoints, wl.sigma, flags=f)
    t_build_box, Gb = timed(lambda: build(0), reps=3)
    t_build_hs, Gh = timed(lambda: build(pump.GRAPH_HSMC), reps=3)
    t_mask_box, _ = timed(Gb.edge_masks)
    t_mask_hs, _ = timed(Gh.edge_masks)
    Gb.close()
    Gh.close()
    rows = []
    for seed in range(args.hsmc_seeds):
        w = inputs.make_workload(args.workload, seed)
        prm = pump.default_plan_params(alpha=w.alpha, eta=w.eta, lam=w.lam, n_mc=w.n_mc, mc_substeps=w.mc_substeps,
                                       mc_seed=w.mc_seed)
        row = {"seed": seed}
        for kind, f in (("box", 0), ("hsmc", pump.GRAPH_HSMC)):
            G = pump.Graph.build(todev(w.states), todev(w.goal_idx), todev(w.boxes), todev(w.xi), w.radius,
                                 w.n_particles, w.n_waypoints, w.sigma, flags=f)
            r = G.plan(prm)
            G.close()
            row[kind] = {"status": r["status"], "cp_hat": r["cp_hat"], "cp_mc": r["cp_mc"], "cost": r["cost"],
                         "partial_plans": r["n_candidates"]}
        rows.append(row)

    def summary(kind):
        ok = [r[kind] for r in rows if r[kind]["status"] == pump.OK]
        if not ok:
            return {"queries_solved": 0}
        err = np.array([x["cp_hat"] - x["cp_mc"] for x in ok])
        return {"queries_solved": len(ok), "mean_cp_hat": float(np.mean([x["cp_hat"] for x in ok])),
                "mean_cp_mc": float(np.mean([x["cp_mc"] for x in ok])), "mean_abs_err": float(np.mean(np.abs(err))),
                "mean_cost": float(np.mean([x["cost"] for x in ok]))}

    return {"workload": args.workload, "build_ms": {"box": t_build_box, "hsmc": t_build_hs},
            "mask_ms": {"box": t_mask_box, "hsmc": t_mask_hs}, "cp_target": wl.alpha,
            "selected_plan_cp": {"box": summary("box"), "hsmc": summary("hsmc")}, "queries": rows,
            "note": "cp_hat = particle estimate used by Explore (N particles); cp_mc = 10^4-rollout Monte Carlo of the same plan"}


def served_measure(pump, args, rank, ws, rate):
    """The served form: args.serve_requests requests with Poisson arrivals at `rate` per
    second (samples U{1000..16000}, boxes U{5..50}, N in {64, 128, 256}, W = 10, CP 1 %), each a
    whole query from host arrays (graph build + masks + Explore + PlanSelection with MC).  Latency
    is arrival to result.  Continuous batching (8 slots, requests admitted as slots and device
    memory free up) against the plain sequential FIFO (1 slot), same arrivals."""
    from paper_1607_06886_gb300 import inputs
    R = args.serve_requests
    wls = inputs.batch_workloads(R, seed=2000 * (rank + 1), n_range=(1000, 16000))
    gaps = np.random.default_rng(12345 + rank).exponential(1.0 / rate, size=R)
    arrivals = np.cumsum(gaps) - gaps[0]
    prms = [pump.default_plan_params(alpha=w.alpha, eta=w.eta, lam=w.lam, n_mc=w.n_mc, mc_substeps=w.mc_substeps,
                                     mc_seed=w.mc_seed) for w in wls]

    def run(slots):
        srv = pump.Server(slots, 64 << 30)
        tickets = []
        t0 = time.perf_counter()
        for k, (w, p) in enumerate(zip(wls, prms)):
            delay = t0 + arrivals[k] - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            tickets.append(srv.submit(w.states, w.goal_idx, w.boxes, w.xi, w.radius, w.n_particles, w.n_waypoints,
                                      w.sigma, p))
        res = [srv.wait(t) for t in tickets]
        wall = time.perf_counter() - t0
        st = srv.stats()
        srv.close()
        lat = np.array([r["latency_ms"] for r in res])
        return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "mean_ms": float(lat.mean()), "throughput_rps": R / wall, "peak_running": st["peak_running"],
                "ok": int(sum(r["rc"] in (pump.OK, pump.ERR_INFEASIBLE) for r in res))}, res

    cont, rc_ = run(8)
    seq, rs_ = run(1)
    keys = ("status", "chosen_plan", "cost", "mc_collisions", "n_candidates", "n_plans")
    same = all(all(a[k] == b[k] for k in keys) for a, b in zip(rc_, rs_))
    cands = sum(r["n_candidates"] for r in rc_)
    errs = {}
    for form, rs in (("continuous", rc_), ("sequential", rs_)):
        for r in rs:
            if r["rc"] not in (pump.OK, pump.ERR_INFEASIBLE):
                errs[f"{form}: {pump.status_str(r['rc'])}"] = errs.get(f"{form}: {pump.status_str(r['rc'])}", 0) + 1
    return {"workload": f"served_{R}_at_{rate:g}rps", "requests": R, "arrival_rate_rps": rate,
            "continuous_batching": dict(cont, slots=8), "sequential_fifo": dict(seq, slots=1),
            "p99_speedup": seq["p99_ms"] / cont["p99_ms"], "results_equal": bool(same), "errors": errs,
            "partial_plans": cands,
            "includes": "graph build from host arrays + masks + Explore + PlanSelection with MC + readback",
            "inputs": "seeded synthetic: samples U{1000..16000}, boxes U{5..50}, N in {64,128,256}, W=10, CP 1%"}


def batched_measure(pump, args, dev, flush, rank, ws):
    """The batched form: args.batch_queries independent queries of uneven size (samples
    U{1000..8000}, boxes U{5..50}, N in {64, 128, 256}, W = 10, CP target 1 %), graphs resident,
    each step = the edge masks of every query in one persistent launch + all Explore runs in
    another (pump_plan_batch, Explore only).  The launch forms come from the autotuner.  Also times
    the same queries one after another through the single-query call."""
    import torch
    from paper_1607_06886_gb300 import autotune, inputs
    nq = args.batch_queries
    wls = inputs.batch_workloads(nq, seed=1000 * (rank + 1))
    todev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    Gs = [pump.Graph.build(todev(w.states), todev(w.goal_idx), todev(w.boxes), todev(w.xi), w.radius, w.n_particles,
                           w.n_waypoints, w.sigma) for w in wls]
    prms = [pump.default_plan_params(alpha=w.alpha, eta=w.eta, lam=w.lam, n_mc=w.n_mc, mc_substeps=w.mc_substeps,
                                     mc_seed=w.mc_seed, flags=pump.EXPLORE_ONLY) for w in wls]
    cfg, rec = autotune.tune_batch(Gs, prms)
    stream = torch.cuda.current_stream()
    # the same queries one at a time through pump_plan (reference for the batched launch)
    flush.zero_()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    single = [G.plan(p) for G, p in zip(Gs, prms)]
    b.record(stream)
    torch.cuda.synchronize()
    seq_ms = a.elapsed_time(b)
    reps, times, res = max(3, min(args.steps, 5)), [], None
    for k in range(reps + 1):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier(ws)
        a.record(stream)
        rc, res = pump.plan_batch(Gs, prms, cfg)
        b.record(stream)
        torch.cuda.synchronize()
        assert rc == pump.OK, rc
        if k:
            times.append(a.elapsed_time(b))
    same = all(r["n_candidates"] == q["n_candidates"] and r["n_plans"] == q["n_plans"] for r, q in zip(res, single))
    ms = max_over_ranks(float(np.median(times)), ws)
    cands = sum(r["n_candidates"] for r in res)
    plans = sum(r["n_plans"] for r in res)
    ms_expl, ms_mask = res[0]["ms_explore"], res[0]["ms_masks"]
    # expansion proper against HBM: algorithmic bytes per candidate and per kept plan (as for the
    # single query), over all queries, divided by the batched Explore launch's time
    nbytes = sum(r["n_candidates"] * (12 + 4 * (G.counts()[4] // 32)) + r["n_plans"] * (28 + 4 * (G.counts()[4] // 32))
                 for r, G in zip(res, Gs))
    hbm = float(load_peaks()["hbm_gbs"])
    # the mask pass against the ALU peak: lane-ops counted exactly on every 16th query, scaled to the
    # batch by edges
    import torch
    edges = [int(G.counts()[1]) for G in Gs]
    samp = list(range(0, nq, 16))
    ops_s = sum(mask_lane_ops(Gs[k], wls[k].boxes)[0] for k in samp)
    ops_mask = ops_s * sum(edges) / max(sum(edges[k] for k in samp), 1)
    props = torch.cuda.get_device_properties(dev)
    alu_peak = props.multi_processor_count * 128 * float(load_peaks().get("sm_max_mhz", 2070.0)) * 1e6
    out = {"workload": f"batch_{nq}", "queries": nq, "value": sum_over_ranks(cands, ws) / (ms / 1e3),
           "unit": "partial_plans/s", "ms_per_batch": ms, "ms_masks": ms_mask, "ms_explore": ms_expl,
           "partial_plans": cands, "plans": plans, "edges": int(sum(int(G.counts()[1]) for G in Gs)),
           "single_queries_ms": seq_ms, "speedup_vs_single_queries": seq_ms / ms, "results_equal_single": bool(same),
           "launch": {"cluster_size": cfg.cluster_size, "mbest_global": cfg.mbest_global, "tuned_ms": rec.get("explore_ms"),
                      "mask_pairs": cfg.mask_pairs, "mask_chunk": cfg.mask_chunk, "mask_span": cfg.mask_span,
                      "mask_tuned_ms": rec.get("mask_ms")},
           "explore_roofline": {"bound": "hbm", "achieved": nbytes / (ms_expl / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                                "frac": nbytes / (ms_expl / 1e3) / 1e9 / hbm},
           "mask_roofline": {"bound": "alu", "achieved": ops_mask / (ms_mask / 1e3) / 1e12, "peak": alu_peak / 1e12,
                             "unit": "Tops/s", "frac": ops_mask / (ms_mask / 1e3) / alu_peak,
                             "work": f"lane-ops counted on {len(samp)} of {nq} queries, scaled by edges",
                             "peak_source": "SMs x 128 lanes x sm_max_mhz (derived)"},
           "inputs": "seeded synthetic: samples U{1000..8000}, boxes U{5..50}, N in {64,128,256}, W=10, CP 1%"}
    for G in Gs:
        G.close()
    return out


def mask_lane_ops(G, boxes):
    """Algorithmic lane-op work of one edge-mask pass over graph G: every edge tests its position
    box against the O obstacles (6 comparisons each); an edge whose box meets k obstacles runs the
    deviation recurrence and position of every particle and waypoint (3 axes x 8 float ops) and
    tests those k obstacles (6 comparisons each, counted in full although a hit ends the scan).
    Returns (lane-ops, live-edge flags)."""
    cnt = G.counts()
    E, N, W = int(cnt[1]), int(cnt[4]), int(cnt[5])
    boxes = np.asarray(boxes, np.float32).reshape(-1, 6)
    O = int(boxes.shape[0])
    ib = G.export("edge_box")
    ov = np.zeros(E, np.int64)
    for o in range(O):
        b = boxes[o]
        ov += ((b[0] <= ib[:, 3]) & (ib[:, 0] <= b[3]) & (b[1] <= ib[:, 4]) & (ib[:, 1] <= b[4]) &
               (b[2] <= ib[:, 5]) & (ib[:, 2] <= b[5])).astype(np.int64)
    live = ov > 0
    return float(E) * 6 * O + float(N) * W * float(np.sum(24 + 6 * ov[live])), live


def roofline_measure(pump, G, prm, wl, dev, flush, steps, fused_ms=None):
    """Average device time of the edge-mask launch and of Explore, each run alone (CUDA events on
    the launching stream, L2 flushed before each launch), with their algorithmic work.  When the
    timed steps ran fused (fused_ms: their mean Explore-launch time, the library's CUDA events on
    the launching stream), the fused kernel is the step's dominant kernel and is reported."""
    import torch
    peaks = load_peaks()
    stream = torch.cuda.current_stream()
    reps = max(5, min(steps, 20))
    # edge masks
    t = []
    for _ in range(reps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        G.edge_masks()
        b.record(stream)
        t.append((a, b))
    torch.cuda.synchronize()
    ms_mask = float(np.mean([a.elapsed_time(b) for a, b in t]))
    # explore alone (persistent kernel + its init/finalize launches)
    t = []
    for _ in range(reps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        st = G.explore(prm)
        b.record(stream)
        t.append((a, b))
    torch.cuda.synchronize()
    ms_expl = float(np.mean([a.elapsed_time(b) for a, b in t]))
    cnt = G.counts()
    E, N, W = int(cnt[1]), int(cnt[4]), int(cnt[5])
    # edge masks: ALU-bound.  Work of the culled query: every edge tests its position box against
    # the O obstacles (6 comparisons each); an edge whose box meets k obstacles runs the deviation
    # recurrence and position for every particle and waypoint (3 axes x 8 float ops = 24) and tests
    # those k obstacles (6 comparisons each, counted in full although a hit ends the scan).
    ops_mask, live = mask_lane_ops(G, wl.boxes)
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    props = torch.cuda.get_device_properties(dev)
    alu_peak = props.multi_processor_count * 128 * sm_mhz * 1e6  # lane-ops/s
    mask_frac = (ops_mask / (ms_mask / 1e3)) / alu_peak
    # explore: algorithmic bytes per candidate (edge id, cost, mask words, dominance slot) and per
    # surviving plan (record)
    w = N // 32
    bytes_expl = float(st["n_candidates"]) * (4 + 4 + 4 * w + 4) + float(st["n_plans"]) * (28 + 4 * w)
    hbm = float(peaks["hbm_gbs"])
    expl_gbs = bytes_expl / (ms_expl / 1e3) / 1e9
    # ablation: the masks recomputed per (plan, edge) pair, as an expansion that evaluates the
    # collision probability per candidate does (the library computes each edge's mask once per
    # query); the pairs are this run's candidates, every out-edge of every expanded plan
    heads, expd, rp = G.export("plan_head"), G.export("plan_expanded"), G.export("row_ptr")
    pairs = np.concatenate([np.arange(rp[h], rp[h + 1], dtype=np.int32) for h in heads[expd >= 0]])
    assert len(pairs) == int(st["n_candidates"]), (len(pairs), st["n_candidates"])
    ed = torch.from_numpy(pairs).to(dev)
    out_rows = torch.empty((len(pairs), w), dtype=torch.int32, device=dev)
    bad = torch.zeros(1, dtype=torch.int32, device=dev)
    t = []
    for _ in range(reps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        rc = G.edge_masks_list(ed.data_ptr(), len(pairs), out_rows.data_ptr(), bad.data_ptr())
        b.record(stream)
        assert rc == pump.OK, rc
        t.append((a, b))
    torch.cuda.synchronize()
    assert int(bad.item()) == 0
    ms_pairs = float(np.mean([a.elapsed_time(b) for a, b in t]))
    del ed, out_rows, bad
    detail = {
        "edge_mask": {"ms": ms_mask, "bound": "alu", "ops": ops_mask, "live_edges": int(live.sum()), "edges": E,
                      "achieved_tops": ops_mask / (ms_mask / 1e3) / 1e12, "peak_tops": alu_peak / 1e12,
                      "frac": mask_frac, "traffic": measured_traffic("k_edge_mask")},
        "explore": {"ms": ms_expl, "bound": "hbm", "bytes": bytes_expl, "achieved_gbs": expl_gbs, "peak_gbs": hbm,
                    "frac": expl_gbs / hbm, "iterations": st["n_iterations"],
                    "traffic": measured_traffic("k_explore_cluster")},
        "per_pair_masks": {"pairs": int(len(pairs)), "edges": E, "ms": ms_pairs, "ms_per_edge_memo": ms_mask,
                           "ratio": ms_pairs / ms_mask,
                           "what": "ablation: every candidate (plan, edge) pair's mask recomputed "
                                   "(pump_edge_masks_list over the run's candidates) against one mask per edge"},
    }
    if fused_ms:
        # one launch does both: the mask workers' lane operations are its throughput work, and
        # Explore's dependent chain (16 SMs) sets its length
        detail["fused"] = {"ms": fused_ms, "bound": "alu", "ops": ops_mask,
                           "achieved_tops": ops_mask / (fused_ms / 1e3) / 1e12, "peak_tops": alu_peak / 1e12,
                           "frac": ops_mask / (fused_ms / 1e3) / alu_peak, "explore_bytes": bytes_expl,
                           "explore_gbs": bytes_expl / (fused_ms / 1e3) / 1e9,
                           "traffic": measured_traffic("k_explore_fused")}
        roof = {"kernel": "k_explore_fused", "bound": "alu", "achieved": ops_mask / (fused_ms / 1e3) / 1e12,
                "peak": alu_peak / 1e12, "unit": "Tops/s", "frac": ops_mask / (fused_ms / 1e3) / alu_peak,
                "traffic": measured_traffic("k_explore_fused"),
                "peak_source": "152 SMs x 128 lanes x sm_max_mhz (derived)"}
    elif ms_expl >= ms_mask:
        roof = {"kernel": "k_explore_cluster", "bound": "hbm", "achieved": expl_gbs, "peak": hbm, "unit": "GB/s",
                "frac": expl_gbs / hbm, "traffic": measured_traffic("k_explore_cluster"),
                "peak_source": peaks["_source"]}
    else:
        roof = {"kernel": "k_edge_mask", "bound": "alu", "achieved": ops_mask / (ms_mask / 1e3) / 1e12,
                "peak": alu_peak / 1e12, "unit": "Tops/s", "frac": mask_frac, "traffic": measured_traffic("k_edge_mask"),
                "peak_source": "152 SMs x 128 lanes x sm_max_mhz (derived)"}
    return roof, detail


if __name__ == "__main__":
    sys.exit(main())
