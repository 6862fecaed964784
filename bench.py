"""Benchmark of the TIM+ hot path on one GB300 (or N, as independent replicas).

Default workload (the largest configuration, the size of the paper's Twitter graph in
Section 7): a directed Chung-Lu graph with 41.6M nodes and 1.4B edges (exponent 2.1),
IC trivalency (p per edge from {0.1, 0.01, 0.001}), k = 50, eps = 0.2, l = 1. One step
= build G^T from the device-resident out-CSR (tim_load_graph_device) and run TIM+
(tim_run: Algorithm 2 -> Algorithm 3 -> theta -> Algorithm 1). The metric is RR sets
generated per second over the whole step. The R-MAT scale-20 workload (IC weighted
cascade then LT 1/indeg, k = 50, eps = 0.1) rides along as a nested object, and is the
headline with --workload c2.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload c3|c2]

Prints one JSON line (rank 0). Under torchrun every rank runs its own independent
TIM+ step on its own GPU with a rank-specific seed (weak scaling, no data exchange).
"""
from __future__ import annotations

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

from paper_1404_0900_gb300 import inputs, start_round  # noqa: E402

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# DRAM bytes (read + write) per RR-set member of the IC sampler passes, from a one-pass
# ncu capture (dram__bytes_read.sum + dram__bytes_write.sum) of the pass's kernel on the
# workload the bench times, divided by the members that pass produced; the traffic of
# one launch is scaled from it by members. None where no capture of the current kernel
# exists.
DRAM_BYTES_PER_MEMBER = {
    # profiles/sampler_dram_c3.md
    "c3": {1: 384.8, 2: 760.1, 3: 561.4},
    "c2": {1: None, 2: None, 3: None},
}
FALLBACK_HBM_GBS = 6800.0
METRIC = "RR sets/s (TIM+ end to end, graph load included)"
L2_FLUSH_BYTES = 512 << 20


def parse_args(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", choices=["c3", "c2"], default="c3",
                   help="c3: TIM+ on the 41.6M-node / 1.4B-edge Chung-Lu graph, IC "
                        "trivalency, k=50, eps=0.2 (the headline; the c2 line rides along "
                        "nested); c2: TIM+ on R-MAT --scale, IC and LT, --k, --eps")
    p.add_argument("--no-c2", action="store_true",
                   help="with --workload c3: skip the nested R-MAT scale-20 line")
    p.add_argument("--scale", type=int, default=20)
    p.add_argument("--k", type=int, default=50)
    p.add_argument("--eps", type=float, default=0.1)
    p.add_argument("--ell", type=float, default=1.0)
    p.add_argument("--seed", type=int, default=1)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=20.0,
                   help="cap on the CPU time of the oracle's RR-set sample (c3 baseline)")
    p.add_argument("--no-batch", action="store_true",
                   help="skip the 64-query batched-vs-plain comparison")
    p.add_argument("--batch-queries", type=int, default=64)
    p.add_argument("--no-learned", action="store_true",
                   help="skip the learned-start-round comparisons")
    p.add_argument("--mode", choices=["timplus", "sample", "batch", "learned", "spread"],
                   default="timplus",
                   help="timplus: the TIM+ step of --workload (default); sample: only RR-set "
                        "generation (tim_sample_rr of --theta NodeSelection sets on R-MAT "
                        "--scale), for profiling; spread: forward Monte-Carlo spread of "
                        "TIM+'s seeds (--cascades) against the RR estimate")
    p.add_argument("--theta", type=int, default=1_000_000)
    p.add_argument("--graph", choices=["rmat", "chunglu-tenth"], default="rmat",
                   help="--mode sample: R-MAT --scale (weighted cascade or LT 1/indeg), or the "
                        "largest configuration's graph at a tenth of its size (4.16M nodes, "
                        "140M edges, IC trivalency), drawn on the GPU")
    p.add_argument("--cascades", type=int, default=10_000)
    p.add_argument("--model", choices=["ic", "lt"], default="ic")
    return p.parse_args(argv)


# ------------------------------------------------------------ distributed glue

def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def init_dist(world: int, backend: str):
    if world <= 1:
        return None
    import torch.distributed as dist
    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    dist.init_process_group(backend=backend)
    return dist


def reduce_step_results(dist, device, seconds: float, sets: float):
    """Max of the timed seconds and sum of the RR sets over ranks."""
    if dist is None:
        return seconds, sets
    import torch
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    s = torch.tensor([sets], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(s, op=dist.ReduceOp.SUM)
    return float(t.item()), float(s.item())


# ------------------------------------------------------------------ workload

def workload(args):
    g = inputs.rmat(args.scale, seed=1)
    return g, inputs.weighted_cascade(g), inputs.lt_inverse_indegree(g)


def config_dict(args, g, world):
    return {"workload": f"TIM+ on directed R-MAT scale {args.scale} (a,b,c,d=.57,.19,.19,.05; "
                        f"n={g.n}, m={g.m}), IC weighted cascade then LT 1/indeg, "
                        f"k={args.k}, eps={args.eps}, l={args.ell}",
            "n": g.n, "m": g.m, "k": args.k, "eps": args.eps, "ell": args.ell,
            "models": ["IC", "LT"], "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
            "l2": f"flushed between timed steps ({L2_FLUSH_BYTES >> 20} MiB write)"}


def measured_peaks():
    try:
        return json.load(open(PEAKS_FILE))
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        loaded = [x for x in sm if mx and x > 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


# ---------------------------------------------------------------- our arm

def run_c2_line(args, nested: bool = False):
    """The R-MAT workload's TIM+ step (IC then LT). nested: a sub-object of the c3
    line (no process group of its own; batched and learned comparisons left out)."""
    import torch

    from paper_1404_0900_gb300 import tim

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    dist = None if nested else init_dist(world, "nccl")
    seed = args.seed + rank
    g, w_ic, w_lt = workload(args)
    stream = torch.cuda.Stream(device=device)
    torch.cuda.set_stream(stream)
    d_rowptr = torch.from_numpy(g.rowptr).to(device)
    d_dst = torch.from_numpy(g.dst).to(device)
    d_w = {tim.TIM_IC: torch.from_numpy(w_ic).to(device), tim.TIM_LT: torch.from_numpy(w_lt).to(device)}
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=device)
    engines = {m: tim.Engine(local, stream) for m in (tim.TIM_IC, tim.TIM_LT)}
    seeds = np.zeros(args.k, dtype=np.int32)

    def step():
        out = {}
        for m, eng in engines.items():
            tim.tim_load_graph_device(eng.ctx, g.n, g.m, d_rowptr, d_dst, d_w[m], m)
            _, frac, st = tim.tim_run(eng.ctx, args.k, args.eps, args.ell, seed, seeds_out=seeds)
            out[m] = st
        return out

    # autotune the sampler on the loaded graphs (settings never change results)
    tuning = {}
    for m, eng in engines.items():
        tim.tim_load_graph_device(eng.ctx, g.n, g.m, d_rowptr, d_dst, d_w[m], m)
        tuning["IC" if m == tim.TIM_IC else "LT"] = tim.tim_autotune(eng.ctx, 1_000_000, seed)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    for eng in engines.values():
        tim.tim_get_profile(eng.ctx, reset=True)
    launches0 = sum(tim.tim_launch_count(e.ctx) for e in engines.values())
    clocks = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    total_ms, total_sets, widths, per_model = 0.0, 0, 0, {}
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = step()
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
        for m, st in out.items():
            total_sets += st["sets_total"]
            widths += st["width_total"]
            per_model.setdefault(m, []).append(st)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    launches = sum(tim.tim_launch_count(e.ctx) for e in engines.values()) - launches0
    prof_ic = tim.tim_get_profile(engines[tim.TIM_IC].ctx)
    prof_lt = tim.tim_get_profile(engines[tim.TIM_LT].ctx)
    sec, sets_all = reduce_step_results(dist, device, total_ms / 1e3, float(total_sets))

    # end to end through the public API with host buffers (pinned), copies timed
    e2e = None
    if not args.no_e2e:
        h_rowptr = torch.from_numpy(g.rowptr).pin_memory()
        h_dst = torch.from_numpy(g.dst).pin_memory()
        h_w = {m: torch.from_numpy(w).pin_memory() for m, w in ((tim.TIM_IC, w_ic), (tim.TIM_LT, w_lt))}
        h_seeds = torch.zeros(args.k, dtype=torch.int32).pin_memory()

        def step_host():
            n_sets = 0
            for m, eng in engines.items():
                tim.lib().tim_load_graph(eng.ctx, g.n, g.m, tim._ptr(h_rowptr), tim._ptr(h_dst),
                                         tim._ptr(h_w[m]), m)
                _, _, st = tim.tim_run(eng.ctx, args.k, args.eps, args.ell, seed,
                                       seeds_out=h_seeds.numpy())
                n_sets += st["sets_total"]
            return n_sets

        step_host()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t_ms, e_sets = 0.0, 0
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            e_sets += step_host()
            torch.cuda.synchronize()
            t_ms += (time.perf_counter() - t0) * 1e3
        esec, esets = reduce_step_results(dist, device, t_ms / 1e3, float(e_sets))
        h2d = 2 * (h_rowptr.numel() * 8 + h_dst.numel() * 4 + g.m * 4)
        e2e = {"value": esets / esec, "unit": "RR sets/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": 2 * args.k * 4, "ms_per_step": t_ms / args.steps}

    for eng in engines.values():
        eng.close()
    if dist:
        dist.destroy_process_group()
    if rank != 0:
        return None
    del flush
    torch.cuda.empty_cache()

    # roofline of the dominant kernel: the IC sampler pass with the most device time
    roofline = sampler_roofline(prof_ic, "c2")
    ic = per_model[tim.TIM_IC][-1]
    lt = per_model[tim.TIM_LT][-1]
    line = {
        "metric": METRIC,
        "value": sets_all / sec,
        "unit": "RR sets/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u32/int64 (FP64 for kappa and theta)",
        "data": "synthetic (seeded R-MAT, no dataset)",
        "config": config_dict(args, g, world),
        "width_rate": {"value": widths / (total_ms / 1e3), "unit": "in-edges of R's nodes "
                       "(w(R), Eq. 1) per second; skipped lists counted in full, so not GTEPS"},
        "gteps_examined": sum(prof_ic[f"pass{i}_examined"] + prof_lt[f"pass{i}_examined"]
                              for i in (1, 2, 3)) / (total_ms / 1e3) / 1e9,
        "tim_plus_ms": {"IC": statistics.mean(s["ms_total"] for s in per_model[tim.TIM_IC]),
                        "LT": statistics.mean(s["ms_total"] for s in per_model[tim.TIM_LT])},
        "phases_ms_IC": {k: ic[k] for k in ("ms_kpt", "ms_refine", "ms_select_sample",
                                             "ms_select_greedy")},
        "phases_ms_LT": {k: lt[k] for k in ("ms_kpt", "ms_refine", "ms_select_sample",
                                             "ms_select_greedy")},
        "theta": {"IC": ic["theta"], "LT": lt["theta"]},
        "kpt_plus": {"IC": ic["kpt_plus"], "LT": lt["kpt_plus"]},
        "roofline": roofline,
        "sampler_profile": {"IC": prof_ic, "LT": prof_lt},
        "autotune": tuning,
        "clocks": clk,
        "gpu_launches": launches,
        "e2e": e2e,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_timplus(args, g, w_ic, w_lt, per_model)
    if nested:
        return line
    if not args.no_batch and world == 1:
        line["batched_vs_plain"] = run_batch_compare(args)
    if not args.no_learned and world == 1:
        line["learned_vs_plain"] = run_learned_compare(args, g, w_ic, w_lt)
    return line


def sampler_bytes(p: dict, i: int) -> float:
    """Algorithmic bytes of IC sampler pass i, per RR set R: 8 (|R| + 1) B of in-CSR
    offsets, 8 B (source and threshold) per examined in-edge, 4 |R| B emitted, 8 B of
    set offsets. Examined in-edges: all in-edges of lists outside the geometric-skip
    rule plus the live ones the rule finds (in-edges it skips are not touched)."""
    return (8.0 * (p[f"pass{i}_members"] + p[f"pass{i}_sets"]) + 8.0 * p[f"pass{i}_examined"]
            + 4.0 * p[f"pass{i}_members"] + 8.0 * p[f"pass{i}_sets"])


def sampler_roofline(p: dict, workload: str) -> dict:
    """Roofline of the IC sampler pass with the most device time. Its time is the
    pass's own kernels (for the heavy-set pass: the persistent launches alone), its
    bytes the algorithmic bytes of sampler_bytes, per launch (heavy pass: per batch)."""
    def kernel_ms(i):
        return p["pass3_ms_kernel"] if i == 3 and p.get("pass3_batches") else p[f"pass{i}_ms"]

    def launches(i):
        return max(p["pass3_batches"] if i == 3 and p.get("pass3_batches")
                   else p[f"pass{i}_launches"], 1)
    dom = max((1, 2, 3), key=kernel_ms)
    names = {1: "rr_team_kernel<IC, Cap<256,9>, pass 1> (shared-memory hash, warp per set)",
             2: "rr_team_kernel<IC, Cap<8192,14>, pass 2> (global-arena hash, team per set)",
             3: "bulk_levels_kernel (heavy sets: all BFS levels of a batch in one "
                "persistent cooperative launch)"}
    alg = sampler_bytes(p, dom)
    ms, n = kernel_ms(dom), launches(dom)
    peaks = measured_peaks()
    if peaks and peaks.get("hbm_gbs"):
        peak, src = float(peaks["hbm_gbs"]), "measured"
    else:
        peak, src = FALLBACK_HBM_GBS, "fallback"
    achieved = alg / (ms / 1e3) / 1e9 if ms > 0 else 0.0
    ratio = DRAM_BYTES_PER_MEMBER.get(workload, {}).get(dom)
    return {"kernel": names[dom], "bound": "hbm", "achieved": achieved, "peak": peak,
            "peak_source": src, "unit": "GB/s", "frac": achieved / peak,
            "bytes_per_launch": alg / n, "ms_per_launch": ms / n, "launches": n,
            "traffic": ratio * p[f"pass{dom}_members"] / n if ratio else None,
            "traffic_note": "DRAM bytes per launch: bytes per member from a one-pass ncu "
                            "capture of this kernel x the members per launch (null: no "
                            "capture of the current kernel)"}


# --------------------------------------------------------- the CPU oracle arm

def oracle_rates(args, g, w_ic, w_lt, seconds: float, nthreads: int):
    """RR sets/s of the oracle (Section 3.1 BFS, NodeSelection set ids) per model, on a
    sample sized to take about `seconds` of wall time in total."""
    from oracle import oracle as O
    rates = {}
    target = seconds / 2
    for name, model, w, probe in (("IC", O.IC, w_ic, 1024), ("LT", O.LT, w_lt, 4096)):
        og = O.load_graph(g.n, g.rowptr, g.dst, w, model)
        O.sample(og, args.seed, O.make_sid(3, 0, 0), probe, nthreads)  # threads warm
        # grow the sample until it takes at least half the target (at most 4 tries)
        count, first = probe, probe
        for _ in range(4):
            t0 = time.perf_counter()
            O.sample(og, args.seed, O.make_sid(3, 0, first), count, nthreads)
            dt = max(time.perf_counter() - t0, 1e-6)
            if dt >= 0.5 * target:
                break
            first += count
            count = max(count * 2, int(count * target / dt))
        rates[name] = (count / dt, count, dt)
    return rates


def mix_rate(rates, n_ic, n_lt):
    """Sets/s for a step with n_ic IC sets and n_lt LT sets."""
    t = n_ic / rates["IC"][0] + n_lt / rates["LT"][0]
    return (n_ic + n_lt) / t


def cpu_baseline_timplus(args, g, w_ic, w_lt, per_model) -> dict:
    """The oracle's TIM+ end to end on the same graph and seed, IC then LT, on all host
    threads, with seconds per phase (Algorithm 2, Algorithm 3, Algorithm 1's sampling
    and greedy together); value = RR sets of all phases / seconds."""
    from oracle import oracle as O
    nth = O.host_threads()
    out, sets_all, secs_all = {}, 0, 0.0
    for name, model, w in (("IC", O.IC, w_ic), ("LT", O.LT, w_lt)):
        og = O.load_graph(g.n, g.rowptr, g.dst, w, model)
        t0 = time.perf_counter()
        kpt = O.kpt_estimation(og, args.k, args.ell, args.seed, nth)
        t1 = time.perf_counter()
        ref = O.refine_kpt(og, args.k, args.ell, args.eps, args.seed, kpt, nth)
        t2 = time.perf_counter()
        theta = O.theta_from(g.n, args.k, args.eps, args.ell, ref.kpt_plus)
        O.node_selection(og, args.k, theta, args.seed, nth)
        t3 = time.perf_counter()
        sets = kpt.sets_generated + ref.theta_prime + theta
        out[name] = {"s_kpt": t1 - t0, "s_refine": t2 - t1, "s_select": t3 - t2,
                     "sets": sets, "theta": theta}
        sets_all += sets
        secs_all += t3 - t0
        del og
    return {"value": sets_all / secs_all, "unit": "RR sets/s", "cores": nth, "kind": "oracle",
            "sample": f"oracle TIM+ end to end, IC and LT, on the same graph and seed "
                      f"({nth} threads): {secs_all:.1f} s for {sets_all} RR sets",
            "phases_s": out}


def cpu_baseline_c3(args, n, rowptr, dst, w) -> dict:
    """The oracle on the largest configuration: a fixed sample of RR sets with
    NodeSelection ids (up to 10^6, in chunks of 50,000, until --cpu-seconds) plus one
    Algorithm 2 round (round 10: c_10 sets, kappa sum), on all host threads; value =
    their RR sets / their seconds. The oracle's own G^T build is not timed."""
    from oracle import oracle as O
    nth = O.host_threads()
    t0 = time.perf_counter()
    og = O.load_graph(n, rowptr, dst, w, O.IC)
    load_s = time.perf_counter() - t0
    done, secs, chunk = 0, 0.0, 50_000
    while done < 1_000_000 and secs < args.cpu_seconds:
        t = time.perf_counter()
        O.sample(og, args.seed, O.make_sid(3, 0, done), chunk, nth)
        secs += time.perf_counter() - t
        done += chunk
    rnd = 10
    c = O.c_i(n, args.ell, rnd)
    t = time.perf_counter()
    O.kappa_sum(og, 50, args.seed, O.make_sid(1, rnd, 0), c, nth)
    rsecs = time.perf_counter() - t
    del og
    return {"value": (done + c) / (secs + rsecs), "unit": "RR sets/s", "cores": nth,
            "kind": "oracle",
            "sample": f"{done} RR sets (NodeSelection ids) in {secs:.1f} s and Algorithm 2 "
                      f"round {rnd} ({c} sets, kappa sum) in {rsecs:.1f} s on the same graph "
                      f"({nth} threads); the oracle's own G^T build ({load_s:.0f} s) untimed"}


def run_reference(args):
    """The reference arm: the CPU oracle as it stands, on the host cores, on the same
    workload. Each step is a bounded sample of the workload's RR sets (NodeSelection set
    ids, fresh ids every step): c3, 50,000 sets of the Chung-Lu graph (drawn with the
    same generator, on the GPU, and copied to the host; the oracle builds its own G^T,
    untimed); c2, about 2 s of IC and LT sets, the rate weighted 7:2 (the GPU step's
    mix). Rank 0 alone runs; the other ranks exit at once."""
    rank, world, _ = dist_env()
    if rank != 0:
        return None
    from oracle import oracle as O
    nth = O.host_threads()
    vals, secs = [], 0.0
    if args.workload == "c3":
        import torch
        g, w = c3_graph(torch.device("cuda", 0))
        n, m = g.n, g.m
        rowptr, dst, wh = g.rowptr.cpu().numpy(), g.dst.cpu().numpy(), w.cpu().numpy()
        del g, w
        torch.cuda.empty_cache()
        og = O.load_graph(n, rowptr, dst, wh, O.IC)
        del rowptr, dst, wh
        per = 50_000
        for i in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            O.sample(og, args.seed, O.make_sid(3, 0, i * per), per, nth)
            dt = time.perf_counter() - t0
            if i >= args.warmup:
                secs += dt
                vals.append(per / dt)
        config = c3_config(world, n, m)
        timed = (f"per step: oracle RR-set generation of {per} sets of the same graph "
                 f"(NodeSelection ids), {nth} threads")
        data = "synthetic (seeded Chung-Lu drawn on the GPU, no dataset)"
    else:
        g, w_ic, w_lt = workload(args)
        per_step = 2.0
        for _ in range(args.warmup):
            oracle_rates(args, g, w_ic, w_lt, per_step / 4, nth)
        for _ in range(args.steps):
            t0 = time.perf_counter()
            r = oracle_rates(args, g, w_ic, w_lt, per_step, nth)
            secs += time.perf_counter() - t0
            vals.append(mix_rate(r, 7, 2))
        config = config_dict(args, g, world)
        timed = ("per step: oracle RR-set generation, IC and LT sets of NodeSelection ids, "
                 f"about 1 s each, rate weighted 7:2, {nth} threads")
        data = "synthetic (seeded R-MAT, no dataset)"
    v = statistics.mean(vals)
    return {"impl": "reference", "metric": METRIC, "timed": timed, "value": v,
            "unit": "RR sets/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": secs * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32/int64 (FP64 for kappa)", "data": data,
            "config": config,
            "cpu_baseline": {"value": v, "unit": "RR sets/s", "cores": nth, "kind": "oracle",
                             "sample": timed},
            "e2e": {"value": v, "unit": "RR sets/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def run_sample_only(args):
    """Time tim_sample_rr alone: --theta RR sets with NodeSelection set ids."""
    import torch

    from paper_1404_0900_gb300 import tim
    model = tim.TIM_IC if args.model == "ic" else tim.TIM_LT
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    sid0 = 3 << 56
    with tim.Engine(0, stream) as eng:
        if args.graph == "chunglu-tenth":
            model = tim.TIM_IC
            dg = inputs.chung_lu_device(4_160_000, 175_000_000, 2.1, seed=1,
                                        m_exact=140_000_000)
            w = inputs.trivalency_device(dg, seed=2)
            tim.tim_load_graph_device(eng.ctx, dg.n, dg.m, dg.rowptr, dg.dst, w, model)
            del dg, w
        else:
            g = inputs.rmat(args.scale, seed=1)
            w = inputs.weighted_cascade(g) if model == tim.TIM_IC else inputs.lt_inverse_indegree(g)
            tim.tim_load_graph(eng.ctx, g.n, g.rowptr, g.dst, w, model)
        for _ in range(args.warmup):
            tim.tim_sample_rr(eng.ctx, args.theta, args.seed, sid0)
        tim.tim_get_profile(eng.ctx, reset=True)
        ms = 0.0
        for _ in range(args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            tim.tim_sample_rr(eng.ctx, args.theta, args.seed, sid0)
            e1.record(stream)
            e1.synchronize()
            ms += e0.elapsed_time(e1)
        prof = tim.tim_get_profile(eng.ctx)
    passes = {}
    for i in (1, 2, 3):
        t = prof[f"pass{i}_ms"]
        b = sampler_bytes(prof, i)
        passes[f"pass{i}"] = {"ms": t, "sets": prof[f"pass{i}_sets"],
                              "width": prof[f"pass{i}_width"],
                              "members": prof[f"pass{i}_members"],
                              "live": prof[f"pass{i}_live"],
                              "examined": prof[f"pass{i}_examined"], "algorithmic_bytes": b,
                              "GB/s": b / (t / 1e3) / 1e9 if t > 0 else 0.0}
    width = sum(prof[f"pass{i}_width"] for i in (1, 2, 3))
    return {"mode": "sample", "model": args.model, "graph": args.graph, "scale": args.scale,
            "theta": args.theta,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "RR sets/s": args.theta * args.steps / (ms / 1e3),
            "GTEPS (in-edges examined)": width / (ms / 1e3) / 1e9, "passes": passes}


def c3_config(world: int, n: int, m: int) -> dict:
    return {"workload": "TIM+ on a directed Chung-Lu graph of Twitter's size (41.6M nodes, "
                        "1.4B edges, exponent 2.1), IC trivalency p in {0.1, 0.01, 0.001}, "
                        "k=50, eps=0.2, l=1; a step = G^T build from the device out-CSR + TIM+",
            "n": n, "m": m, "k": 50, "eps": 0.2, "ell": 1.0, "models": ["IC"],
            "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
            "l2": f"inputs larger than L2 (G^T about 11 GB), and {L2_FLUSH_BYTES >> 20} MiB "
                  f"written between timed steps"}


def c3_graph(device):
    """The largest configuration's graph and trivalency weights, drawn on `device`."""
    g = inputs.chung_lu_c3_device(seed=1, device=device)
    return g, inputs.trivalency_device(g, seed=2)


def run_c3_line(args):
    """The headline: TIM+ on the largest configuration (see the module comment)."""
    import torch

    from paper_1404_0900_gb300 import tim

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    dist = init_dist(world, "nccl")
    seed = args.seed + rank
    k, eps, ell = 50, 0.2, args.ell
    stream = torch.cuda.Stream(device=device)
    torch.cuda.set_stream(stream)
    t0 = time.perf_counter()
    g, w = c3_graph(device)
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    n, m = g.n, g.m
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=device)
    eng = tim.Engine(local, stream)

    def step():
        tim.tim_load_graph_device(eng.ctx, n, m, g.rowptr, g.dst, w, tim.TIM_IC)
        return tim.tim_run(eng.ctx, k, eps, ell, seed)

    tim.tim_load_graph_device(eng.ctx, n, m, g.rowptr, g.dst, w, tim.TIM_IC)
    tuning = tim.tim_autotune(eng.ctx, 200_000, seed)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    tim.tim_get_profile(eng.ctx, reset=True)
    launches0 = tim.tim_launch_count(eng.ctx)
    clocks = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    total_ms, total_sets, runs = 0.0, 0, []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        seeds, frac, st = step()
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
        total_sets += st["sets_total"]
        runs.append(st)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    launches = tim.tim_launch_count(eng.ctx) - launches0
    prof = tim.tim_get_profile(eng.ctx)
    sec, sets_all = reduce_step_results(dist, device, total_ms / 1e3, float(total_sets))

    # end to end through the public API with host buffers (pinned), copies timed
    e2e, host = None, None
    if not args.no_e2e or (rank == 0 and not args.no_cpu_baseline):
        host = (g.rowptr.cpu().pin_memory(), g.dst.cpu().pin_memory(), w.cpu().pin_memory())
    del g, w
    torch.cuda.empty_cache()
    if not args.no_e2e:
        # a serving loop through the public API: every step uploads its graph from pinned
        # host memory (tim_load_graph builds G^T from it) and reads its seeds back. Two
        # contexts on two streams take the steps in turn, and the next step's upload and
        # build are issued from a second host thread while this step's TIM+ runs, so the
        # copies over the host link overlap the other context's kernels (the library
        # releases the interpreter lock in its calls; each context is used by one thread
        # at a time). Every copy of every step is inside the timed region.
        import threading

        h_rowptr, h_dst, h_w = host
        eng2 = tim.Engine(local, torch.cuda.Stream(device=device))
        for e in (eng, eng2):
            tim.tim_set_width_budget(e.ctx, tuning["width_budget"])
            tim.tim_set_chunk(e.ctx, tuning["chunk"])
            tim.tim_set_team_factor(e.ctx, tuning["team_factor"])
            tim.tim_set_pass1_capacity(e.ctx, tuning["pass1_capacity"])
        engs = (eng, eng2)
        h_seeds = [torch.zeros(k, dtype=torch.int32).pin_memory() for _ in engs]

        def load(e):
            rc = tim.lib().tim_load_graph(e.ctx, n, m, tim._ptr(h_rowptr), tim._ptr(h_dst),
                                          tim._ptr(h_w), tim.TIM_IC)
            if rc != 0:
                raise RuntimeError(f"tim_load_graph failed ({rc})")

        def run(i):
            _, _, st = tim.tim_run(engs[i % 2].ctx, k, eps, ell, seed,
                                   seeds_out=h_seeds[i % 2].numpy())
            return st["sets_total"]

        for i in range(2):  # both contexts allocate their buffers once
            load(engs[i])
            run(i)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        flush.zero_()
        torch.cuda.synchronize()
        e_sets = 0
        t1 = time.perf_counter()
        load(engs[0])
        for i in range(args.steps):
            nxt = None
            if i + 1 < args.steps:
                nxt = threading.Thread(target=load, args=(engs[(i + 1) % 2],))
                nxt.start()
            e_sets += run(i)
            if nxt:
                nxt.join()
        torch.cuda.synchronize()
        t_ms = (time.perf_counter() - t1) * 1e3
        eng2.close()
        esec, esets = reduce_step_results(dist, device, t_ms / 1e3, float(e_sets))
        h2d = h_rowptr.numel() * 8 + h_dst.numel() * 4 + h_w.numel() * 4
        e2e = {"value": esets / esec, "unit": "RR sets/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": k * 4, "ms_per_step": t_ms / args.steps,
               "pipeline": "two contexts; step i+1's upload and build overlap step i's TIM+"}
    eng.close()
    del flush
    torch.cuda.empty_cache()
    if dist:
        dist.destroy_process_group()
    if rank != 0:
        return None
    st = runs[-1]
    line = {
        "metric": METRIC,
        "value": sets_all / sec,
        "unit": "RR sets/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u32/int64 (FP64 for kappa and theta)",
        "data": "synthetic (seeded Chung-Lu drawn on the GPU, no dataset)",
        "config": c3_config(world, n, m),
        "gteps_examined": sum(prof[f"pass{i}_examined"] for i in (1, 2, 3)) / sec / 1e9,
        "tim_plus_ms": statistics.mean(r["ms_total"] for r in runs),
        "phases_ms": {x: st[x] for x in ("ms_kpt", "ms_refine", "ms_select_sample",
                                         "ms_select_greedy")},
        "kpt_round": st["kpt_round"], "kpt_star": st["kpt_star"], "kpt_plus": st["kpt_plus"],
        "theta": st["theta"], "sets_per_step": st["sets_total"],
        "members_select": st["members_select"],
        "roofline": sampler_roofline(prof, "c3"),
        "sampler_profile": prof,
        "autotune": tuning,
        "generate_s": gen_s,
        "clocks": clk,
        "gpu_launches": launches,
        "e2e": e2e,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_c3(args, n, host[0].numpy(), host[1].numpy(),
                                               host[2].numpy())
    del host
    if world == 1 and not args.no_c2:
        line["c2"] = run_c2_line(args, nested=True)
    if not args.no_batch and world == 1:
        line["batched_vs_plain"] = run_batch_compare(args)
    if not args.no_learned and world == 1:
        line["learned_vs_plain"] = run_learned_compare(args)
    return line


def run_spread(args):
    """Forward Monte-Carlo spread (Section 2.1; Section 7 averages 10^5 cascades) of the
    seeds TIM+ returns on the bench graph, IC and LT: --cascades cascades per timed run,
    CUDA events on the library's stream; the mean against the RR-set estimate n * F_R(S)
    of the same run (Corollary 1)."""
    import torch

    from paper_1404_0900_gb300 import tim
    g = inputs.rmat(args.scale, seed=1)
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    out = {"mode": "spread", "scale": args.scale, "k": args.k, "eps": args.eps,
           "cascades": args.cascades, "steps": args.steps, "warmup": args.warmup,
           "models": {}}
    sid0 = 7 << 56
    for name, model, w in (("IC", tim.TIM_IC, inputs.weighted_cascade(g)),
                           ("LT", tim.TIM_LT, inputs.lt_inverse_indegree(g))):
        with tim.Engine(0, stream) as eng:
            tim.tim_load_graph(eng.ctx, g.n, g.rowptr, g.dst, w, model)
            seeds, frac, st = tim.tim_run(eng.ctx, args.k, args.eps, args.ell, args.seed)
            for _ in range(max(args.warmup, 1)):
                tim.tim_spread_mc(eng.ctx, seeds, args.cascades, args.seed, sid0)
            ms = 0.0
            totals = []
            for s in range(args.steps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                mean, total, counts = tim.tim_spread_mc(eng.ctx, seeds, args.cascades, args.seed,
                                                        sid0 + s * args.cascades,
                                                        want_counts=True)
                e1.record(stream)
                e1.synchronize()
                ms += e0.elapsed_time(e1)
                totals.append(counts.astype(np.float64))
            allc = np.concatenate(totals)
            rr = g.n * frac
            out["models"][name] = {
                "cascades_per_s": args.cascades * args.steps / (ms / 1e3),
                "activated_per_s": float(allc.sum()) / (ms / 1e3),
                "ms_per_run": ms / args.steps, "spread_mc": float(allc.mean()),
                "spread_mc_stderr": float(allc.std() / np.sqrt(allc.size)),
                "spread_rr": rr, "rel_diff": float(allc.mean()) / rr - 1.0,
                "theta": st["theta"]}
    return out


def batch_specs(nq: int):
    """The batched workload: query q has an R-MAT graph of scale U{12..20} (graph seed
    q + 1), k ~ U{1..50}, eps from {0.1, 0.2, 0.3, 0.5}; even q use IC weighted cascade,
    odd q LT with 1/indeg in-weights."""
    rng = np.random.Generator(np.random.Philox(20140900))
    out = []
    for q in range(nq):
        scale = int(rng.integers(12, 21))
        k = int(rng.integers(1, 51))
        eps = float(rng.choice([0.1, 0.2, 0.3, 0.5]))
        out.append((scale, q + 1, q % 2, k, eps))
    return out


def run_batch_compare(args, reps: int = 2):
    """End-to-end TIM+ seconds for nq queries: one after another with tim_run (plain)
    against tim_run_batch (batched), both on graphs already loaded; the seeds of every
    query must be the same both ways."""
    import torch

    from paper_1404_0900_gb300 import tim
    specs = batch_specs(args.batch_queries)
    graphs = []
    for scale, gseed, model, k, eps in specs:
        g = inputs.rmat(scale, seed=gseed)
        w = inputs.weighted_cascade(g) if model == 0 else inputs.lt_inverse_indegree(g)
        graphs.append((g, w, model, k, eps))
    stream = torch.cuda.Stream()
    engines = [tim.Engine(0, stream) for _ in graphs]
    try:
        for (g, w, model, _, _), e in zip(graphs, engines):
            tim.tim_load_graph(e.ctx, g.n, g.rowptr, g.dst, w, model)
        queries = [{"ctx": e.ctx, "k": k, "eps": eps, "ell": 1.0, "tag": i + 1}
                   for i, (e, (_, _, _, k, eps)) in enumerate(zip(engines, graphs))]
        for i, e in enumerate(engines):
            tim.tim_set_query_tag(e.ctx, i + 1)
        # autotune on the largest IC query, then use its settings everywhere
        big = max((i for i, sp in enumerate(specs) if sp[2] == 0), key=lambda i: specs[i][0])
        tuning = tim.tim_autotune(engines[big].ctx, 500_000, args.seed)
        for e in engines:
            tim.tim_set_width_budget(e.ctx, tuning["width_budget"])
            tim.tim_set_team_size(e.ctx, tuning["team_size"])
            tim.tim_set_chunk(e.ctx, tuning["chunk"])
            tim.tim_set_team_factor(e.ctx, tuning["team_factor"])
            tim.tim_set_pass1_capacity(e.ctx, tuning["pass1_capacity"])

        def plain():
            outs = []
            for q in queries:
                seeds, _, st = tim.tim_run(q["ctx"], q["k"], q["eps"], 1.0, args.seed)
                outs.append((seeds, st))
            return outs

        def timed(fn):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            out = fn()
            e1.record(stream)
            e1.synchronize()
            return out, e0.elapsed_time(e1)

        mlp = None
        if not getattr(args, "no_learned", False) and start_round.available():
            mlp, _ = start_round.load(engines[0].ctx)
        plain()
        tim.tim_run_batch(queries, args.seed)
        if mlp is not None:
            tim.tim_run_batch(queries, args.seed, mlp=mlp)
        t_plain, t_batch, t_learn = [], [], []
        for _ in range(reps):
            p_out, tp = timed(plain)
            (b_out, bst), tb = timed(lambda: tim.tim_run_batch(queries, args.seed))
            t_plain.append(tp)
            t_batch.append(tb)
            if mlp is not None:
                (l_out, lst), tl = timed(lambda: tim.tim_run_batch(queries, args.seed, mlp=mlp))
                t_learn.append(tl)
        same = all(np.array_equal(p[0], b[0]) and p[1]["theta"] == b[2]["theta"]
                   for p, b in zip(p_out, b_out))
        sets = sum(st["sets_total"] for _, st in p_out)
        learned = None
        if mlp is not None:
            ident = [bool(np.array_equal(p[0], l[0])) for p, l in zip(p_out, l_out)]
            # spread of differing seed sets: coverage of fresh RR sets (set-id phase 6)
            rel = []
            for i, (p, l) in enumerate(zip(p_out, l_out)):
                if ident[i]:
                    continue
                ctx = queries[i]["ctx"]
                cnt = 200_000
                cp = tim.tim_covered_count(ctx, p[0], args.seed + 7, 6 << 56, cnt)
                cl = tim.tim_covered_count(ctx, l[0], args.seed + 7, 6 << 56, cnt)
                rel.append((cl - cp) / max(cp, 1))
            tl = min(t_learn)
            learned = {
                "learned_batched_ms": tl, "speedup_vs_plain": min(t_plain) / tl,
                "speedup_vs_batched": min(t_batch) / tl,
                "accepted": lst["learned_accepted"], "fallback_rate":
                    1.0 - lst["learned_accepted"] / len(specs),
                "seeds_identical_to_plain": int(sum(ident)),
                "spread_rel_diff_of_differing": rel,
                "kpt_launch_rounds": {"batched": bst["kpt_launch_rounds"],
                                      "learned_batched": lst["kpt_launch_rounds"]},
                "phase_ms": {k: lst[k] for k in ("ms_kpt", "ms_predict", "ms_refine",
                                                 "ms_select_sample", "ms_select_greedy")},
                "kpt_rr_sets": {"batched": sum(b[2]["kpt_sets"] for b in b_out),
                                "learned_batched": sum(x[2]["kpt_sets"] for x in l_out)},
            }
            tim.tim_mlp_destroy(mlp)
    finally:
        for e in engines:
            e.close()
    tp, tb = min(t_plain), min(t_batch)
    out = {"queries": len(specs), "scales": "R-MAT U{12..20}", "plain_ms": tp,
           "batched_ms": tb, "speedup": tp / tb, "seeds_identical": bool(same),
           "rr_sets": sets, "batched_rr_sets_per_s": sets / (tb / 1e3),
           "batched_phase_ms": {k: bst[k] for k in ("ms_kpt", "ms_refine", "ms_select_sample",
                                                    "ms_select_greedy")},
           "autotune": tuning}
    if learned is not None:
        out["learned"] = learned
    return out


def run_learned_compare(args, g20=None, w_ic=None, w_lt=None, reps: int = 2):
    """Plain TIM+ against TIM+ from the learned start round on held-out graphs (the
    network was trained on device-drawn graphs of scales 12-18): the host R-MAT scale-20
    graph of the main workload and a device-drawn R-MAT scale-22 graph (seed 2022), IC
    weighted cascade and LT 1/indeg each, k = 50, eps = 0.1. Reports device times, the
    predicted and plain stopping rounds, acceptance (fallback rate) and the spread of
    both seed sets estimated on 10^6 fresh RR sets (set-id phase 6)."""
    import torch

    from paper_1404_0900_gb300 import tim
    if not start_round.available():
        return {"unavailable": "no trained start-round network in the package"}
    if g20 is None:
        g20 = inputs.rmat(20, seed=1)
        w_ic, w_lt = inputs.weighted_cascade(g20), inputs.lt_inverse_indegree(g20)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    k, eps, ell, seed = 50, 0.1, 1.0, args.seed
    cases = []
    with tim.Engine(0, stream) as eng:
        mlp, rec = start_round.load(eng.ctx)
        try:
            g22 = inputs.rmat_device(22, seed=2022)
            w22 = inputs.weighted_cascade_device(g22)  # IC 1/indeg; LT 1/indeg is the same
            graphs = [("rmat20", g20.n, g20.m, torch.from_numpy(g20.rowptr).cuda(),
                       torch.from_numpy(g20.dst).cuda(),
                       {0: torch.from_numpy(w_ic).cuda(), 1: torch.from_numpy(w_lt).cuda()}),
                      ("rmat22", g22.n, g22.m, g22.rowptr, g22.dst, {0: w22, 1: w22})]
            for name, n, m, rp, dst, ws in graphs:
                for model in (tim.TIM_IC, tim.TIM_LT):
                    torch.cuda.synchronize()
                    tim.tim_load_graph_device(eng.ctx, n, m, rp, dst, ws[model], model)
                    tim.tim_autotune(eng.ctx, 500_000, seed)
                    tim.tim_run(eng.ctx, k, eps, ell, seed)
                    tim.tim_run_learned(eng.ctx, mlp, k, eps, ell, seed)
                    tp, tl = [], []
                    for _ in range(reps):
                        ps, _, pst = tim.tim_run(eng.ctx, k, eps, ell, seed)
                        ls, _, lst = tim.tim_run_learned(eng.ctx, mlp, k, eps, ell, seed)
                        tp.append(pst)
                        tl.append(lst)
                    bp = min(tp, key=lambda s: s["ms_total"])
                    bl = min(tl, key=lambda s: s["ms_total"])
                    cnt = 1_000_000
                    cp = tim.tim_covered_count(eng.ctx, ps, seed + 7, 6 << 56, cnt)
                    cl = tim.tim_covered_count(eng.ctx, ls, seed + 7, 6 << 56, cnt)
                    cases.append({
                        "graph": name, "model": "IC" if model == tim.TIM_IC else "LT",
                        "n": n, "m": m,
                        "plain_ms": bp["ms_total"], "learned_ms": bl["ms_total"],
                        "plain_kpt_ms": bp["ms_kpt"], "learned_kpt_ms": bl["ms_kpt"],
                        "plain_round": bp["kpt_round"], "predicted_round": bl["kpt_predicted_round"],
                        "accepted": bool(bl["kpt_accepted"]),
                        "kpt_rr_sets": {"plain": bp["kpt_sets"], "learned": bl["kpt_sets"]},
                        "seeds_identical": bool(np.array_equal(ps, ls)),
                        "spread_estimate": {"plain": n * cp / cnt, "learned": n * cl / cnt},
                    })
        finally:
            tim.tim_mlp_destroy(mlp)
    acc = sum(c["accepted"] for c in cases)
    return {"k": k, "eps": eps, "cases": cases, "fallback_rate": 1.0 - acc / len(cases),
            "plain_ms_total": sum(c["plain_ms"] for c in cases),
            "learned_ms_total": sum(c["learned_ms"] for c in cases),
            "training": {key: rec.get(key) for key in ("graphs", "samples", "held_out", "seconds")}}


def main(argv=None):
    args = parse_args(argv)
    if args.mode == "sample" and args.impl == "ours":
        print(json.dumps(run_sample_only(args)), flush=True)
        return
    if args.mode == "batch" and args.impl == "ours":
        print(json.dumps(run_batch_compare(args)), flush=True)
        return
    if args.mode == "learned" and args.impl == "ours":
        print(json.dumps(run_learned_compare(args)), flush=True)
        return
    if args.mode == "spread" and args.impl == "ours":
        print(json.dumps(run_spread(args)), flush=True)
        return
    if args.impl == "reference":
        line = run_reference(args)
    else:
        line = run_c3_line(args) if args.workload == "c3" else run_c2_line(args)
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
