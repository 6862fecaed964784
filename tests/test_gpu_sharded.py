"""One TIM+ query split over ranks by set id, through the C ABI (tim_run_sharded): two
and three processes (gloo on 127.0.0.1 for the all-reduces, which run on the host),
each with its own context on the one GPU, every rank generating its share of each
phase's RR sets. Every rank's result must equal tim_run on one context and the
oracle's TIM+ bit for bit: stopping round, KPT*, theta', Algorithm 3's covered count,
KPT+, theta, the seeds and the covered count. The stepwise greedy calls it uses
(tim_select_begin / counts / take) are checked against tim_node_select on one store."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

from oracle import oracle as O
from paper_1404_0900_gb300 import inputs, tim

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RANK_CODE = r"""
import json, os, sys
import numpy as np
import torch
import torch.distributed as dist
from paper_1404_0900_gb300 import inputs, tim
rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
dist.init_process_group("gloo")
torch.cuda.set_device(0)
red = tim.torch_allreduce(dist)
out = {}
for name, (scale, kind, model, k, eps) in json.loads(sys.argv[1]).items():
    g = inputs.rmat(scale, seed=6)
    if kind == "tri":
        w = inputs.trivalency(g, seed=2)
    elif kind != "trig":
        w = inputs.weighted_cascade(g) if model == 0 else inputs.lt_inverse_indegree(g)
    with tim.Engine(0) as eng:
        if kind == "trig":
            tim.tim_load_graph_triggering(eng.ctx, g.n, g.rowptr, g.dst,
                                          *inputs.triggering_random(g, seed=3))
        else:
            tim.tim_load_graph(eng.ctx, g.n, g.rowptr, g.dst, w, model)
        seeds, frac, st = tim.tim_run_sharded(eng.ctx, k, eps, 1.0, 23, rank, world, red)
    out[name] = {"seeds": seeds.tolist(), "frac": frac,
                 **{x: st[x] for x in ("kpt_round", "kpt_star", "theta_prime",
                                       "covered_prime", "kpt_plus", "theta", "covered",
                                       "members_select", "sets_total")}}
dist.barrier()
dist.destroy_process_group()
print(json.dumps({"rank": rank, "out": out}))
"""

CASES = {"wc_ic": (14, "wc", 0, 20, 0.3), "lt": (14, "wc", 1, 10, 0.5),
         "tri_ic": (13, "tri", 0, 8, 0.5), "triggering": (13, "trig", 2, 8, 0.5)}


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _run_ranks(world: int):
    port = _free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE=str(world),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", RANK_CODE, json.dumps(CASES)],
                                      cwd=ROOT, env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=900)
        assert p.returncode == 0, err[-3000:]
        outs.append(json.loads(out.strip().splitlines()[-1]))
    return outs


def _graph(scale, kind, model):
    g = inputs.rmat(scale, seed=6)
    if kind == "trig":
        return g, inputs.triggering_random(g, seed=3)
    if kind == "tri":
        return g, inputs.trivalency(g, seed=2)
    return g, inputs.weighted_cascade(g) if model == O.IC else inputs.lt_inverse_indegree(g)


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_tim_plus_equals_one_context_and_the_oracle(world):
    outs = _run_ranks(world)
    for name, (scale, kind, model, k, eps) in CASES.items():
        g, w = _graph(scale, kind, model)
        with tim.Engine(0) as eng:
            if kind == "trig":
                tim.tim_load_graph_triggering(eng.ctx, g.n, g.rowptr, g.dst, *w)
                og = O.load_graph_triggering(g.n, g.rowptr, g.dst, *w)
            else:
                tim.tim_load_graph(eng.ctx, g.n, g.rowptr, g.dst, w, model)
                og = O.load_graph(g.n, g.rowptr, g.dst, w, model)
            seeds, frac, st = tim.tim_run(eng.ctx, k, eps, 1.0, 23)
        ref = O.tim_plus(og, k, eps, 1.0, 23)
        assert np.array_equal(seeds, ref.seeds) and st["theta"] == ref.theta
        for o in outs:
            r = o["out"][name]
            assert r["kpt_round"] == st["kpt_round"] == ref.kpt.stop_round, (name, world)
            assert r["kpt_star"] == st["kpt_star"] == ref.kpt.kpt_star
            assert r["theta_prime"] == st["theta_prime"] == ref.refine.theta_prime
            assert r["covered_prime"] == st["covered_prime"] == ref.refine.covered
            assert r["kpt_plus"] == st["kpt_plus"]
            assert abs(r["kpt_plus"] - ref.refine.kpt_plus) <= 1e-9 * ref.refine.kpt_plus
            assert r["theta"] == st["theta"]
            assert np.array_equal(np.array(r["seeds"], dtype=np.int32), seeds), (name, world)
            assert r["covered"] == st["covered"] == ref.covered
            assert r["frac"] == frac
            assert r["members_select"] == st["members_select"]
            assert r["sets_total"] == st["sets_total"]


def test_stepwise_greedy_equals_node_select():
    g = inputs.rmat(12, seed=5)
    w = inputs.weighted_cascade(g)
    with tim.Engine(0) as eng:
        tim.tim_load_graph(eng.ctx, g.n, g.rowptr, g.dst, w, tim.TIM_IC)
        tim.tim_sample_rr(eng.ctx, 30000, 3, 0)
        seeds, _, cov = tim.tim_node_select(eng.ctx, 12)
        tim.tim_select_begin(eng.ctx)
        first = tim.tim_coverage_counts(eng.ctx, g.n)
        covered, chosen = 0, []
        for _ in range(12):
            c = tim.tim_select_counts(eng.ctx, g.n).astype(np.int64)
            c[chosen] = -1
            v = int(np.argmax(c))
            chosen.append(v)
            covered += tim.tim_select_take(eng.ctx, v)
        assert chosen == seeds.tolist() and covered == cov
        assert first.sum() > 0
        # sampling ends the open selection
        tim.tim_sample_rr(eng.ctx, 10, 3, 0)
        with pytest.raises(tim.TimError) as ei:
            tim.tim_select_take(eng.ctx, 0)
        assert ei.value.code == tim.TIM_ERR_STATE
