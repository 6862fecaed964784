"""One TIM+ query split over CPU ranks by set id (gloo, 127.0.0.1), on the oracle: the
graph is replicated, every rank generates its share of each phase's RR sets, and the
ranks all-reduce the exact kappa sum of every Algorithm 2 round, the covered count of
Algorithm 3 and the coverage counts of every greedy round. The result must equal the
single-process oracle TIM+ exactly: stopping round, KPT*, theta', the covered count of
Algorithm 3, KPT+, theta, the seeds and the covered count."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

from oracle import oracle as O
from paper_1404_0900_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RANK_CODE = r"""
import json, os, sys
import numpy as np
import torch.distributed as dist
from oracle import oracle as O, sharded
from paper_1404_0900_gb300 import inputs
rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
dist.init_process_group("gloo")
import torch

def allreduce(arr):
    t = torch.from_numpy(arr)
    dist.all_reduce(t)

out = {}
for name, (scale, model, k, eps) in json.loads(sys.argv[1]).items():
    g = inputs.rmat(scale, seed=4)
    w = inputs.weighted_cascade(g) if model == 0 else inputs.lt_inverse_indegree(g)
    og = O.load_graph(g.n, g.rowptr, g.dst, w, model)
    r = sharded.tim_plus_sharded(og, k, eps, 1.0, 17, rank, world, allreduce, nthreads=2)
    r["seeds"] = r["seeds"].tolist()
    out[name] = r
dist.barrier()
dist.destroy_process_group()
print(json.dumps({"rank": rank, "out": out}))
"""

CASES = {"ic": (11, O.IC, 10, 0.3), "lt": (11, O.LT, 5, 0.5)}


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _run_ranks(world: int):
    port = _free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE=str(world),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, "-c", RANK_CODE, json.dumps(CASES)],
                                      cwd=ROOT, env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=600)
        assert p.returncode == 0, err[-3000:]
        outs.append(json.loads(out.strip().splitlines()[-1]))
    return outs


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_oracle_tim_plus_equals_single_process(world):
    outs = _run_ranks(world)
    for name, (scale, model, k, eps) in CASES.items():
        g = inputs.rmat(scale, seed=4)
        w = inputs.weighted_cascade(g) if model == O.IC else inputs.lt_inverse_indegree(g)
        og = O.load_graph(g.n, g.rowptr, g.dst, w, model)
        ref = O.tim_plus(og, k, eps, 1.0, 17, nthreads=2)
        for o in outs:
            r = o["out"][name]
            assert r["kpt_round"] == ref.kpt.stop_round, (name, world)
            assert r["kpt_star"] == ref.kpt.kpt_star
            assert r["theta_prime"] == ref.refine.theta_prime
            assert r["covered_prime"] == ref.refine.covered
            assert r["kpt_plus"] == ref.refine.kpt_plus
            assert r["theta"] == ref.theta
            assert np.array_equal(np.array(r["seeds"]), ref.seeds), (name, world)
            assert r["covered"] == ref.covered


def test_shard_ranges_partition_every_phase():
    from oracle import sharded
    for c in (0, 1, 7, 1000, 12345677):
        for world in (1, 2, 3, 8):
            spans = [sharded.shard(c, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == c
            assert all(spans[i][1] == spans[i + 1][0] for i in range(world - 1))


def test_limb_all_reduce_is_exact():
    from oracle import sharded
    vals = [(1 << 127) - 12345, (1 << 96) + 7, 0, (1 << 64) - 1]

    def fake(arr, parts=vals):
        # the sum over "ranks" whose values are parts[i], as the limbs would add
        tot = np.zeros_like(arr)
        for v in parts:
            tot += np.array([(v >> (32 * i)) & 0xFFFFFFFF for i in range(4)], dtype=np.int64)
        arr[:] = tot
    assert sharded.allreduce_int(vals[0], fake) == sum(vals)
