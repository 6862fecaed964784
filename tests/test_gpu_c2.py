"""GPU parity of the bench's own workload at full size and in the bench's launch
configuration: TIM+ on the directed R-MAT scale-20 graph (n = 1,048,576, ~16M edges),
k = 50, eps = 0.1, l = 1, seed 1, IC weighted cascade and LT 1/indeg, the graph loaded
from device memory and the sampler autotuned first, exactly as `bench.py` runs it.
Compared with the oracle's TIM+ on the same graph: stopping round, KPT*, theta', the
covered count of Algorithm 3, KPT+ (1e-9), lambda, theta, the 50 seeds, Algorithm 1's
covered count and member total."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1404_0900_gb300 import inputs, tim

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def graph():
    return inputs.rmat(20, seed=1)


@pytest.mark.parametrize("model", [O.IC, O.LT])
def test_bench_workload_tim_plus_full_size(graph, model):
    import torch
    g = graph
    w = inputs.weighted_cascade(g) if model == O.IC else inputs.lt_inverse_indegree(g)
    k, eps, ell, seed = 50, 0.1, 1.0, 1
    with tim.Engine(0) as eng:
        d_rowptr = torch.from_numpy(g.rowptr).cuda()
        d_dst = torch.from_numpy(g.dst).cuda()
        d_w = torch.from_numpy(w).cuda()
        torch.cuda.synchronize()
        tim.tim_load_graph_device(eng.ctx, g.n, g.m, d_rowptr, d_dst, d_w, model)
        tim.tim_autotune(eng.ctx, 1_000_000, seed)
        seeds, frac, st = tim.tim_run(eng.ctx, k, eps, ell, seed)
    og = O.load_graph(g.n, g.rowptr, g.dst, w, model)
    ref = O.tim_plus(og, k, eps, ell, seed)
    assert st["kpt_round"] == ref.kpt.stop_round
    assert st["kpt_star"] == ref.kpt.kpt_star
    assert st["theta_prime"] == ref.refine.theta_prime
    assert st["covered_prime"] == ref.refine.covered
    assert abs(st["kpt_plus"] - ref.refine.kpt_plus) <= 1e-9 * ref.refine.kpt_plus
    lam = O.lam(g.n, k, eps, ell)
    assert abs(st["lambda"] - lam) <= 1e-9 * lam
    q = lam / ref.refine.kpt_plus
    assert st["theta"] == ref.theta or abs(q - round(q)) <= 1e-9 * q
    if st["theta"] == ref.theta:
        assert np.array_equal(seeds, ref.seeds)
        assert st["covered"] == ref.covered
        assert frac == ref.covered / ref.theta
        assert st["members_select"] == ref.extra["members"]
