"""GPU parity of the forward Monte-Carlo spread (Section 2.1: E[I(S)] as the average
number of nodes reachable from S in random graphs; triggering form of Section 4.2):
per-cascade activated counts through the C ABI against the oracle, bit for bit, on the
same seeded graphs, seed sets and set ids -- small graphs of every kind, hubs of a large
out-degree, ragged and empty inputs, the bench's R-MAT 20 graph with TIM+'s own seeds --
and the argument errors."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1404_0900_gb300 import inputs, tim

pytestmark = pytest.mark.gpu
MC = O.make_sid(7, 0, 0)


@pytest.fixture(scope="module")
def eng():
    import torch
    assert torch.cuda.is_available()
    e = tim.Engine(0)
    yield e
    e.close()


def _case(name):
    if name == "rmat12_wc":
        g = inputs.rmat(12, seed=5)
        return g, inputs.weighted_cascade(g), O.IC
    if name == "rmat12_tri":
        g = inputs.rmat(12, seed=6)
        return g, inputs.trivalency(g, seed=3), O.IC
    if name == "rmat12_lt":
        g = inputs.rmat(12, seed=7)
        return g, inputs.lt_inverse_indegree(g), O.LT
    if name == "rmat12_lt_rand":
        g = inputs.rmat(12, seed=8)
        return g, inputs.lt_random_normalised(g, 4), O.LT
    if name == "rand_p1":
        g = inputs.random_small(2000, 6000, seed=2)
        return g, inputs.constant(g, 1.0), O.IC
    if name == "out_star":  # node 0 points to every other node: one 20,000-edge out-list
        g = inputs.from_edges(20001, [(0, i) for i in range(1, 20001)])
        return g, inputs.constant(g, 0.5), O.IC
    if name == "chain_lt":
        g = inputs.chain(3000)
        return g, inputs.lt_inverse_indegree(g), O.LT
    raise KeyError(name)


@pytest.mark.parametrize("name", ["rmat12_wc", "rmat12_tri", "rmat12_lt", "rmat12_lt_rand",
                                  "rand_p1", "out_star", "chain_lt"])
def test_cascade_counts_bit_exact(eng, name):
    g, w, model = _case(name)
    tim.tim_load_graph(eng.ctx, g.n, g.rowptr, g.dst, w, model)
    og = O.load_graph(g.n, g.rowptr, g.dst, w, model)
    rng = np.random.default_rng(1)
    for seeds in ([0], rng.choice(g.n, 20, replace=False).tolist(), [3, 3, 7]):
        for count, sid0 in ((1031, MC + 5), (1, MC + 77)):
            mean, total, counts = tim.tim_spread_mc(eng.ctx, seeds, count, 17, sid0,
                                                    want_counts=True)
            ref, rtot = O.spread_mc(og, seeds, count, 17, sid0)
            assert np.array_equal(counts.astype(np.int64), ref), (name, seeds)
            assert total == rtot and mean == rtot / count


def test_empty_inputs(eng):
    g = inputs.rmat(10, seed=1)
    tim.tim_load_graph(eng.ctx, g.n, g.rowptr, g.dst, inputs.weighted_cascade(g), tim.TIM_IC)
    assert tim.tim_spread_mc(eng.ctx, [1, 2], 0, 1, MC, want_counts=True)[:2] == (0.0, 0)
    mean, total, counts = tim.tim_spread_mc(eng.ctx, [], 50, 1, MC, want_counts=True)
    assert total == 0 and mean == 0.0 and not counts.any()
    # every node a seed: every cascade activates all of them
    mean, total, _ = tim.tim_spread_mc(eng.ctx, list(range(g.n)), 7, 1, MC)
    assert total == 7 * g.n


def test_errors(eng):
    g = inputs.rmat(10, seed=1)
    tim.tim_load_graph(eng.ctx, g.n, g.rowptr, g.dst, inputs.weighted_cascade(g), tim.TIM_IC)
    with pytest.raises(tim.TimError) as e:
        tim.tim_spread_mc(eng.ctx, [0, g.n], 10, 1, MC)
    assert e.value.code == tim.TIM_ERR_ARG
    with pytest.raises(tim.TimError) as e:
        tim.tim_spread_mc(eng.ctx, [-1], 10, 1, MC)
    assert e.value.code == tim.TIM_ERR_ARG
    with tim.Engine(0) as fresh:
        with pytest.raises(tim.TimError) as e:
            tim.tim_spread_mc(fresh.ctx, [0], 10, 1, MC)
        assert e.value.code == tim.TIM_ERR_STATE


@pytest.mark.parametrize("model", [O.IC, O.LT])
def test_full_size_rmat20_with_timplus_seeds(eng, model):
    g = inputs.rmat(20, seed=1)
    w = inputs.weighted_cascade(g) if model == O.IC else inputs.lt_inverse_indegree(g)
    tim.tim_load_graph(eng.ctx, g.n, g.rowptr, g.dst, w, model)
    seeds, frac, _ = tim.tim_run(eng.ctx, 50, 0.1, 1.0, 1)
    mean, total, counts = tim.tim_spread_mc(eng.ctx, seeds, 96, 1, MC, want_counts=True)
    og = O.load_graph(g.n, g.rowptr, g.dst, w, model)
    ref, rtot = O.spread_mc(og, seeds, 96, 1, MC)
    assert np.array_equal(counts.astype(np.int64), ref) and total == rtot
    # the cascades and the RR sets estimate the same E[I(S)] (Corollary 1): within a
    # generous 5 standard errors of the cascades plus 2 % for the RR estimate
    sd = float(ref.std())
    assert abs(mean - g.n * frac) <= 5 * sd / np.sqrt(96) + 0.02 * g.n * frac
