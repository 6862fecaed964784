"""Pins for the oracle's forward Monte-Carlo spread (Section 2.1: the estimate of E[I(S)]
as the average number of nodes reachable from S in random graphs g; triggering form of
Section 4.2): exact spreads by enumerating every world on tiny graphs, the worked
spread example of Section 2.1, p = 1 (forward reachability) and p = 0 (the seeds), and
the RR-set duality world by world (the root of an RR set is activated from S exactly
when the set meets S, Definitions 1-2) wherever both walks read the same coins."""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import breadth_first_order

from oracle import exact as X
from oracle import oracle as O
from paper_1404_0900_gb300 import inputs

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
MC = O.make_sid(7, 0, 0)

TINY_IC = [(0, 1, 0.5), (1, 2, 0.4), (2, 0, 0.3), (3, 0, 0.7), (3, 4, 0.2), (4, 1, 0.6),
           (1, 3, 0.25), (2, 4, 0.5)]
TINY_LT = [(0, 1, 0.5), (4, 1, 0.4), (1, 2, 0.9), (2, 0, 0.3), (3, 0, 0.6), (3, 4, 0.2),
           (2, 4, 0.7), (1, 3, 1.0)]


def _og(n, edges, model):
    g = inputs.from_edges(n, [(u, v) for u, v, _ in edges])
    pmap = {(u, v): p for u, v, p in edges}
    w = np.array([pmap[(int(u), int(v))] for u, v in zip(g.src(), g.dst)], dtype=np.float32)
    return O.load_graph(n, g.rowptr, g.dst, w, model)


@pytest.mark.parametrize("model,edges", [(O.IC, TINY_IC), (O.LT, TINY_LT)])
def test_mean_matches_exact_spread(model, edges):
    og = _og(5, edges, model)
    cascades = 200_000
    for seeds in ([0], [3], [1, 4], [0, 2, 3]):
        exact = X.spread(5, edges, seeds, model)
        counts, total = O.spread_mc(og, seeds, cascades, 11, MC)
        assert total == int(counts.sum())
        sd = max(float(counts.std()), 1e-9)
        assert abs(total / cascades - exact) <= 5.0 * sd / np.sqrt(cascades), (seeds, exact)


def test_golden_spread_example_of_section_2_1():
    gold = json.load(open(os.path.join(GOLD, "example1_fig1.json")))
    n, ex = gold["n"], gold["spread_example"]
    live = {tuple(e) for e in ex["live_edges"]}
    # the example's world: the two edges it names as taken are live, the rest dead
    edges = [(u, v, 1.0 if (u, v) in live else 0.0) for u, v, _ in gold["edges"]]
    og = _og(n, edges, O.IC)
    counts, _ = O.spread_mc(og, ex["seeds"], 50, 1, MC)
    assert counts.tolist() == [ex["spread"]] * 50
    assert O.cascade_one(og, ex["seeds"], 1, MC).tolist() == [0, 1, 3]


def test_p1_cascades_are_forward_reachability():
    g = inputs.random_small(300, 900, seed=6)
    og = O.load_graph(g.n, g.rowptr, g.dst, inputs.constant(g, 1.0), O.IC)
    a = sp.csr_matrix((np.ones(g.m), g.dst, g.rowptr), shape=(g.n, g.n))
    rng = np.random.default_rng(2)
    for _ in range(5):
        seeds = rng.choice(g.n, size=3, replace=False)
        reach = set()
        for s in seeds:
            reach |= set(breadth_first_order(a, int(s), directed=True,
                                             return_predecessors=False).tolist())
        counts, _ = O.spread_mc(og, seeds, 20, 3, MC)
        assert counts.tolist() == [len(reach)] * 20
        assert O.cascade_one(og, seeds, 3, MC + 5).tolist() == sorted(reach)


def test_p0_cascades_are_the_distinct_seeds():
    g = inputs.random_small(100, 400, seed=7)
    og = O.load_graph(g.n, g.rowptr, g.dst, inputs.constant(g, 0.0), O.IC)
    counts, total = O.spread_mc(og, [5, 9, 5, 40], 30, 4, MC)
    assert counts.tolist() == [3] * 30 and total == 90


def _duality(og, seeds, seed, sids):
    s = set(int(x) for x in seeds)
    for sid in sids:
        root = O.root(seed, sid, og.n)
        rr, _ = O.rr_one(og, seed, sid)
        act = O.cascade_one(og, seeds, seed, sid)
        assert (root in set(act.tolist())) == bool(s & set(rr.tolist())), sid


@pytest.mark.parametrize("weights", ["inv_indeg", "random_normalised"])
def test_lt_rr_duality_world_by_world(weights):
    g = inputs.rmat(10, seed=5)
    w = inputs.lt_inverse_indegree(g) if weights == "inv_indeg" else inputs.lt_random_normalised(g, 8)
    og = O.load_graph(g.n, g.rowptr, g.dst, w, O.LT)
    for seeds in ([0], [3, 17, 100], list(range(0, 1000, 50))):
        _duality(og, seeds, 9, [O.make_sid(3, 0, j) for j in range(400)])


def test_ic_rr_duality_world_by_world_without_skipped_lists():
    # trivalency: no in-list carries one shared probability, so RR sampling flips the
    # same per-edge coins as the cascades
    g = inputs.rmat(11, seed=6)
    og = O.load_graph(g.n, g.rowptr, g.dst, inputs.trivalency(g, seed=2), O.IC)
    for seeds in ([0], [1, 2, 3], list(range(0, 2048, 64))):
        _duality(og, seeds, 13, [O.make_sid(3, 0, j) for j in range(400)])
    # weighted cascade on a graph whose in-degrees stay below the skip rule's 512
    g = inputs.rmat(9, seed=2)
    assert int(np.bincount(g.dst, minlength=g.n).max()) < 512
    og = O.load_graph(g.n, g.rowptr, g.dst, inputs.weighted_cascade(g), O.IC)
    _duality(og, [0, 7, 30], 5, [O.make_sid(3, 0, j) for j in range(400)])


def test_threads_do_not_change_counts():
    g = inputs.rmat(10, seed=4)
    og = O.load_graph(g.n, g.rowptr, g.dst, inputs.weighted_cascade(g), O.IC)
    c1, t1 = O.spread_mc(og, [0, 1, 2], 700, 3, MC, nthreads=1)
    c4, t4 = O.spread_mc(og, [0, 1, 2], 700, 3, MC, nthreads=4)
    assert np.array_equal(c1, c4) and t1 == t4
    for c in (0, 13, 699):
        assert len(O.cascade_one(og, [0, 1, 2], 3, MC + c)) == c1[c]
