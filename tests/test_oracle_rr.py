"""Pins for the oracle's RR sets (Definitions 1-2, Section 3.1 BFS, Section 4.2 and the
LT setting of Section 6), the in-CSR transpose and the thresholds."""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import breadth_first_order

from oracle import oracle as O
from paper_1404_0900_gb300 import inputs

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _reverse_reach(n, us, vs, root):
    """Nodes that can reach `root` along edges us -> vs, via scipy's BFS on G^T."""
    if len(us) == 0:
        return np.array([root])
    a = sp.csr_matrix((np.ones(len(us)), (vs, us)), shape=(n, n))
    order = breadth_first_order(a, root, directed=True, return_predecessors=False)
    return np.sort(order)


def _graph(g, w, model):
    return O.load_graph(g.n, g.rowptr, g.dst, w, model)


def test_transpose_matches_scipy_and_is_sorted_by_source():
    g = inputs.random_small(50, 400, seed=3)
    w = inputs.uniform_random(g, seed=4)
    og = _graph(g, w, O.IC)
    a = sp.csr_matrix((w, g.dst, g.rowptr), shape=(g.n, g.n)).tocsc()  # columns = dst
    assert np.array_equal(og.rowptr, a.indptr.astype(np.int64))
    for v in range(g.n):
        seg = og.src[og.rowptr[v]:og.rowptr[v + 1]]
        assert np.all(np.diff(seg) > 0)
        col = a[:, v]
        assert np.array_equal(seg, np.sort(col.indices))
        ww = og.in_w[og.rowptr[v]:og.rowptr[v + 1]]
        assert np.array_equal(ww, np.asarray(col.toarray()).ravel()[seg].astype(np.float32))


@pytest.mark.parametrize("bad", ["selfloop", "dup", "range"])
def test_transpose_rejects_bad_graphs(bad):
    rowptr = np.array([0, 2, 3, 3], dtype=np.int64)
    dst = {"selfloop": [1, 0, 2], "dup": [1, 1, 2], "range": [1, 5, 2]}[bad]
    with pytest.raises(ValueError):
        O.load_graph(3, rowptr, np.array(dst, dtype=np.int32), np.full(3, 0.5, np.float32), O.IC)


def test_ic_thresholds_exact():
    ps = np.array([0.0, 1e-9, 0.1, 0.25, 0.5, 0.999999, 1.0], dtype=np.float32)
    g = inputs.star_in(len(ps) + 1)
    og = _graph(g, ps, O.IC)
    for j in range(len(ps)):
        p = Fraction(float(og.in_w[j]))
        want = 0xFFFFFFFF if p >= 1 else math.floor(p * 2 ** 32)
        assert int(og.thr[j]) == want


def test_lt_cumulative_thresholds_exact():
    w = np.array([0.2, 0.3, 0.4], dtype=np.float32)
    g = inputs.star_in(4)
    og = _graph(g, w, O.LT)
    acc = 0
    for j in range(3):
        acc += math.floor(Fraction(float(og.in_w[j])) * 2 ** 32)
        assert int(og.thr[j]) == min(acc, 2 ** 32 - 1)
    with pytest.raises(ValueError):
        _graph(g, np.array([0.5, 0.5, 0.5], dtype=np.float32), O.LT)


def test_p1_rr_set_is_exact_reverse_reachability():
    g = inputs.random_small(60, 150, seed=5)
    og = _graph(g, inputs.constant(g, 1.0), O.IC)
    src = g.src()
    for j in range(200):
        sid = O.make_sid(3, 0, j)
        r, w = O.rr_one(og, 9, sid)
        root = O.root(9, sid, g.n)
        want = _reverse_reach(g.n, src, g.dst, root)
        assert np.array_equal(r, want)
        assert w == int(og.indeg()[want].sum())


def test_p0_rr_set_is_root_alone():
    g = inputs.random_small(40, 200, seed=6)
    for model, w in ((O.IC, inputs.constant(g, 0.0)), (O.LT, inputs.constant(g, 0.0))):
        og = _graph(g, w, model)
        for j in range(100):
            sid = O.make_sid(1, 3, j)
            r, wid = O.rr_one(og, 2, sid)
            root = O.root(2, sid, g.n)
            assert r.tolist() == [root]
            assert wid == int(og.indeg()[root])


def _ic_world(og, seed, sid):
    """Live edges of the random graph g for this set id, from the coins (Python)."""
    us, vs = [], []
    for v in range(og.n):
        for j in range(og.rowptr[v], og.rowptr[v + 1]):
            thr = int(og.thr[j])
            x = O.ic_word(seed, sid, j)
            if thr == 0xFFFFFFFF or x < thr:
                us.append(int(og.src[j]))
                vs.append(v)
    return us, vs


def _lt_world(og, seed, sid):
    us, vs = [], []
    for v in range(og.n):
        lo, hi = og.rowptr[v], og.rowptr[v + 1]
        if hi == lo:
            continue
        x = O.lt_word(seed, sid, v)
        j = int(np.searchsorted(og.thr[lo:hi], x, side="right"))
        if j < hi - lo:
            us.append(int(og.src[lo + j]))
            vs.append(v)
    return us, vs


@pytest.mark.parametrize("model", [O.IC, O.LT])
def test_bfs_equals_definition_and_scipy_world(model):
    g = inputs.random_small(40, 160, seed=8)
    w = inputs.uniform_random(g, 0.0, 0.6, seed=9) if model == O.IC else \
        inputs.lt_random_normalised(g, seed=9) * np.float32(0.95)
    og = _graph(g, w, model)
    world = _ic_world if model == O.IC else _lt_world
    for j in range(60):
        sid = O.make_sid(2, 0, j)
        r_bfs, w_bfs = O.rr_one(og, 4, sid)
        r_def, w_def = O.rr_by_definition(og, 4, sid)
        assert np.array_equal(r_bfs, r_def) and w_bfs == w_def
        us, vs = world(og, 4, sid)
        want = _reverse_reach(g.n, np.array(us), np.array(vs), O.root(4, sid, g.n))
        assert np.array_equal(r_bfs, want)


def test_lt_rr_set_is_the_backward_chain_of_its_world():
    # In an LT world every node keeps at most one live in-edge (Section 6), so the
    # nodes that reach the root form the chain root <- u1 <- u2 <- ... (Section 4.2).
    g = inputs.rmat(9)
    og = _graph(g, inputs.lt_inverse_indegree(g), O.LT)
    for j in range(300):
        sid = O.make_sid(3, 0, j)
        r, _ = O.rr_one(og, 1, sid)
        us, vs = _lt_world(og, 1, sid)
        pred = dict(zip(vs, us))
        chain = [O.root(1, sid, g.n)]
        while chain[-1] in pred and pred[chain[-1]] not in chain:
            chain.append(pred[chain[-1]])
        assert r.tolist() == sorted(chain)


def test_lt_pick_frequencies():
    w = np.array([0.2, 0.3, 0.4], dtype=np.float32)  # none: 0.1
    g = inputs.star_in(4)
    og = _graph(g, w, O.LT)
    counts = np.zeros(4)
    N = 20000
    for j in range(N):
        x = O.lt_word(5, O.make_sid(3, 0, j), 0)
        idx = int(np.searchsorted(og.thr[0:3], x, side="right"))
        counts[idx] += 1
    for c, p in zip(counts, [0.2, 0.3, 0.4, 0.1]):
        assert abs(c / N - p) < 5 * math.sqrt(p * (1 - p) / N)


def test_sample_matches_single_sets_and_thread_count():
    g = inputs.rmat(10)
    og = _graph(g, inputs.weighted_cascade(g), O.IC)
    off1, mem1, w1 = O.sample(og, 3, O.make_sid(3, 0, 0), 5000, nthreads=1)
    off4, mem4, w4 = O.sample(og, 3, O.make_sid(3, 0, 0), 5000, nthreads=4)
    assert np.array_equal(off1, off4) and np.array_equal(mem1, mem4) and np.array_equal(w1, w4)
    for j in range(0, 5000, 97):
        r, w = O.rr_one(og, 3, O.make_sid(3, 0, j))
        assert np.array_equal(np.sort(mem1[off1[j]:off1[j + 1]]), r) and w == w1[j]


def test_golden_example1_rr_sets_and_spread():
    gold = json.load(open(os.path.join(GOLD, "example1_fig1.json")))
    n = gold["n"]
    # deterministic worlds: p = 1 on the live edges, 0 elsewhere
    for key, live_key in (("example1", "live_edges"), ("spread_example", "live_edges")):
        live = {tuple(e) for e in gold[key][live_key]}
        g = inputs.from_edges(n, [(u, v) for u, v, _ in gold["edges"]])
        p = np.array([1.0 if (int(u), int(v)) in live else 0.0
                      for u, v in zip(g.src(), g.dst)], dtype=np.float32)
        og = _graph(g, p, O.IC)
        by_root = {}
        j = 0
        while len(by_root) < n:
            sid = O.make_sid(3, 0, j)
            by_root.setdefault(O.root(1, sid, n), O.rr_one(og, 1, sid)[0].tolist())
            j += 1
        if key == "example1":
            for r, members in gold["example1"]["rr_sets"].items():
                assert by_root[int(r)] == members
            sets = [by_root[r] for r in range(n)]
            off = np.cumsum([0] + [len(s) for s in sets]).astype(np.int64)
            seeds, _, _ = O.greedy(n, off, np.concatenate(sets).astype(np.int32),
                                   gold["example1"]["k"])
            assert seeds.tolist() == gold["example1"]["greedy"]
        else:
            s = gold["spread_example"]["seeds"][0]
            # spread of {s} in this world = number of roots whose RR set holds s
            assert sum(1 for r in range(n) if s in by_root[r]) == gold["spread_example"]["spread"]
