"""Pins of the oracle's general triggering model (Section 4.2): node v picks one of its
options (a set of in-edges) with the option's probability, or none; an RR set is then
the set of nodes that reach the root through picked in-edges. Pinned by:
  - the LT model written as singleton options equals the LT model set by set (the pick
    uses the same draw and the same cumulative thresholds);
  - the IC model written as all subsets of each in-list has IC's exact spread (every
    world enumerated), so IC and LT are special cases;
  - BFS = the definition with every node's option drawn first (Definitions 1-2);
  - the exact RR-set distribution and Corollary 1 on tiny graphs, every trigger world
    enumerated;
  - world by world, the RR set of an id meets S iff the forward cascade of S with the
    same id reaches the root;
  - invalid distributions are rejected."""
import itertools
import math

import numpy as np
import pytest

from oracle import exact
from oracle import oracle as O
from paper_1404_0900_gb300 import inputs


def _tiny_graph(n, edges):
    """A graph from (u, v) pairs and its out-CSR edge ids, in out-CSR order."""
    g = inputs.from_edges(n, edges)
    src = g.src()
    return g, [(int(src[e]), int(g.dst[e])) for e in range(g.m)]


def _options_arrays(n, opts):
    """opts[v] = [(prob, [edge ids]), ...] -> the loader's arrays."""
    orow, prob, erow, edges = [0], [], [0], []
    for v in range(n):
        for p, es in opts.get(v, []):
            prob.append(p)
            edges.extend(es)
            erow.append(len(edges))
        orow.append(len(prob))
    return (np.array(orow, np.int64), np.array(prob, np.float32), np.array(erow, np.int64),
            np.array(edges, np.int64))


def _exact_options(n, opts, pairs):
    """The same distribution for exact.trig_worlds: in-neighbours instead of edge ids; the
    probabilities as the float32 values the oracle reads."""
    return [[(float(np.float32(p)), [pairs[e][0] for e in es]) for p, es in opts.get(v, [])]
            for v in range(n)]


def test_lt_as_singleton_options_is_the_lt_model():
    g = inputs.rmat(10, seed=2)
    for w in (inputs.lt_inverse_indegree(g), inputs.lt_random_normalised(g, 3)):
        ot = O.load_graph_triggering(g.n, g.rowptr, g.dst, *inputs.triggering_from_lt(g, w))
        ol = O.load_graph(g.n, g.rowptr, g.dst, w, O.LT)
        a = O.sample(ot, 5, O.make_sid(3, 0, 0), 20000)
        b = O.sample(ol, 5, O.make_sid(3, 0, 0), 20000)
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
        ra, rb = O.tim_plus(ot, 5, 0.5, 1.0, 9), O.tim_plus(ol, 5, 0.5, 1.0, 9)
        assert np.array_equal(ra.seeds, rb.seeds) and ra.theta == rb.theta


def _ic_as_triggering(n, pairs, p):
    """IC with probability p per edge: node v's options are the non-empty subsets T of its
    in-edges with probability prod_{e in T} p_e prod_{e not in T} (1 - p_e)."""
    opts = {}
    for v in range(n):
        ins = [e for e, (_, dv) in enumerate(pairs) if dv == v]
        lst = []
        for r in range(1, len(ins) + 1):
            for sub in itertools.combinations(ins, r):
                pr = 1.0
                for e in ins:
                    pr *= p[e] if e in sub else 1.0 - p[e]
                lst.append((pr, list(sub)))
        if lst:
            opts[v] = lst
    return opts


def test_ic_as_all_subsets_has_the_ic_spread():
    g, pairs = _tiny_graph(6, [(0, 1), (0, 2), (1, 2), (2, 3), (3, 1), (1, 4), (4, 5), (2, 5),
                               (5, 0)])
    rng = np.random.default_rng(3)
    p = [float(x) for x in rng.uniform(0.1, 0.9, len(pairs))]
    opts = _ic_as_triggering(g.n, pairs, p)
    ex_opts = [[(pr, [pairs[e][0] for e in es]) for pr, es in opts.get(v, [])]
               for v in range(g.n)]
    ic_edges = [(u, v, p[e]) for e, (u, v) in enumerate(pairs)]
    for S in ([0], [2], [1, 4], [0, 3, 5]):
        a = exact.spread(g.n, None, S, model=2, options=ex_opts)
        b = exact.spread(g.n, ic_edges, S, model=0)
        assert abs(a - b) <= 1e-12 * b


def _random_tiny_distribution(seed):
    rng = np.random.default_rng(seed)
    g, pairs = _tiny_graph(6, [(0, 1), (2, 1), (3, 1), (1, 2), (4, 2), (0, 3), (2, 3), (5, 4),
                               (3, 4), (1, 5), (0, 5), (4, 0)])
    opts = {}
    for v in range(g.n):
        ins = [e for e, (_, dv) in enumerate(pairs) if dv == v]
        k = int(rng.integers(1, 4))
        r = rng.random(k)
        r *= rng.uniform(0.4, 1.0) / r.sum()
        opts[v] = []
        for i in range(k):
            size = int(rng.integers(1, len(ins) + 1))
            opts[v].append((float(r[i]), sorted(rng.choice(ins, size, replace=False).tolist())))
    return g, pairs, opts


@pytest.mark.parametrize("seed", [1, 2])
def test_rr_distribution_and_corollary_1_by_enumeration(seed):
    g, pairs, opts = _random_tiny_distribution(seed)
    og = O.load_graph_triggering(g.n, g.rowptr, g.dst, *_options_arrays(g.n, opts))
    ex_opts = _exact_options(g.n, opts, pairs)
    count = 400_000
    off, mem, _ = O.sample(og, 11, O.make_sid(3, 0, 0), count)
    sets = [frozenset(mem[off[j]:off[j + 1]].tolist()) for j in range(count)]
    # the exact distribution of a random RR set against the frequencies
    dist = exact.rr_distribution(g.n, None, model=2, options=ex_opts)
    freq = {}
    for r in sets:
        freq[r] = freq.get(r, 0) + 1
    assert set(freq) <= set(dist)
    for r, pr in dist.items():
        se = math.sqrt(pr * (1 - pr) / count)
        assert abs(freq.get(r, 0) / count - pr) <= 5 * se + 1e-9, (r, pr)
    # Corollary 1: n F_R(S) estimates E[I(S)]
    for S in ([0], [1, 4], [2, 3, 5]):
        ex = exact.spread(g.n, None, S, model=2, options=ex_opts)
        cov = sum(1 for r in sets if r & set(S))
        f = ex / g.n
        assert abs(cov / count - f) <= 5 * math.sqrt(f * (1 - f) / count), (S, cov, ex)


def test_bfs_equals_definition_and_the_cascade_duality():
    g = inputs.rmat(10, seed=5)
    og = O.load_graph_triggering(g.n, g.rowptr, g.dst, *inputs.triggering_random(g, seed=6))
    S = [0, 1, 2, 7, 100]
    for j in range(300):
        sid = O.make_sid(3, 0, j)
        bfs, wb = O.rr_one(og, 4, sid)
        ref, wr = O.rr_by_definition(og, 4, sid)
        assert np.array_equal(bfs, ref) and wb == wr
        # width: in-degrees of the members (Eq. 1)
        assert wb == int(og.indeg()[bfs].sum())
        casc = O.cascade_one(og, S, 4, sid)
        root = O.root(4, sid, g.n)
        assert (root in set(casc.tolist())) == bool(set(bfs.tolist()) & set(S))


def test_forward_spread_matches_the_exact_spread():
    g, pairs, opts = _random_tiny_distribution(3)
    og = O.load_graph_triggering(g.n, g.rowptr, g.dst, *_options_arrays(g.n, opts))
    ex_opts = _exact_options(g.n, opts, pairs)
    for S in ([0], [3, 5]):
        counts, tot = O.spread_mc(og, S, 200_000, 2, O.make_sid(7, 0, 0))
        ex = exact.spread(g.n, None, S, model=2, options=ex_opts)
        se = counts.std() / math.sqrt(counts.size)
        assert abs(counts.mean() - ex) <= 5 * se + 1e-9


def test_invalid_triggering_distributions_are_rejected():
    g, pairs = _tiny_graph(4, [(0, 1), (2, 1), (1, 3), (0, 3)])
    into = {v: [e for e, (_, dv) in enumerate(pairs) if dv == v] for v in range(g.n)}
    good = {1: [(0.5, into[1])], 3: [(0.3, [into[3][0]]), (0.6, [into[3][1]])]}
    O.load_graph_triggering(g.n, g.rowptr, g.dst, *_options_arrays(g.n, good))
    bad = [
        {1: [(0.7, into[1]), (0.4, [into[1][0]])]},  # probabilities sum above 1
        {1: [(0.5, [into[3][0]])]},                    # an edge into another node
        {1: [(0.5, [into[1][0], into[1][0]])]},        # a repeated edge
        {1: [(-0.1, into[1])]},                        # negative probability
    ]
    for b in bad:
        with pytest.raises(ValueError):
            O.load_graph_triggering(g.n, g.rowptr, g.dst, *_options_arrays(g.n, b))
