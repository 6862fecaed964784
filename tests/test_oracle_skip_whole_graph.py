"""Whole-graph pin of the oracle's geometric-skip rule for IC in-lists.

Section 3.1 samples an RR set by drawing one coin per examined in-edge. For long in-lists
whose in-edges share one probability the oracle finds the live in-edges instead from
geometric gaps (tim_oracle.c, skip_iter). Other tests pin that rule on isolated lists.
Here the oracle's one-coin-per-in-edge mode (Section 3.1 as printed, no skipping)
serves as the reference on whole graphs, where many skip lists and ordinary lists meet
in one BFS. The two modes use different random numbers, so their sets differ one by
one. What must agree is their law, measured on disjoint set-id ranges:
  - mean |R| and mean w(R) (Eq. 1);
  - the histogram of |R|;
  - how often each of the 20 highest-degree nodes lies in a set;
  - the fraction of sets that fixed seed sets cover (F_R(S) of Corollary 1).
Every difference must stay within 5 standard errors (two-sample z), and the histograms
must pass a chi-square homogeneity test at p > 1e-6. A sensitivity check shows that
the same statistics reject a 2 % error in the live probability of the skip lists.

Graphs: a weighted-cascade R-MAT scale-14 graph (15 lists under the rule, which hold
the hubs every set reaches), and a graph of 4,096 nodes with 2,048 in-lists of 512 to
1,023 in-edges beside 2,048 short ones, p = 0.5 / indeg(v)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1404_0900_gb300 import inputs

Z_MAX = 5.0


def _sets(og, count, sid0, per_edge):
    off, mem, wid = O.sample(og, 1, sid0, count, per_edge=per_edge)
    return off, mem, wid


def _z_mean(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    se = np.sqrt(a.var() / a.size + b.var() / b.size)
    return (a.mean() - b.mean()) / se


def _z_prop(ka, na, kb, nb):
    p = (ka + kb) / (na + nb)
    se = np.sqrt(p * (1 - p) * (1 / na + 1 / nb))
    return 0.0 if se == 0 else (ka / na - kb / nb) / se


def _cover_flags(off, mem, in_s):
    """Per set: does it meet the node set in_s (bool[n])?"""
    return np.logical_or.reduceat(in_s[mem], off[:-1])


def law_statistics(og, a, b, seed_sets, top_nodes):
    """z-scores (and the histogram p-value) of every statistic compared between two
    samples a, b = (off, mem, widths)."""
    from scipy.stats import chi2_contingency
    (oa, ma, wa), (ob, mb, wb) = a, b
    na, nb = oa.size - 1, ob.size - 1
    sa, sb = np.diff(oa), np.diff(ob)
    out = {"size": _z_mean(sa, sb), "width": _z_mean(wa, wb)}
    ca = np.bincount(ma, minlength=og.n)
    cb = np.bincount(mb, minlength=og.n)
    for v in top_nodes:
        out[f"node{v}"] = _z_prop(int(ca[v]), na, int(cb[v]), nb)
    for name, s in seed_sets.items():
        in_s = np.zeros(og.n, dtype=bool)
        in_s[s] = True
        out[f"cover_{name}"] = _z_prop(int(_cover_flags(oa, ma, in_s).sum()), na,
                                       int(_cover_flags(ob, mb, in_s).sum()), nb)
    top = 12
    ha = np.bincount(np.minimum(sa, top), minlength=top + 1)[1:]
    hb = np.bincount(np.minimum(sb, top), minlength=top + 1)[1:]
    keep = (ha + hb) > 0
    out["hist_p"] = chi2_contingency(np.vstack([ha[keep], hb[keep]]))[1]
    return out


def _check(stats):
    bad = {k: v for k, v in stats.items() if k != "hist_p" and abs(v) > Z_MAX}
    assert not bad, bad
    assert stats["hist_p"] > 1e-6, stats["hist_p"]


def _top_and_seeds(g, og, rng_seed):
    deg = g.indeg() + np.diff(g.rowptr)
    top = np.argsort(-deg, kind="stable")[:20]
    rng = np.random.Generator(np.random.Philox(rng_seed))
    indeg = og.indeg()
    seeds = {"top_in": np.argsort(-indeg, kind="stable")[:10],
             "top_out": np.argsort(-np.diff(g.rowptr), kind="stable")[:10],
             "random50": rng.choice(g.n, size=50, replace=False),
             "random500": rng.choice(g.n, size=500, replace=False)}
    return top, seeds


@pytest.fixture(scope="module")
def rmat14():
    g = inputs.rmat(14, seed=1)
    og = O.load_graph(g.n, g.rowptr, g.dst, inputs.weighted_cascade(g), O.IC)
    return g, og


@pytest.fixture(scope="module")
def mixed():
    g = inputs.mixed_in_degree(4096, seed=5)
    w = (0.5 * inputs.weighted_cascade(g)).astype(np.float32)
    return g, w, O.load_graph(g.n, g.rowptr, g.dst, w, O.IC)


def _skip_lists(og):
    d = og.indeg()
    return sum(1 for v in range(og.n)
               if d[v] and O.skip_applies(int(d[v]), int(og.thr[og.rowptr[v]]))
               and np.all(og.thr[og.rowptr[v]:og.rowptr[v + 1]] == og.thr[og.rowptr[v]]))


def test_rmat14_weighted_cascade_skip_rule_has_the_per_edge_law(rmat14):
    g, og = rmat14
    assert _skip_lists(og) >= 10
    count = 200_000
    a = _sets(og, count, O.make_sid(9, 1, 0), per_edge=False)
    b = _sets(og, count, O.make_sid(9, 2, 0), per_edge=True)
    top, seeds = _top_and_seeds(g, og, 11)
    _check(law_statistics(og, a, b, seeds, top))


def test_many_skip_lists_have_the_per_edge_law(mixed):
    g, _, og = mixed
    assert _skip_lists(og) == 2048
    count = 1_000_000
    a = _sets(og, count, O.make_sid(9, 3, 0), per_edge=False)
    b = _sets(og, count, O.make_sid(9, 4, 0), per_edge=True)
    top, seeds = _top_and_seeds(g, og, 12)
    _check(law_statistics(og, a, b, seeds, top))


def test_statistics_reject_a_two_percent_error_on_the_skip_lists(mixed):
    """Sensitivity: per-edge sets of the same graph whose long lists carry 2 % more
    probability must fail the comparison with the skip rule's sets."""
    g, w, og = mixed
    indeg = g.indeg()
    w2 = w.copy()
    w2[indeg[g.dst] >= O.SKIP_MIN_INDEG] *= np.float32(1.02)
    og2 = O.load_graph(g.n, g.rowptr, g.dst, w2, O.IC)
    count = 1_000_000
    a = _sets(og, count, O.make_sid(9, 3, 0), per_edge=False)
    b = _sets(og2, count, O.make_sid(9, 5, 0), per_edge=True)
    top, seeds = _top_and_seeds(g, og, 12)
    st = law_statistics(og, a, b, seeds, top)
    assert abs(st["size"]) > Z_MAX and abs(st["width"]) > Z_MAX, st


def test_per_edge_mode_is_the_definition_and_leaves_other_lists_alone(mixed):
    g, _, og = mixed
    # BFS = Definitions 1-2 with the whole world drawn, in the per-edge mode too
    for j in range(40):
        sid = O.make_sid(9, 6, j)
        bfs, wb = O.rr_one(og, 3, sid, per_edge=True)
        ref, wr = O.rr_by_definition(og, 3, sid, per_edge=True)
        assert np.array_equal(bfs, ref) and wb == wr
    # graphs with no list under the rule: both modes give the same sets
    h = inputs.rmat(10, seed=2)
    for w, model in ((inputs.trivalency(h, seed=3), O.IC), (inputs.lt_inverse_indegree(h), O.LT),
                     (inputs.weighted_cascade(h), O.IC)):
        oh = O.load_graph(h.n, h.rowptr, h.dst, w, model)
        if model == O.IC and _skip_lists(oh):
            continue
        a = O.sample(oh, 5, O.make_sid(3, 0, 0), 3000)
        b = O.sample(oh, 5, O.make_sid(3, 0, 0), 3000, per_edge=True)
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
