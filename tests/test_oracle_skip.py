"""Pins for the geometric-skip rule of IC in-lists that share one threshold t (at least
512 in-edges, t (2 bitlength(d) + 2) < 2^32): each in-edge must be live with
probability t / 2^32, independently, exactly as with one coin per edge.

- The fixed-point powers Q_b against q^(2^b) computed to 80 digits.
- The digit decision against the exact rational comparison U (2^64 + Q) < Q 2^64.
- Live counts, per-position frequencies, pair frequencies and the first-gap law against
  Bernoulli(t / 2^32) per edge, for several t.
- A restatement of the gap procedure in Python (independent of the C code) on a few
  lists, and RR sets by BFS against RR sets from the drawn world on graphs with hubs.
"""
import math
from decimal import Decimal, getcontext

import numpy as np
import pytest

from oracle import oracle as O
from paper_1404_0900_gb300 import inputs

M64 = 1 << 64


def test_q_powers_against_high_precision():
    getcontext().prec = 80
    for t in (1, 85899, 1 << 20, 0x7FFFFFFF, 0xFFFFFF00, 4294967294):
        q = Decimal((1 << 32) - t) / Decimal(1 << 32)
        x = q
        for b in range(0, 32):
            want = x * Decimal(M64)
            got = O.skip_q(t, b)
            assert abs(Decimal(got) - want) <= Decimal(2 ** b), (t, b)
            x = x * x
    assert O.skip_q(85899, 0) == ((1 << 32) - 85899) << 32  # exact at b = 0


def test_digit_decision_is_the_exact_rational_test():
    rng = np.random.default_rng(11)
    qs = [1, 2, 3, M64 - 1, M64 - (1 << 32), 1 << 63, (1 << 63) + 12345]
    qs += [int(x) for x in rng.integers(0, 2**63, size=40, dtype=np.uint64)] + \
          [int(x) << 1 | 1 for x in rng.integers(0, 2**63, size=40, dtype=np.uint64)]
    for q in qs:
        cut = q * M64 // (M64 + q)  # largest u with u (2^64 + q) < q 2^64 is near here
        us = [0, 1, max(cut - 1, 0), cut, cut + 1, q - 1, q, q + 1, M64 - 1]
        us += [int(x) for x in rng.integers(0, 2**63, size=8, dtype=np.uint64)]
        for u in us:
            if not 0 <= u < M64:
                continue
            assert O.skip_bit(u, q) == (u * (M64 + q) < q * M64), (u, q)


def _samples(t, d, n, seed=3, beg=0):
    return [O.skip_live(seed, O.make_sid(3, 0, j), beg, d, t) for j in range(n)]


@pytest.mark.parametrize("t,d,n", [(4294967296 // 3000, 3000, 4000), (42949672, 3000, 1500),
                                   (1288490188, 1500, 800)])
def test_live_edges_are_independent_bernoulli(t, d, n):
    p = t / 2**32
    sets = _samples(t, d, n)
    counts = np.array([len(s) for s in sets], dtype=np.float64)
    mean, var = d * p, d * p * (1 - p)
    assert abs(counts.mean() - mean) < 5 * math.sqrt(var / n)
    assert 0.8 < counts.var() / var < 1.2
    hits = np.zeros(d)
    for s in sets:
        hits[s] += 1
    # per-position frequencies: chi-square with d degrees of freedom
    chi = np.sum((hits - n * p) ** 2 / (n * p * (1 - p)))
    assert abs(chi - d) < 6 * math.sqrt(2 * d), chi
    if p > 0.1:
        # pairs at distance 1 and 7 are live together with probability p^2
        for dist in (1, 7):
            both = sum(np.intersect1d(s, s + dist).size for s in sets)
            pairs = n * (d - dist)
            assert abs(both / pairs - p * p) < 5 * math.sqrt(p * p / pairs)


def test_first_gap_is_geometric():
    t, d, n = 42949672, 5000, 6000  # p = 0.01
    q = 1 - t / 2**32
    first = np.array([s[0] if len(s) else d for s in _samples(t, d, n, seed=9)])
    for g in (0, 10, 50, 100, 200, 400):
        want = q ** g
        got = np.mean(first >= g)
        assert abs(got - want) < 5 * math.sqrt(want * (1 - want) / n) + 1e-9, (g, got, want)


def _python_skip(seed, sid, beg, d, t):
    """The gap procedure restated with Python integers (Philox from the oracle)."""
    qs = [((1 << 32) - t) << 32]
    for _ in range(32):
        qs.append(qs[-1] * qs[-1] >> 64)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    out, pos, r = [], 0, 0
    while pos < d:
        rem = d - pos
        B = rem.bit_length()

        def uni(b):
            w = O.philox([sid & 0xFFFFFFFF, sid >> 32, beg + (r >> 1), 0x100 + b], key)
            lo, hi = (int(w[2]), int(w[3])) if r & 1 else (int(w[0]), int(w[1]))
            return hi << 32 | lo

        if uni(B) < qs[B]:
            break
        gap = 0
        for b in range(B):
            u = uni(b)
            if u * (M64 + qs[b]) < qs[b] * M64:
                gap |= 1 << b
        if gap >= rem:
            break
        out.append(pos + gap)
        pos += gap + 1
        r += 1
    return out


def test_python_restatement_agrees():
    for j, (t, d, beg) in enumerate([(1288490188, 1200, 0), (42949672, 2000, 77),
                                     (4294967296 // 1100, 1100, 123456)]):
        for k in range(6):
            sid = O.make_sid(3, 0, 1000 * j + k)
            assert O.skip_live(5, sid, beg, d, t).tolist() == _python_skip(5, sid, beg, d, t)


def _star_plus(n_leaves, extra_edges):
    edges = [(i, 0) for i in range(1, n_leaves + 1)] + extra_edges
    return inputs.from_edges(n_leaves + 1, edges)


@pytest.mark.parametrize("weights", ["wc", "mixed", "p_half"])
def test_bfs_equals_definition_with_skip_lists(weights):
    # node 0: 1500 in-edges (a skip list unless its thresholds differ); a few chains
    g = _star_plus(1500, [(0, 7), (7, 9), (3, 1), (5, 1), (2, 1)])
    if weights == "wc":
        w = inputs.weighted_cascade(g)
    elif weights == "mixed":
        w = inputs.weighted_cascade(g)
        w[3] = np.float32(0.5)  # one different threshold into node 0: per-edge coins
    else:
        w = inputs.constant(g, 0.5)
    og = O.load_graph(g.n, g.rowptr, g.dst, w, O.IC)
    for j in range(300):
        sid = O.make_sid(3, 0, j)
        r_bfs, w_bfs = O.rr_one(og, 4, sid)
        r_def, w_def = O.rr_by_definition(og, 4, sid)
        assert np.array_equal(r_bfs, r_def) and w_bfs == w_def


def test_hub_rr_sets_follow_the_binomial():
    # RR sets rooted at the hub of a weighted-cascade star: |R| - 1 ~ Binomial(n-1, p)
    n_leaves = 1999
    g = _star_plus(n_leaves, [])
    og = O.load_graph(g.n, g.rowptr, g.dst, inputs.weighted_cascade(g), O.IC)
    t = int(og.thr[0])
    p = t / 2**32
    sizes = []
    j = 0
    while len(sizes) < 3000:
        sid = O.make_sid(3, 0, j)
        j += 1
        if O.root(8, sid, g.n) != 0:
            continue
        r, _ = O.rr_one(og, 8, sid)
        sizes.append(len(r) - 1)
    sizes = np.array(sizes)
    for kk in range(4):
        want = math.comb(n_leaves, kk) * p ** kk * (1 - p) ** (n_leaves - kk)
        got = np.mean(sizes == kk)
        assert abs(got - want) < 5 * math.sqrt(want * (1 - want) / len(sizes)), (kk, got, want)


def test_rule_boundaries():
    # length and probability bounds of the rule
    assert not O.skip_applies(511, 1000) and O.skip_applies(512, 1000)
    assert not O.skip_applies(5000, 0)
    for d in (512, 1000, 1023, 1024, 40000):
        bl = d.bit_length()
        lim = ((1 << 32) - 1) // (2 * bl + 2)  # largest t with t (2 bl + 2) < 2^32
        assert O.skip_applies(d, lim) and not O.skip_applies(d, lim + 1)
    # weighted cascade: every in-list of 32 or more in-edges qualifies
    for d in (512, 513, 1000, 4096, 10 ** 6):
        t = int(np.float32(1.0 / d) * np.float64(2 ** 32))
        assert O.skip_applies(d, t)


def test_lists_at_the_length_bound_follow_the_rule_in_bfs():
    # nodes with 511 and 512 in-edges under weighted cascade (coins, then skip) and one
    # with 600 in-edges at p = 0.3 (coins): BFS and the drawn world agree
    edges = [(i, 0) for i in range(3, 515)] + [(i, 1) for i in range(515, 1115)] + \
        [(i, 2) for i in range(1115, 1626)] + [(0, 1), (2, 0)]
    g = inputs.from_edges(1626, edges)
    w = inputs.weighted_cascade(g)
    w[g.dst == 1] = np.float32(0.3)
    og = O.load_graph(g.n, g.rowptr, g.dst, w, O.IC)
    for j in range(400):
        sid = O.make_sid(3, 0, j)
        a, wa = O.rr_one(og, 6, sid)
        b, wb = O.rr_by_definition(og, 6, sid)
        assert np.array_equal(a, b) and wa == wb
