"""Pins for the oracle's greedy maximum coverage (the selection of Algorithm 1), RefineKPT
(Algorithm 3) and the TIM / TIM+ drivers (Sections 3.3 and 4.1)."""
import itertools
import math

import numpy as np
import pytest

from oracle import exact as X
from oracle import oracle as O
from paper_1404_0900_gb300 import inputs


def _csr(sets):
    off = np.cumsum([0] + [len(s) for s in sets]).astype(np.int64)
    mem = np.concatenate([np.asarray(s, dtype=np.int32) for s in sets]) if sets else \
        np.zeros(0, dtype=np.int32)
    return off, mem


def _marginal_trace(n, sets, k):
    """Greedy by explicit marginal gains with Python sets; ties to the smallest id."""
    uncovered = [set(s) for s in sets]
    chosen = []
    for _ in range(k):
        gains = {v: sum(1 for s in uncovered if v in s) for v in range(n) if v not in chosen}
        best = max(gains.values())
        v = min(u for u, gv in gains.items() if gv == best)
        chosen.append(v)
        uncovered = [s for s in uncovered if v not in s]
    return chosen, len(sets) - len(uncovered)


@pytest.mark.parametrize("seed", range(12))
def test_greedy_marginal_gains_and_approximation(seed):
    rng = np.random.default_rng(seed)
    n = 9
    sets = [sorted(set(rng.integers(0, n, size=rng.integers(1, 4)).tolist()))
            for _ in range(rng.integers(5, 30))]
    off, mem = _csr(sets)
    for k in (1, 2, 3, 4):
        seeds, cov, counts = O.greedy(n, off, mem, k)
        want, wcov = _marginal_trace(n, sets, k)
        assert seeds.tolist() == want and cov == wcov
        assert cov >= (1 - 1 / math.e) * X.max_coverage_brute(n, sets, k) - 1e-9
        if k == 1:
            assert counts.tolist() == [sum(1 for s in sets if v in s) for v in range(n)]


def test_greedy_ties_and_exhaustion():
    # equal counts -> smallest id; once everything is covered the smallest unchosen ids
    off, mem = _csr([[4, 2], [2, 4], [7], [7]])
    seeds, cov, _ = O.greedy(10, off, mem, 5)
    assert seeds.tolist() == [2, 7, 0, 1, 3] and cov == 4
    off, mem = _csr([])
    seeds, cov, _ = O.greedy(4, off, mem, 4)
    assert seeds.tolist() == [0, 1, 2, 3] and cov == 0
    with pytest.raises(ValueError):
        O.greedy(3, off, mem, 4)


def test_refine_on_strongly_connected_p1():
    # every RR set is V, so S'_k covers all theta' sets: f = 1, KPT' = n / (1 + eps')
    g = inputs.complete(8)
    og = O.load_graph(g.n, g.rowptr, g.dst, inputs.constant(g, 1.0), O.IC)
    kpt = O.kpt_estimation(og, 2, 1.0, 3)
    ref = O.refine_kpt(og, 2, 1.0, 0.5, 3, kpt)
    assert ref.covered == ref.theta_prime
    assert ref.kpt_prime == g.n / (1 + ref.eps_prime)
    assert ref.kpt_plus == max(ref.kpt_prime, kpt.kpt_star)
    assert ref.theta_prime == math.ceil(O.lam_prime(g.n, ref.eps_prime, 1.0) / kpt.kpt_star)


def _ring_of_stars(copies=4):
    """Disjoint copies of a 6-node graph with a clear best seed per copy."""
    base = [(0, 1, 0.6), (0, 2, 0.6), (0, 3, 0.6), (3, 4, 0.5), (4, 5, 0.5), (5, 0, 0.1),
            (2, 5, 0.3)]
    return 6 * copies, [(u + 6 * c, v + 6 * c, p) for c in range(copies) for u, v, p in base], base


def test_tim_plus_approximation_and_kpt_plus_bounds():
    n, edges, base = _ring_of_stars(3)
    g = inputs.from_edges(n, [(u, v) for u, v, _ in edges])
    pmap = {(u, v): p for u, v, p in edges}
    w = np.array([pmap[(int(u), int(v))] for u, v in zip(g.src(), g.dst)], dtype=np.float32)
    og = O.load_graph(n, g.rowptr, g.dst, w, O.IC)
    k, eps = 3, 0.3
    # OPT of a disjoint union with k = copies: the best single seed in each copy
    opt1, _ = X.opt_exact(6, base, 1, O.IC)
    opt = 3 * opt1
    for seed in (1, 2, 3):
        r = O.tim_plus(og, k, eps, 1.0, seed)
        val = sum(X.spread(6, base, [s - 6 * c for s in r.seeds if 6 * c <= s < 6 * c + 6], O.IC)
                  for c in range(3))
        assert val >= (1 - 1 / math.e - eps) * opt
        assert r.kpt.kpt_star <= r.refine.kpt_plus <= opt * (1 + 1e-9)
        assert r.theta == math.ceil(O.lam(n, k, eps, 1.0) / r.refine.kpt_plus)
        t = O.tim(og, k, eps, 1.0, seed)
        assert t.theta >= r.theta
