"""Pins for the oracle's estimators: Corollary 1 (n * F_R(S) is unbiased for E[I(S)]),
Lemma 5 (KPT = n * E[kappa(R)]), kappa itself (Eq. 6), the fixed-point round sums,
c_i (Eq. 7), lambda (Eq. 4), eps' and lambda' (Section 4.1) and Algorithm 2's
closed-form cases."""
import math
from fractions import Fraction

import numpy as np
import pytest
from scipy.special import gammaln

from oracle import exact as X
from oracle import oracle as O
from paper_1404_0900_gb300 import inputs

TINY_IC = [  # (u, v, p): 5 nodes, 8 edges, a cycle and a hub
    (0, 1, 0.5), (1, 2, 0.4), (2, 0, 0.3), (3, 0, 0.7), (3, 4, 0.2), (4, 1, 0.6),
    (1, 3, 0.25), (2, 4, 0.5)]
TINY_LT = [  # in-weights per node sum to <= 1
    (0, 1, 0.5), (4, 1, 0.4), (1, 2, 0.9), (2, 0, 0.3), (3, 0, 0.6), (3, 4, 0.2),
    (2, 4, 0.7), (1, 3, 1.0)]


def _og(n, edges, model):
    g = inputs.from_edges(n, [(u, v) for u, v, _ in edges])
    pmap = {(u, v): p for u, v, p in edges}
    w = np.array([pmap[(int(u), int(v))] for u, v in zip(g.src(), g.dst)], dtype=np.float32)
    return O.load_graph(n, g.rowptr, g.dst, w, model), g


@pytest.mark.parametrize("model,edges", [(O.IC, TINY_IC), (O.LT, TINY_LT)])
def test_corollary1_coverage_fraction_estimates_exact_spread(model, edges):
    n = 5
    og, _ = _og(n, edges, model)
    theta = 200000
    off, mem, _ = O.sample(og, 17, O.make_sid(3, 0, 0), theta)
    for seeds in ([0], [3], [1, 4], [0, 2, 3]):
        exact = X.spread(n, edges, seeds, model)
        hit = np.zeros(theta, dtype=bool)
        sid_of = np.repeat(np.arange(theta), np.diff(off))
        hit[sid_of[np.isin(mem, seeds)]] = True
        rho = exact / n
        est = hit.mean()
        assert abs(est - rho) < 5 * math.sqrt(rho * (1 - rho) / theta) + 1e-12, (seeds, est, rho)


@pytest.mark.parametrize("model,edges", [(O.IC, TINY_IC), (O.LT, TINY_LT)])
def test_rr_set_distribution_matches_definition(model, edges):
    n = 5
    og, _ = _og(n, edges, model)
    dist = X.rr_distribution(n, edges, model)
    theta = 100000
    off, mem, _ = O.sample(og, 23, O.make_sid(3, 0, 0), theta)
    emp = {}
    for j in range(theta):
        r = frozenset(mem[off[j]:off[j + 1]].tolist())
        emp[r] = emp.get(r, 0) + 1
    for r, p in dist.items():
        c = emp.get(r, 0) / theta
        assert abs(c - p) < 5 * math.sqrt(p * (1 - p) / theta) + 2e-5, (r, c, p)
    assert set(emp) <= set(dist)


@pytest.mark.parametrize("model,edges,k", [(O.IC, TINY_IC, 1), (O.IC, TINY_IC, 2),
                                           (O.LT, TINY_LT, 2)])
def test_lemma5_kpt_equals_n_mean_kappa(model, edges, k):
    n = 5
    lhs = X.kpt_exact(n, edges, k, model)
    rhs = X.kappa_mean_exact(n, edges, k, model, kappa=O.kappa)
    assert abs(lhs - rhs) <= 1e-12 * lhs
    # and the ordering n/m * EPT <= KPT <= OPT (Eq. 8)
    m = len(edges)
    ept = X.kappa_mean_exact(n, edges, 1, model, kappa=lambda w, mm, kk: w / mm) * m / n
    opt, _ = X.opt_exact(n, edges, k, model)
    assert n / m * ept <= lhs + 1e-12 and lhs <= opt + 1e-12


@pytest.mark.parametrize("w,m,k", [(0, 10, 5), (10, 10, 5), (3, 17, 1), (1, 1_400_000_000, 50),
                                   (21000, 16_084_614, 50), (7, 1000, 37), (999, 1000, 64),
                                   (123456, 262144, 10)])
def test_kappa_matches_exact_rational(w, m, k):
    got = Fraction(O.kappa(w, m, k))
    want = X.kappa_exact(w, m, k)
    if want == 0:
        assert got == 0
    else:
        assert abs(got - want) / want < Fraction(1, 10 ** 13)


def test_kappa_fixed_is_floor_times_2_63():
    for x in (0.0, 1.0, 0.5, 1e-9, 0.3333333333333333, 2.0 ** -70, 0.9999999999999999):
        assert O.kappa_fixed(x) == math.floor(Fraction(x) * 2 ** 63)


def test_round_sum_is_exact_sum_of_fixed_kappas():
    g = inputs.rmat(10)
    og = O.load_graph(g.n, g.rowptr, g.dst, inputs.weighted_cascade(g), O.IC)
    sid0 = O.make_sid(1, 2, 0)
    off, mem, widths = O.sample(og, 7, sid0, 3000)
    s, wsum = O.kappa_sum(og, 9, 7, sid0, 3000, nthreads=3)
    assert wsum == int(widths.sum())
    want = sum(math.floor(Fraction(O.kappa(int(w), og.m, 9)) * 2 ** 63) for w in widths)
    assert s == want
    exact = sum(X.kappa_exact(int(w), og.m, 9) for w in widths)
    assert abs(Fraction(s, 2 ** 63) - exact) < Fraction(3000 * 64, 2 ** 52)


def test_c_i_eq7_rounded_up_and_round_count():
    for n in (4, 16384, 1 << 20, 41_600_000):
        for ell in (0.5, 1.0, 1.3):
            for i in (1, 5, 12):
                c = O.c_i(n, ell, i)
                real = (6 * ell * math.log(n) + 6 * math.log(math.log2(n))) * 2 ** i
                assert c - 1 < real <= c
    assert O.kpt_rounds(2) == 0 and O.kpt_rounds(3) == 0 and O.kpt_rounds(4) == 1
    assert O.kpt_rounds(16384) == 13 and O.kpt_rounds(1 << 20) == 19
    assert O.kpt_rounds(41_600_000) == 24  # log2 41.6M = 25.3


@pytest.mark.parametrize("n,k,eps,ell", [(16384, 10, 0.5, 1.0), (1 << 20, 50, 0.1, 1.0),
                                         (41_600_000, 50, 0.2, 1.0), (100, 100, 1.0, 0.5)])
def test_lambda_eq4_against_exact_binomial(n, k, eps, ell):
    lnb = math.log(math.comb(n, k))  # exact big integer, then one correctly rounded log
    assert abs(lnb - (gammaln(n + 1) - gammaln(k + 1) - gammaln(n - k + 1))) < 1e-6 * max(1, lnb)
    want = (8 + 2 * eps) * n * (ell * math.log(n) + lnb + math.log(2)) / eps ** 2
    assert abs(O.lam(n, k, eps, ell) - want) <= 1e-9 * want
    assert abs(O.log_binom(n, k) - lnb) <= 1e-13 * max(1.0, lnb)


def test_eps_prime_and_lambda_prime():
    for eps, k, ell in ((0.1, 50, 1.0), (0.5, 10, 1.0), (0.2, 1, 2.0)):
        ep = O.eps_prime(eps, k, ell)
        assert abs(ep ** 3 - 125 * ell * eps ** 2 / (k + ell)) < 1e-12 * ep ** 3
        n = 1 << 20
        assert abs(O.lam_prime(n, ep, ell) * ep ** 2 / ((2 + ep) * ell * n * math.log(n)) - 1) < 1e-12


def test_kpt_strongly_connected_p1_stops_at_round1_with_n_over_2():
    # p = 1 on a strongly connected graph: every RR set is V, w = m, kappa = 1, so
    # sum/c_1 = 1 > 1/2 and Algorithm 2 returns n * c_1 / (2 c_1) = n / 2.
    for g in (inputs.cycle(64), inputs.complete(9)):
        og = O.load_graph(g.n, g.rowptr, g.dst, inputs.constant(g, 1.0), O.IC)
        r = O.kpt_estimation(og, 3, 1.0, 5)
        assert r.stop_round == 1 and r.kpt_star == g.n / 2


def test_kpt_tiny_graph_has_no_rounds():
    g = inputs.chain(3)
    og = O.load_graph(g.n, g.rowptr, g.dst, inputs.constant(g, 0.5), O.IC)
    r = O.kpt_estimation(og, 1, 1.0, 5)
    assert r.kpt_star == 1.0 and r.stop_round == 0 and r.last_round == 0


def test_kpt_p0_closed_form():
    # p = 0: R = {root}, so E[kappa] = mean over v of 1 - (1 - indeg(v)/m)^k.
    g = inputs.rmat(11)
    og = O.load_graph(g.n, g.rowptr, g.dst, inputs.constant(g, 0.0), O.IC)
    k = 5
    indeg = og.indeg()
    kv = np.array([O.kappa(int(d), og.m, k) for d in indeg])
    mu = kv.mean()
    cnt = 400000
    s, _ = O.kappa_sum(og, k, 3, O.make_sid(1, 1, 0), cnt)
    est = s / 2 ** 63 / cnt
    assert abs(est - mu) < 5 * kv.std() / math.sqrt(cnt)


def test_theorem2_kpt_star_within_quarter_kpt_and_opt():
    # Theorem 2: KPT* in [KPT/4, OPT] with probability >= 1 - n^-l. The graph is a
    # disjoint union of copies of TINY_IC, so both sides are exact: an RR set lives in
    # one copy (Lemma 5 with m of the union gives KPT), and OPT for k = 2 puts the two
    # seeds in two different copies (spread adds across copies; submodularity).
    n, edges, copies, k = 5, TINY_IC, 8, 2
    big = [(u + n * c, v + n * c, p) for c in range(copies) for u, v, p in edges]
    N, M = n * copies, len(big)
    og, _ = _og(N, big, O.IC)
    d = X.indegrees(n, edges)
    kpt = N * sum(pr * O.kappa(sum(d[v] for v in r), M, k)
                  for r, pr in X.rr_distribution(n, edges, O.IC).items())
    opt = 2 * X.opt_exact(n, edges, 1, O.IC)[0]
    bad = 0
    for seed in range(40):
        r = O.kpt_estimation(og, k, 1.0, seed)
        bad += not (kpt / 4 <= r.kpt_star <= opt)
    assert bad <= 3  # expected at most 40 * N^-1 = 1
