"""Exact quantities by brute-force enumeration on tiny graphs (test infrastructure).

Pure Python, written straight from the paper's definitions, used to pin the oracle:

  spread                 -- E[I(S)] (Section 2.1; live-edge view of Section 2.2 and the
                            triggering model of Section 4.2: IC, LT or a general
                            triggering distribution), by enumerating every random graph g
                            with its probability.
  rr_distribution        -- the exact distribution of a random RR set (Definitions 1-2)
  kpt_exact              -- KPT = E[I(S*)] for S* = k draws from the in-degree
                            distribution V (Section 3.2, before Lemma 5)
  kappa_mean_exact       -- n * E[kappa(R)] (Lemma 5) from rr_distribution
  opt_exact              -- OPT = max over |S| = k of E[I(S)]
  max_coverage_brute     -- best k-subset for a set system

Edges are (u, v, p) triples meaning u -> v with probability / LT weight p.
"""
from __future__ import annotations

import itertools
from fractions import Fraction


def _reach_from(n, live_edges, sources):
    """Nodes reachable from `sources` along live edges u -> v."""
    out = [[] for _ in range(n)]
    for u, v in live_edges:
        out[u].append(v)
    seen = set(sources)
    stack = list(sources)
    while stack:
        u = stack.pop()
        for v in out[u]:
            if v not in seen:
                seen.add(v)
                stack.append(v)
    return seen


def ic_worlds(edges):
    """Every live-edge graph g of the IC model with its probability (Section 2.2)."""
    m = len(edges)
    for mask in range(1 << m):
        pr = 1.0
        live = []
        for i, (u, v, p) in enumerate(edges):
            if mask >> i & 1:
                pr *= p
                live.append((u, v))
            else:
                pr *= 1.0 - p
        if pr > 0.0:
            yield pr, live


def lt_worlds(n, edges):
    """Every triggering-set choice of the LT model with its probability: node v picks
    in-edge (u, v) with probability b(u, v) and nothing with 1 - sum b (Section 6)."""
    ins = [[] for _ in range(n)]
    for u, v, b in edges:
        ins[v].append((u, b))
    choices = []
    for v in range(n):
        opts = [(None, 1.0 - sum(b for _, b in ins[v]))] + [(u, b) for u, b in ins[v]]
        choices.append([(u, b) for u, b in opts if b > 0.0])
    for combo in itertools.product(*choices):
        pr = 1.0
        live = []
        for v, (u, b) in enumerate(combo):
            pr *= b
            if u is not None:
                live.append((u, v))
        yield pr, live


def trig_worlds(n, options):
    """Every choice of a general triggering model (Section 4.2) with its probability:
    options[v] = [(probability, [in-neighbours u ...]), ...]; node v picks one option, or
    none with 1 - the sum of its probabilities; the live edges are u -> v for the picked
    option's u."""
    choices = []
    for v in range(n):
        opts = list(options[v]) if v < len(options) else []
        rest = 1.0 - sum(p for p, _ in opts)
        ch = [(p, us) for p, us in opts if p > 0.0]
        if rest > 0.0:
            ch.append((rest, []))
        choices.append(ch)
    for combo in itertools.product(*choices):
        pr = 1.0
        live = []
        for v, (p, us) in enumerate(combo):
            pr *= p
            live.extend((u, v) for u in us)
        yield pr, live


def worlds(n, edges, model, options=None):
    if model == 2:
        return trig_worlds(n, options)
    return ic_worlds(edges) if model == 0 else lt_worlds(n, edges)


def spread(n, edges, seeds, model=0, options=None):
    """E[I(S)]: expected number of nodes reachable from S in a random graph g."""
    return sum(pr * len(_reach_from(n, live, seeds))
               for pr, live in worlds(n, edges, model, options))


def rr_distribution(n, edges, model=0, options=None):
    """Exact distribution of a random RR set: {frozenset R: probability}."""
    dist = {}
    for pr, live in worlds(n, edges, model, options):
        rev = [(v, u) for u, v in live]
        for root in range(n):
            r = frozenset(_reach_from(n, rev, [root]))
            dist[r] = dist.get(r, 0.0) + pr / n
    return dist


def indegrees(n, edges):
    d = [0] * n
    for _, v, _ in edges:
        d[v] += 1
    return d


def kappa_mean_exact(n, edges, k, model=0, kappa=None):
    """n * E[kappa(R)] with kappa(R) = 1 - (1 - w(R)/m)^k (Eq. 6, Lemma 5).
    `kappa(w, m, k)` may be supplied to evaluate kappa with a given routine."""
    m = len(edges)
    d = indegrees(n, edges)
    if kappa is None:
        kappa = lambda w, mm, kk: 1.0 - (1.0 - w / mm) ** kk  # noqa: E731
    tot = 0.0
    for r, pr in rr_distribution(n, edges, model).items():
        w = sum(d[v] for v in r)
        tot += pr * kappa(w, m, k)
    return n * tot


def kpt_exact(n, edges, k, model=0):
    """KPT: mean spread of S*, the set of k independent draws from V (the in-degree
    distribution), duplicates removed (Section 3.2)."""
    m = len(edges)
    d = indegrees(n, edges)
    support = [v for v in range(n) if d[v] > 0]
    cache = {}
    tot = 0.0
    for combo in itertools.product(support, repeat=k):
        pr = 1.0
        for v in combo:
            pr *= d[v] / m
        s = frozenset(combo)
        if s not in cache:
            cache[s] = spread(n, edges, s, model)
        tot += pr * cache[s]
    return tot


def opt_exact(n, edges, k, model=0):
    best, arg = -1.0, None
    for s in itertools.combinations(range(n), k):
        val = spread(n, edges, s, model)
        if val > best + 1e-15:
            best, arg = val, s
    return best, arg


def max_coverage_brute(n, sets, k):
    """Largest number of sets hit by any k nodes."""
    best = 0
    for s in itertools.combinations(range(n), k):
        ss = set(s)
        best = max(best, sum(1 for r in sets if ss & set(r)))
    return best


def kappa_exact(w, m, k) -> Fraction:
    """kappa(R) as an exact rational."""
    q = 1 - Fraction(w, m)
    return 1 - q ** k
