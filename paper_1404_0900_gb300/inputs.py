"""Seeded synthetic inputs: directed graphs and per-edge weights.

This module produces inputs only. It holds none of the influence-maximisation
arithmetic (no coins, thresholds, RR sets, widths or estimators): both the CUDA
path and the CPU oracle consume what it returns, and neither is imported here.

Every graph is returned as an out-CSR of G with sources sorted ascending and, within
one source, destinations sorted ascending; self-loops and duplicate edges removed:

    rowptr : int64[n+1]   out-edge offsets of each source node
    dst    : int32[m]     destination of each edge
    weight : float32[m]   p(e) for IC, or the LT in-weight of e

The shapes follow the paper's workloads (Section 6, Table 2): sparse directed
social graphs with skewed degrees. R-MAT stands in for the benchmark graphs and a
directed Chung-Lu power-law graph for the billion-edge Twitter crawl; the datasets
themselves are not available. Randomness comes from numpy's Philox bit generator
seeded by the caller.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Graph:
    n: int
    rowptr: np.ndarray  # int64[n+1]
    dst: np.ndarray  # int32[m]
    name: str = ""

    @property
    def m(self) -> int:
        return int(self.dst.shape[0])

    def src(self) -> np.ndarray:
        """Source node of every edge, int32[m] (edge order)."""
        deg = np.diff(self.rowptr)
        return np.repeat(np.arange(self.n, dtype=np.int32), deg)

    def indeg(self) -> np.ndarray:
        return np.bincount(self.dst, minlength=self.n).astype(np.int64)


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(seed))


def csr_from_pairs(n: int, src: np.ndarray, dst: np.ndarray, name: str = "") -> Graph:
    """Drop self-loops and duplicate pairs, sort by (src, dst), build an out-CSR."""
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    keep = src != dst
    key = np.sort(src[keep] * np.int64(n) + dst[keep])
    if key.size:
        key = key[np.concatenate(([True], key[1:] != key[:-1]))]
    s = key // n
    d = (key % n).astype(np.int32)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(s, minlength=n), out=rowptr[1:])
    return Graph(n=n, rowptr=rowptr, dst=d, name=name)


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19,
         c: float = 0.19, seed: int = 1) -> Graph:
    """Directed R-MAT graph: 2**scale nodes, edge_factor * 2**scale edge draws.

    Each draw descends `scale` levels of the adjacency matrix, picking the
    (src-bit, dst-bit) quadrant (0,0) w.p. a, (0,1) w.p. b, (1,0) w.p. c and
    (1,1) w.p. 1-a-b-c (each probability rounded to a multiple of 2^-16: one 16-bit
    draw per level picks the quadrant through a lookup table). No noise, no
    relabelling; self-loops and duplicates are removed afterwards, so m is below the
    number of draws.
    """
    n = 1 << scale
    draws = edge_factor * n
    rng = _rng(seed)
    cut = np.round(np.array([a, a + b, a + b + c]) * 65536).astype(np.int64)
    lut = np.zeros(65536, dtype=np.uint8)
    lut[cut[0]:cut[1]] = 1  # (0, 1)
    lut[cut[1]:cut[2]] = 2  # (1, 0)
    lut[cut[2]:] = 3        # (1, 1)
    sdt = np.int32 if scale <= 30 else np.int64
    src = np.empty(draws, dtype=np.int64)
    dst = np.empty(draws, dtype=np.int64)
    chunk = 1 << 23
    for lo in range(0, draws, chunk):
        hi = min(draws, lo + chunk)
        s = np.zeros(hi - lo, dtype=sdt)
        d = np.zeros(hi - lo, dtype=sdt)
        for _ in range(scale):
            q = lut[rng.integers(0, 65536, size=hi - lo, dtype=np.uint16)]
            s <<= 1
            d <<= 1
            s |= q >> 1
            d |= q & 1
        src[lo:hi] = s
        dst[lo:hi] = d
    return csr_from_pairs(n, src, dst, name=f"rmat{scale}")


def chung_lu(n: int, m_target: int, gamma: float = 2.1, seed: int = 1,
             max_rounds: int = 64) -> Graph:
    """Directed Chung-Lu power-law graph with about m_target distinct edges.

    Node weights w_i ~ (i+1)^(-1/(gamma-1)); sources are drawn proportional to w
    on the node ids, destinations proportional to w on a seeded permutation of the
    ids. Self-loops and duplicates are dropped and draws repeat until m_target
    distinct edges exist (or max_rounds is hit).
    """
    rng = _rng(seed)
    w = (np.arange(n, dtype=np.float64) + 1.0) ** (-1.0 / (gamma - 1.0))
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    perm = rng.permutation(n)
    have = np.zeros(0, dtype=np.int64)
    for _ in range(max_rounds):
        need = m_target - have.shape[0]
        if need <= 0:
            break
        k = int(need * 1.1) + 16
        s = np.searchsorted(cdf, rng.random(k), side="right")
        d = perm[np.searchsorted(cdf, rng.random(k), side="right")]
        s = np.minimum(s, n - 1)
        d = np.minimum(d, n - 1)
        keep = s != d
        key = np.sort(np.concatenate([have, s[keep].astype(np.int64) * n + d[keep]]))
        have = key[np.concatenate(([True], key[1:] != key[:-1]))] if key.size else key
    if have.shape[0] > m_target:
        pick = np.sort(rng.choice(have.shape[0], size=m_target, replace=False))
        have = have[pick]
    s = have // n
    d = have % n
    return csr_from_pairs(n, s, d, name=f"chunglu{n}")


def mixed_in_degree(n: int, hub_range=(512, 1023), light_range=(1, 64), seed: int = 1) -> Graph:
    """Directed graph whose even nodes have in-degree drawn uniformly from hub_range and
    odd nodes from light_range, each in-neighbour set drawn uniformly at random among
    the other nodes (a graph with thousands of long in-lists beside short ones)."""
    rng = _rng(seed)
    src, dst = [], []
    for v in range(n):
        lo, hi = hub_range if v % 2 == 0 else light_range
        d = int(rng.integers(lo, hi + 1))
        u = rng.choice(n - 1, size=d, replace=False)
        u = u + (u >= v)  # skip v itself
        src.append(u)
        dst.append(np.full(d, v, dtype=np.int64))
    return csr_from_pairs(n, np.concatenate(src), np.concatenate(dst), name=f"mixed{n}")


def from_edges(n: int, edges, name: str = "") -> Graph:
    """Graph from an explicit list of (u, v) pairs (u -> v)."""
    if len(edges) == 0:
        return Graph(n=n, rowptr=np.zeros(n + 1, dtype=np.int64),
                     dst=np.zeros(0, dtype=np.int32), name=name)
    e = np.asarray(edges, dtype=np.int64)
    return csr_from_pairs(n, e[:, 0], e[:, 1], name=name)


# ---------------------------------------------------------------- edge weights

def weighted_cascade(g: Graph) -> np.ndarray:
    """IC weighted cascade: p(u, v) = 1 / indeg(v), as float32 (Section 6)."""
    indeg = g.indeg()
    return (1.0 / indeg[g.dst].astype(np.float64)).astype(np.float32)


def lt_inverse_indegree(g: Graph) -> np.ndarray:
    """LT in-weights b(u, v) = 1 / indeg(v), as float32."""
    return weighted_cascade(g)


def lt_random_normalised(g: Graph, seed: int = 1) -> np.ndarray:
    """LT in-weights drawn uniformly in [0, 1] per edge, then normalised so that
    the in-weights of every node sum to one (Section 6, LT setting)."""
    rng = _rng(seed)
    r = rng.random(g.m)
    tot = np.bincount(g.dst, weights=r, minlength=g.n)
    return (r / tot[g.dst]).astype(np.float32)


def trivalency(g: Graph, seed: int = 1) -> np.ndarray:
    """IC trivalency: p(e) uniform over {0.1, 0.01, 0.001}, drawn per edge."""
    rng = _rng(seed)
    vals = np.array([0.1, 0.01, 0.001], dtype=np.float32)
    return vals[rng.integers(0, 3, size=g.m)]


def constant(g: Graph, p: float) -> np.ndarray:
    return np.full(g.m, p, dtype=np.float32)


def uniform_random(g: Graph, lo: float = 0.0, hi: float = 1.0, seed: int = 1) -> np.ndarray:
    rng = _rng(seed)
    return rng.uniform(lo, hi, size=g.m).astype(np.float32)


# ----------------------------------------------------- triggering distributions
#
# A triggering distribution (Section 4.2) as arrays over the out-CSR of G:
#   opt_rowptr      int64[n+1]   options of node v: opt_rowptr[v] .. opt_rowptr[v+1]
#   opt_prob        float32[k]   probability of each option (a node's sum <= 1)
#   opt_edge_rowptr int64[k+1]   edges of option o: opt_edge_rowptr[o] .. [o+1]
#   opt_edges       int64[..]    out-CSR edge ids, each an edge into the option's node

def _in_edges_by_node(g: Graph):
    """Out-CSR edge ids into each node, ascending by source (edge id order)."""
    order = np.argsort(g.dst, kind="stable")
    starts = np.zeros(g.n + 1, dtype=np.int64)
    np.cumsum(np.bincount(g.dst, minlength=g.n), out=starts[1:])
    return order.astype(np.int64), starts


def triggering_from_lt(g: Graph, w: np.ndarray):
    """The LT model as a triggering distribution: node v picks the single in-edge e with
    probability w[e], its options in the order of their sources."""
    order, starts = _in_edges_by_node(g)
    return (starts, np.asarray(w, dtype=np.float32)[order],
            np.arange(g.m + 1, dtype=np.int64), order)


def triggering_random(g: Graph, max_options: int = 3, max_size: int = 4,
                      mass=(0.5, 1.0), seed: int = 1):
    """Random triggering distributions: a node with in-edges gets 1..max_options options,
    each a uniform random subset of 1..max_size of its in-edges (distinct within the
    option), with probabilities drawn uniformly and scaled to a total mass drawn from
    `mass` (the rest: no in-edge)."""
    rng = _rng(seed)
    order, starts = _in_edges_by_node(g)
    orow = [0]
    probs, erow, edges = [], [0], []
    for v in range(g.n):
        ins = order[starts[v]:starts[v + 1]]
        if ins.size:
            k = int(rng.integers(1, max_options + 1))
            r = rng.random(k)
            r *= rng.uniform(mass[0], mass[1]) / r.sum()
            for i in range(k):
                size = int(rng.integers(1, min(max_size, ins.size) + 1))
                pick = np.sort(rng.choice(ins.size, size=size, replace=False))
                edges.extend(ins[pick].tolist())
                erow.append(len(edges))
                probs.append(r[i])
        orow.append(len(probs))
    return (np.array(orow, dtype=np.int64), np.array(probs, dtype=np.float32),
            np.array(erow, dtype=np.int64), np.array(edges, dtype=np.int64))


def triggering_all_in(g: Graph, p: float):
    """One option per node with in-edges: all of them, with probability p (the node's
    in-edges are live together or not at all)."""
    order, starts = _in_edges_by_node(g)
    has = np.diff(starts) > 0
    orow = np.zeros(g.n + 1, dtype=np.int64)
    np.cumsum(has, out=orow[1:])
    erow = np.concatenate([[0], starts[1:][has]]).astype(np.int64)
    return orow, np.full(int(has.sum()), p, dtype=np.float32), erow, order


# ------------------------------------------------------------ small hand graphs

def star_in(n: int) -> Graph:
    """Nodes 1..n-1 all point to node 0."""
    return from_edges(n, [(i, 0) for i in range(1, n)], name=f"star{n}")


def chain(n: int) -> Graph:
    """0 -> 1 -> ... -> n-1."""
    return from_edges(n, [(i, i + 1) for i in range(n - 1)], name=f"chain{n}")


def cycle(n: int) -> Graph:
    return from_edges(n, [(i, (i + 1) % n) for i in range(n)], name=f"cycle{n}")


def complete(n: int) -> Graph:
    return from_edges(n, [(i, j) for i in range(n) for j in range(n) if i != j],
                      name=f"complete{n}")


def random_small(n: int, m: int, seed: int) -> Graph:
    """Uniform random directed graph with (at most) m distinct edges."""
    rng = _rng(seed)
    pairs = set()
    tries = 0
    while len(pairs) < m and tries < 50 * m + 100:
        u, v = (int(x) for x in rng.integers(0, n, size=2))
        tries += 1
        if u != v:
            pairs.add((u, v))
    return from_edges(n, sorted(pairs), name=f"rand{n}_{m}_{seed}")


# ------------------------------------------------------- generators on the GPU
#
# The same graph families drawn with torch on a CUDA device, for workloads of many
# graphs (the start-round training set) where host generation would dominate. The
# draws come from torch's generator, so a device graph differs from the host graph of
# the same seed; each is a fixed function of its seed on one software stack.

@dataclass
class DeviceGraph:
    n: int
    rowptr: "object"  # torch int64[n+1] on the device
    dst: "object"     # torch int32[m] on the device
    name: str = ""

    @property
    def m(self) -> int:
        return int(self.dst.shape[0])

    def to_host(self) -> Graph:
        return Graph(n=self.n, rowptr=self.rowptr.cpu().numpy(), dst=self.dst.cpu().numpy(),
                     name=self.name)


def _torch_gen(seed: int, device):
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def csr_from_pairs_device(n: int, src, dst, name: str = "", m_exact: int | None = None,
                          gen=None) -> DeviceGraph:
    """Device version of csr_from_pairs (self-loops and duplicates dropped). With m_exact,
    a uniform random subset of exactly m_exact of the distinct edges is kept (drawn
    with `gen`); fewer distinct edges than that is an error."""
    import torch
    keep = src != dst
    key = torch.unique(src[keep].to(torch.int64) * n + dst[keep].to(torch.int64), sorted=True)
    del keep
    if m_exact is not None:
        if key.numel() < m_exact:
            raise ValueError(f"only {key.numel()} distinct edges, {m_exact} asked for")
        # the m_exact smallest of one uniform key per edge (a sort, not a permutation)
        r = torch.rand(key.numel(), generator=gen, device=key.device, dtype=torch.float64)
        pick = torch.argsort(r, stable=True)[:m_exact]
        del r
        key = key[torch.sort(pick).values]
        del pick
    s = key // n
    d = (key % n).to(torch.int32)
    rowptr = torch.zeros(n + 1, dtype=torch.int64, device=key.device)
    rowptr[1:] = torch.cumsum(torch.bincount(s, minlength=n), 0)
    return DeviceGraph(n=n, rowptr=rowptr, dst=d.contiguous(), name=name)


def rmat_device(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19,
                c: float = 0.19, seed: int = 1, device="cuda") -> DeviceGraph:
    """R-MAT as in rmat(), drawn on the device (16-bit quadrant draws per level)."""
    import torch
    n = 1 << scale
    draws = edge_factor * n
    gen = _torch_gen(seed, device)
    cut = [int(round(v * 65536)) for v in (a, a + b, a + b + c)]
    lut = torch.zeros(65536, dtype=torch.int64, device=device)
    lut[cut[0]:cut[1]] = 1
    lut[cut[1]:cut[2]] = 2
    lut[cut[2]:] = 3
    src = torch.zeros(draws, dtype=torch.int64, device=device)
    dst = torch.zeros(draws, dtype=torch.int64, device=device)
    for _ in range(scale):
        q = lut[torch.randint(0, 65536, (draws,), generator=gen, device=device)]
        src = (src << 1) | (q >> 1)
        dst = (dst << 1) | (q & 1)
    return csr_from_pairs_device(n, src, dst, name=f"rmat{scale}_dev")


def chung_lu_device(n: int, m_draws: int, gamma: float = 2.1, seed: int = 1,
                    device="cuda", m_exact: int | None = None) -> DeviceGraph:
    """Directed Chung-Lu power-law graph from m_draws edge draws (node weights
    (i+1)^(-1/(gamma-1)), destinations on a seeded permutation of the ids); self-loops
    and duplicates dropped, so m is below m_draws (or exactly m_exact: a uniform subset
    of the distinct edges)."""
    import torch
    gen = _torch_gen(seed, device)
    # the weight CDF on the host: a device float scan may round differently run to run
    w = (np.arange(n, dtype=np.float64) + 1.0) ** (-1.0 / (gamma - 1.0))
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    cdf = torch.from_numpy(cdf).to(device)
    del w
    # a seeded permutation: the stable order of one uniform key per id (reproducible
    # whatever the device's sort does with equal keys)
    perm = torch.argsort(torch.rand(n, generator=gen, device=device, dtype=torch.float64),
                         stable=True)
    u = torch.rand(m_draws, generator=gen, device=device, dtype=torch.float64)
    s = torch.searchsorted(cdf, u, right=True).clamp_(max=n - 1)
    u = torch.rand(m_draws, generator=gen, device=device, dtype=torch.float64)
    d = perm[torch.searchsorted(cdf, u, right=True).clamp_(max=n - 1)]
    del u, perm, cdf
    return csr_from_pairs_device(n, s, d, name=f"chunglu{n}_dev", m_exact=m_exact, gen=gen)


# The largest configuration: a Chung-Lu graph of Twitter's size (Section 7, Table 2):
# 41.6M nodes, 1.4B edges, exponent 2.1. 1.75B draws leave about 1.44B distinct edges.
C3_N, C3_M, C3_DRAWS = 41_600_000, 1_400_000_000, 1_750_000_000


def chung_lu_c3_device(seed: int = 1, device="cuda") -> DeviceGraph:
    return chung_lu_device(C3_N, C3_DRAWS, 2.1, seed=seed, device=device, m_exact=C3_M)


def weighted_cascade_device(g: DeviceGraph):
    """p(u, v) = 1 / indeg(v) as a device float32 tensor."""
    import torch
    indeg = torch.bincount(g.dst.to(torch.int64), minlength=g.n).to(torch.float64)
    return (1.0 / indeg[g.dst.to(torch.int64)]).to(torch.float32)


def trivalency_device(g: DeviceGraph, seed: int = 1):
    import torch
    gen = _torch_gen(seed, g.dst.device)
    vals = torch.tensor([0.1, 0.01, 0.001], dtype=torch.float32, device=g.dst.device)
    return vals[torch.randint(0, 3, (g.m,), generator=gen, device=g.dst.device)]


def lt_random_normalised_device(g: DeviceGraph, seed: int = 1):
    """Uniform random in-weights normalised to sum to one per node. The draws are
    integers in [1, 2^40) so that the per-node sums are exact whatever order the device
    adds them in (reproducible weights)."""
    import torch
    gen = _torch_gen(seed, g.dst.device)
    r = torch.randint(1, 1 << 40, (g.m,), generator=gen, device=g.dst.device, dtype=torch.int64)
    d = g.dst.to(torch.int64)
    tot = torch.zeros(g.n, dtype=torch.int64, device=g.dst.device).index_add_(0, d, r)
    return (r.to(torch.float64) / tot[d].to(torch.float64)).to(torch.float32)
