"""TIM+ for one query split over several ranks by set id, on the CPU oracle.

TEST INFRASTRUCTURE (like the rest of oracle/): the multi-rank tests use it to pin the
partition of one query that the GPU library implements in tim_run_sharded. The paper's
RR sets are independent given their set ids (Section 3), so rank r of W generates only
the sets j in [c r / W, c (r+1) / W) of each phase's c sets, and the ranks combine:

  - Algorithm 2: per round, the exact 2^-63 fixed-point kappa sum (a Python integer;
    carried through the all-reduce in 32-bit limbs so that int64 sums are exact);
  - Algorithm 3: greedy on R' (below), then the covered count of the theta' sets;
  - Algorithm 1: the greedy over the union of the ranks' sets.

The greedy is the plain definition of Algorithm 1's selection: every round counts, for
every node, the uncovered sets that contain it (here: the count of each rank's own sets,
summed over the ranks), takes the node with the largest count (ties: the smallest id;
chosen nodes excluded) and marks the sets that contain it.

`allreduce(arr)` sums an int64 numpy array over the ranks in place.
"""
from __future__ import annotations

import math

import numpy as np

from . import oracle as O


def shard(c: int, rank: int, world: int) -> tuple[int, int]:
    return c * rank // world, c * (rank + 1) // world


def allreduce_int(value: int, allreduce) -> int:
    """Exact sum of a non-negative integer below 2^128 over the ranks."""
    limbs = np.array([(value >> (32 * i)) & 0xFFFFFFFF for i in range(4)], dtype=np.int64)
    allreduce(limbs)
    return sum(int(limbs[i]) << (32 * i) for i in range(4))


def greedy_sharded(n: int, off: np.ndarray, mem: np.ndarray, k: int, allreduce):
    """(seeds, covered count over all ranks) of the greedy on the union of the ranks'
    CSR-of-sets (off, mem)."""
    n_sets = off.shape[0] - 1
    set_of = np.repeat(np.arange(n_sets, dtype=np.int64), np.diff(off))
    covered = np.zeros(n_sets, dtype=bool)
    chosen = np.zeros(n, dtype=bool)
    seeds = np.zeros(k, dtype=np.int32)
    for r in range(k):
        live = ~covered[set_of]
        counts = np.bincount(mem[live], minlength=n).astype(np.int64)
        allreduce(counts)
        counts[chosen] = -1
        v = int(np.argmax(counts))  # first maximum: the smallest id
        chosen[v] = True
        seeds[r] = v
        covered[np.unique(set_of[mem == v])] = True
    tot = np.array([int(covered.sum())], dtype=np.int64)
    allreduce(tot)
    return seeds, int(tot[0])


def tim_plus_sharded(g: O.OracleGraph, k: int, eps: float, ell: float, seed: int, rank: int,
                     world: int, allreduce, nthreads: int = 0, tag: int = 0) -> dict:
    n = g.n
    # Algorithm 2
    kpt_star, stop, last, last_c = 1.0, 0, 0, 0
    for i in range(1, O.kpt_rounds(n) + 1):
        c = O.c_i(n, ell, i)
        lo, hi = shard(c, rank, world)
        s, _ = O.kappa_sum(g, k, seed, O.make_sid(O.PHASE_KPT, i, tag << 32) + lo, hi - lo,
                           nthreads)
        S = allreduce_int(s, allreduce)
        last, last_c = i, c
        if S > (c << (63 - i)):
            kpt_star = float(n) * math.ldexp(float(S), -63) / (2.0 * float(c))
            stop = i
            break
    # Algorithm 3
    if last:
        lo, hi = shard(last_c, rank, world)
        off, mem, _ = O.sample(g, seed, O.make_sid(O.PHASE_KPT, last, tag << 32) + lo, hi - lo,
                               nthreads)
    else:
        off, mem = np.zeros(1, dtype=np.int64), np.zeros(0, dtype=np.int32)
    seeds_p, _ = greedy_sharded(n, off, mem, k, allreduce)
    ep = O.eps_prime(eps, k, ell)
    theta_p = int(math.ceil(O.lam_prime(n, ep, ell) / kpt_star))
    lo, hi = shard(theta_p, rank, world)
    cov = np.array([O.covered_count(g, seed, O.make_sid(O.PHASE_REFINE, 0, tag << 32) + lo,
                                    hi - lo, seeds_p, nthreads)], dtype=np.int64)
    allreduce(cov)
    cov_p = int(cov[0])
    kpt_prime = cov_p / theta_p * n / (1.0 + ep)
    kpt_plus = max(kpt_prime, kpt_star)
    # Algorithm 1
    theta = O.theta_from(n, k, eps, ell, kpt_plus)
    lo, hi = shard(theta, rank, world)
    off, mem, _ = O.sample(g, seed, O.make_sid(O.PHASE_SELECT, 0, tag << 32) + lo, hi - lo,
                           nthreads)
    seeds, covered = greedy_sharded(n, off, mem, k, allreduce)
    return {"seeds": seeds, "covered": covered, "theta": theta, "kpt_star": kpt_star,
            "kpt_round": stop, "kpt_plus": kpt_plus, "theta_prime": theta_p,
            "covered_prime": cov_p}
