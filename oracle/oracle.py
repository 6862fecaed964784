"""Python face of the CPU oracle for TIM / TIM+ (Tang, Xiao, Shi, SIGMOD'14).

TEST INFRASTRUCTURE. Only the tests, the smoke check and the benchmark's CPU
baseline use this module; the GPU library never imports it and it never imports the
GPU library. The arithmetic lives in tim_oracle.c (plain C, see its header for the
readings of the paper that it fixes); this file marshals numpy arrays and strings the
paper's algorithms together in the paper's order:

  kpt_estimation  -- Algorithm 2 (Section 3.2), c_i of Eq. 7
  refine_kpt      -- Algorithm 3 (Section 4.1), eps' of Section 4.1
  node_selection  -- Algorithm 1 (Section 3.1), theta from Eq. 4 / Eq. 5
  tim_plus        -- TIM+ (Section 4.1): Algorithm 2 -> 3 -> theta -> Algorithm 1
  tim             -- TIM (Section 3.3): Algorithm 2 -> theta -> Algorithm 1
  spread_mc       -- forward Monte-Carlo estimate of E[I(S)] (Section 2.1; Section 7)
"""
from __future__ import annotations

import ctypes as C
import math
import os
from dataclasses import dataclass, field

import numpy as np

from . import build as _build

IC, LT, TRIG = 0, 1, 2
PHASE_KPT, PHASE_REFINE, PHASE_SELECT = 1, 2, 3

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        i64, u64, i32, u32, dbl = C.c_int64, C.c_uint64, C.c_int, C.c_uint32, C.c_double
        P = C.c_void_p
        sig = {
            "or_philox4x32_10": (None, [P, P, P]),
            "or_make_sid": (u64, [u64, u64, u64]),
            "or_root": (i64, [u64, u64, i64]),
            "or_ic_word": (u32, [u64, u64, i64]),
            "or_lt_word": (u32, [u64, u64, i64]),
            "or_transpose": (i32, [i64, i64, P, P, P, P, P, P]),
            "or_ic_thresholds": (i32, [i64, P, P]),
            "or_lt_thresholds": (i32, [i64, P, P, P]),
            "or_rr_by_definition": (i64, [P, P, P, i64, i64, i32, P, u64, u64, P, P]),
            "or_rr_one": (i64, [P, P, P, i64, i64, i32, P, u64, u64, P, P]),
            "or_rr_one_mode": (i64, [P, P, P, i64, i64, i32, P, i32, u64, u64, P, P]),
            "or_rr_by_definition_mode": (i64, [P, P, P, i64, i64, i32, P, i32, u64, u64, P, P]),
            "or_sample_mode": (i64, [P, P, P, i64, i64, i32, P, i32, u64, u64, i64, P, P, i64, P,
                                     i32]),
            "or_kappa": (dbl, [i64, i64, i32]),
            "or_kappa_fixed": (u64, [dbl]),
            "or_sample": (i64, [P, P, P, i64, i64, i32, P, u64, u64, i64, P, P, i64, P, i32]),
            "or_kappa_sum": (i32, [P, P, P, i64, i64, i32, P, i32, u64, u64, i64, P, P, P, i32]),
            "or_log_binom": (dbl, [i64, i64]),
            "or_lambda": (dbl, [i64, i32, dbl, dbl]),
            "or_eps_prime": (dbl, [dbl, i32, dbl]),
            "or_lambda_prime": (dbl, [i64, dbl, dbl]),
            "or_c_i": (i64, [i64, dbl, i32]),
            "or_kpt_rounds": (i32, [i64]),
            "or_kpt_estimate": (i32, [P, P, P, i64, i64, i32, P, i32, dbl, u64, u64, i32,
                                      P, P, P, P, P, P]),
            "or_greedy": (i64, [i64, i64, P, P, i32, P, P]),
            "or_covered_count": (i64, [P, P, P, i64, i64, i32, P, u64, u64, i64, P, i32]),
            "or_skip_q": (u64, [u32, i32]),
            "or_skip_bit": (i32, [u64, u64]),
            "or_skip_live": (i64, [u64, u64, i64, i64, u32, P]),
            "or_trig_build": (i32, [i64, i64, P, P, P, P, P, P, P, P, P]),
            "or_out_positions": (i32, [i64, i64, P, P, P, P, P]),
            "or_cascade_one": (i64, [P, P, P, i64, i64, i32, P, P, P, P, u64, u64, P, i32, P]),
            "or_spread_mc": (i64, [P, P, P, i64, i64, i32, P, P, P, P, u64, u64, i64, P, i32, P,
                                   i32]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


# ------------------------------------------------------------------ primitives

def philox(ctr, key) -> np.ndarray:
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def make_sid(phase: int, rnd: int, j: int) -> int:
    return int(lib().or_make_sid(phase, rnd, j))


def root(seed: int, sid: int, n: int) -> int:
    return int(lib().or_root(seed, sid, n))


def ic_word(seed: int, sid: int, j: int) -> int:
    return int(lib().or_ic_word(seed, sid, j))


def lt_word(seed: int, sid: int, v: int) -> int:
    return int(lib().or_lt_word(seed, sid, v))


SKIP_MIN_INDEG = 512  # shortest IC in-list that can take the geometric-skip rule


def skip_applies(d: int, t: int) -> bool:
    """The skip rule's condition on a list of d in-edges sharing threshold t."""
    return d >= SKIP_MIN_INDEG and t > 0 and t * (2 * d.bit_length() + 2) < (1 << 32)


def skip_q(t: int, b: int) -> int:
    """Q_b of the geometric-skip rule: (1 - t/2^32)^(2^b) in 0.64 fixed point."""
    return int(lib().or_skip_q(t, b))


def skip_bit(u: int, q: int) -> bool:
    """Digit decision of the geometric-skip rule: U / 2^64 < Q / (2^64 + Q)."""
    return bool(lib().or_skip_bit(u, q))


def skip_live(seed: int, sid: int, beg: int, d: int, t: int) -> np.ndarray:
    """Live relative positions of a d-edge in-list starting at in-CSR position beg
    whose in-edges share threshold t, under the geometric-skip rule."""
    out = np.zeros(max(d, 1), dtype=np.int64)
    r = lib().or_skip_live(seed, sid, beg, d, t, _p(out))
    if r < 0:
        raise ValueError("invalid skip list")
    return out[:r]


def kappa(w: int, m: int, k: int) -> float:
    """kappa(R) of Eq. 6 in FP64."""
    return float(lib().or_kappa(w, m, k))


def kappa_fixed(x: float) -> int:
    return int(lib().or_kappa_fixed(x))


def lam(n: int, k: int, eps: float, ell: float) -> float:
    """lambda of Eq. 4."""
    return float(lib().or_lambda(n, k, eps, ell))


def log_binom(n: int, k: int) -> float:
    return float(lib().or_log_binom(n, k))


def eps_prime(eps: float, k: int, ell: float) -> float:
    return float(lib().or_eps_prime(eps, k, ell))


def lam_prime(n: int, eps_p: float, ell: float) -> float:
    return float(lib().or_lambda_prime(n, eps_p, ell))


def c_i(n: int, ell: float, i: int) -> int:
    return int(lib().or_c_i(n, ell, i))


def kpt_rounds(n: int) -> int:
    return int(lib().or_kpt_rounds(n))


# ------------------------------------------------------------------- the graph

@dataclass
class OracleGraph:
    """G^T as an in-CSR plus the per-edge thresholds of one diffusion model."""
    n: int
    m: int
    model: int
    rowptr: np.ndarray  # int64[n+1]
    src: np.ndarray  # int32[m]
    thr: np.ndarray  # uint32[m]
    in_w: np.ndarray  # float32[m]
    out: tuple | None = None  # (out_rowptr, out_pos, pos_dst), built on first use
    trig: object = None  # triggering model: (or_trig structure, the arrays it points to)

    def indeg(self) -> np.ndarray:
        return np.diff(self.rowptr)

    def out_positions(self):
        """G as an out-CSR of in-CSR positions, and each position's destination."""
        if self.out is None:
            orow = np.zeros(self.n + 1, dtype=np.int64)
            opos = np.zeros(max(self.m, 1), dtype=np.int64)
            pdst = np.zeros(max(self.m, 1), dtype=np.int32)
            rc = lib().or_out_positions(self.n, self.m, _p(self.rowptr), _p(self.src), _p(orow),
                                        _p(opos), _p(pdst))
            if rc != 0:
                raise MemoryError
            self.out = (orow, opos, pdst)
        return self.out

    def args(self):
        t = C.byref(self.trig[0]) if self.trig is not None else None
        return (_p(self.rowptr), _p(self.src), _p(self.thr), self.n, self.m, self.model, t)


def load_graph(n: int, rowptr, dst, weight, model: int) -> OracleGraph:
    """Build G^T (Table 1) from an out-CSR of G and the model's thresholds."""
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    weight = np.ascontiguousarray(weight, dtype=np.float32)
    m = int(dst.shape[0])
    in_rowptr = np.zeros(n + 1, dtype=np.int64)
    in_src = np.zeros(max(m, 1), dtype=np.int32)
    in_w = np.zeros(max(m, 1), dtype=np.float32)
    rc = lib().or_transpose(n, m, _p(rowptr), _p(dst), _p(weight), _p(in_rowptr), _p(in_src),
                            _p(in_w))
    if rc != 0:
        raise ValueError(f"invalid graph (code {rc})")
    thr = np.zeros(max(m, 1), dtype=np.uint32)
    if model == IC:
        rc = lib().or_ic_thresholds(m, _p(in_w), _p(thr))
    else:
        rc = lib().or_lt_thresholds(n, _p(in_rowptr), _p(in_w), _p(thr))
    if rc != 0:
        raise ValueError(f"invalid weights (code {rc})")
    return OracleGraph(n, m, model, in_rowptr, in_src, thr, in_w)


class or_trig(C.Structure):
    _fields_ = [("node_opt", C.c_void_p), ("opt_cum", C.c_void_p), ("opt_off", C.c_void_p),
                ("opt_pos", C.c_void_p)]


def load_graph_triggering(n: int, rowptr, dst, opt_rowptr, opt_prob, opt_edge_rowptr,
                          opt_edges) -> OracleGraph:
    """G^T with a triggering model (Section 4.2): node v picks option o in opt_rowptr[v] ..
    opt_rowptr[v+1] with probability opt_prob[o] (none with the rest); option o is the set
    of out-CSR edges opt_edges[opt_edge_rowptr[o] .. opt_edge_rowptr[o+1]) into v."""
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    m = int(dst.shape[0])
    in_rowptr = np.zeros(n + 1, dtype=np.int64)
    in_src = np.zeros(max(m, 1), dtype=np.int32)
    in_w = np.zeros(max(m, 1), dtype=np.float32)
    rc = lib().or_transpose(n, m, _p(rowptr), _p(dst), None, _p(in_rowptr), _p(in_src), _p(in_w))
    if rc != 0:
        raise ValueError(f"invalid graph (code {rc})")
    orow = np.ascontiguousarray(opt_rowptr, dtype=np.int64)
    oprob = np.ascontiguousarray(opt_prob, dtype=np.float32)
    oer = np.ascontiguousarray(opt_edge_rowptr, dtype=np.int64)
    oe = np.ascontiguousarray(opt_edges, dtype=np.int64)
    if orow.shape[0] != n + 1 or oer.shape[0] != oprob.shape[0] + 1:
        raise ValueError("triggering arrays of the wrong length")
    cum = np.zeros(max(oprob.shape[0], 1), dtype=np.uint32)
    pos = np.zeros(max(oe.shape[0], 1), dtype=np.int64)
    if oe.shape[0] == 0:
        oe = np.zeros(1, dtype=np.int64)
    rc = lib().or_trig_build(n, m, _p(rowptr), _p(dst), _p(in_rowptr), _p(orow), _p(oprob),
                             _p(oer), _p(oe), _p(cum), _p(pos))
    if rc != 0:
        raise ValueError(f"invalid triggering distribution (code {rc})")
    t = or_trig(orow.ctypes.data, cum.ctypes.data, oer.ctypes.data, pos.ctypes.data)
    thr = np.zeros(max(m, 1), dtype=np.uint32)
    return OracleGraph(n, m, TRIG, in_rowptr, in_src, thr, in_w, trig=(t, orow, cum, oer, pos))


# ------------------------------------------------------------------- RR sets

def rr_one(g: OracleGraph, seed: int, sid: int, per_edge: bool = False):
    """One RR set by randomised BFS: (sorted members, width). per_edge: one coin per
    in-edge in every list, without the geometric-skip rule (Section 3.1 as printed;
    for statistical checks of the rule only)."""
    buf = np.zeros(g.n, dtype=np.int32)
    w = np.zeros(1, dtype=np.int64)
    cnt = lib().or_rr_one_mode(*g.args(), int(per_edge), seed, sid, _p(buf), _p(w))
    if cnt < 0:
        raise MemoryError
    return np.sort(buf[:cnt]), int(w[0])


def rr_by_definition(g: OracleGraph, seed: int, sid: int, per_edge: bool = False):
    """The same RR set from Definitions 1-2 (whole random graph drawn first)."""
    buf = np.zeros(g.n, dtype=np.int32)
    w = np.zeros(1, dtype=np.int64)
    cnt = lib().or_rr_by_definition_mode(*g.args(), int(per_edge), seed, sid, _p(buf), _p(w))
    if cnt < 0:
        raise MemoryError
    return buf[:cnt].copy(), int(w[0])


def sample(g: OracleGraph, seed: int, sid0: int, count: int, nthreads: int = 0,
           per_edge: bool = False):
    """RR sets sid0 .. sid0+count-1 as (off int64[count+1], mem int32, widths int64).
    per_edge: see rr_one."""
    off = np.zeros(count + 1, dtype=np.int64)
    widths = np.zeros(max(count, 1), dtype=np.int64)
    cap = max(16, count * 8)
    while True:
        mem = np.zeros(cap, dtype=np.int32)
        tot = lib().or_sample_mode(*g.args(), int(per_edge), seed, sid0, count, _p(off), _p(mem),
                                   cap, _p(widths), nthreads)
        if tot < 0:
            raise MemoryError
        if tot <= cap:
            return off, mem[:tot], widths[:count]
        cap = tot


def kappa_sum(g: OracleGraph, k: int, seed: int, sid0: int, count: int, nthreads: int = 0):
    """Exact 2^-63 fixed-point sum of kappa over a range of set ids (Python int) and
    the sum of widths."""
    hi = np.zeros(1, dtype=np.uint64)
    lo = np.zeros(1, dtype=np.uint64)
    ws = np.zeros(1, dtype=np.int64)
    rc = lib().or_kappa_sum(*g.args(), k, seed, sid0, count, _p(hi), _p(lo), _p(ws), nthreads)
    if rc != 0:
        raise MemoryError
    return (int(hi[0]) << 64) | int(lo[0]), int(ws[0])


def greedy(n: int, off, mem, k: int):
    """Greedy max coverage (the selection of Algorithm 1): (seeds, covered count,
    first-round coverage counts)."""
    off = np.ascontiguousarray(off, dtype=np.int64)
    mem = np.ascontiguousarray(mem, dtype=np.int32)
    if mem.shape[0] == 0:
        mem = np.zeros(1, dtype=np.int32)
    seeds = np.zeros(max(k, 1), dtype=np.int32)
    counts = np.zeros(n, dtype=np.int64)
    cov = lib().or_greedy(n, off.shape[0] - 1, _p(off), _p(mem), k, _p(seeds), _p(counts))
    if cov < 0:
        raise ValueError(f"greedy failed ({cov})")
    return seeds[:k].copy(), int(cov), counts


def covered_count(g: OracleGraph, seed: int, sid0: int, count: int, seeds,
                  nthreads: int = 0) -> int:
    in_s = np.zeros(g.n, dtype=np.uint8)
    in_s[np.asarray(seeds, dtype=np.int64)] = 1
    r = lib().or_covered_count(*g.args(), seed, sid0, count, _p(in_s), nthreads)
    if r < 0:
        raise MemoryError
    return int(r)


# ------------------------------------------------------ forward Monte Carlo

def _seed_array(g: OracleGraph, seeds) -> np.ndarray:
    s = np.ascontiguousarray(seeds, dtype=np.int32)
    if s.size and (s.min() < 0 or s.max() >= g.n):
        raise ValueError("seed out of range")
    return s if s.size else np.zeros(1, dtype=np.int32)


def cascade_one(g: OracleGraph, seeds, seed: int, sid: int) -> np.ndarray:
    """The nodes activated from `seeds` in the world of set id sid (sorted)."""
    orow, opos, pdst = g.out_positions()
    s = _seed_array(g, seeds)
    buf = np.zeros(g.n + 1, dtype=np.int32)
    cnt = lib().or_cascade_one(*g.args(), _p(orow), _p(opos), _p(pdst), seed, sid, _p(s),
                               len(seeds), _p(buf))
    if cnt < 0:
        raise ValueError(f"cascade failed ({cnt})")
    return np.sort(buf[:cnt])


def spread_mc(g: OracleGraph, seeds, count: int, seed: int, sid0: int, nthreads: int = 0):
    """Forward Monte-Carlo spread (Section 2.1): activated-node counts of cascades sid0 ..
    sid0 + count - 1 (int64[count]) and their exact total; total / count estimates
    E[I(S)]."""
    orow, opos, pdst = g.out_positions()
    s = _seed_array(g, seeds)
    counts = np.zeros(max(count, 1), dtype=np.int64)
    tot = lib().or_spread_mc(*g.args(), _p(orow), _p(opos), _p(pdst), seed, sid0, count, _p(s),
                             len(seeds), _p(counts), nthreads)
    if tot < 0:
        raise ValueError(f"spread failed ({tot})")
    return counts[:count], int(tot)


# --------------------------------------------------------------- Algorithm 2

@dataclass
class KptResult:
    kpt_star: float
    stop_round: int  # 0: no round stopped, KPT* = 1
    last_round: int  # the round whose sets form R' of Algorithm 3 (0: none ran)
    last_c: int
    last_sum: int  # exact 2^-63 fixed-point kappa sum of the last round
    sets_generated: int = 0


def kpt_estimation(g: OracleGraph, k: int, ell: float, seed: int, nthreads: int = 0,
                   tag: int = 0) -> KptResult:
    out = [np.zeros(1, dtype=t) for t in (np.float64, np.int32, np.int32, np.int64, np.uint64,
                                          np.uint64)]
    rc = lib().or_kpt_estimate(*g.args(), k, ell, seed, tag, nthreads, *[_p(a) for a in out])
    if rc != 0:
        raise MemoryError
    last_round = int(out[2][0])
    gen = sum(c_i(g.n, ell, i) for i in range(1, last_round + 1))
    return KptResult(kpt_star=float(out[0][0]), stop_round=int(out[1][0]), last_round=last_round,
                     last_c=int(out[3][0]), last_sum=(int(out[4][0]) << 64) | int(out[5][0]),
                     sets_generated=gen)


def kpt_estimation_from(g: OracleGraph, k: int, ell: float, seed: int, i0: int,
                        nthreads: int = 0, tag: int = 0) -> tuple[KptResult, bool]:
    """Algorithm 2 started at a predicted round i0 (a rule the paper does not have).

    The prediction is accepted when round i0 - 1 fails the stop test of Algorithm 2
    and round i0 passes it (for i0 = 1: when round 1 passes); the result is then
    round i0's estimate KPT* = n sum / (2 c_i0), with round i0's sets as R'. Otherwise
    the result is plain Algorithm 2's. Rounds use the same set ids as the plain sweep,
    so round i's sets do not depend on which rounds ran. Returns (result, accepted)."""
    rounds = kpt_rounds(g.n)
    if rounds < 1 or i0 < 1:
        return kpt_estimation(g, k, ell, seed, nthreads, tag), False
    i0 = min(i0, rounds)

    def round_sum(i):
        c = c_i(g.n, ell, i)
        s, _ = kappa_sum(g, k, seed, make_sid(PHASE_KPT, i, tag << 32), c, nthreads)
        return s, c

    lo_pass = False
    if i0 >= 2:
        s, c = round_sum(i0 - 1)
        lo_pass = s > (c << (63 - (i0 - 1)))
    s, c = round_sum(i0)
    if not lo_pass and s > (c << (63 - i0)):
        kpt = float(g.n) * math.ldexp(float(s), -63) / (2.0 * float(c))
        return KptResult(kpt_star=kpt, stop_round=i0, last_round=i0, last_c=c, last_sum=s), True
    return kpt_estimation(g, k, ell, seed, nthreads, tag), False


# --------------------------------------------------------------- Algorithm 3

@dataclass
class RefineResult:
    kpt_plus: float
    kpt_prime: float
    eps_prime: float
    theta_prime: int
    covered: int
    seeds_prime: np.ndarray


def refine_kpt(g: OracleGraph, k: int, ell: float, eps: float, seed: int, kpt: KptResult,
               nthreads: int = 0, tag: int = 0) -> RefineResult:
    # R' = the RR sets of the last iteration of Algorithm 2
    if kpt.last_round > 0:
        off, mem, _ = sample(g, seed, make_sid(PHASE_KPT, kpt.last_round, tag << 32), kpt.last_c,
                             nthreads)
    else:
        off, mem = np.zeros(1, dtype=np.int64), np.zeros(0, dtype=np.int32)
    # greedy on R'
    seeds_p, _, _ = greedy(g.n, off, mem, k)
    # eps' and theta'
    ep = eps_prime(eps, k, ell)
    lp = lam_prime(g.n, ep, ell)
    theta_p = int(math.ceil(lp / kpt.kpt_star))
    # fraction of theta' fresh RR sets covered by S'_k
    cov = covered_count(g, seed, make_sid(PHASE_REFINE, 0, tag << 32), theta_p, seeds_p, nthreads)
    f = cov / theta_p
    # KPT' and KPT+
    kpt_prime = f * g.n / (1.0 + ep)
    return RefineResult(kpt_plus=max(kpt_prime, kpt.kpt_star), kpt_prime=kpt_prime,
                        eps_prime=ep, theta_prime=theta_p, covered=cov, seeds_prime=seeds_p)


# --------------------------------------------------------------- Algorithm 1

@dataclass
class SelectResult:
    seeds: np.ndarray
    covered: int
    theta: int
    members: int


def node_selection(g: OracleGraph, k: int, theta: int, seed: int, nthreads: int = 0,
                   tag: int = 0) -> SelectResult:
    off, mem, _ = sample(g, seed, make_sid(PHASE_SELECT, 0, tag << 32), theta, nthreads)
    seeds, cov, _ = greedy(g.n, off, mem, k)
    return SelectResult(seeds=seeds, covered=cov, theta=theta, members=int(mem.shape[0]))


def theta_from(n: int, k: int, eps: float, ell: float, kpt_lower: float) -> int:
    """theta = lambda / KPT, rounded up (Eq. 5 with OPT replaced by its lower bound)."""
    return int(math.ceil(lam(n, k, eps, ell) / kpt_lower))


@dataclass
class TimResult:
    seeds: np.ndarray
    covered: int
    theta: int
    kpt: KptResult
    refine: RefineResult | None
    extra: dict = field(default_factory=dict)

    @property
    def covered_fraction(self) -> float:
        return self.covered / self.theta if self.theta else 0.0


def tim_plus(g: OracleGraph, k: int, eps: float, ell: float, seed: int, nthreads: int = 0,
             theta_override: int | None = None, tag: int = 0,
             start_round: int | None = None) -> TimResult:
    """TIM+ (Section 4.1); with start_round, Algorithm 2 is kpt_estimation_from."""
    if start_round is None:
        kpt = kpt_estimation(g, k, ell, seed, nthreads, tag)
    else:
        kpt, _ = kpt_estimation_from(g, k, ell, seed, start_round, nthreads, tag)
    ref = refine_kpt(g, k, ell, eps, seed, kpt, nthreads, tag)
    theta = theta_override if theta_override is not None else theta_from(g.n, k, eps, ell,
                                                                          ref.kpt_plus)
    sel = node_selection(g, k, theta, seed, nthreads, tag)
    return TimResult(seeds=sel.seeds, covered=sel.covered, theta=theta, kpt=kpt, refine=ref,
                     extra={"members": sel.members})


def tim(g: OracleGraph, k: int, eps: float, ell: float, seed: int, nthreads: int = 0,
        tag: int = 0) -> TimResult:
    kpt = kpt_estimation(g, k, ell, seed, nthreads, tag)
    theta = theta_from(g.n, k, eps, ell, kpt.kpt_star)
    sel = node_selection(g, k, theta, seed, nthreads, tag)
    return TimResult(seeds=sel.seeds, covered=sel.covered, theta=theta, kpt=kpt, refine=None,
                     extra={"members": sel.members})


def host_threads() -> int:
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
