"""ctypes binding of libtim.so (include/tim.h): the same names, argument marshalling only.

Every computation runs in the CUDA library; this module converts numpy arrays / torch
tensors to pointers and status codes to exceptions. There is no fallback: if the
library is missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

from . import build as _build

TIM_IC, TIM_LT, TIM_TRIG = 0, 1, 2
TIM_OK = 0
TIM_ERR_ARG, TIM_ERR_OOM, TIM_ERR_OVERFLOW = -1, -2, -3
TIM_ERR_TIMEOUT, TIM_ERR_CUDA, TIM_ERR_STATE = -4, -5, -6

STATUS = {0: "TIM_OK", -1: "TIM_ERR_ARG", -2: "TIM_ERR_OOM", -3: "TIM_ERR_OVERFLOW",
          -4: "TIM_ERR_TIMEOUT", -5: "TIM_ERR_CUDA", -6: "TIM_ERR_STATE"}

HEADER = os.path.join(_build.ROOT, "include", "tim.h")


class TimError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class tim_stats(C.Structure):
    _fields_ = [
        ("kpt_round", C.c_int), ("kpt_last_round", C.c_int),
        ("kpt_star", C.c_double), ("kpt_prime", C.c_double), ("kpt_plus", C.c_double),
        ("eps_prime", C.c_double), ("lambda_", C.c_double),
        ("theta_prime", C.c_uint64), ("covered_prime", C.c_uint64), ("theta", C.c_uint64),
        ("covered", C.c_uint64), ("sets_total", C.c_uint64), ("members_select", C.c_uint64),
        ("width_total", C.c_uint64), ("width_select", C.c_uint64),
        ("ms_kpt", C.c_double), ("ms_refine", C.c_double), ("ms_select_sample", C.c_double),
        ("ms_select_greedy", C.c_double), ("ms_total", C.c_double),
        ("kpt_sets", C.c_uint64), ("kpt_predicted_round", C.c_int), ("kpt_accepted", C.c_int),
    ]

    def as_dict(self) -> dict:
        d = {name: getattr(self, name) for name, _ in self._fields_}
        d["lambda"] = d.pop("lambda_")
        return d


class tim_profile(C.Structure):
    _fields_ = [
        ("pass1_launches", C.c_uint64), ("pass1_ms", C.c_double),
        ("pass1_sets", C.c_uint64), ("pass1_width", C.c_uint64), ("pass1_live", C.c_uint64),
        ("pass1_members", C.c_uint64),
        ("pass2_launches", C.c_uint64), ("pass2_ms", C.c_double),
        ("pass2_sets", C.c_uint64), ("pass2_width", C.c_uint64), ("pass2_live", C.c_uint64),
        ("pass2_members", C.c_uint64),
        ("pass3_launches", C.c_uint64), ("pass3_ms", C.c_double),
        ("pass3_sets", C.c_uint64), ("pass3_width", C.c_uint64), ("pass3_live", C.c_uint64),
        ("pass3_members", C.c_uint64),
        ("pass1_examined", C.c_uint64), ("pass2_examined", C.c_uint64),
        ("pass3_examined", C.c_uint64),
        ("pass3_batches", C.c_uint64), ("pass3_levels", C.c_uint64),
        ("pass3_ms_offsets", C.c_double), ("pass3_ms_expand", C.c_double),
        ("pass3_ms_wait", C.c_double), ("pass3_ms_kernel", C.c_double),
    ]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class tim_query(C.Structure):
    _fields_ = [("ctx", C.c_void_p), ("k", C.c_int), ("eps", C.c_double), ("ell", C.c_double),
                ("tag", C.c_uint32), ("seeds", C.c_void_p), ("covered_fraction", C.c_double),
                ("stats", tim_stats)]


class tim_batch_stats(C.Structure):
    _fields_ = [("queries", C.c_int), ("kpt_launch_rounds", C.c_int), ("sets_total", C.c_uint64),
                ("ms_kpt", C.c_double), ("ms_refine", C.c_double), ("ms_select_sample", C.c_double),
                ("ms_select_greedy", C.c_double), ("ms_total", C.c_double),
                ("learned_accepted", C.c_int), ("ms_predict", C.c_double)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class tim_tuning(C.Structure):
    _fields_ = [("width_budget", C.c_uint64), ("team_size", C.c_int), ("chunk", C.c_int),
                ("trials", C.c_int), ("best_ms", C.c_double), ("default_ms", C.c_double),
                ("team_factor", C.c_int), ("pass1_capacity", C.c_int)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


_lib = None
_P = C.c_void_p
_SIGS = {
    "tim_create": (C.c_int, [C.POINTER(_P), C.c_int, _P]),
    "tim_destroy": (C.c_int, [_P]),
    "tim_strerror": (C.c_char_p, [C.c_int]),
    "tim_last_error_message": (C.c_char_p, [_P]),
    "tim_load_graph": (C.c_int, [_P, C.c_int64, C.c_int64, _P, _P, _P, C.c_int]),
    "tim_load_graph_device": (C.c_int, [_P, C.c_int64, C.c_int64, _P, _P, _P, C.c_int]),
    "tim_load_graph_triggering": (C.c_int, [_P, C.c_int64, C.c_int64, _P, _P, _P, _P, _P,
                                            _P]),
    "tim_get_graph": (C.c_int, [_P, _P, _P, _P]),
    "tim_sample_rr": (C.c_int, [_P, C.c_uint64, C.c_uint64, C.c_uint64, _P]),
    "tim_get_rr": (C.c_int, [_P, _P, _P, C.c_uint64, _P]),
    "tim_rr_size": (C.c_int, [_P, _P, _P]),
    "tim_kappa_sum": (C.c_int, [_P, C.c_int, C.c_uint64, C.c_uint64, C.c_uint64, _P, _P, _P]),
    "tim_kpt_estimate": (C.c_int, [_P, C.c_int, C.c_double, C.c_uint64, _P, _P]),
    "tim_refine_kpt": (C.c_int, [_P, C.c_int, C.c_double, C.c_double, C.c_uint64, _P, _P, _P]),
    "tim_node_select": (C.c_int, [_P, C.c_int, _P, _P, _P]),
    "tim_coverage_counts": (C.c_int, [_P, _P]),
    "tim_covered_count": (C.c_int, [_P, _P, C.c_int, C.c_uint64, C.c_uint64, C.c_uint64, _P]),
    "tim_run": (C.c_int, [_P, C.c_int, C.c_double, C.c_double, C.c_uint64, _P, _P, _P,
                          C.c_uint64]),
    "tim_run_tim": (C.c_int, [_P, C.c_int, C.c_double, C.c_double, C.c_uint64, _P, _P, _P]),
    "tim_launch_count": (C.c_uint64, [_P]),
    "tim_spread_mc": (C.c_int, [_P, _P, C.c_int, C.c_uint64, C.c_uint64, C.c_uint64, _P, _P,
                                _P]),
    "tim_get_profile": (C.c_int, [_P, _P, C.c_int]),
    "tim_set_width_budget": (C.c_int, [_P, C.c_uint64]),
    "tim_set_team_size": (C.c_int, [_P, C.c_int]),
    "tim_set_team_factor": (C.c_int, [_P, C.c_int]),
    "tim_set_pass1_capacity": (C.c_int, [_P, C.c_int]),
    "tim_set_wait_limit": (C.c_int, [_P, C.c_uint32]),
    "tim_set_pass2_budget": (C.c_int, [_P, C.c_uint64]),
    "tim_set_heavy_pass": (C.c_int, [_P, C.c_int]),
    "tim_set_query_tag": (C.c_int, [_P, C.c_uint32]),
    "tim_set_chunk": (C.c_int, [_P, C.c_int]),
    "tim_run_batch": (C.c_int, [_P, C.c_int, C.c_uint64, C.c_int, _P]),
    "tim_autotune": (C.c_int, [_P, C.c_uint64, C.c_uint64, _P]),
    "tim_node_select_noalloc": (C.c_int, [C.c_int, _P, C.c_int64, C.c_uint64, _P, _P, C.c_int,
                                          _P, _P]),
    "tim_graph_features": (C.c_int, [_P, _P]),
    "tim_select_begin": (C.c_int, [_P]),
    "tim_select_counts": (C.c_int, [_P, _P]),
    "tim_select_take": (C.c_int, [_P, C.c_int32, _P]),
    "tim_run_sharded": (C.c_int, [_P, C.c_int, C.c_double, C.c_double, C.c_uint64, C.c_int,
                                  C.c_int, _P, _P, _P, _P, _P]),
    "tim_mlp_create": (C.c_int, [C.POINTER(_P), _P, C.c_int]),
    "tim_mlp_destroy": (C.c_int, [_P]),
    "tim_mlp_param_count": (C.c_uint64, [_P]),
    "tim_mlp_set_params": (C.c_int, [_P, _P, C.c_uint64]),
    "tim_mlp_get_params": (C.c_int, [_P, _P, C.c_uint64]),
    "tim_mlp_set_scaling": (C.c_int, [_P, _P, _P, C.c_float, C.c_float]),
    "tim_mlp_grad": (C.c_int, [_P, _P, _P, C.c_uint64, _P, _P]),
    "tim_mlp_train": (C.c_int, [_P, _P, _P, C.c_uint64, C.c_int, C.c_float, _P]),
    "tim_mlp_predict": (C.c_int, [_P, _P, C.c_uint64, _P]),
    "tim_kpt_estimate_learned": (C.c_int, [_P, _P, C.c_int, C.c_double, C.c_uint64, _P, _P, _P,
                                           _P]),
    "tim_run_learned": (C.c_int, [_P, _P, C.c_int, C.c_double, C.c_double, C.c_uint64, _P, _P,
                                  _P]),
    "tim_run_batch_learned": (C.c_int, [_P, C.c_int, C.c_uint64, C.c_int, _P, _P]),
}

TIM_GRAPH_FEATURES, TIM_START_FEATURES, TIM_MLP_HIDDEN, TIM_MLP_MAX_IN = 8, 12, 64, 32


def library_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = True) -> C.CDLL:
    """Load libtim.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is None:
        path = _build.build() if build_if_missing else _build.LIB
        if not os.path.exists(path):
            raise OSError(f"libtim.so not found at {path}")
        L = C.CDLL(path)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def declared_functions() -> list[str]:
    """Names of the functions include/tim.h declares."""
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\S.*?\b(tim_[a-z_0-9]+)\(", text, flags=re.M)))


def _ptr(a) -> C.c_void_p:
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data_as(_P)
    if hasattr(a, "data_ptr"):  # torch tensor
        return _P(a.data_ptr())
    return _P(int(a))


def _check(ctx, rc: int):
    if rc != TIM_OK:
        msg = lib().tim_last_error_message(ctx).decode() if ctx else ""
        raise TimError(rc, msg or lib().tim_strerror(rc).decode())


# ---------------------------------------------------------------- the calls

# cudaStreamLegacy: the legacy default stream as an explicit handle
CUDA_STREAM_LEGACY = 0x1


def tim_create(device: int = 0, stream=None):
    """stream: a torch.cuda.Stream, a raw cudaStream_t int, or None (the context creates
    its own stream). A torch stream whose handle is 0 is the legacy default stream: it
    is passed as cudaStreamLegacy, so that the context's work is ordered after the work
    torch queued there (handle 0 alone would mean "create an own stream")."""
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream or CUDA_STREAM_LEGACY
    h = _P()
    rc = lib().tim_create(C.byref(h), device, _P(stream) if stream else None)
    if rc != TIM_OK:
        raise TimError(rc, lib().tim_strerror(rc).decode())
    return h


def tim_destroy(ctx):
    _check(None, lib().tim_destroy(ctx))


def tim_load_graph(ctx, n: int, rowptr, dst, weight, model: int):
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    weight = np.ascontiguousarray(weight, dtype=np.float32)
    _check(ctx, lib().tim_load_graph(ctx, n, dst.shape[0], _ptr(rowptr), _ptr(dst),
                                     _ptr(weight), model))


def tim_load_graph_device(ctx, n: int, m: int, d_rowptr, d_dst, d_weight, model: int):
    """Device arrays: torch CUDA tensors (int64, int32, float32) or raw pointers."""
    _check(ctx, lib().tim_load_graph_device(ctx, n, m, _ptr(d_rowptr), _ptr(d_dst),
                                            _ptr(d_weight), model))


def tim_load_graph_triggering(ctx, n: int, rowptr, dst, opt_rowptr, opt_prob, opt_edge_rowptr,
                              opt_edges):
    """G (out-CSR) and each node's triggering options (Section 4.2): node v's options
    opt_rowptr[v] .. opt_rowptr[v+1], option o with probability opt_prob[o] and the out-CSR
    edge ids opt_edges[opt_edge_rowptr[o] .. opt_edge_rowptr[o+1])."""
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    opt_rowptr = np.ascontiguousarray(opt_rowptr, dtype=np.int64)
    opt_prob = np.ascontiguousarray(opt_prob, dtype=np.float32)
    opt_edge_rowptr = np.ascontiguousarray(opt_edge_rowptr, dtype=np.int64)
    opt_edges = np.ascontiguousarray(opt_edges, dtype=np.int64)
    _check(ctx, lib().tim_load_graph_triggering(ctx, n, dst.shape[0], _ptr(rowptr), _ptr(dst),
                                                _ptr(opt_rowptr), _ptr(opt_prob),
                                                _ptr(opt_edge_rowptr), _ptr(opt_edges)))


def tim_get_graph(ctx, n: int, m: int):
    """G^T of the loaded graph: (rowptr uint64[n+1], src uint32[m], thr uint32[m])."""
    rowptr = np.zeros(n + 1, dtype=np.uint64)
    src = np.zeros(max(m, 1), dtype=np.uint32)
    thr = np.zeros(max(m, 1), dtype=np.uint32)
    _check(ctx, lib().tim_get_graph(ctx, rowptr.ctypes.data_as(_P), src.ctypes.data_as(_P),
                                    thr.ctypes.data_as(_P)))
    return rowptr, src[:m], thr[:m]


def tim_select_begin(ctx):
    _check(ctx, lib().tim_select_begin(ctx))


def tim_select_counts(ctx, n: int) -> np.ndarray:
    counts = np.zeros(max(n, 1), dtype=np.int32)
    _check(ctx, lib().tim_select_counts(ctx, counts.ctypes.data_as(_P)))
    return counts[:n]


def tim_select_take(ctx, node: int) -> int:
    newly = C.c_uint64()
    _check(ctx, lib().tim_select_take(ctx, node, C.byref(newly)))
    return newly.value


ALLREDUCE_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.POINTER(C.c_int64), C.c_uint64)


def torch_allreduce(dist):
    """An all-reduce for tim_run_sharded over a torch.distributed process group: sums an
    int64 numpy array in place (gloo on host memory)."""
    import torch

    def reduce(arr: np.ndarray):
        t = torch.from_numpy(arr)
        dist.all_reduce(t)
    return reduce


def tim_run_sharded(ctx, k: int, eps: float, ell: float, seed: int, rank: int, world: int,
                    allreduce):
    """TIM+ for one query over `world` ranks by set id; allreduce(arr) sums an int64 numpy
    array over the ranks in place. Returns (seeds, covered_fraction, stats dict)."""
    def cb(user, data, count):
        try:
            allreduce(np.ctypeslib.as_array(data, shape=(count,)))
            return 0
        except Exception:  # reported by the library as a failed call
            return -1
    fn = ALLREDUCE_FN(cb)
    seeds = np.zeros(k, dtype=np.int32)
    frac = C.c_double()
    st = tim_stats()
    _check(ctx, lib().tim_run_sharded(ctx, k, eps, ell, seed, rank, world,
                                      C.cast(fn, _P), None, seeds.ctypes.data_as(_P),
                                      C.byref(frac), C.byref(st)))
    return seeds, frac.value, st.as_dict()


def tim_sample_rr(ctx, theta: int, seed: int, first_set_id: int) -> int:
    tot = C.c_uint64()
    _check(ctx, lib().tim_sample_rr(ctx, theta, seed, first_set_id, C.byref(tot)))
    return tot.value


def tim_rr_size(ctx) -> tuple[int, int]:
    a, b = C.c_uint64(), C.c_uint64()
    _check(ctx, lib().tim_rr_size(ctx, C.byref(a), C.byref(b)))
    return a.value, b.value


def tim_get_rr(ctx):
    """The RR-set store as (off int64[theta+1], mem int32, widths int64[theta])."""
    ns, nm = tim_rr_size(ctx)
    off = np.zeros(ns + 1, dtype=np.int64)
    mem = np.zeros(max(nm, 1), dtype=np.int32)
    widths = np.zeros(max(ns, 1), dtype=np.int64)
    _check(ctx, lib().tim_get_rr(ctx, _ptr(off), _ptr(mem), nm, _ptr(widths)))
    return off, mem[:nm], widths[:ns]


def tim_kappa_sum(ctx, k: int, seed: int, first_set_id: int, count: int) -> tuple[int, int]:
    hi, lo, ws = C.c_uint64(), C.c_uint64(), C.c_uint64()
    _check(ctx, lib().tim_kappa_sum(ctx, k, seed, first_set_id, count, C.byref(hi), C.byref(lo),
                                    C.byref(ws)))
    return (hi.value << 64) | lo.value, ws.value


def tim_kpt_estimate(ctx, k: int, ell: float, seed: int) -> tuple[float, int]:
    kpt, rnd = C.c_double(), C.c_int()
    _check(ctx, lib().tim_kpt_estimate(ctx, k, ell, seed, C.byref(kpt), C.byref(rnd)))
    return kpt.value, rnd.value


def tim_refine_kpt(ctx, k: int, ell: float, eps: float, seed: int) -> tuple[float, float, int]:
    kp, ep, tp = C.c_double(), C.c_double(), C.c_uint64()
    _check(ctx, lib().tim_refine_kpt(ctx, k, ell, eps, seed, C.byref(kp), C.byref(ep),
                                     C.byref(tp)))
    return kp.value, ep.value, tp.value


def tim_node_select(ctx, k: int):
    seeds = np.zeros(k, dtype=np.int32)
    frac, cov = C.c_double(), C.c_uint64()
    _check(ctx, lib().tim_node_select(ctx, k, _ptr(seeds), C.byref(frac), C.byref(cov)))
    return seeds, frac.value, cov.value


def tim_coverage_counts(ctx, n: int) -> np.ndarray:
    counts = np.zeros(n, dtype=np.int32)
    _check(ctx, lib().tim_coverage_counts(ctx, _ptr(counts)))
    return counts


def tim_covered_count(ctx, seeds, seed: int, first_set_id: int, count: int) -> int:
    s = np.ascontiguousarray(seeds, dtype=np.int32)
    cov = C.c_uint64()
    _check(ctx, lib().tim_covered_count(ctx, _ptr(s), s.shape[0], seed, first_set_id, count,
                                        C.byref(cov)))
    return cov.value


def tim_run(ctx, k: int, eps: float, ell: float, seed: int, theta_override: int = 0,
            seeds_out: np.ndarray | None = None):
    """TIM+ end to end. Returns (seeds int32[k], covered fraction, stats dict)."""
    seeds = seeds_out if seeds_out is not None else np.zeros(k, dtype=np.int32)
    frac = C.c_double()
    st = tim_stats()
    _check(ctx, lib().tim_run(ctx, k, eps, ell, seed, _ptr(seeds), C.byref(frac), C.byref(st),
                              theta_override))
    return seeds, frac.value, st.as_dict()


def tim_run_tim(ctx, k: int, eps: float, ell: float, seed: int):
    """Plain TIM end to end. Returns (seeds, covered fraction, stats dict)."""
    seeds = np.zeros(k, dtype=np.int32)
    frac = C.c_double()
    st = tim_stats()
    _check(ctx, lib().tim_run_tim(ctx, k, eps, ell, seed, _ptr(seeds), C.byref(frac),
                                  C.byref(st)))
    return seeds, frac.value, st.as_dict()


def tim_node_select_noalloc(device: int, stream, n: int, n_sets: int, d_off, d_mem, k: int,
                            d_seeds, d_covered):
    """Greedy selection on caller-owned device buffers, without any device allocation
    by the library (torch CUDA tensors or raw device pointers)."""
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    rc = lib().tim_node_select_noalloc(device, _P(stream) if stream else None, n, n_sets,
                                       _ptr(d_off), _ptr(d_mem), k, _ptr(d_seeds),
                                       _ptr(d_covered))
    if rc != TIM_OK:
        raise TimError(rc, lib().tim_strerror(rc).decode())


def tim_launch_count(ctx) -> int:
    return int(lib().tim_launch_count(ctx))


def tim_spread_mc(ctx, seeds, count: int, seed: int, first_set_id: int,
                  want_counts: bool = False):
    """Forward Monte-Carlo spread of `seeds` over `count` cascades (set ids first_set_id
    + c). Returns (mean, total, per-cascade counts as uint32 or None)."""
    s = np.ascontiguousarray(seeds, dtype=np.int32)
    total, mean = C.c_uint64(), C.c_double()
    counts = np.zeros(max(count, 1), dtype=np.uint32) if want_counts else None
    _check(ctx, lib().tim_spread_mc(ctx, _ptr(s) if s.size else None, int(s.size), count, seed,
                                    first_set_id, C.byref(total), C.byref(mean),
                                    _ptr(counts) if want_counts else None))
    return mean.value, total.value, (counts[:count] if want_counts else None)


def tim_set_width_budget(ctx, budget: int):
    _check(ctx, lib().tim_set_width_budget(ctx, budget))


def tim_set_query_tag(ctx, tag: int):
    _check(ctx, lib().tim_set_query_tag(ctx, tag))


def tim_set_chunk(ctx, sets: int):
    _check(ctx, lib().tim_set_chunk(ctx, sets))


def tim_run_batch(queries, seed: int, plus: bool = True, mlp=None):
    """queries: list of dicts {ctx, k, eps, ell, tag}. Returns (list of (seeds, covered
    fraction, stats dict), batch stats dict). With `mlp` (a tim_mlp handle), Algorithm 2
    starts from learned rounds (tim_run_batch_learned)."""
    nq = len(queries)
    arr = (tim_query * nq)()
    seeds = []
    for i, q in enumerate(queries):
        s = np.zeros(q["k"], dtype=np.int32)
        seeds.append(s)
        arr[i].ctx = q["ctx"]
        arr[i].k = q["k"]
        arr[i].eps = q["eps"]
        arr[i].ell = q.get("ell", 1.0)
        arr[i].tag = q.get("tag", i + 1)
        arr[i].seeds = s.ctypes.data_as(_P)
    bst = tim_batch_stats()
    ctx0 = queries[0]["ctx"] if nq else None
    if mlp is None:
        _check(ctx0, lib().tim_run_batch(C.cast(arr, _P), nq, seed, 1 if plus else 0,
                                         C.byref(bst)))
    else:
        _check(ctx0, lib().tim_run_batch_learned(C.cast(arr, _P), nq, seed, 1 if plus else 0, mlp,
                                                 C.byref(bst)))
    out = [(seeds[i], arr[i].covered_fraction, arr[i].stats.as_dict()) for i in range(nq)]
    return out, bst.as_dict()


def tim_autotune(ctx, sample_sets: int, seed: int = 1) -> dict:
    t = tim_tuning()
    _check(ctx, lib().tim_autotune(ctx, sample_sets, seed, C.byref(t)))
    return t.as_dict()


def tim_set_team_size(ctx, warps: int):
    _check(ctx, lib().tim_set_team_size(ctx, warps))


def tim_set_team_factor(ctx, factor: int):
    _check(ctx, lib().tim_set_team_factor(ctx, factor))


def tim_set_pass1_capacity(ctx, members: int):
    _check(ctx, lib().tim_set_pass1_capacity(ctx, members))


def tim_set_pass2_budget(ctx, budget: int):
    _check(ctx, lib().tim_set_pass2_budget(ctx, budget))


def tim_set_wait_limit(ctx, polls: int):
    _check(ctx, lib().tim_set_wait_limit(ctx, polls))


def tim_set_heavy_pass(ctx, stepped: bool):
    _check(ctx, lib().tim_set_heavy_pass(ctx, int(bool(stepped))))


def tim_get_profile(ctx, reset: bool = False) -> dict:
    p = tim_profile()
    _check(ctx, lib().tim_get_profile(ctx, C.byref(p), 1 if reset else 0))
    return p.as_dict()


def tim_graph_features(ctx) -> np.ndarray:
    out = np.zeros(TIM_GRAPH_FEATURES, dtype=np.float32)
    _check(ctx, lib().tim_graph_features(ctx, _ptr(out)))
    return out


def tim_mlp_create(ctx, d_in: int = TIM_START_FEATURES):
    h = _P()
    _check(ctx, lib().tim_mlp_create(C.byref(h), ctx, d_in))
    return h


def tim_mlp_destroy(mlp):
    lib().tim_mlp_destroy(mlp)


def tim_mlp_param_count(mlp) -> int:
    return int(lib().tim_mlp_param_count(mlp))


def tim_mlp_set_params(ctx, mlp, params):
    p = np.ascontiguousarray(params, dtype=np.float32)
    _check(ctx, lib().tim_mlp_set_params(mlp, _ptr(p), p.size))


def tim_mlp_get_params(ctx, mlp) -> np.ndarray:
    p = np.zeros(tim_mlp_param_count(mlp), dtype=np.float32)
    _check(ctx, lib().tim_mlp_get_params(mlp, _ptr(p), p.size))
    return p


def tim_mlp_set_scaling(ctx, mlp, in_mu, in_isd, out_mu: float, out_sd: float):
    mu = np.ascontiguousarray(in_mu, dtype=np.float32)
    isd = np.ascontiguousarray(in_isd, dtype=np.float32)
    _check(ctx, lib().tim_mlp_set_scaling(mlp, _ptr(mu), _ptr(isd), out_mu, out_sd))


def tim_mlp_grad(ctx, mlp, x, y) -> tuple[float, np.ndarray]:
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.ascontiguousarray(y, dtype=np.float32)
    loss = C.c_float()
    g = np.zeros(tim_mlp_param_count(mlp), dtype=np.float32)
    _check(ctx, lib().tim_mlp_grad(mlp, _ptr(x), _ptr(y), y.shape[0], C.byref(loss), _ptr(g)))
    return float(loss.value), g


def tim_mlp_train(ctx, mlp, x, y, steps: int, lr: float) -> np.ndarray:
    """Full-batch Adam on the device; returns the loss before each step."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.ascontiguousarray(y, dtype=np.float32)
    hist = np.zeros(max(steps, 1), dtype=np.float32)
    _check(ctx, lib().tim_mlp_train(mlp, _ptr(x), _ptr(y), y.shape[0], steps, lr, _ptr(hist)))
    return hist[:steps]


def tim_mlp_predict(ctx, mlp, x) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float32)
    out = np.zeros(x.shape[0], dtype=np.float32)
    _check(ctx, lib().tim_mlp_predict(mlp, _ptr(x), x.shape[0], _ptr(out)))
    return out


def tim_kpt_estimate_learned(ctx, mlp, k: int, ell: float, seed: int):
    """Returns (KPT*, stopping round, predicted start round, accepted)."""
    kpt, rnd, pred, acc = C.c_double(), C.c_int(), C.c_int(), C.c_int()
    _check(ctx, lib().tim_kpt_estimate_learned(ctx, mlp, k, ell, seed, C.byref(kpt), C.byref(rnd),
                                               C.byref(pred), C.byref(acc)))
    return kpt.value, rnd.value, pred.value, bool(acc.value)


def tim_run_learned(ctx, mlp, k: int, eps: float, ell: float, seed: int):
    """TIM+ with the learned start round. Returns (seeds, covered fraction, stats)."""
    seeds = np.zeros(k, dtype=np.int32)
    frac = C.c_double()
    st = tim_stats()
    _check(ctx, lib().tim_run_learned(ctx, mlp, k, eps, ell, seed, _ptr(seeds), C.byref(frac),
                                      C.byref(st)))
    return seeds, frac.value, st.as_dict()


class Engine:
    """Owns one tim_ctx; closes it on exit."""

    def __init__(self, device: int = 0, stream=None):
        self.ctx = tim_create(device, stream)

    def close(self):
        if self.ctx:
            tim_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
