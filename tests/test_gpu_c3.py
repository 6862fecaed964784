"""GPU parity at the paper's largest scale (Section 7, Table 2: a network of Twitter's
size): a directed Chung-Lu graph with 41.6M nodes and exactly 1.4B edges (exponent 2.1),
IC with p drawn per edge from {0.1, 0.01, 0.001} (trivalency), k = 50, eps = 0.2, l = 1.

The graph is drawn on the device, loaded through the C ABI from device memory, and --
copied to the host -- loaded into the oracle, which builds its own G^T. Compared bit for
bit: a spread of RR sets and the heaviest ones the GPU drew (up to ~10^6 members, the
level-synchronous third pass), and TIM+ end to end (stopping round, KPT*, R' greedy,
theta', KPT+, theta, seeds, covered count), and G^T itself against the oracle's
transpose. The module takes a few minutes: the oracle transposes 1.4B edges and runs
TIM+ on all host threads."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1404_0900_gb300 import inputs, tim

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c3():
    import torch
    assert torch.cuda.is_available()
    g = inputs.chung_lu_c3_device(seed=1)
    w = inputs.trivalency_device(g, seed=2)
    eng = tim.Engine(0, torch.cuda.current_stream())
    tim.tim_load_graph_device(eng.ctx, g.n, g.m, g.rowptr, g.dst, w, tim.TIM_IC)
    indeg = torch.bincount(g.dst.to(torch.int64), minlength=g.n)
    shape = {"n": g.n, "m": g.m, "max_indeg": int(indeg.max()),
             "max_outdeg": int((g.rowptr[1:] - g.rowptr[:-1]).max())}
    del indeg
    og = O.load_graph(g.n, g.rowptr.cpu().numpy(), g.dst.cpu().numpy(), w.cpu().numpy(), O.IC)
    del g, w
    torch.cuda.empty_cache()
    yield eng, og, shape
    eng.close()


def test_c3_graph_shape_and_transpose(c3):
    eng, og, shape = c3
    assert shape["n"] == 41_600_000 and shape["m"] == 1_400_000_000
    assert og.n == shape["n"] and og.m == shape["m"]
    # power law with exponent 2.1: hubs of millions of in- and out-edges
    assert shape["max_indeg"] > 10**6 and shape["max_outdeg"] > 10**6
    # G^T (offsets, sources, thresholds) bit for bit against the oracle's transpose
    rowptr, src, thr = tim.tim_get_graph(eng.ctx, og.n, og.m)
    assert np.array_equal(rowptr, og.rowptr.astype(np.uint64))
    assert np.array_equal(src, og.src[:og.m].astype(np.uint32))
    assert np.array_equal(thr, og.thr[:og.m])


def test_c3_rr_sets_spread_and_heaviest(c3):
    eng, og, _ = c3
    seed, sid0, count = 7, O.make_sid(3, 0, 0) + 12345, 200_000
    tim.tim_sample_rr(eng.ctx, count, seed, sid0)
    off, mem, wid = tim.tim_get_rr(eng.ctx)
    sizes = np.diff(off)
    heaviest = np.argsort(sizes, kind="stable")[-8:]
    assert sizes[heaviest[-1]] > 8192  # at least one set beyond the second pass
    for j in sorted(set(range(0, count, 500)) | set(int(x) for x in heaviest)):
        ref, rw = O.rr_one(og, seed, sid0 + j)
        assert np.array_equal(np.sort(mem[off[j]:off[j + 1]]), ref), j
        assert int(wid[j]) == rw, j


def test_c3_tim_plus_end_to_end(c3):
    eng, og, _ = c3
    k, eps, ell, seed = 50, 0.2, 1.0, 1
    seeds, frac, st = tim.tim_run(eng.ctx, k, eps, ell, seed)
    ref = O.tim_plus(og, k, eps, ell, seed)
    assert st["kpt_round"] == ref.kpt.stop_round
    assert st["kpt_star"] == ref.kpt.kpt_star
    assert st["theta_prime"] == ref.refine.theta_prime
    assert st["covered_prime"] == ref.refine.covered
    assert abs(st["kpt_plus"] - ref.refine.kpt_plus) <= 1e-9 * ref.refine.kpt_plus
    lam = O.lam(og.n, k, eps, ell)
    assert abs(st["lambda"] - lam) <= 1e-9 * lam
    # theta may differ by one only when lambda / KPT+ is within 1e-9 of an integer
    q = lam / ref.refine.kpt_plus
    assert st["theta"] == ref.theta or abs(q - round(q)) <= 1e-9 * q
    if st["theta"] == ref.theta:
        assert np.array_equal(seeds, ref.seeds)
        assert st["covered"] == ref.covered
        assert st["members_select"] == ref.extra["members"]
