"""GPU parity: the CUDA path through the C ABI against the CPU oracle, on the same
seeded inputs. RR sets (sorted), widths, coverage counts, covered counts and seed
sets are compared bit for bit; the kappa sums are exact integers, so KPT*, KPT', KPT+
and theta are compared exactly too (theta may differ by one only when lambda / KPT+
lies within 1e-9 relative of an integer)."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1404_0900_gb300 import inputs, tim

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eng():
    import torch
    assert torch.cuda.is_available()
    e = tim.Engine(0)
    yield e
    e.close()


def _load(eng, g, w, model):
    tim.tim_load_graph(eng.ctx, g.n, g.rowptr, g.dst, w, model)
    return O.load_graph(g.n, g.rowptr, g.dst, w, model)


def _sets(off, mem):
    return [np.sort(mem[off[j]:off[j + 1]]) for j in range(len(off) - 1)]


def _compare_store(eng, og, seed, sid0, count):
    tot = tim.tim_sample_rr(eng.ctx, count, seed, sid0)
    off, mem, wid = tim.tim_get_rr(eng.ctx)
    roff, rmem, rwid = O.sample(og, seed, sid0, count)
    assert tot == rmem.shape[0]
    assert np.array_equal(np.diff(off), np.diff(roff))
    assert np.array_equal(wid, rwid)
    for a, b in zip(_sets(off, mem), _sets(roff, rmem)):
        assert np.array_equal(a, b)
    return off


GRAPHS = {
    "rmat12_wc": lambda: (inputs.rmat(12, seed=5), "wc"),
    "rmat14_wc": lambda: (inputs.rmat(14, seed=1), "wc"),
    "rand_p1": lambda: (inputs.random_small(3000, 9000, seed=2), "p1"),
    "star": lambda: (inputs.star_in(40000), "wc"),
    "chain": lambda: (inputs.chain(3000), "p1"),
    "rmat10_tri": lambda: (inputs.rmat(10, seed=9), "tri"),
    "rmat13_mixed": lambda: (inputs.rmat(13, seed=4), "mixed"),
    # 500 roots reach node 0, whose 6000 in-edges are all live: one frontier batch
    # inserts 6000 members into a set whose visited hash starts small and must grow
    "fan_p1": lambda: (inputs.from_edges(6501, [(i, 0) for i in range(1, 6001)]
                                         + [(0, j) for j in range(6001, 6501)]), "p1"),
}


def _weights(g, kind, model):
    if kind == "p1":  # LT weights must sum to <= 1 per node: use 1/indeg there
        return inputs.constant(g, 1.0) if model == O.IC else inputs.lt_inverse_indegree(g)
    if kind == "tri":
        return inputs.trivalency(g, seed=3) if model == O.IC else inputs.lt_random_normalised(g, 3)
    if kind == "mixed":
        # in-lists with one shared probability (even nodes), per-edge probabilities (odd
        # nodes), some p = 0 and p = 1 in-lists
        w = inputs.weighted_cascade(g).copy()
        if model == O.IC:
            odd = (g.dst % 2) == 1
            w[odd] = inputs.trivalency(g, seed=5)[odd]
            w[g.dst % 7 == 0] = 1.0
            w[g.dst % 11 == 0] = 0.0
        return w
    return inputs.weighted_cascade(g)


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("model", [O.IC, O.LT])
def test_rr_sets_bit_exact(eng, name, model):
    g, kind = GRAPHS[name]()
    w = _weights(g, kind, model)
    og = _load(eng, g, w, model)
    count = 3000 if name in ("rand_p1", "chain", "fan_p1") else 20000
    _compare_store(eng, og, 11, O.make_sid(3, 0, 0), count)
    # a second seed and a set-id range that does not start at zero
    _compare_store(eng, og, 12345678901, (5 << 40) + 17, 777)


@pytest.mark.parametrize("budget,team,cap,factor", [(0, 0, 256, 2), (64, 1, 256, 2),
                                                    (1 << 40, 0, 256, 2), (0, 2, 256, 2),
                                                    (0, 4, 256, 2), (0, 8, 256, 2),
                                                    (300, 8, 256, 2), (1024, 0, 128, 1),
                                                    (1024, 0, 512, 8), (1 << 40, 0, 512, 64),
                                                    (2048, 0, 128, 4)])
def test_ic_rr_sets_bit_exact_for_any_split(eng, budget, team, cap, factor):
    # which pass expands a set, its queue capacity in pass 1 and how many warps share it
    # must not matter
    g = inputs.rmat(13, seed=3)
    w = inputs.weighted_cascade(g)
    og = _load(eng, g, w, O.IC)
    tim.tim_set_width_budget(eng.ctx, budget)
    tim.tim_set_team_size(eng.ctx, team)
    tim.tim_set_pass1_capacity(eng.ctx, cap)
    tim.tim_set_team_factor(eng.ctx, factor)
    try:
        _compare_store(eng, og, 5, O.make_sid(3, 0, 0), 6000)
        k = O.kappa_sum(og, 10, 5, O.make_sid(1, 3, 0), 4000)
        assert tim.tim_kappa_sum(eng.ctx, 10, 5, O.make_sid(1, 3, 0), 4000) == k
        seeds = np.array([0, 1, 2, 5], dtype=np.int32)
        assert tim.tim_covered_count(eng.ctx, seeds, 5, 77, 5000) == \
            O.covered_count(og, 5, 77, 5000, seeds)
    finally:
        tim.tim_set_width_budget(eng.ctx, 16384)
        tim.tim_set_team_size(eng.ctx, 0)
        tim.tim_set_pass1_capacity(eng.ctx, 256)
        tim.tim_set_team_factor(eng.ctx, 2)


def test_rr_sets_ragged_and_empty(eng):
    g = inputs.rmat(11, seed=4)
    w = inputs.weighted_cascade(g)
    og = _load(eng, g, w, O.IC)
    for count in (0, 1, 2, 31, 33, 4097):
        tot = tim.tim_sample_rr(eng.ctx, count, 3, 99)
        off, mem, wid = tim.tim_get_rr(eng.ctx)
        assert off.shape[0] == count + 1
        if count:
            roff, rmem, rwid = O.sample(og, 3, 99, count)
            assert np.array_equal(wid, rwid) and tot == rmem.shape[0]


def test_edge_free_and_tiny_graphs(eng):
    for g in (inputs.from_edges(2, []), inputs.from_edges(2, [(0, 1)]),
              inputs.from_edges(5, [(4, 0), (3, 0)])):
        for model in (O.IC, O.LT):
            w = inputs.constant(g, 1.0 if model == O.IC else 0.5)
            og = _load(eng, g, w, model)
            _compare_store(eng, og, 1, 0, 500)


@pytest.mark.parametrize("model", [O.IC, O.LT])
def test_kappa_sum_exact(eng, model):
    g = inputs.rmat(13, seed=7)
    w = inputs.weighted_cascade(g)
    og = _load(eng, g, w, model)
    for k, count in ((1, 5000), (10, 20000), (50, 7777), (1000, 3000)):
        sid0 = O.make_sid(1, 4, 0)
        got = tim.tim_kappa_sum(eng.ctx, k, 5, sid0, count)
        want = O.kappa_sum(og, k, 5, sid0, count)
        assert got == want, (k, got, want)


@pytest.mark.parametrize("model", [O.IC, O.LT])
def test_coverage_counts_and_covered_count(eng, model):
    g = inputs.rmat(12, seed=8)
    w = inputs.weighted_cascade(g)
    og = _load(eng, g, w, model)
    sid0 = O.make_sid(3, 0, 0)
    tim.tim_sample_rr(eng.ctx, 30000, 21, sid0)
    counts = tim.tim_coverage_counts(eng.ctx, g.n)
    roff, rmem, _ = O.sample(og, 21, sid0, 30000)
    seeds, cov, counts0 = O.greedy(g.n, roff, rmem, 7)
    assert np.array_equal(counts.astype(np.int64), counts0)
    gs, frac, gcov = tim.tim_node_select(eng.ctx, 7)
    assert np.array_equal(gs, seeds) and gcov == cov
    assert frac == cov / 30000
    c = tim.tim_covered_count(eng.ctx, seeds[:3], 21, O.make_sid(2, 0, 0), 25000)
    assert c == O.covered_count(og, 21, O.make_sid(2, 0, 0), 25000, seeds[:3])


@pytest.mark.parametrize("team", [1, 2, 4, 8])
def test_covered_count_with_every_set_in_teams(eng, team):
    # budget 0 hands every set, light or heavy, to the second pass, where teams of
    # `team` warps stop each set at its first seed (Algorithm 3's coverage test)
    g = inputs.rmat(13, seed=4)
    w = inputs.weighted_cascade(g)
    og = _load(eng, g, w, O.IC)
    rng = np.random.default_rng(team)
    try:
        tim.tim_set_width_budget(eng.ctx, 0)
        tim.tim_set_team_size(eng.ctx, team)
        for seeds in ([0], rng.choice(g.n, 5, replace=False).tolist(),
                      rng.choice(g.n, 60, replace=False).tolist()):
            for count in (3000, 777):
                c = tim.tim_covered_count(eng.ctx, seeds, 5, O.make_sid(2, 0, 9), count)
                assert c == O.covered_count(og, 5, O.make_sid(2, 0, 9), count, seeds), (team, seeds)
    finally:
        tim.tim_set_width_budget(eng.ctx, 16384)
        tim.tim_set_team_size(eng.ctx, 0)


@pytest.mark.parametrize("k", [1, 3, 16])
def test_greedy_ties_and_k_equals_n(eng, k):
    g = inputs.complete(16)
    og = _load(eng, g, inputs.constant(g, 0.0), O.IC)
    tim.tim_sample_rr(eng.ctx, 64, 2, 0)
    roff, rmem, _ = O.sample(og, 2, 0, 64)
    seeds, cov, _ = O.greedy(g.n, roff, rmem, k)
    gs, _, gcov = tim.tim_node_select(eng.ctx, k)
    assert np.array_equal(gs, seeds) and gcov == cov


@pytest.mark.parametrize("p", [1.0, 0.3])
def test_greedy_with_sets_of_many_member_chunks(eng, p):
    # p = 1: every set is the root's whole reverse-reachable part of an R-MAT 14 graph,
    # thousands of members, so the cooperative greedy splits the sets its first seed
    # covers into chunks of members that all warps share; p = 0.3 mixes small and large
    g = inputs.rmat(14, seed=3)
    og = _load(eng, g, inputs.constant(g, p), O.IC)
    tim.tim_sample_rr(eng.ctx, 3000, 7, O.make_sid(3, 0, 5))
    roff, rmem, _ = O.sample(og, 7, O.make_sid(3, 0, 5), 3000)
    assert np.diff(roff).max() > 4096
    for k in (1, 10):
        seeds, cov, _ = O.greedy(g.n, roff, rmem, k)
        gs, frac, gcov = tim.tim_node_select(eng.ctx, k)
        assert np.array_equal(gs, seeds) and gcov == cov, (p, k)
    # after the last round the counts are the uncovered sets each node is in
    tim.tim_select_begin(eng.ctx)
    left = tim.tim_select_counts(eng.ctx, g.n).astype(np.int64)
    for v in seeds:
        tim.tim_select_take(eng.ctx, int(v))
    after = tim.tim_select_counts(eng.ctx, g.n).astype(np.int64)
    covered = np.zeros(3000, bool)
    for j in range(3000):
        covered[j] = np.isin(rmem[roff[j]:roff[j + 1]], seeds).any()
    want = np.zeros(g.n, np.int64)
    for j in np.nonzero(~covered)[0]:
        want[rmem[roff[j]:roff[j + 1]]] += 1
    assert np.array_equal(after, want) and left.sum() == rmem.shape[0]


def _theta_equal(a, b, lam, kpt):
    if a == b:
        return True
    x = lam / kpt
    return abs(a - b) == 1 and abs(x - round(x)) <= 1e-9 * x


@pytest.mark.parametrize("model", [O.IC, O.LT])
@pytest.mark.parametrize("scale,k,eps", [(12, 5, 0.5), (14, 10, 0.5)])
def test_tim_plus_end_to_end(eng, model, scale, k, eps):
    g = inputs.rmat(scale, seed=1)
    w = inputs.weighted_cascade(g)
    og = _load(eng, g, w, model)
    seeds, frac, st = tim.tim_run(eng.ctx, k, eps, 1.0, 1)
    ref = O.tim_plus(og, k, eps, 1.0, 1)
    assert st["kpt_round"] == ref.kpt.stop_round
    assert st["kpt_last_round"] == ref.kpt.last_round
    assert st["kpt_star"] == ref.kpt.kpt_star
    assert st["theta_prime"] == ref.refine.theta_prime
    assert st["covered_prime"] == ref.refine.covered
    assert abs(st["eps_prime"] - ref.refine.eps_prime) <= 1e-15
    assert abs(st["kpt_plus"] - ref.refine.kpt_plus) <= 1e-9 * ref.refine.kpt_plus
    lam = O.lam(g.n, k, eps, 1.0)
    assert abs(st["lambda"] - lam) <= 1e-9 * lam
    assert _theta_equal(st["theta"], ref.theta, lam, ref.refine.kpt_plus)
    if st["theta"] == ref.theta:
        assert np.array_equal(seeds, ref.seeds)
        assert st["covered"] == ref.covered
        assert frac == ref.covered / ref.theta
        assert st["members_select"] == ref.extra["members"]


@pytest.mark.parametrize("model", [O.IC, O.LT])
def test_plain_tim_end_to_end(eng, model):
    g = inputs.rmat(12, seed=2)
    w = inputs.weighted_cascade(g)
    og = _load(eng, g, w, model)
    seeds, frac, st = tim.tim_run_tim(eng.ctx, 4, 0.5, 1.0, 3)
    ref = O.tim(og, 4, 0.5, 1.0, 3)
    assert st["kpt_star"] == ref.kpt.kpt_star
    lam = O.lam(g.n, 4, 0.5, 1.0)
    assert _theta_equal(st["theta"], ref.theta, lam, ref.kpt.kpt_star)
    if st["theta"] == ref.theta:
        assert np.array_equal(seeds, ref.seeds) and st["covered"] == ref.covered


def test_kpt_strongly_connected_closed_form(eng):
    g = inputs.complete(12)
    _load(eng, g, inputs.constant(g, 1.0), O.IC)
    kpt, rnd = tim.tim_kpt_estimate(eng.ctx, 3, 1.0, 5)
    assert rnd == 1 and kpt == g.n / 2


def test_invalid_inputs_are_rejected(eng):
    rowptr = np.array([0, 2, 3, 3], dtype=np.int64)
    for dst in ([1, 0, 2], [1, 1, 2], [1, 7, 2]):
        with pytest.raises(tim.TimError) as ei:
            tim.tim_load_graph(eng.ctx, 3, rowptr, np.array(dst, np.int32),
                               np.full(3, 0.5, np.float32), O.IC)
        assert ei.value.code == -1
    with pytest.raises(tim.TimError):
        tim.tim_load_graph(eng.ctx, 3, rowptr, np.array([1, 2, 0], np.int32),
                           np.array([0.5, 1.5, 0.5], np.float32), O.IC)
    g = inputs.star_in(4)
    with pytest.raises(tim.TimError):
        tim.tim_load_graph(eng.ctx, 4, g.rowptr, g.dst, np.full(3, 0.5, np.float32), O.LT)
    with pytest.raises(tim.TimError) as ei:
        tim.tim_kpt_estimate(eng.ctx, 1, 1.0, 1)  # graph was not loaded
    assert ei.value.code == -6
    g = inputs.rmat(8)
    _load(eng, g, inputs.weighted_cascade(g), O.IC)
    with pytest.raises(tim.TimError):
        tim.tim_node_select(eng.ctx, g.n + 1)


def test_device_resident_load_matches_host_load(eng):
    import torch
    g = inputs.rmat(12, seed=6)
    w = inputs.weighted_cascade(g)
    tim.tim_load_graph(eng.ctx, g.n, g.rowptr, g.dst, w, O.IC)
    a = tim.tim_sample_rr(eng.ctx, 5000, 4, 0)
    off_a, mem_a, wid_a = tim.tim_get_rr(eng.ctx)
    dr = torch.from_numpy(g.rowptr).cuda()
    dd = torch.from_numpy(g.dst).cuda()
    dw = torch.from_numpy(w).cuda()
    torch.cuda.synchronize()
    tim.tim_load_graph_device(eng.ctx, g.n, g.m, dr, dd, dw, O.IC)
    b = tim.tim_sample_rr(eng.ctx, 5000, 4, 0)
    off_b, mem_b, wid_b = tim.tim_get_rr(eng.ctx)
    assert a == b and np.array_equal(off_a, off_b) and np.array_equal(wid_a, wid_b)
    for x, y in zip(_sets(off_a, mem_a), _sets(off_b, mem_b)):
        assert np.array_equal(x, y)


def test_autotune_keeps_results(eng):
    g = inputs.rmat(13, seed=2)
    w = inputs.weighted_cascade(g)
    og = _load(eng, g, w, O.IC)
    before = tim.tim_run(eng.ctx, 5, 0.5, 1.0, 9)
    t = tim.tim_autotune(eng.ctx, 20000, 9)
    assert t["trials"] >= 3 and t["best_ms"] <= t["default_ms"] + 1e-9
    after = tim.tim_run(eng.ctx, 5, 0.5, 1.0, 9)
    assert np.array_equal(before[0], after[0]) and before[2]["theta"] == after[2]["theta"]
    ref = O.tim_plus(og, 5, 0.5, 1.0, 9)
    assert np.array_equal(after[0], ref.seeds)
    assert t["team_factor"] in (1, 2, 4, 8) and t["pass1_capacity"] in (128, 256, 512)
    assert t["trials"] == 20
    tim.tim_set_width_budget(eng.ctx, 16384)
    tim.tim_set_team_size(eng.ctx, 0)
    tim.tim_set_chunk(eng.ctx, 2)
    tim.tim_set_team_factor(eng.ctx, 2)
    tim.tim_set_pass1_capacity(eng.ctx, 256)


def _hub_graph(n, m_background, hub_degrees, seed):
    """Random background graph plus hubs 0, 1, ... with the given in-degrees (their
    in-lists then fall under the geometric-skip rule when they share a threshold)."""
    rng = np.random.default_rng(seed)
    src = [rng.integers(0, n, m_background)]
    dst = [rng.integers(len(hub_degrees), n, m_background)]  # hubs get exactly their degree
    for h, d in enumerate(hub_degrees):
        src.append(rng.choice(np.arange(len(hub_degrees), n), size=d, replace=False))
        dst.append(np.full(d, h))
        # out-edges, so that RR sets often reach the hub
        src.append(np.full(300, h))
        dst.append(rng.choice(np.arange(len(hub_degrees), n), size=300, replace=False))
    return inputs.csr_from_pairs(n, np.concatenate(src), np.concatenate(dst), name="hubs")


@pytest.mark.parametrize("weights", ["wc", "p0.002", "p0.3_heavy", "mixed"])
@pytest.mark.parametrize("budget,team", [(16384, 0), (64, 1), (0, 8), (1 << 40, 0)])
def test_skip_lists_bit_exact_in_every_pass(eng, weights, budget, team):
    if weights == "p0.3_heavy":  # sets beyond the pass-2 queue: the batched third pass
        g = _hub_graph(20000, 100000, [1024, 1500, 3000, 5000], seed=1)
        w = inputs.constant(g, 0.3)
        count = 600
    else:
        g = _hub_graph(12000, 60000, [511, 512, 1500, 3000, 9000], seed=2)
        if weights == "wc":
            w = inputs.weighted_cascade(g)
        elif weights == "p0.002":
            w = inputs.constant(g, 0.002)
        else:  # hub 2's in-list gets one different probability: per-edge coins there
            w = inputs.weighted_cascade(g)
            w[np.flatnonzero(g.dst == 2)[7]] = np.float32(0.25)
        count = 20000
    og = _load(eng, g, w, O.IC)
    tim.tim_set_width_budget(eng.ctx, budget)
    tim.tim_set_team_size(eng.ctx, team)
    try:
        _compare_store(eng, og, 5, O.make_sid(3, 0, 0), count)
        k = O.kappa_sum(og, 10, 5, O.make_sid(1, 3, 0), count)
        assert tim.tim_kappa_sum(eng.ctx, 10, 5, O.make_sid(1, 3, 0), count) == k
        seeds = np.array([0, 1, 7, 11], dtype=np.int32)
        assert tim.tim_covered_count(eng.ctx, seeds, 5, 77, count) == \
            O.covered_count(og, 5, 77, count, seeds)
    finally:
        tim.tim_set_width_budget(eng.ctx, 16384)
        tim.tim_set_team_size(eng.ctx, 0)


def _heavy_skip_graph():
    """Sets far beyond pass 2's queue (p = 0.3 on a background of mean in-degree 5) that
    also reach hubs whose in-lists take the skip rule (weighted cascade, 600-9000
    in-edges): the heavy-set pass meets both kinds of list."""
    g = _hub_graph(30000, 150000, [600, 1500, 3000, 9000], seed=3)
    w = inputs.constant(g, 0.3)
    hub = g.dst < 4
    w[hub] = inputs.weighted_cascade(g)[hub]
    return g, w


@pytest.mark.parametrize("stepped", [0, 1])
def test_heavy_pass_persistent_and_stepped_bit_exact(eng, stepped):
    g, w = _heavy_skip_graph()
    og = _load(eng, g, w, O.IC)
    tim.tim_set_heavy_pass(eng.ctx, stepped)
    try:
        tim.tim_get_profile(eng.ctx, reset=True)
        off = _compare_store(eng, og, 5, O.make_sid(3, 0, 0), 400)
        assert np.diff(off).max() > 8192
        assert tim.tim_get_profile(eng.ctx)["pass3_sets"] > 0
        k = O.kappa_sum(og, 10, 5, O.make_sid(1, 3, 0), 300)
        assert tim.tim_kappa_sum(eng.ctx, 10, 5, O.make_sid(1, 3, 0), 300) == k
        seeds = np.array([0, 1, 7, 11], dtype=np.int32)
        assert tim.tim_covered_count(eng.ctx, seeds, 5, 77, 300) == \
            O.covered_count(og, 5, 77, 300, seeds)
    finally:
        tim.tim_set_heavy_pass(eng.ctx, 0)


def test_grid_barrier_timeout_is_reported_and_the_context_recovers(eng):
    """A poll limit of zero makes every block that waits at a grid barrier give up at
    once: the heavy-set pass and the greedy return TIM_ERR_TIMEOUT (no fault, no hang),
    and with the default limit the same context gives the oracle's results again."""
    g, w = _heavy_skip_graph()
    og = _load(eng, g, w, O.IC)
    sid0 = O.make_sid(3, 0, 0)
    tim.tim_set_wait_limit(eng.ctx, 0)
    try:
        with pytest.raises(tim.TimError) as ei:
            tim.tim_sample_rr(eng.ctx, 400, 5, sid0)
        assert ei.value.code == -4
    finally:
        tim.tim_set_wait_limit(eng.ctx, 1 << 24)
    _compare_store(eng, og, 5, sid0, 400)
    # the greedy's cooperative launch
    h = inputs.rmat(12, seed=5)
    wh = inputs.weighted_cascade(h)
    oh = _load(eng, h, wh, O.IC)
    tim.tim_sample_rr(eng.ctx, 20000, 5, sid0)
    tim.tim_set_wait_limit(eng.ctx, 0)
    try:
        with pytest.raises(tim.TimError) as ei:
            tim.tim_node_select(eng.ctx, 10)
        assert ei.value.code == -4
    finally:
        tim.tim_set_wait_limit(eng.ctx, 1 << 24)
    seeds, _, cov = tim.tim_node_select(eng.ctx, 10)
    roff, rmem, _ = O.sample(oh, 5, sid0, 20000)
    rseeds, rcov, _ = O.greedy(h.n, roff, rmem, 10)
    assert np.array_equal(seeds, rseeds) and cov == rcov


def _oracle_graph_arrays(og):
    return og.rowptr.astype(np.uint64), og.src[:og.m].astype(np.uint32), og.thr[:og.m]


@pytest.mark.parametrize("name", ["rmat12_wc", "rmat10_tri", "rmat13_mixed", "star", "chain",
                                  "rand_p1"])
@pytest.mark.parametrize("model", [O.IC, O.LT])
def test_graph_load_equals_the_oracle_transpose(eng, name, model):
    """Row A1 directly: the in-CSR offsets, sources (ascending per in-list) and thresholds
    of G^T bit for bit against the oracle's own transpose (Table 1)."""
    g, kind = GRAPHS[name]()
    w = _weights(g, kind, model)
    og = _load(eng, g, w, model)
    rowptr, src, thr = tim.tim_get_graph(eng.ctx, g.n, g.m)
    r0, s0, t0 = _oracle_graph_arrays(og)
    assert np.array_equal(rowptr, r0) and np.array_equal(src, s0) and np.array_equal(thr, t0)


@pytest.mark.parametrize("n", [(1 << 20) + 3, 1 << 21, (1 << 21) + 1, 3 << 21])
def test_graph_load_key_widths(eng, n):
    """Node counts around powers of two change the number of sort passes (odd and even)."""
    rng = np.random.default_rng(n)
    m = 200_000
    g = inputs.csr_from_pairs(n, rng.integers(0, n, m), rng.integers(0, n, m))
    w = inputs.uniform_random(g, 0.0, 1.0, seed=4)
    og = _load(eng, g, w, O.IC)
    rowptr, src, thr = tim.tim_get_graph(eng.ctx, g.n, g.m)
    r0, s0, t0 = _oracle_graph_arrays(og)
    assert np.array_equal(rowptr, r0) and np.array_equal(src, s0) and np.array_equal(thr, t0)


def test_device_load_on_the_default_stream_follows_pending_work():
    """An engine on torch's default stream (handle 0) runs on that stream: a device load
    right after the kernels that produce its inputs, with no synchronisation, sees
    their results."""
    import torch
    g = inputs.rmat(16, seed=8)
    w = inputs.trivalency(g, seed=9)
    og = O.load_graph(g.n, g.rowptr, g.dst, w, O.IC)
    with tim.Engine(0, torch.cuda.current_stream()) as e:
        for _ in range(2):
            d_rowptr = torch.from_numpy(g.rowptr).cuda()
            d_dst = torch.from_numpy(g.dst).cuda()
            d_w = torch.from_numpy(w).cuda()
            # a long chain of work on the default stream that ends in the weights
            for _ in range(200):
                d_w = d_w * 1.0 + 0.0
            tim.tim_load_graph_device(e.ctx, g.n, g.m, d_rowptr, d_dst, d_w, tim.TIM_IC)
            rowptr, src, thr = tim.tim_get_graph(e.ctx, g.n, g.m)
            r0, s0, t0 = _oracle_graph_arrays(og)
            assert np.array_equal(rowptr, r0) and np.array_equal(src, s0)
            assert np.array_equal(thr, t0)
