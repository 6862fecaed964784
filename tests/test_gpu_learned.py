"""GPU parity of the learned start round of Algorithm 2 against the CPU oracle.

- Graph features (tim_graph_features) against oracle.mlp.graph_features.
- The network's forward, loss and gradient (tim_mlp_grad / tim_mlp_predict) against the
  fp64 oracle with the same bfloat16 weight rounding; Adam steps (tim_mlp_train)
  against the oracle's Adam.
- The accept-or-sweep rule (tim_kpt_estimate_learned, tim_run_learned,
  tim_run_batch_learned) against oracle.kpt_estimation_from / tim_plus(start_round),
  with a network forced to a chosen start round.
- The trained network (when its file is present) on held-out graphs: how often its
  start round is accepted and how many sampling rounds it saves.
"""
import math

import numpy as np
import pytest

from oracle import mlp as M
from oracle import oracle as O
from paper_1404_0900_gb300 import inputs, start_round, tim

pytestmark = pytest.mark.gpu
D = tim.TIM_START_FEATURES


@pytest.fixture(scope="module")
def eng():
    import torch
    assert torch.cuda.is_available()
    e = tim.Engine(0)
    yield e
    e.close()


@pytest.fixture()
def net(eng):
    h = tim.tim_mlp_create(eng.ctx, D)
    yield h
    tim.tim_mlp_destroy(h)


def _feature_graphs():
    r = inputs.rmat(12, seed=5)
    cl = inputs.chung_lu(3000, 20000, seed=3)
    iso = inputs.from_edges(20, [(0, 1), (2, 1), (5, 7), (7, 5), (19, 0)])
    return [
        ("rmat12_wc", r, inputs.weighted_cascade(r), tim.TIM_IC),
        ("rmat12_lt", r, inputs.lt_inverse_indegree(r), tim.TIM_LT),
        ("rmat12_tri", r, inputs.trivalency(r, seed=2), tim.TIM_IC),
        ("chunglu_ltr", cl, inputs.lt_random_normalised(cl, seed=4), tim.TIM_LT),
        ("chunglu_p1", cl, inputs.constant(cl, 1.0), tim.TIM_IC),
        ("star", inputs.star_in(50), inputs.weighted_cascade(inputs.star_in(50)), tim.TIM_IC),
        ("isolated", iso, inputs.uniform_random(iso, seed=1), tim.TIM_IC),
        ("no_edges", inputs.from_edges(16, []), np.zeros(0, dtype=np.float32), tim.TIM_IC),
    ]


@pytest.mark.parametrize("case", range(8))
def test_graph_features_match_oracle(eng, case):
    name, g, w, model = _feature_graphs()[case]
    tim.tim_load_graph(eng.ctx, g.n, g.rowptr, g.dst, w, model)
    got = tim.tim_graph_features(eng.ctx)
    want = M.graph_features(g.n, g.rowptr, g.dst, w)
    # the GPU sums thresholds floor(p 2^32) 2^-32 (LT: the saturated cumulative one)
    assert np.allclose(got, want, rtol=2e-6, atol=2e-6), (name, got, want)
    # cached: a second call returns the same values; a reload recomputes
    assert np.array_equal(tim.tim_graph_features(eng.ctx), got)


def _random_case(N, seed, d=D):
    rng = np.random.default_rng(seed)
    p = rng.normal(0, 0.25, size=M.param_count(d)).astype(np.float32)
    x = rng.normal(1.0, 2.0, size=(N, d)).astype(np.float32)
    y = rng.normal(0.5, 1.5, size=N).astype(np.float32)
    mu = rng.normal(size=d).astype(np.float32)
    isd = rng.uniform(0.3, 1.5, size=d).astype(np.float32)
    return p, x, y, mu, isd, 0.25, 1.75


@pytest.mark.parametrize("N", [1, 31, 32, 100, 1000])
def test_mlp_gradient_matches_oracle(eng, net, N):
    p, x, y, mu, isd, omu, osd = _random_case(N, N)
    tim.tim_mlp_set_params(eng.ctx, net, p)
    tim.tim_mlp_set_scaling(eng.ctx, net, mu, isd, omu, osd)
    loss, g = tim.tim_mlp_grad(eng.ctx, net, x, y)
    sc = M.Scaling(D, mu.astype(np.float64), isd.astype(np.float64), omu, osd)
    want_loss, want_g = M.loss_and_grads(p, x.astype(np.float64), y.astype(np.float64), D, sc)
    assert abs(loss - want_loss) <= 2e-5 * abs(want_loss) + 1e-7
    scale = np.max(np.abs(want_g))
    err = np.abs(g - want_g)
    assert np.all(err <= 1e-4 * np.abs(want_g) + 2e-5 * scale), (np.max(err), scale)
    pred = tim.tim_mlp_predict(eng.ctx, net, x)
    want_pred = M.predict(p, x.astype(np.float64), D, sc)
    assert np.allclose(pred, want_pred, rtol=1e-5, atol=1e-5 * np.max(np.abs(want_pred)))
    # deterministic: the same call twice gives the same bits
    loss2, g2 = tim.tim_mlp_grad(eng.ctx, net, x, y)
    assert loss2 == loss and np.array_equal(g2, g)


def test_adam_steps_match_oracle(eng, net):
    N, steps, lr = 200, 5, 1e-2
    p, x, y, mu, isd, omu, osd = _random_case(N, 77)
    p = M.bf16_round(p)  # start on bfloat16 values
    tim.tim_mlp_set_params(eng.ctx, net, p)
    tim.tim_mlp_set_scaling(eng.ctx, net, mu, isd, omu, osd)
    hist = tim.tim_mlp_train(eng.ctx, net, x, y, steps, lr)
    got = tim.tim_mlp_get_params(eng.ctx, net)
    sc = M.Scaling(D, mu.astype(np.float64), isd.astype(np.float64), omu, osd)
    w = p.astype(np.float64)
    m = np.zeros_like(w)
    v = np.zeros_like(w)
    losses = []
    for t in range(1, steps + 1):
        loss, g = M.loss_and_grads(w.astype(np.float32), x.astype(np.float64),
                                   y.astype(np.float64), D, sc)
        losses.append(loss)
        w, m, v = M.adam_step(w, m, v, g, t, lr)
    assert np.allclose(hist, losses, rtol=1e-4)
    assert np.allclose(got, w, rtol=0, atol=2e-5), np.max(np.abs(got - w))
    assert hist[-1] < hist[0]


# ---------------------------------------------------------------- learned start rule

def _forced(eng, net, g, k, i0):
    """Make the network output a constant that maps to start round i0 on graph g."""
    p = np.zeros(M.param_count(D), dtype=np.float32)
    p[-1] = (i0 - 0.5) - math.log2(max(g.m, 1) / k)
    tim.tim_mlp_set_params(eng.ctx, net, p)
    tim.tim_mlp_set_scaling(eng.ctx, net, np.zeros(D), np.ones(D), 0.0, 1.0)


@pytest.mark.parametrize("model", [tim.TIM_IC, tim.TIM_LT])
def test_learned_kpt_matches_oracle(eng, net, model):
    g = inputs.rmat(12, seed=9)
    w = inputs.weighted_cascade(g) if model == tim.TIM_IC else inputs.lt_inverse_indegree(g)
    tim.tim_load_graph(eng.ctx, g.n, g.rowptr, g.dst, w, model)
    og = O.load_graph(g.n, g.rowptr, g.dst, w, model)
    k, seed = 10, 3
    plain = O.kpt_estimation(og, k, 1.0, seed)
    i_star = plain.stop_round
    assert i_star >= 2
    rounds = O.kpt_rounds(g.n)
    for i0 in sorted({1, i_star - 1, i_star, i_star + 1, rounds}):
        _forced(eng, net, g, k, i0)
        kpt, rnd, pred, acc = tim.tim_kpt_estimate_learned(eng.ctx, net, k, 1.0, seed)
        want, want_acc = O.kpt_estimation_from(og, k, 1.0, seed, i0)
        assert pred == i0
        assert acc == want_acc, i0
        assert rnd == want.stop_round
        assert abs(kpt - want.kpt_star) <= 1e-9 * want.kpt_star
        # R' in the store: the sets of the stopping round
        off, mem, _ = tim.tim_get_rr(eng.ctx)
        roff, rmem, _ = O.sample(og, seed, O.make_sid(O.PHASE_KPT, want.last_round, 0),
                                 want.last_c)
        assert np.array_equal(np.diff(off), np.diff(roff))
        for j in range(0, len(off) - 1, max(1, (len(off) - 1) // 97)):
            assert np.array_equal(np.sort(mem[off[j]:off[j + 1]]),
                                  np.sort(rmem[roff[j]:roff[j + 1]]))
    # TIM+ end to end from a start round: seeds bit-exact with the oracle
    for i0 in (i_star, i_star + 1):
        _forced(eng, net, g, k, i0)
        seeds, frac, st = tim.tim_run_learned(eng.ctx, net, k, 0.5, 1.0, seed)
        ref = O.tim_plus(og, k, 0.5, 1.0, seed, start_round=i0)
        assert np.array_equal(seeds, ref.seeds)
        assert st["theta"] == ref.theta and st["covered"] == ref.covered
        assert st["kpt_predicted_round"] == i0
        assert st["kpt_accepted"] == (i0 == i_star)


def test_batch_learned_equals_single_learned(eng, net):
    specs = [(12, 1, tim.TIM_IC, 5), (11, 2, tim.TIM_LT, 3), (10, 3, tim.TIM_IC, 20),
             (12, 4, tim.TIM_LT, 10), (9, 5, tim.TIM_IC, 1)]
    graphs = []
    for scale, gs, model, k in specs:
        g = inputs.rmat(scale, seed=gs)
        w = inputs.weighted_cascade(g) if model == tim.TIM_IC else inputs.lt_inverse_indegree(g)
        graphs.append((g, w, model, k))
    # one constant output for every query: start rounds differ with n, m and k
    p = np.zeros(M.param_count(D), dtype=np.float32)
    p[-1] = -1.3
    tim.tim_mlp_set_params(eng.ctx, net, p)
    tim.tim_mlp_set_scaling(eng.ctx, net, np.zeros(D), np.ones(D), 0.0, 1.0)
    engines = [tim.Engine(0) for _ in graphs]
    try:
        queries = []
        for i, ((g, w, model, k), e) in enumerate(zip(graphs, engines)):
            tim.tim_load_graph(e.ctx, g.n, g.rowptr, g.dst, w, model)
            queries.append({"ctx": e.ctx, "k": k, "eps": 0.5, "ell": 1.0, "tag": 40 + i})
        res, bst = tim.tim_run_batch(queries, seed=5, plus=True, mlp=net)
        plain, _ = tim.tim_run_batch(queries, seed=5, plus=True)
        accepted = 0
        for i, (g, w, model, k) in enumerate(graphs):
            with tim.Engine(0) as one:
                tim.tim_load_graph(one.ctx, g.n, g.rowptr, g.dst, w, model)
                tim.tim_set_query_tag(one.ctx, 40 + i)
                seeds, frac, st = tim.tim_run_learned(one.ctx, net, k, 0.5, 1.0, 5)
            bseeds, bfrac, bs = res[i]
            assert np.array_equal(bseeds, seeds), i
            for key in ("kpt_round", "kpt_star", "kpt_plus", "theta", "covered", "kpt_sets",
                        "kpt_predicted_round", "kpt_accepted"):
                assert bs[key] == st[key], (i, key, bs[key], st[key])
            i0 = bs["kpt_predicted_round"]
            og = O.load_graph(g.n, g.rowptr, g.dst, w, model)
            want, want_acc = O.kpt_estimation_from(og, k, 1.0, 5, i0, tag=40 + i)
            assert bool(bs["kpt_accepted"]) == want_acc and bs["kpt_round"] == want.stop_round
            accepted += bs["kpt_accepted"]
            if not bs["kpt_accepted"]:  # a rejected start returns exactly the plain run
                assert np.array_equal(bseeds, plain[i][0])
                assert bs["kpt_star"] == plain[i][2]["kpt_star"]
        assert bst["learned_accepted"] == accepted
    finally:
        for e in engines:
            e.close()


def test_learned_rejects_bad_arguments(eng, net):
    g = inputs.rmat(8, seed=1)
    tim.tim_load_graph(eng.ctx, g.n, g.rowptr, g.dst, inputs.weighted_cascade(g), tim.TIM_IC)
    with pytest.raises(tim.TimError):
        tim.tim_kpt_estimate_learned(eng.ctx, net, 0, 1.0, 1)
    small = tim.tim_mlp_create(eng.ctx, 5)
    try:
        with pytest.raises(tim.TimError):  # not a 12-feature network
            tim.tim_kpt_estimate_learned(eng.ctx, small, 3, 1.0, 1)
    finally:
        tim.tim_mlp_destroy(small)
    with pytest.raises(tim.TimError):
        tim.tim_mlp_set_params(eng.ctx, net, np.zeros(3, dtype=np.float32))
    with pytest.raises(tim.TimError):
        tim.tim_mlp_create(eng.ctx, 33)


# ---------------------------------------------------------------- the trained network

HELD_OUT = [(s, gs, model) for s, gs in ((15, 101), (16, 102), (17, 103), (18, 104))
            for model in (tim.TIM_IC, tim.TIM_LT)]


@pytest.mark.skipif(not start_round.available(), reason="no trained start-round network")
def test_trained_network_gain_on_held_out_graphs(eng):
    """Host-generated R-MAT graphs (the training set was drawn on the device), k = 50:
    the learned start must be accepted on most of them, every result must equal what
    the rule defines, and the sampling launches of Algorithm 2 must drop."""
    mlp, rec = start_round.load(eng.ctx)
    try:
        acc = 0
        launches_plain = launches_learned = 0
        for scale, gs, model in HELD_OUT:
            g = inputs.rmat(scale, seed=gs)
            w = inputs.weighted_cascade(g) if model == tim.TIM_IC else inputs.lt_inverse_indegree(g)
            tim.tim_load_graph(eng.ctx, g.n, g.rowptr, g.dst, w, model)
            kpt, rnd = tim.tim_kpt_estimate(eng.ctx, 50, 1.0, 1)
            lkpt, lrnd, pred, a = tim.tim_kpt_estimate_learned(eng.ctx, mlp, 50, 1.0, 1)
            launches_plain += rnd if rnd else O.kpt_rounds(g.n)
            if a:
                acc += 1
                launches_learned += 1
                assert lrnd == pred
                if pred == rnd:
                    assert lkpt == kpt
            else:  # the plain sweep ran after the two-round try
                assert lrnd == rnd and lkpt == kpt
                launches_learned += 1 + rnd
        assert acc >= len(HELD_OUT) // 2, acc
        assert launches_learned < launches_plain
    finally:
        tim.tim_mlp_destroy(mlp)
