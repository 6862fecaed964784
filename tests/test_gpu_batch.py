"""Batched queries (tim_run_batch): every query's result must equal a single run of
the same query with the same seed and set-id tag, and tagged runs must match the
oracle. Queries mix IC and LT, graph sizes, k and eps."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1404_0900_gb300 import inputs, tim

pytestmark = pytest.mark.gpu

SPECS = [  # (scale, graph seed, model, k, eps)
    (12, 1, tim.TIM_IC, 5, 0.5), (11, 2, tim.TIM_LT, 3, 0.3), (13, 3, tim.TIM_IC, 20, 0.5),
    (10, 4, tim.TIM_LT, 1, 0.2), (9, 5, tim.TIM_IC, 7, 0.5), (12, 6, tim.TIM_LT, 10, 0.5),
    (3, 7, tim.TIM_IC, 2, 0.5), (13, 8, tim.TIM_LT, 4, 0.5),
]


def _weights(g, model):
    return inputs.weighted_cascade(g) if model == tim.TIM_IC else inputs.lt_inverse_indegree(g)


def _graphs():
    out = []
    for scale, gseed, model, k, eps in SPECS:
        g = inputs.rmat(scale, seed=gseed) if scale > 3 else inputs.complete(5)
        out.append((g, _weights(g, model), model, k, eps))
    return out


@pytest.mark.parametrize("plus", [True, False])
def test_batch_equals_single_tagged_runs(plus):
    graphs = _graphs()
    engines = [tim.Engine(0) for _ in graphs]
    try:
        queries = []
        for i, ((g, w, model, k, eps), e) in enumerate(zip(graphs, engines)):
            tim.tim_load_graph(e.ctx, g.n, g.rowptr, g.dst, w, model)
            queries.append({"ctx": e.ctx, "k": k, "eps": eps, "ell": 1.0, "tag": 100 + i})
        res, bst = tim.tim_run_batch(queries, seed=7, plus=plus)
        assert bst["queries"] == len(graphs)
        for i, (g, w, model, k, eps) in enumerate(graphs):
            with tim.Engine(0) as one:
                tim.tim_load_graph(one.ctx, g.n, g.rowptr, g.dst, w, model)
                tim.tim_set_query_tag(one.ctx, 100 + i)
                if plus:
                    seeds, frac, st = tim.tim_run(one.ctx, k, eps, 1.0, 7)
                else:
                    seeds, frac, st = tim.tim_run_tim(one.ctx, k, eps, 1.0, 7)
            bseeds, bfrac, bst_i = res[i]
            assert np.array_equal(bseeds, seeds), i
            assert bfrac == frac
            for key in ("kpt_round", "kpt_last_round", "kpt_star", "kpt_prime", "kpt_plus",
                        "theta_prime", "covered_prime", "theta", "covered", "sets_total",
                        "members_select", "width_total"):
                assert bst_i[key] == st[key], (i, key, bst_i[key], st[key])
    finally:
        for e in engines:
            e.close()


def test_tagged_run_matches_oracle():
    g = inputs.rmat(12, seed=9)
    for model in (tim.TIM_IC, tim.TIM_LT):
        w = _weights(g, model)
        og = O.load_graph(g.n, g.rowptr, g.dst, w, model)
        with tim.Engine(0) as e:
            tim.tim_load_graph(e.ctx, g.n, g.rowptr, g.dst, w, model)
            tim.tim_set_query_tag(e.ctx, 4321)
            seeds, frac, st = tim.tim_run(e.ctx, 6, 0.5, 1.0, 3)
        ref = O.tim_plus(og, 6, 0.5, 1.0, 3, tag=4321)
        assert st["kpt_star"] == ref.kpt.kpt_star and st["theta"] == ref.theta
        assert np.array_equal(seeds, ref.seeds) and st["covered"] == ref.covered


def test_batch_rejects_bad_queries():
    g = inputs.rmat(8)
    with tim.Engine(0) as e:
        tim.tim_load_graph(e.ctx, g.n, g.rowptr, g.dst, _weights(g, tim.TIM_IC), tim.TIM_IC)
        with pytest.raises(tim.TimError):
            tim.tim_run_batch([{"ctx": e.ctx, "k": g.n + 1, "eps": 0.5}], seed=1)
        with pytest.raises(tim.TimError):  # the same context twice
            tim.tim_run_batch([{"ctx": e.ctx, "k": 2, "eps": 0.5, "tag": 1},
                               {"ctx": e.ctx, "k": 2, "eps": 0.5, "tag": 2}], seed=1)


def test_batch_long_lt_chains_with_wide_teams():
    # LT chains longer than the shared-memory queue reach pass 2; a team of several warps
    # must give the same sets (and widths) as one warp
    graphs = [inputs.chain(3000), inputs.rmat(12, seed=3), inputs.cycle(2000)]
    models = [tim.TIM_LT, tim.TIM_IC, tim.TIM_LT]
    engines = [tim.Engine(0) for _ in graphs]
    try:
        queries = []
        for i, (g, model, e) in enumerate(zip(graphs, models, engines)):
            w = _weights(g, model)
            tim.tim_load_graph(e.ctx, g.n, g.rowptr, g.dst, w, model)
            queries.append({"ctx": e.ctx, "k": 3, "eps": 0.5, "ell": 1.0, "tag": 7 + i})
        for team in (8, 2):
            tim.tim_set_team_size(engines[0].ctx, team)
            res, _ = tim.tim_run_batch(queries, seed=11)
            for i, (g, model) in enumerate(zip(graphs, models)):
                og = O.load_graph(g.n, g.rowptr, g.dst, _weights(g, model), model)
                ref = O.tim_plus(og, 3, 0.5, 1.0, 11, tag=7 + i)
                seeds, _, st = res[i]
                assert st["kpt_star"] == ref.kpt.kpt_star, (team, i)
                assert st["theta"] == ref.theta and np.array_equal(seeds, ref.seeds), (team, i)
    finally:
        for e in engines:
            e.close()
