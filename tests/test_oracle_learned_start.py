"""Pins for the oracle's Algorithm 2 from a predicted start round: with the plain
sweep's own stopping round as the prediction it is accepted and returns the plain
result; a prediction one round late or early is rejected (the round before it passes,
or it fails) and the plain result comes back; and an accepted prediction is exactly
one whose two rounds bracket the stop test, checked against the round sums."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1404_0900_gb300 import inputs


def _graph(scale, seed, model):
    g = inputs.rmat(scale, seed=seed)
    w = inputs.weighted_cascade(g) if model == 0 else inputs.lt_inverse_indegree(g)
    return O.load_graph(g.n, g.rowptr, g.dst, w, model)


def _round_passes(og, k, seed, i, tag=0):
    c = O.c_i(og.n, 1.0, i)
    s, _ = O.kappa_sum(og, k, seed, O.make_sid(O.PHASE_KPT, i, tag << 32), c)
    return s > (c << (63 - i))


@pytest.mark.parametrize("model", [0, 1])
def test_start_rounds_around_the_plain_stop(model):
    og = _graph(10, 3, model)
    k, seed = 5, 11
    plain = O.kpt_estimation(og, k, 1.0, seed)
    assert plain.stop_round >= 2
    i_star = plain.stop_round
    res, acc = O.kpt_estimation_from(og, k, 1.0, seed, i_star)
    assert acc and res.stop_round == i_star and res.kpt_star == plain.kpt_star
    assert res.last_sum == plain.last_sum and res.last_c == plain.last_c
    for i0 in (i_star - 1, i_star + 1):
        res, acc = O.kpt_estimation_from(og, k, 1.0, seed, i0)
        assert not acc
        assert res.stop_round == plain.stop_round and res.kpt_star == plain.kpt_star


def test_acceptance_is_the_bracketing_condition():
    og = _graph(9, 5, 0)
    rounds = O.kpt_rounds(og.n)
    for k in (1, 8):
        passes = [None] + [_round_passes(og, k, 2, i) for i in range(1, rounds + 1)]
        for i0 in range(1, rounds + 1):
            _, acc = O.kpt_estimation_from(og, k, 1.0, 2, i0)
            want = passes[i0] and (i0 == 1 or not passes[i0 - 1])
            assert acc == want, (k, i0)


def test_out_of_range_predictions():
    og = _graph(8, 1, 0)
    plain = O.kpt_estimation(og, 3, 1.0, 4)
    res, acc = O.kpt_estimation_from(og, 3, 1.0, 4, 0)
    assert not acc and res.kpt_star == plain.kpt_star
    # beyond the last round: clamped to it
    r = O.kpt_rounds(og.n)
    a, acc_a = O.kpt_estimation_from(og, 3, 1.0, 4, 10 * r)
    b, acc_b = O.kpt_estimation_from(og, 3, 1.0, 4, r)
    assert acc_a == acc_b and a.kpt_star == b.kpt_star and a.stop_round == b.stop_round
