"""Pins for the CPU oracle of the start-round predictor: the analytic gradient equals
central finite differences of the loss, bfloat16 rounding and GELU match their
definitions, Adam's first step has its closed form, the graph features of small hand
graphs are counted by hand, and the start-round mapping inverts the stop test."""
import math

import numpy as np
from scipy import integrate

from oracle import mlp as M
from paper_1404_0900_gb300 import inputs


def test_bf16_round_is_nearest_even():
    vals = np.array([1.0, 1.00390625, 1.005859375, 1.0078125, -3.14159, 65504.0, 1e-30,
                     0.1, 0.333333], dtype=np.float32)
    got = M.bf16_round(vals)
    for v, g in zip(vals, got):
        # the two bfloat16 neighbours: low 16 bits cleared, or cleared plus one ulp
        u = int(np.float32(v).view(np.uint32))
        lo = np.uint32(u & 0xFFFF0000).view(np.float32)
        hi = np.uint32((u & 0xFFFF0000) + 0x10000).view(np.float32)
        dlo, dhi = abs(float(v) - float(lo)), abs(float(v) - float(hi))
        want = lo if dlo < dhi else hi if dhi < dlo else (lo if ((u >> 16) & 1) == 0 else hi)
        assert g == want, (v, g, want)
    # exact ties: 1 + 2^-8 lies halfway between 1 and 1 + 2^-7 -> even (1.0)
    assert M.bf16_round(np.float32(1.0 + 2 ** -8)) == np.float32(1.0)
    assert M.bf16_round(np.float32(1.0 + 3 * 2 ** -8)) == np.float32(1.0 + 2 ** -6)


def test_gelu_is_t_times_normal_cdf():
    for t in (-3.0, -0.7, 0.0, 0.4, 2.5):
        cdf = integrate.quad(lambda s: math.exp(-s * s / 2) / math.sqrt(2 * math.pi), -40, t)[0]
        assert abs(M.gelu(np.float64(t)) - t * cdf) < 1e-10
        eps = 1e-6
        num = (M.gelu(np.float64(t + eps)) - M.gelu(np.float64(t - eps))) / (2 * eps)
        assert abs(M.gelu_grad(np.float64(t)) - num) < 1e-7


def _case(d=12, B=37, seed=3):
    rng = np.random.default_rng(seed)
    # weights already representable in bfloat16, so rounding is the identity
    p = M.bf16_round(rng.normal(0, 0.3, size=M.param_count(d)).astype(np.float32))
    x = rng.normal(2.0, 3.0, size=(B, d))
    y = rng.normal(1.0, 2.0, size=B)
    sc = M.Scaling(d, in_mu=rng.normal(size=d), in_isd=rng.uniform(0.2, 2.0, size=d),
                   out_mu=0.7, out_sd=1.9)
    return p, x, y, sc


def test_gradient_matches_finite_differences():
    d = 12
    p, x, y, sc = _case(d)
    loss, g = M.loss_and_grads(p, x, y, d, sc)
    pf = p.astype(np.float64)
    assert abs(loss - M.loss_unrounded(pf, x, y, d, sc)) < 1e-12
    rng = np.random.default_rng(5)
    # every bias and output weight, plus a sample of the hidden weights
    h = M.HIDDEN
    nW1, nW2 = h * d, h * h
    fixed = list(range(nW1, nW1 + h)) + list(range(nW1 + h + nW2, pf.size))
    idx = fixed + list(rng.choice(nW1, 40, replace=False)) + \
        list(nW1 + h + rng.choice(nW2, 60, replace=False))
    for i in idx:
        e = np.zeros_like(pf)
        e[i] = 1e-6
        num = (M.loss_unrounded(pf + e, x, y, d, sc) - M.loss_unrounded(pf - e, x, y, d, sc)) / 2e-6
        assert abs(num - g[i]) <= 2e-7 + 1e-5 * abs(num), (i, num, g[i])


def test_zero_network_loss_is_half_mean_square():
    d = 5
    p = np.zeros(M.param_count(d), dtype=np.float32)
    x = np.random.default_rng(1).normal(size=(10, d))
    y = np.arange(10, dtype=np.float64)
    sc = M.Scaling(d, out_mu=2.0, out_sd=4.0)
    loss, g = M.loss_and_grads(p, x, y, d, sc)
    assert abs(loss - 0.5 * np.mean(((y - 2.0) / 4.0) ** 2)) < 1e-12
    # only b3 sees a gradient when every weight is zero: d loss / d b3 = mean(z - yn)
    assert abs(g[-1] - np.mean(-(y - 2.0) / 4.0)) < 1e-12
    assert np.all(g[:-1] == 0)
    assert np.allclose(M.predict(p, x, d, sc), 2.0)


def test_adam_first_step_is_lr_times_sign():
    g = np.array([3.0, -0.5, 1e-3, -7.0])
    p0 = np.zeros(4)
    p1, m, v = M.adam_step(p0, np.zeros(4), np.zeros(4), g, 1, 0.01)
    assert np.allclose(p1, -0.01 * np.sign(g), rtol=1e-4)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)
    # constant gradient: every step moves by lr (bias-corrected moments equal g, g^2)
    p, m, v = p0, np.zeros(4), np.zeros(4)
    for t in range(1, 6):
        q, m, v = M.adam_step(p, m, v, g, t, 0.01)
        assert np.allclose(q - p, -0.01 * np.sign(g), rtol=1e-4)
        p = q


def test_graph_features_by_hand():
    # 0 -> 2, 1 -> 2, 2 -> 3, 0 -> 3 with IC weights 0.5, 0.25, 1.0, 0.125
    g = inputs.from_edges(4, [(0, 2), (1, 2), (2, 3), (0, 3)])
    # out-CSR order: (0,2), (0,3), (1,2), (2,3)
    w = np.array([0.5, 0.125, 0.25, 1.0])
    f = M.graph_features(4, g.rowptr, g.dst, w)
    indeg = np.array([0, 0, 2, 2.0])
    outdeg = np.array([2, 1, 1, 0.0])
    insum = np.array([0, 0, 0.75, 1.125])
    hop2 = np.array([0, 0, 0 + 0, 2 + 0.0])  # in(3) = {2 (indeg 2), 0 (indeg 0)}
    want = []
    for a in (np.log1p(indeg), np.log1p(outdeg), insum, np.log1p(hop2)):
        want += [a.mean(), a.max()]
    assert np.allclose(f, want, rtol=0, atol=1e-15)
    # star into node 0: the hub has indeg n-1, every leaf outdeg 1
    s = inputs.star_in(9)
    fs = M.graph_features(9, s.rowptr, s.dst, inputs.weighted_cascade(s))
    assert abs(fs[0] - math.log(9) / 9) < 1e-15 and abs(fs[1] - math.log(9)) < 1e-15
    assert abs(fs[2] - 8 * math.log(2) / 9) < 1e-15 and abs(fs[3] - math.log(2)) < 1e-15
    assert abs(fs[4] - 1 / 9) < 1e-7 and abs(fs[5] - 1.0) < 1e-7
    assert fs[6] == 0 and fs[7] == 0  # every in-neighbour of the hub has indeg 0


def test_start_round_inverts_the_stop_test():
    # if KPT* sits strictly inside (n 2^-i / 2, n 2^-(i-1) / 2], round i is the first to pass
    n, m, k, rounds = 1 << 20, 16 << 20, 50, 19
    for i in range(1, rounds + 1):
        for frac in (0.51, 0.75, 0.99):
            kpt = n * 2.0 ** -i * (1 + frac)  # in (n 2^-i, 2 n 2^-i) = (lo, hi) of round i
            kpt /= 2
            assert n * 2.0 ** -i / 2 < kpt < n * 2.0 ** -(i - 1) / 2
            t = M.start_round_target(n, m, k, kpt)
            assert M.start_round(t, n, m, k, rounds) == i
    assert M.start_round(-100.0, n, m, k, rounds) == 1
    assert M.start_round(100.0, n, m, k, rounds) == rounds
