"""CPU oracle of the KptEstimation start-round predictor (test infrastructure: only the
tests, the smoke check and the CPU baseline of the benchmark import it).

The method (Algorithm 2) tries rounds i = 1, 2, ... until the mean of kappa over c_i
RR sets exceeds 2^-i. The predictor guesses the stopping round from graph features so
that the sweep can start there; this module states, in plain fp64 NumPy, everything the
GPU computes for it:

graph features (per node v of G, then pooled over all nodes as mean and max)
    log(1 + indeg v), log(1 + outdeg v), sum of p(u, v) over the in-edges of v
    (the total LT in-weight under LT), log(1 + sum of indeg u over the in-edges (u, v))
query features
    ln n, ln max(m, 1), ln k, model (0 = IC, 1 = LT)

network (three layers, GELU after the first two, one output)
    xn = (x - in_mu) * in_isd
    h1 = gelu(W1 xn + b1),  h2 = gelu(W2 h1 + b2),  z = W3 h2 + b3
    prediction = out_mu + out_sd * z
with gelu(t) = t * Phi(t) (Phi the standard normal CDF, through erf). The weight
matrices take part in bfloat16: each W is rounded to the nearest bfloat16 (ties to
even) before use; biases, activations and sums stay in higher precision.

loss (regression of a target y given in prediction units)
    yn = (y - out_mu) / out_sd,   loss = (1 / 2B) * sum_b (z_b - yn_b)^2
and its gradient with respect to the flat parameter vector, taken with respect to
the rounded weight values.

Adam (Kingma and Ba, ICLR 2015, Algorithm 1) with bias correction updates the fp32
master parameters.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

HIDDEN = 64


def bf16_round(x) -> np.ndarray:
    """float32 -> nearest bfloat16 (ties to even), returned as float32 values."""
    a = np.ascontiguousarray(x, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).reshape(a.shape)


def gelu(t):
    return 0.5 * t * (1.0 + erf(t / math.sqrt(2.0)))


def gelu_grad(t):
    return 0.5 * (1.0 + erf(t / math.sqrt(2.0))) + t * np.exp(-0.5 * t * t) / math.sqrt(2 * math.pi)


def param_count(d: int, h: int = HIDDEN, r: int = 1) -> int:
    return h * d + h + h * h + h + r * h + r


def unpack(params: np.ndarray, d: int, h: int = HIDDEN, r: int = 1):
    """Flat parameter vector -> W1[h,d], b1[h], W2[h,h], b2[h], W3[r,h], b3[r]."""
    sizes = [(h, d), (h,), (h, h), (h,), (r, h), (r,)]
    out, o = [], 0
    for s in sizes:
        k = int(np.prod(s))
        out.append(params[o:o + k].reshape(s))
        o += k
    assert o == params.size
    return out


class Scaling:
    """Input standardisation and output scale of the network."""

    def __init__(self, d, in_mu=None, in_isd=None, out_mu=0.0, out_sd=1.0):
        self.in_mu = np.zeros(d) if in_mu is None else np.asarray(in_mu, dtype=np.float64)
        self.in_isd = np.ones(d) if in_isd is None else np.asarray(in_isd, dtype=np.float64)
        self.out_mu = float(out_mu)
        self.out_sd = float(out_sd)


def _layers(params, d, h, r):
    W1, b1, W2, b2, W3, b3 = unpack(np.asarray(params, dtype=np.float32), d, h, r)
    W1, W2, W3 = (bf16_round(w).astype(np.float64) for w in (W1, W2, W3))
    return W1, b1.astype(np.float64), W2, b2.astype(np.float64), W3, b3.astype(np.float64)


def forward(params, x, d, sc: Scaling | None = None, h: int = HIDDEN, r: int = 1):
    """Raw network output z[B, r] and the intermediate values."""
    sc = sc or Scaling(d)
    W1, b1, W2, b2, W3, b3 = _layers(params, d, h, r)
    xn = (np.asarray(x, dtype=np.float64) - sc.in_mu) * sc.in_isd
    a1 = xn @ W1.T + b1
    h1 = gelu(a1)
    a2 = h1 @ W2.T + b2
    h2 = gelu(a2)
    z = h2 @ W3.T + b3
    return z, (xn, a1, h1, a2, h2, W1, W2, W3)


def predict(params, x, d, sc: Scaling | None = None):
    sc = sc or Scaling(d)
    z, _ = forward(params, x, d, sc)
    return sc.out_mu + sc.out_sd * z[:, 0]


def loss_and_grads(params, x, y, d, sc: Scaling | None = None, h: int = HIDDEN, r: int = 1):
    """Loss (1/2B) sum (z - yn)^2 and its gradient w.r.t. the flat parameters."""
    sc = sc or Scaling(d)
    z, (xn, a1, h1, a2, h2, W1, W2, W3) = forward(params, x, d, sc, h, r)
    B = xn.shape[0]
    yn = (np.asarray(y, dtype=np.float64).reshape(B, r) - sc.out_mu) / sc.out_sd
    diff = z - yn
    loss = float(0.5 * np.sum(diff * diff) / B)
    dz = diff / B
    gW3 = dz.T @ h2
    gb3 = dz.sum(axis=0)
    da2 = (dz @ W3) * gelu_grad(a2)
    gW2 = da2.T @ h1
    gb2 = da2.sum(axis=0)
    da1 = (da2 @ W2) * gelu_grad(a1)
    gW1 = da1.T @ xn
    gb1 = da1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return loss, g


def loss_unrounded(weights_f64, x, y, d, sc: Scaling | None = None, h: int = HIDDEN, r: int = 1):
    """The loss as a function of weights used as given (no bfloat16 rounding): the
    function whose finite differences pin loss_and_grads."""
    sc = sc or Scaling(d)
    W1, b1, W2, b2, W3, b3 = unpack(np.asarray(weights_f64, dtype=np.float64), d, h, r)
    xn = (np.asarray(x, dtype=np.float64) - sc.in_mu) * sc.in_isd
    z = gelu(gelu(xn @ W1.T + b1) @ W2.T + b2) @ W3.T + b3
    B = xn.shape[0]
    yn = (np.asarray(y, dtype=np.float64).reshape(B, r) - sc.out_mu) / sc.out_sd
    return float(0.5 * np.sum((z - yn) ** 2) / B)


ADAM_B1, ADAM_B2, ADAM_EPS = 0.9, 0.999, 1e-8


def adam_step(params, m, v, g, t, lr):
    """One Adam update (step t >= 1) of fp64 copies; returns (params, m, v)."""
    m = ADAM_B1 * m + (1 - ADAM_B1) * g
    v = ADAM_B2 * v + (1 - ADAM_B2) * g * g
    mhat = m / (1 - ADAM_B1 ** t)
    vhat = v / (1 - ADAM_B2 ** t)
    return params - lr * mhat / (np.sqrt(vhat) + ADAM_EPS), m, v


def init_params(d: int, seed: int, h: int = HIDDEN, r: int = 1) -> np.ndarray:
    """Seeded fp32 initial parameters (uniform +-1/sqrt(fan_in), zero biases)."""
    rng = np.random.Generator(np.random.Philox(seed))
    parts = []
    for fan_out, fan_in in ((h, d), (h, h), (r, h)):
        lim = 1.0 / math.sqrt(fan_in)
        parts.append(rng.uniform(-lim, lim, size=fan_out * fan_in))
        parts.append(np.zeros(fan_out))
    return np.concatenate(parts).astype(np.float32)


# ------------------------------------------------------------------ graph features

def graph_features(n, rowptr, dst, weight):
    """The 8 pooled graph features (mean and max over nodes of the four per-node
    features, in the order indeg, outdeg, in-weight sum, 2-hop in-degree) of the
    out-CSR graph (rowptr, dst) with per-edge weights."""
    rowptr = np.asarray(rowptr, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    w = np.asarray(weight, dtype=np.float64)
    outdeg = np.diff(rowptr).astype(np.float64)
    src = np.repeat(np.arange(n), np.diff(rowptr))
    indeg = np.bincount(dst, minlength=n).astype(np.float64)
    insum = np.bincount(dst, weights=w, minlength=n)
    hop2 = np.bincount(dst, weights=indeg[src], minlength=n)
    per = [np.log1p(indeg), np.log1p(outdeg), insum, np.log1p(hop2)]
    out = []
    for f in per:
        out += [float(np.mean(f)), float(np.max(f))]
    return np.array(out)


def query_features(gfeat, n, m, k, model):
    return np.concatenate([gfeat, [math.log(n), math.log(max(m, 1)), math.log(k), float(model)]])


def start_round_target(n, m, k, kpt_star):
    """Regression target of the predictor: log2(n / (2 KPT*)) - log2(max(m,1) / k).
    The first round i whose test passes satisfies i - 1 <= log2(n / (2 KPT*)) < i when
    the estimates of consecutive rounds agree, and KPT* grows about like n k / m times
    the mean RR-set width, so the difference stays bounded across graph sizes."""
    return math.log2(n / (2.0 * kpt_star)) - math.log2(max(m, 1) / k)


def start_round(pred, n, m, k, rounds):
    """Start round i0 from a prediction of start_round_target: floor(t) + 1, clamped
    to the rounds of Algorithm 2."""
    t = pred + math.log2(max(m, 1) / k)
    return int(min(max(math.floor(t) + 1, 1), max(rounds, 1)))
