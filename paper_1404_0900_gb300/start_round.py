"""The trained start-round network of Algorithm 2: file format and loading.

The file (JSON) holds the flat fp32 parameter vector in the layout of tim_mlp
(W1[64][12] b1[64] W2[64][64] b2[64] W3[1][64] b3[1]), the input standardisation
(in_mu, in_isd), the output scale (out_mu, out_sd), and a record of how it was trained.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np

from . import tim as T

DEFAULT_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "start_round_mlp.json")


def init_params(d: int, seed: int, hidden: int = T.TIM_MLP_HIDDEN) -> np.ndarray:
    """Seeded initial parameters: weights uniform in +-1/sqrt(fan_in), zero biases."""
    rng = np.random.Generator(np.random.Philox(seed))
    parts = []
    for fan_out, fan_in in ((hidden, d), (hidden, hidden), (1, hidden)):
        lim = 1.0 / math.sqrt(fan_in)
        parts.append(rng.uniform(-lim, lim, size=fan_out * fan_in))
        parts.append(np.zeros(fan_out))
    return np.concatenate(parts).astype(np.float32)


def save(path: str, params, in_mu, in_isd, out_mu: float, out_sd: float, record: dict):
    doc = {"d_in": int(len(in_mu)), "hidden": T.TIM_MLP_HIDDEN,
           "params": [float(v) for v in np.asarray(params, dtype=np.float32)],
           "in_mu": [float(v) for v in in_mu], "in_isd": [float(v) for v in in_isd],
           "out_mu": float(out_mu), "out_sd": float(out_sd), "record": record}
    with open(path, "w") as f:
        json.dump(doc, f)


def available(path: str = DEFAULT_PATH) -> bool:
    return os.path.exists(path)


def load(ctx, path: str = DEFAULT_PATH):
    """Create a tim_mlp on ctx's device holding the trained network; returns
    (handle, record). Free the handle with tim.tim_mlp_destroy."""
    with open(path) as f:
        doc = json.load(f)
    d = int(doc["d_in"])
    if d != T.TIM_START_FEATURES or int(doc.get("hidden", T.TIM_MLP_HIDDEN)) != T.TIM_MLP_HIDDEN:
        raise ValueError(f"{path}: not a start-round network")
    mlp = T.tim_mlp_create(ctx, d)
    try:
        T.tim_mlp_set_params(ctx, mlp, np.asarray(doc["params"], dtype=np.float32))
        T.tim_mlp_set_scaling(ctx, mlp, doc["in_mu"], doc["in_isd"], doc["out_mu"], doc["out_sd"])
    except Exception:
        T.tim_mlp_destroy(mlp)
        raise
    return mlp, doc.get("record", {})
