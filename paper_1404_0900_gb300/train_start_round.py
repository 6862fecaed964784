"""Train the start-round network of Algorithm 2 on graphs the method labels itself.

    python -m paper_1404_0900_gb300.train_start_round --graphs 2000 --out start_round_mlp.json

Training set: seeded synthetic graphs drawn on the GPU, scales 12..18 -- R-MAT with
varied (a, b, c) and edge factor, and directed Chung-Lu power-law graphs with varied
exponent and mean degree -- each under IC (weighted cascade or trivalency) or LT
(1/indeg or random normalised weights), with two values of k each. Every (graph, k) is
labelled by the plain KptEstimation (Algorithm 2, l = 1) of this library: the target is
log2(n / (2 KPT*)) - log2(m / k). Features come from tim_graph_features; the network is
trained by full-batch Adam in the library's own forward/backward kernels
(tim_mlp_train). A tenth of the graphs is held out to report the error and how often
the predicted start round equals the plain stopping round.
"""
from __future__ import annotations

import argparse
import math
import time

import numpy as np

from . import inputs, start_round, tim as T


def graph_spec(i: int, base_seed: int) -> dict:
    r = np.random.Generator(np.random.Philox(base_seed + i))
    spec = {"index": i, "scale": int(r.integers(12, 19))}
    if r.random() < 0.6:
        a = float(r.uniform(0.45, 0.65))
        b = float(r.uniform(0.08, min(0.25, (0.95 - a) / 2)))
        spec.update(family="rmat", a=a, b=b, c=b, edge_factor=int(r.choice([4, 8, 16, 32])))
    else:
        spec.update(family="chung_lu", gamma=float(r.uniform(2.0, 3.0)),
                    mean_degree=int(r.choice([4, 8, 16, 32])))
    spec["model"] = int(r.random() < 0.5)
    if spec["model"] == T.TIM_IC:
        spec["weights"] = "wc" if r.random() < 0.7 else "trivalency"
    else:
        spec["weights"] = "inv_indeg" if r.random() < 0.7 else "random_normalised"
    k1 = 50 if r.random() < 0.3 else int(math.exp(r.uniform(0.0, math.log(50.0))))
    k2 = int(math.exp(r.uniform(0.0, math.log(50.0))))
    spec["ks"] = sorted({max(1, k1), max(1, k2)})
    spec["graph_seed"] = int(r.integers(1, 2**31))
    return spec


def make_graph(spec: dict, device="cuda"):
    s = spec["scale"]
    if spec["family"] == "rmat":
        g = inputs.rmat_device(s, spec["edge_factor"], spec["a"], spec["b"], spec["c"],
                               seed=spec["graph_seed"], device=device)
    else:
        n = 1 << s
        g = inputs.chung_lu_device(n, n * spec["mean_degree"], spec["gamma"],
                                   seed=spec["graph_seed"], device=device)
    w = spec["weights"]
    if w in ("wc", "inv_indeg"):
        wt = inputs.weighted_cascade_device(g)
    elif w == "trivalency":
        wt = inputs.trivalency_device(g, seed=spec["graph_seed"] + 1)
    else:
        wt = inputs.lt_random_normalised_device(g, seed=spec["graph_seed"] + 1)
    return g, wt


def build_dataset(n_graphs: int, base_seed: int, log=print):
    import torch
    stream = torch.cuda.current_stream()
    eng = T.Engine(0, stream)
    X, Y, rounds, meta = [], [], [], []
    t_gen = t_lab = 0.0
    try:
        for i in range(n_graphs):
            spec = graph_spec(i, base_seed)
            t0 = time.perf_counter()
            g, wt = make_graph(spec)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            T.tim_load_graph_device(eng.ctx, g.n, g.m, g.rowptr, g.dst, wt, spec["model"])
            f = T.tim_graph_features(eng.ctx)
            for k in spec["ks"]:
                if k > g.n:
                    continue
                kpt, rnd = T.tim_kpt_estimate(eng.ctx, k, 1.0, 1000 + i)
                x = np.concatenate([f, [math.log(g.n), math.log(max(g.m, 1)), math.log(k),
                                        float(spec["model"])]]).astype(np.float32)
                y = math.log2(g.n / (2.0 * kpt)) - math.log2(max(g.m, 1) / k)
                X.append(x)
                Y.append(y)
                rounds.append(rnd)
                meta.append((i, g.n, g.m, k))
            t_lab += time.perf_counter() - t1
            t_gen += t1 - t0
            del g, wt
            if (i + 1) % 200 == 0:
                log(f"  {i + 1}/{n_graphs} graphs  gen {t_gen:.1f}s  label {t_lab:.1f}s")
    finally:
        eng.close()
    return (np.array(X, dtype=np.float32), np.array(Y, dtype=np.float64),
            np.array(rounds), np.array(meta, dtype=np.int64), t_gen, t_lab)


def start_rounds(pred, meta):
    out = []
    for p, (_, n, m, k) in zip(pred, meta):
        rounds = max(int(math.floor(math.log2(n))) - 1, 1)
        t = float(p) + math.log2(max(m, 1) / k)
        out.append(min(max(math.floor(t) + 1, 1), rounds))
    return np.array(out)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--graphs", type=int, default=2000)
    ap.add_argument("--seed", type=int, default=14040900)
    ap.add_argument("--steps", type=int, default=6000)
    ap.add_argument("--lr", type=float, default=3e-3)
    ap.add_argument("--out", default=start_round.DEFAULT_PATH)
    a = ap.parse_args(argv)

    t0 = time.perf_counter()
    X, Y, R, meta, t_gen, t_lab = build_dataset(a.graphs, a.seed)
    gid = meta[:, 0]
    val = gid >= int(a.graphs * 0.9)
    tr = ~val
    mu = X[tr].mean(axis=0)
    sd = X[tr].std(axis=0)
    isd = np.where(sd > 1e-6, 1.0 / np.maximum(sd, 1e-6), 1.0).astype(np.float32)
    out_mu, out_sd = float(Y[tr].mean()), float(max(Y[tr].std(), 1e-3))

    eng = T.Engine(0)
    mlp = T.tim_mlp_create(eng.ctx, T.TIM_START_FEATURES)
    t1 = time.perf_counter()
    T.tim_mlp_set_params(eng.ctx, mlp, start_round.init_params(T.TIM_START_FEATURES, a.seed))
    T.tim_mlp_set_scaling(eng.ctx, mlp, mu, isd, out_mu, out_sd)
    first = a.steps * 2 // 3
    h1 = T.tim_mlp_train(eng.ctx, mlp, X[tr], Y[tr], first, a.lr)
    h2 = T.tim_mlp_train(eng.ctx, mlp, X[tr], Y[tr], a.steps - first, a.lr / 3)
    t_train = time.perf_counter() - t1
    params = T.tim_mlp_get_params(eng.ctx, mlp)

    def report(mask):
        p = T.tim_mlp_predict(eng.ctx, mlp, X[mask])
        err = p - Y[mask]
        i0 = start_rounds(p, meta[mask])
        stop = R[mask]
        return {"samples": int(mask.sum()), "rmse": float(np.sqrt(np.mean(err ** 2))),
                "round_match": float(np.mean(i0 == stop)),
                "round_within_1": float(np.mean(np.abs(i0 - stop) <= 1)),
                "mean_stop_round": float(np.mean(stop))}

    rec = {
        "graphs": a.graphs, "samples": int(len(Y)), "seed": a.seed, "steps": a.steps,
        "lr": a.lr, "loss_first": float(h1[0]) if len(h1) else None,
        "loss_last": float(h2[-1]) if len(h2) else None,
        "train": report(tr), "held_out": report(val),
        "seconds": {"generate": round(t_gen, 2), "label": round(t_lab, 2),
                    "train": round(t_train, 2), "total": round(time.perf_counter() - t0, 2)},
        "recipe": "R-MAT (60%; a in [0.45,0.65], b=c in [0.08,0.25], edge factor 4-32) and "
                  "Chung-Lu (40%; gamma in [2,3], mean degree 4-32), scales 12-18; IC "
                  "weighted cascade / trivalency, LT 1/indeg / random normalised; two k "
                  "in [1,50] per graph; labels from plain KptEstimation, l = 1",
    }
    start_round.save(a.out, params, mu, isd, out_mu, out_sd, rec)
    T.tim_mlp_destroy(mlp)
    eng.close()
    print({k: rec[k] for k in ("samples", "loss_first", "loss_last", "train", "held_out",
                               "seconds")})


if __name__ == "__main__":
    main()
