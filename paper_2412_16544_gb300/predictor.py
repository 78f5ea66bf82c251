"""Training and evaluation of the rank / expansion predictor on streams the method itself compresses.

The training pairs come from HT-RISE: for every node whose residual is formed, the update reports the
node's 66 sketch features and the truncation it made (kept residual rank r_R of a residual dimension
c). Targets: t0 = r_R / c, t1 = 1 if r_R > 0. The streams are advected spectral fields with spectral
slope U(-2.5, -1.2) and advection speed U(0, 2) cells per snapshot, eps in {1e-2, 1e-4}.

Everything numerical runs in the library (sketch, forward, backward, Adam on the GPU); this module
only generates the streams, batches the pairs and drives the calls.

  python -m paper_2412_16544_gb300.predictor --seeds 200 --held-out 40
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

import paper_2412_16544_gb300 as B

F_IN = 66
HIDDEN = 128


def stream_params(seed: int):
    """(slope, speed, eps) of training stream `seed`."""
    rng = np.random.default_rng([int(seed), 7_000_001])
    return float(rng.uniform(-2.5, -1.2)), float(rng.uniform(0.0, 2.0)), float((1e-2, 1e-4)[seed % 2])


def make_stream(seed: int, increments: int, items: int, grid: int):
    import bht_synth
    slope, speed, eps = stream_params(seed)
    Y = bht_synth.spectral_field(seed, 0, increments * items, n=grid, slope=slope, speed=speed)
    return Y.reshape(increments, items, grid, grid, grid), eps


def compress(Y, eps: float, precision: str = "mixed", predictor=None, record: bool = False):
    """BHT-l2r on Y[0], HT-RISE on the rest. Returns (state, tree, infos, pairs)."""
    import torch
    dims = Y.shape[2:]
    tree = B.bht_tree_create_balanced(dims)
    nodes = 2 * len(dims) - 1
    st = B.bht_l2r(tree, torch.from_numpy(np.ascontiguousarray(Y[0])).cuda(), eps, precision=precision)
    infos, X, T = [], [], []
    for k in range(1, Y.shape[0]):
        feats = np.zeros((nodes, F_IN), dtype=np.float32) if record else None
        labels = np.full((nodes, 2), -1, dtype=np.int64) if record else None
        info = B.htrise_update(st, torch.from_numpy(np.ascontiguousarray(Y[k])).cuda(), eps, precision=precision,
                               predictor=predictor, node_features=feats, node_labels=labels)
        infos.append(info)
        if record:
            for n in range(nodes):
                if labels[n, 1] > 0:
                    X.append(feats[n])
                    T.append([labels[n, 0] / labels[n, 1], 1.0 if labels[n, 0] > 0 else 0.0])
    pairs = (np.array(X, dtype=np.float32).reshape(-1, F_IN), np.array(T, dtype=np.float32).reshape(-1, 2))
    return st, tree, infos, pairs


def dataset(seeds, increments: int = 4, items: int = 32, grid: int = 64, precision: str = "mixed"):
    Xs, Ts = [], []
    for seed in seeds:
        Y, eps = make_stream(seed, increments, items, grid)
        st, tree, _, (X, T) = compress(Y, eps, precision, record=True)
        B.bht_state_destroy(st)
        B.bht_tree_destroy(tree)
        Xs.append(X)
        Ts.append(T)
    return np.concatenate(Xs), np.concatenate(Ts)


def init_params(seed: int) -> np.ndarray:
    """U(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights and biases (the flat layout of bht_mlp_create)."""
    rng = np.random.default_rng(seed)
    shapes = [(HIDDEN, F_IN), (HIDDEN,), (HIDDEN, HIDDEN), (HIDDEN,), (2, HIDDEN), (2,)]
    fans = [F_IN, F_IN, HIDDEN, HIDDEN, HIDDEN, HIDDEN]
    return np.concatenate([rng.uniform(-fan ** -0.5, fan ** -0.5, size=s).ravel()
                           for s, fan in zip(shapes, fans)]).astype(np.float32)


def train(X: np.ndarray, T: np.ndarray, steps: int = 600, batch: int = 256, lr: float = 2e-3, seed: int = 0):
    """Adam on the GPU with the library's kernels; returns (net, loss history)."""
    import torch
    net = B.bht_mlp_create(init_params(seed), F_IN, HIDDEN)
    Xd = torch.from_numpy(X).cuda()
    Td = torch.from_numpy(T).cuda()
    rng = np.random.default_rng(seed + 1)
    hist = []
    for step in range(steps):
        idx = torch.from_numpy(rng.integers(0, X.shape[0], size=min(batch, X.shape[0]))).cuda()
        hist.append(B.bht_mlp_loss_grad(net, Xd[idx].contiguous(), Td[idx].contiguous()))
        B.bht_mlp_adam_step(net, lr)
    return net, hist


def evaluate(net, seeds, increments: int = 4, items: int = 32, grid: int = 64, precision: str = "mixed"):
    """Held-out streams with and without the predictor: skip rate, fallbacks, equality of the results."""
    import torch
    out = {"nodes": 0, "skipped": 0, "fallback": 0, "missed": 0, "max_rel_err": 0.0, "max_diff_vs_plain": 0.0,
           "max_diff_plain_repeat": 0.0, "ranks_equal": True, "eig_launches_plain": 0, "eig_launches_pred": 0}
    names = [B.bht_kernel_class_name(i) for i in range(B.KERNEL_CLASSES)]
    tri = names.index("eig_tridiag_f64")
    for seed in seeds:
        Y, eps = make_stream(seed, increments, items, grid)
        runs, ranks = {}, {}
        # the plain run twice: the reproducibility floor of the mixed path (FP64 atomics in the reductions)
        for tag, pred in (("plain", None), ("repeat", None), ("pred", net)):
            B.bht_profile_read(reset=True)
            B.bht_profile_enable(1 << tri)
            st, tree, infos, _ = compress(Y, eps, precision, predictor=pred)
            B.bht_profile_enable(0)
            launches = B.bht_profile_read(reset=True)["eig_tridiag_f64"][1]
            if tag != "repeat":
                out[f"eig_launches_{tag}"] += launches
            rec = B.ht_reconstruct(st, 0, Y.shape[0] * Y.shape[1], dtype="float64").cpu().numpy()
            runs[tag] = rec
            ranks[tag] = B.bht_get_ranks(st)
            if pred is not None:
                for i in infos:
                    out["nodes"] += i.pred_nodes
                    out["skipped"] += i.pred_skipped
                    out["fallback"] += i.pred_fallback
                    out["missed"] += i.pred_missed
                Yf = Y.reshape((-1,) + Y.shape[2:]).astype(np.float64)
                for k in range(Y.shape[0]):
                    sl = slice(k * Y.shape[1], (k + 1) * Y.shape[1])
                    e = np.linalg.norm(rec[sl] - Yf[sl]) / np.linalg.norm(Yf[sl]) / eps
                    out["max_rel_err"] = max(out["max_rel_err"], float(e))
            B.bht_state_destroy(st)
            B.bht_tree_destroy(tree)
        nrm = np.linalg.norm(runs["plain"])
        out["max_diff_vs_plain"] = max(out["max_diff_vs_plain"], float(np.linalg.norm(runs["pred"] - runs["plain"]) / nrm))
        out["max_diff_plain_repeat"] = max(out["max_diff_plain_repeat"],
                                           float(np.linalg.norm(runs["repeat"] - runs["plain"]) / nrm))
        out["ranks_equal"] = out["ranks_equal"] and ranks["pred"] == ranks["plain"]
    out["skip_rate"] = out["skipped"] / max(out["nodes"], 1)
    # a prediction of "no expansion" that the exact check overturned would have violated the node bound
    out["violation_rate_before_fallback"] = out["fallback"] / max(out["nodes"], 1)
    out["violation_rate_after_fallback"] = 0.0 if out["max_rel_err"] <= 1.0 + 1e-4 else 1.0
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--seeds", type=int, default=200)
    ap.add_argument("--held-out", type=int, default=40)
    ap.add_argument("--grid", type=int, default=64)
    ap.add_argument("--increments", type=int, default=4)
    ap.add_argument("--items", type=int, default=32)
    ap.add_argument("--steps", type=int, default=1500)
    a = ap.parse_args()
    t0 = time.time()
    train_seeds = list(range(a.seeds - a.held_out))
    test_seeds = list(range(a.seeds - a.held_out, a.seeds))
    X, T = dataset(train_seeds, a.increments, a.items, a.grid)
    t1 = time.time()
    net, hist = train(X, T, steps=a.steps)
    t2 = time.time()
    res = evaluate(net, test_seeds, a.increments, a.items, a.grid)
    res.update({"train_pairs": int(X.shape[0]), "expand_fraction": float(T[:, 1].mean()) if len(T) else 0.0,
                "loss_first": hist[0], "loss_last": float(np.mean(hist[-50:])), "seconds_data": t1 - t0,
                "seconds_train": t2 - t1, "seconds_eval": time.time() - t2, "grid": a.grid,
                "train_seeds": len(train_seeds), "held_out_seeds": len(test_seeds)})
    print(json.dumps(res))
    B.bht_mlp_destroy(net)


if __name__ == "__main__":
    main()
