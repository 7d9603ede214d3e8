"""Trains the source-order model on farness computed by the library itself.

Training set: R-MAT graphs (scale 14 by default, edge factor 16, the R-MAT
parameters of the benchmark, seeds derived from the base seed), the exact
farness of every vertex with out-degree >= 1 from tkc_distance_sums (full
BFS on the GPU), standardized log-farness per graph as the target, and the
library's standardized vertex features as the input.  Training runs the
library's own forward/backward/Adam kernels (tkc_mlp_train_step); this
script only moves arrays.  Writes the fp32 master weights (TKC_MLP_PARAMS
little-endian floats) and a JSON note next to them.

    python -m paper_1704_01077_gb300.train_order --graphs 200 --scale 14
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

from . import graphgen as gg
from . import tkc

HERE = os.path.dirname(os.path.abspath(__file__))
WEIGHTS = os.path.join(HERE, "weights", "source_order_mlp.f32")


def training_set(ctx, graphs: int, scale: int, seed_offset: int = 1000):
    import torch

    xs, ts = [], []
    for i in range(graphs):
        g = gg.rmat(scale, 16, seed=gg.splitmix64(gg.BASE_SEED + seed_offset + i))
        h = tkc.tkc_load_csr(ctx, g.n, g.offsets, g.cols, g.directed)
        try:
            x = tkc.tkc_vertex_features(h, g.n)
            src = np.flatnonzero(g.outdeg() > 0).astype(np.uint32)
            S, r = tkc.tkc_distance_sums(h, src)
        finally:
            tkc.tkc_free_graph(h)
        keep = r >= 2
        src, S, r = src[keep], S[keep].astype(np.float64), r[keep].astype(np.float64)
        logf = np.log((g.n - 1) * S / (r - 1) ** 2)
        z = (logf - logf.mean()) / max(logf.std(), 1e-9)
        xs.append(x[torch.from_numpy(src.astype(np.int64)).cuda()])
        ts.append(torch.from_numpy(z.astype(np.float32)).cuda())
    return torch.cat(xs).contiguous(), torch.cat(ts).contiguous()


def train(ctx, X, T, epochs: int, batch: int, lr: float, seed: int):
    import torch

    gen = torch.Generator(device="cpu").manual_seed(seed)
    tkc.tkc_mlp_init(ctx, seed)
    history = []
    m = X.shape[0]
    for ep in range(epochs):
        perm = torch.randperm(m, generator=gen).cuda()
        Xp, Tp = X[perm].contiguous(), T[perm].contiguous()
        losses = []
        for i in range(0, m - batch + 1, batch):
            losses.append(tkc.tkc_mlp_train_step(ctx, Xp[i:i + batch], Tp[i:i + batch], lr))
        history.append(float(np.mean(losses)))
    return history


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--graphs", type=int, default=200)
    ap.add_argument("--scale", type=int, default=14)
    ap.add_argument("--epochs", type=int, default=12)
    ap.add_argument("--batch", type=int, default=2048)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--seed", type=int, default=1704)
    ap.add_argument("--out", default=WEIGHTS)
    a = ap.parse_args(argv)
    ctx = tkc.tkc_create(tkc.Options())
    t0 = time.time()
    X, T = training_set(ctx, a.graphs, a.scale)
    t1 = time.time()
    hist = train(ctx, X, T, a.epochs, a.batch, a.lr, a.seed)
    t2 = time.time()
    w = tkc.tkc_get_source_model(ctx)
    tkc.tkc_destroy(ctx)
    os.makedirs(os.path.dirname(a.out), exist_ok=True)
    w.astype("<f4").tofile(a.out)
    note = {"graphs": a.graphs, "scale": a.scale, "edge_factor": 16, "samples": int(X.shape[0]),
            "epochs": a.epochs, "batch": a.batch, "lr": a.lr, "seed": a.seed, "loss_per_epoch": hist,
            "seconds_data": round(t1 - t0, 1), "seconds_train": round(t2 - t1, 1),
            "target": "per-graph standardized log farness", "params": int(w.size)}
    with open(os.path.splitext(a.out)[0] + ".json", "w") as f:
        json.dump(note, f, indent=1)
    print(json.dumps(note))


def load_weights(path: str = WEIGHTS) -> np.ndarray | None:
    if not os.path.exists(path):
        return None
    w = np.fromfile(path, dtype="<f4")
    return w if w.size == tkc.TKC_MLP_PARAMS else None


if __name__ == "__main__":
    main()
