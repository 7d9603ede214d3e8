"""CPU oracle of the learned order's vertex features -- TEST INFRASTRUCTURE.

Plain numpy/Python, float64: log1p of out-degree, in-degree, the 2-walk count
(sum of out-degrees of out-neighbours), an h-index core estimate (4 steps from
the degree over out- and, if directed, in-neighbours: the largest h such that
at least h neighbours have a value >= h), and the SCC size (oracle.scc); each
standardized to mean 0 and variance 1 over the graph."""
from __future__ import annotations

import numpy as np

import oracle


def _h_index(vals):
    s = np.sort(np.asarray(vals))[::-1]
    h = 0
    for i, v in enumerate(s):
        if v >= i + 1:
            h = i + 1
        else:
            break
    return h


def raw_features(g):
    n = g.n
    off = g.offsets.astype(np.int64)
    col = g.cols.astype(np.int64)
    outd = np.diff(off)
    ind = np.bincount(col, minlength=n) if n else np.zeros(0, np.int64)
    w2 = np.array([outd[col[off[v]:off[v + 1]]].sum() for v in range(n)], dtype=np.float64)
    rows_out = [col[off[v]:off[v + 1]] for v in range(n)]
    rows_in = [[] for _ in range(n)]
    if g.directed:
        for v in range(n):
            for w in rows_out[v]:
                rows_in[w].append(v)
    c = outd + (ind if g.directed else 0)
    for _ in range(4):
        c = np.array([min(_h_index(np.concatenate([c[rows_out[v]], c[np.array(rows_in[v], np.int64)]])), c[v])
                      for v in range(n)], dtype=np.int64)
    comp, nc = oracle.scc(g)
    size = np.bincount(comp, minlength=nc)[comp]
    return np.stack([np.log1p(outd), np.log1p(ind), np.log1p(w2), np.log1p(c), np.log1p(size)], axis=1)


def features(g):
    x = raw_features(g)
    m = x.mean(axis=0)
    sd = np.sqrt(np.maximum(x.var(axis=0), 1e-12))
    return (x - m) / sd
