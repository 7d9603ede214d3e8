"""CPU oracle of the learned order's vertex features -- TEST INFRASTRUCTURE.

Plain numpy/Python, float64: log1p of out-degree, in-degree, the 2-walk count
(sum of out-degrees of out-neighbours), the core number of the graph with arc
directions dropped (core_numbers: peeling by increasing degree), and the SCC
size (oracle.scc); each standardized to mean 0 and variance 1 over the graph.

core_numbers is pinned against networkx.core_number (which takes in-degree +
out-degree and both neighbour lists for a directed graph, as here)."""
from __future__ import annotations

import numpy as np

import oracle


def core_numbers(g):
    """Core number of every vertex: the largest k such that the vertex lies in
    a subgraph whose vertices all keep degree >= k.  Degrees and neighbours
    are those of the graph with arc directions dropped: out-arcs, plus in-arcs
    when directed (a pair linked both ways counts twice).  Peeling: repeatedly
    remove a vertex of least remaining degree; its core number is the largest
    such least degree seen so far."""
    n = g.n
    off = g.offsets.astype(np.int64)
    col = g.cols.astype(np.int64)
    nbrs = [list(col[off[v]:off[v + 1]]) for v in range(n)]
    if g.directed:
        for v in range(n):
            for w in col[off[v]:off[v + 1]]:
                nbrs[w].append(v)
    deg = [len(x) for x in nbrs]
    core = [0] * n
    removed = [False] * n
    import heapq

    heap = [(deg[v], v) for v in range(n)]
    heapq.heapify(heap)
    k = 0
    while heap:
        d, v = heapq.heappop(heap)
        if removed[v] or d != deg[v]:
            continue
        removed[v] = True
        k = max(k, d)
        core[v] = k
        for w in nbrs[v]:
            if not removed[w]:
                deg[w] -= 1
                heapq.heappush(heap, (deg[w], w))
    return np.array(core, dtype=np.int64)


def raw_features(g):
    n = g.n
    off = g.offsets.astype(np.int64)
    col = g.cols.astype(np.int64)
    outd = np.diff(off)
    ind = np.bincount(col, minlength=n) if n else np.zeros(0, np.int64)
    w2 = np.array([outd[col[off[v]:off[v + 1]]].sum() for v in range(n)], dtype=np.float64)
    c = core_numbers(g)
    comp, nc = oracle.scc(g)
    size = np.bincount(comp, minlength=nc)[comp]
    return np.stack([np.log1p(outd), np.log1p(ind), np.log1p(w2), np.log1p(c), np.log1p(size)], axis=1)


def features(g):
    x = raw_features(g)
    m = x.mean(axis=0)
    sd = np.sqrt(np.maximum(x.var(axis=0), 1e-12))
    return (x - m) / sd
