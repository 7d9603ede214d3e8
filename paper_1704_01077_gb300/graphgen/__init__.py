"""Seeded synthetic graphs for tests and benchmarks.

This module generates inputs only; it computes no distances, reach counts or
bounds, and it is shared by the CUDA path's tests and by the CPU oracle's tests.

Large generators (Barabasi-Albert, R-MAT, Erdos-Renyi) are plain C in
``graphgen.c`` (built by :func:`build`); small closed-form families are numpy.

Every graph is returned as ``Graph(n, offsets, cols, directed)`` with uint32
CSR arrays, rows sorted, no self-loops or duplicate arcs; undirected graphs hold
both arc directions.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB = os.path.join(_HERE, "libgraphgen.so")

# Base seed of the synthetic workloads; each workload derives its own sub-seed
# as splitmix64(BASE_SEED ^ workload_index).
BASE_SEED = 1704010770


@dataclass
class Graph:
    n: int
    offsets: np.ndarray  # uint32[n+1]
    cols: np.ndarray  # uint32[arcs]
    directed: bool
    name: str = ""

    @property
    def arcs(self) -> int:
        return int(self.offsets[-1]) if self.n > 0 else 0

    def outdeg(self) -> np.ndarray:
        return np.diff(self.offsets.astype(np.int64))


def build(force: bool = False) -> str:
    """Compile libgraphgen.so next to its source (gcc, OpenMP)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        u32p = ctypes.POINTER(ctypes.c_uint32)
        pp = ctypes.POINTER(u32p)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        lib.gg_barabasi_albert.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64, pp, pp, u64p]
        lib.gg_rmat.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_double, ctypes.c_double,
                                ctypes.c_double, ctypes.c_uint64, ctypes.c_int, ctypes.c_int, pp, pp, u64p]
        lib.gg_erdos_renyi.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int,
                                       pp, pp, u64p]
        lib.gg_from_arcs.argtypes = [ctypes.c_uint32, ctypes.c_uint64, u32p, u32p, ctypes.c_int, pp, pp, u64p]
        lib.gg_splitmix64.argtypes = [ctypes.c_uint64]
        lib.gg_splitmix64.restype = ctypes.c_uint64
        lib.gg_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        lib.gg_uniform.restype = ctypes.c_double
        lib.gg_free.argtypes = [ctypes.c_void_p]
        _lib = lib
    return _lib


def _take(n, call, *args) -> tuple[np.ndarray, np.ndarray]:
    lib = _load()
    off_p = ctypes.POINTER(ctypes.c_uint32)()
    col_p = ctypes.POINTER(ctypes.c_uint32)()
    m = ctypes.c_uint64(0)
    rc = call(*args, ctypes.byref(off_p), ctypes.byref(col_p), ctypes.byref(m))
    if rc != 0:
        raise RuntimeError(f"graph generator failed with code {rc}")
    try:
        off = np.ctypeslib.as_array(off_p, shape=(n + 1,)).copy()
        cols = np.ctypeslib.as_array(col_p, shape=(max(int(m.value), 1),))[: int(m.value)].copy()
    finally:
        lib.gg_free(off_p)
        lib.gg_free(col_p)
    return off, cols


def splitmix64(x: int) -> int:
    return int(_load().gg_splitmix64(ctypes.c_uint64(x & 0xFFFFFFFFFFFFFFFF)))


def workload_seed(index: int) -> int:
    return splitmix64(BASE_SEED ^ index)


def barabasi_albert(n: int, m: int, seed: int) -> Graph:
    off, cols = _take(n, _load().gg_barabasi_albert, n, m, seed)
    return Graph(n, off, cols, False, f"ba_n{n}_m{m}")


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 1, permute: bool = True, directed: bool = True) -> Graph:
    n = 1 << scale
    off, cols = _take(n, _load().gg_rmat, scale, edge_factor, a, b, c, seed, int(permute),
                      0 if directed else 1)
    return Graph(n, off, cols, directed, f"rmat{scale}_ef{edge_factor}")


def erdos_renyi(n: int, narcs: int, seed: int, directed: bool = True) -> Graph:
    off, cols = _take(n, _load().gg_erdos_renyi, n, narcs, seed, 0 if directed else 1)
    return Graph(n, off, cols, directed, f"er_n{n}_a{narcs}")


def from_arcs(n: int, src, dst, directed: bool, name: str = "") -> Graph:
    src = np.ascontiguousarray(np.asarray(src, dtype=np.uint32))
    dst = np.ascontiguousarray(np.asarray(dst, dtype=np.uint32))
    if n == 0:
        return Graph(0, np.zeros(1, np.uint32), np.zeros(0, np.uint32), directed, name)
    u32p = ctypes.POINTER(ctypes.c_uint32)
    off, cols = _take(n, _load().gg_from_arcs, n, len(src),
                      src.ctypes.data_as(u32p) if len(src) else u32p(),
                      dst.ctypes.data_as(u32p) if len(dst) else u32p(), 0 if directed else 1)
    return Graph(n, off, cols, directed, name)


# --------------------------------------------------------------------------
# Small families with closed-form distance sums (used as oracle pins)
# --------------------------------------------------------------------------

def path(n: int, directed: bool = False) -> Graph:
    i = np.arange(max(n - 1, 0))
    return from_arcs(n, i, i + 1, directed, f"path{n}")


def cycle(n: int, directed: bool = False) -> Graph:
    i = np.arange(n)
    return from_arcs(n, i, (i + 1) % n, directed, f"cycle{n}")


def star(n: int) -> Graph:
    i = np.arange(1, n)
    return from_arcs(n, np.zeros_like(i), i, False, f"star{n}")


def complete(n: int, directed: bool = False) -> Graph:
    a, b = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    mask = a != b
    return from_arcs(n, a[mask], b[mask], directed, f"K{n}")


def complete_bipartite(p: int, q: int) -> Graph:
    a, b = np.meshgrid(np.arange(p), np.arange(p, p + q), indexing="ij")
    return from_arcs(p + q, a.ravel(), b.ravel(), False, f"K{p},{q}")


def hypercube(d: int) -> Graph:
    n = 1 << d
    src, dst = [], []
    for v in range(n):
        for j in range(d):
            w = v ^ (1 << j)
            if v < w:
                src.append(v)
                dst.append(w)
    return from_arcs(n, src, dst, False, f"Q{d}")


def grid(rows: int, cols: int, directed: bool = False, seed: int | None = None, drop: float = 0.0) -> Graph:
    """rows x cols 4-neighbour grid, a street-network stand-in.  With a seed,
    each undirected edge is dropped with probability `drop`; directed grids
    keep each direction of an edge independently with probability 1 - drop
    (one-way streets)."""
    v = np.arange(rows * cols).reshape(rows, cols)
    a = np.concatenate([v[:, :-1].ravel(), v[:-1, :].ravel()])
    b = np.concatenate([v[:, 1:].ravel(), v[1:, :].ravel()])
    if directed:
        src, dst = np.concatenate([a, b]), np.concatenate([b, a])
        if seed is not None and drop > 0:
            keep = np.random.default_rng(seed).random(src.size) >= drop
            src, dst = src[keep], dst[keep]
        return from_arcs(rows * cols, src, dst, True, f"grid{rows}x{cols}d")
    if seed is not None and drop > 0:
        keep = np.random.default_rng(seed).random(a.size) >= drop
        a, b = a[keep], b[keep]
    return from_arcs(rows * cols, a, b, False, f"grid{rows}x{cols}")


def disjoint_union(*gs: Graph) -> Graph:
    src, dst, base = [], [], 0
    directed = any(g.directed for g in gs)
    for g in gs:
        deg = g.outdeg()
        s = np.repeat(np.arange(g.n), deg) + base
        src.append(s)
        dst.append(g.cols.astype(np.int64) + base)
        base += g.n
    s = np.concatenate(src) if src else np.zeros(0)
    d = np.concatenate(dst) if dst else np.zeros(0)
    # arcs are already both-direction for undirected parts; keep them as given
    return from_arcs(base, s, d, True, "union") if directed else _as_undirected_union(base, s, d)


def _as_undirected_union(n, s, d) -> Graph:
    g = from_arcs(n, s, d, True, "union")
    g.directed = False
    return g


def random_tree(n: int, seed: int) -> Graph:
    """Random recursive tree: vertex v>0 attaches to a uniform earlier vertex."""
    if n <= 1:
        return from_arcs(n, [], [], False, f"tree{n}")
    rng = np.random.default_rng(seed)
    v = np.arange(1, n)
    parent = (rng.random(n - 1) * v).astype(np.int64)
    return from_arcs(n, v, parent, False, f"tree{n}")


def random_graph(n: int, p: float, seed: int, directed: bool) -> Graph:
    """G(n, p): each ordered (directed) or unordered pair is an arc/edge with
    probability p, from one seeded numpy stream."""
    rng = np.random.default_rng(seed)
    mask = rng.random((n, n)) < p
    np.fill_diagonal(mask, False)
    if not directed:
        mask = np.triu(mask, 1)
    a, b = np.nonzero(mask)
    return from_arcs(n, a, b, directed, f"gnp{n}")


def reduction_graph(X: int, sets: list[set[int]], p: int = 7, q: int = 36) -> tuple[Graph, dict]:
    """Directed graph of the hardness reduction (Section 3): layers Z, Y, C_0,
    X_1, X_2, C_1..C_p.  Returns the graph and a dict of vertex-id ranges."""
    nc = len(sets)
    ids = {}
    cur = 0

    def alloc(name, size):
        nonlocal cur
        ids[name] = (cur, cur + size)
        cur += size

    alloc("Z", q * nc)
    alloc("Y", q)
    alloc("C0", nc)
    alloc("X1", X)
    alloc("X2", X)
    for i in range(1, p + 1):
        alloc(f"C{i}", nc)
    src, dst = [], []
    z0, y0, c0 = ids["Z"][0], ids["Y"][0], ids["C0"][0]
    x1, x2 = ids["X1"][0], ids["X2"][0]
    for j in range(q):  # each Y vertex owns |C| distinct Z vertices
        for t in range(nc):
            src.append(y0 + j)
            dst.append(z0 + j * nc + t)
    for ci in range(nc):  # C_0 vertices link to every Y vertex
        for j in range(q):
            src.append(c0 + ci)
            dst.append(y0 + j)
    for ci, cset in enumerate(sets):
        for x in range(X):
            if x in cset:
                src.append(c0 + ci)
                dst.append(x1 + x)
                src.append(x1 + x)
                dst.append(ids["C1"][0] + ci)
            else:
                src.append(c0 + ci)
                dst.append(x2 + x)
    for i in range(1, p):
        for ci in range(nc):
            src.append(ids[f"C{i}"][0] + ci)
            dst.append(ids[f"C{i + 1}"][0] + ci)
    return from_arcs(cur, src, dst, True, "reduction"), ids


def log_uniform_sizes(count: int, lo: float, hi: float, seed: int) -> list[int]:
    """n_i = floor(exp(U(ln lo, ln hi))) from one seeded uniform per graph."""
    lib = _load()
    return [int(math.floor(math.exp(math.log(lo) + lib.gg_uniform(seed, i) * (math.log(hi) - math.log(lo)))))
            for i in range(count)]
