"""CPU oracle for exact top-k closeness (arXiv 1704.01077) -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg
may import this module.  It wraps ``oracle.c`` (plain C, built with gcc) through
ctypes and shares nothing with the CUDA library.

Functions and what pins them (see ``tests/test_oracle.py``):
  bfs_sums        textbook BFS per source        Floyd-Warshall, closed forms, networkx
  floyd_warshall  all pairs on <= 64 vertices    exhaustive small graphs vs BFS
  topk            exact (S, r) ordering          Fraction-based brute force
  farness         IEEE doubles from integers     Python float arithmetic on the same ops
  degree_order    computeBoundsDeg               numpy lexsort
  scc             Tarjan                         mutual reachability by brute force
  alpha_omega     Algorithm 6                    alpha <= r <= omega, exact hand-built DAGs
  tree_sums       Algorithm 2                    BFS on random trees
  cut_bounds      Sec. 6 lemma / level           invariants: <= S, non-decreasing, ends at S
  bfscut          Algorithm 1 + Algorithm 4      textbook top-k on thousands of graphs
  bfscut_batched  the same, B searches per step  equals bfscut at B = 1 (all counters), textbook
                                                 top-k at every B, hand-counted star at B = 2
  nb_bounds       Algorithm 3, Eq. 3, Eq. 6      brute-force walk counts, exact on trees and
                                                 cycles, hand-computed hypercube, <= S/(r-1)^2,
                                                 minimum over every r in [alpha, omega]
  lb_level_bounds Section 7, Eq. 4, Eq. 5         <= S on the reach class, per-vertex form of the
                                                 equation, the Section 7 difference lemma
  bfsbound        Algorithm 1 + Algorithm 5      textbook top-k, DegBound and NBBound
  harmonic_*      Section 9 (harmonic centrality) exact rationals from Floyd-Warshall within
                                                 the rounding bound, networkx, closed forms;
                                                 BFSCut/NBCut equal to the textbook top-k
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                           "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


class Counters(ctypes.Structure):
    _fields_ = [("edges_visited", ctypes.c_uint64), ("bfs_started", ctypes.c_uint64),
                ("bfs_cut", ctypes.c_uint64), ("bfs_finished", ctypes.c_uint64)]


class BCounters(ctypes.Structure):
    _fields_ = [("edges_visited", ctypes.c_uint64), ("bfs_started", ctypes.c_uint64),
                ("bfs_cut", ctypes.c_uint64), ("bfs_finished", ctypes.c_uint64), ("levels", ctypes.c_uint64)]


_lib = None
_u32p = ctypes.POINTER(ctypes.c_uint32)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_dp = ctypes.POINTER(ctypes.c_double)


def _bind(lib):
    """Declares the C signatures on a loaded oracle library."""
    lib.orc_bfs_sums.argtypes = [ctypes.c_uint32, _u32p, _u32p, ctypes.c_uint32, _u32p, _u64p, _u32p,
                                 ctypes.c_int]
    lib.orc_floyd_warshall.argtypes = [ctypes.c_uint32, _u32p, _u32p, _u64p, _u32p]
    lib.orc_topk.argtypes = [ctypes.c_uint32, _u64p, _u32p, ctypes.c_uint32, _u32p, _u32p]
    lib.orc_cmp_farness.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint32]
    lib.orc_farness.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint32, _dp, _dp]
    lib.orc_farness.restype = None
    lib.orc_degree_order.argtypes = [ctypes.c_uint32, _u32p, _u32p]
    lib.orc_scc.argtypes = [ctypes.c_uint32, _u32p, _u32p, _u32p]
    lib.orc_scc.restype = ctypes.c_int64
    lib.orc_alpha_omega.argtypes = [ctypes.c_uint32, _u32p, _u32p, ctypes.c_int, _u32p, _u32p]
    lib.orc_cut_min.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64,
                                ctypes.c_uint64, ctypes.c_uint64, _u64p, _u64p]
    lib.orc_cut_min.restype = None
    lib.orc_tree_sums.argtypes = [ctypes.c_uint32, _u32p, _u32p, _u64p]
    lib.orc_cut_bounds.argtypes = [ctypes.c_uint32, _u32p, _u32p, ctypes.c_int, ctypes.c_uint32, _u64p,
                                   ctypes.c_int]
    lib.orc_bfscut.argtypes = [ctypes.c_uint32, _u32p, _u32p, ctypes.c_int, ctypes.c_uint32, _u32p, _u32p,
                               _u64p, _u32p, _u32p, ctypes.POINTER(Counters), _u64p, _u32p, ctypes.c_uint32,
                               _u64p]
    lib.orc_bfscut_batched.argtypes = [ctypes.c_uint32, _u32p, _u32p, ctypes.c_int, ctypes.c_uint32, _u32p,
                                       ctypes.c_uint32, _u64p, ctypes.c_uint32, _u32p, _u64p, _u32p, _u32p,
                                       ctypes.POINTER(BCounters), _u64p, _u32p]
    lib.orc_nb_bounds.argtypes = [ctypes.c_uint32, _u32p, _u32p, ctypes.c_int, _u32p, _u32p, ctypes.c_uint32,
                                  _u64p, _u32p, _u64p, _u64p, ctypes.c_uint32, _dp]
    lib.orc_harmonic_sums.argtypes = [ctypes.c_uint32, _u32p, _u32p, ctypes.c_uint32, _u32p, _dp, _u32p,
                                      ctypes.c_int]
    lib.orc_harmonic_topk.argtypes = [ctypes.c_uint32, _dp, ctypes.c_uint32, _u32p, _u32p]
    lib.orc_bfscut_harmonic.argtypes = [ctypes.c_uint32, _u32p, _u32p, ctypes.c_int, ctypes.c_uint32, _u32p, _dp,
                                        _u32p, _dp, _u32p, _u32p, ctypes.POINTER(Counters), _dp, _u32p,
                                        ctypes.c_uint32]
    lib.orc_lb_level_bounds.argtypes = [ctypes.c_uint32, _u32p, _u32p, ctypes.c_int, ctypes.c_uint32, _u32p, _u64p]
    lib.orc_bfsbound.argtypes = [ctypes.c_uint32, _u32p, _u32p, ctypes.c_int, ctypes.c_uint32, _u32p, _u64p, _u32p,
                                 _u32p, _u64p, _u32p, _u32p, ctypes.POINTER(Counters), ctypes.c_uint32]
    lib.orc_harmonic_cut_bounds.argtypes = [ctypes.c_uint32, _u32p, _u32p, ctypes.c_int, ctypes.c_uint32,
                                            ctypes.c_uint32, _dp, ctypes.c_int]
    return lib


def _load():
    global _lib
    if _lib is None:
        _lib = _bind(ctypes.CDLL(build()))
    return _lib


def _p(a, t):
    if a is None:
        return ctypes.cast(None, t)
    return a.ctypes.data_as(t)


def _csr(g):
    off = np.ascontiguousarray(g.offsets, dtype=np.uint32)
    col = np.ascontiguousarray(g.cols, dtype=np.uint32)
    if col.size == 0:
        col = np.zeros(1, np.uint32)
    return off, col


def _full_order(g, order):
    """A caller's source order as the C side reads it: exactly n vertex ids."""
    if order is None:
        return None
    a = np.ascontiguousarray(order, dtype=np.uint32)
    if a.shape != (g.n,):
        raise ValueError(f"order must list all {g.n} vertices (got {a.size}); see nb_full_order")
    return a


def _per_vertex(g, x, dtype):
    if x is None:
        return None
    a = np.ascontiguousarray(x, dtype=dtype)
    if a.shape != (g.n,):
        raise ValueError(f"expected one value per vertex ({g.n}), got {a.size}")
    return a


def _check(rc):
    if rc < 0:
        raise RuntimeError(f"oracle call failed with code {rc}")
    return rc


def bfs_sums(g, sources=None, threads: int = 0):
    """Textbook BFS: (S, r) for each source (all vertices by default)."""
    off, col = _csr(g)
    srcs = None if sources is None else np.ascontiguousarray(sources, dtype=np.uint32)
    cnt = g.n if srcs is None else len(srcs)
    S = np.zeros(max(cnt, 1), np.uint64)
    r = np.zeros(max(cnt, 1), np.uint32)
    _check(_load().orc_bfs_sums(g.n, _p(off, _u32p), _p(col, _u32p), cnt, _p(srcs, _u32p),
                                _p(S, _u64p), _p(r, _u32p), threads))
    return S[:cnt], r[:cnt]


def floyd_warshall(g):
    off, col = _csr(g)
    S = np.zeros(max(g.n, 1), np.uint64)
    r = np.zeros(max(g.n, 1), np.uint32)
    _check(_load().orc_floyd_warshall(g.n, _p(off, _u32p), _p(col, _u32p), _p(S, _u64p), _p(r, _u32p)))
    return S[: g.n], r[: g.n]


def topk(S, r, k):
    """Exact top-k ids by farness then id, and the count of vertices tied with the k-th."""
    n = len(S)
    S = np.ascontiguousarray(S, dtype=np.uint64)
    r = np.ascontiguousarray(r, dtype=np.uint32)
    ids = np.zeros(max(min(k, n), 1), np.uint32)
    tied = ctypes.c_uint32(0)
    cnt = _check(_load().orc_topk(n, _p(S, _u64p), _p(r, _u32p), k, _p(ids, _u32p), ctypes.byref(tied)))
    return ids[:cnt], int(tied.value)


def cmp_farness(Sa, ra, Sb, rb) -> int:
    return int(_load().orc_cmp_farness(Sa, ra, Sb, rb))


def farness(n, S, r):
    f = ctypes.c_double()
    c = ctypes.c_double()
    _load().orc_farness(n, int(S), int(r), ctypes.byref(f), ctypes.byref(c))
    return f.value, c.value


def degree_order(g):
    off, _ = _csr(g)
    order = np.zeros(max(g.n, 1), np.uint32)
    _check(_load().orc_degree_order(g.n, _p(off, _u32p), _p(order, _u32p)))
    return order[: g.n]


def scc(g):
    off, col = _csr(g)
    comp = np.zeros(max(g.n, 1), np.uint32)
    nc = _check(_load().orc_scc(g.n, _p(off, _u32p), _p(col, _u32p), _p(comp, _u32p)))
    return comp[: g.n], int(nc)


def alpha_omega(g):
    off, col = _csr(g)
    a = np.zeros(max(g.n, 1), np.uint32)
    o = np.zeros(max(g.n, 1), np.uint32)
    _check(_load().orc_alpha_omega(g.n, _p(off, _u32p), _p(col, _u32p), int(g.directed), _p(a, _u32p),
                                   _p(o, _u32p)))
    return a[: g.n], o[: g.n]


def tree_sums(g):
    off, col = _csr(g)
    S = np.zeros(max(g.n, 1), np.uint64)
    _check(_load().orc_tree_sums(g.n, _p(off, _u32p), _p(col, _u32p), _p(S, _u64p)))
    return S[: g.n]


def cut_bounds(g, v, maxlev=256):
    off, col = _csr(g)
    L = np.zeros(maxlev, np.uint64)
    cnt = _check(_load().orc_cut_bounds(g.n, _p(off, _u32p), _p(col, _u32p), int(g.directed), v,
                                        _p(L, _u64p), maxlev))
    return L[:cnt]


def cut_min(Sd, d, nd, g, lo, hi):
    """(L, r): the r in [max(lo, nd), hi] minimising the Section 6 lemma's farness bound."""
    L = ctypes.c_uint64()
    r = ctypes.c_uint64()
    _load().orc_cut_min(Sd, d, nd, g, lo, hi, ctypes.byref(L), ctypes.byref(r))
    return int(L.value), int(r.value)


@dataclass
class TopK:
    ids: np.ndarray
    S: np.ndarray
    r: np.ndarray
    n_tied: int
    counters: Counters | None = None
    all_S: np.ndarray | None = None
    all_r: np.ndarray | None = None


def bfscut(g, k, order=None, want_all=False, max_sources=0, lb_key=None) -> TopK:
    """Algorithm 1 + BFSCut, one source at a time, in degree order (or `order`).
    max_sources > 0 examines only that prefix of the order (for timing samples).
    lb_key (with `order` sorted by it): NBCut's stop at the first source whose
    neighbourhood bound exceeds the k-th farness."""
    off, col = _csr(g)
    kk = min(k, g.n)
    ids = np.zeros(max(kk, 1), np.uint32)
    S = np.zeros(max(kk, 1), np.uint64)
    r = np.zeros(max(kk, 1), np.uint32)
    tied = ctypes.c_uint32(0)
    ctr = Counters()
    order_a = _full_order(g, order)
    allS = np.zeros(max(g.n, 1), np.uint64) if want_all else None
    allr = np.zeros(max(g.n, 1), np.uint32) if want_all else None
    key_a = _per_vertex(g, lb_key, np.uint64)
    cnt = _check(_load().orc_bfscut(g.n, _p(off, _u32p), _p(col, _u32p), int(g.directed), k,
                                    _p(order_a, _u32p), _p(ids, _u32p), _p(S, _u64p), _p(r, _u32p),
                                    ctypes.byref(tied), ctypes.byref(ctr), _p(allS, _u64p), _p(allr, _u32p),
                                    max_sources, _p(key_a, _u64p)))
    return TopK(ids[:cnt], S[:cnt], r[:cnt], int(tied.value), ctr,
                None if allS is None else allS[: g.n], None if allr is None else allr[: g.n])


def bfscut_batched(g, k, B, order=None, lb_key=None, nocut_prefix=0, want_all=False) -> TopK:
    """Algorithm 1 + BFSCut with B searches advancing one level per step and
    the threshold refreshed between steps (the batched schedule; B = 1 is
    `bfscut`).  Counters are BCounters (with `levels`, the number of steps)."""
    off, col = _csr(g)
    kk = min(k, g.n)
    ids = np.zeros(max(kk, 1), np.uint32)
    S = np.zeros(max(kk, 1), np.uint64)
    r = np.zeros(max(kk, 1), np.uint32)
    tied = ctypes.c_uint32(0)
    ctr = BCounters()
    order_a = _full_order(g, order)
    key_a = _per_vertex(g, lb_key, np.uint64)
    allS = np.zeros(max(g.n, 1), np.uint64) if want_all else None
    allr = np.zeros(max(g.n, 1), np.uint32) if want_all else None
    cnt = _check(_load().orc_bfscut_batched(g.n, _p(off, _u32p), _p(col, _u32p), int(g.directed), k,
                                            _p(order_a, _u32p), B, _p(key_a, _u64p), nocut_prefix, _p(ids, _u32p),
                                            _p(S, _u64p), _p(r, _u32p), ctypes.byref(tied), ctypes.byref(ctr),
                                            _p(allS, _u64p), _p(allr, _u32p)))
    return TopK(ids[:cnt], S[:cnt], r[:cnt], int(tied.value), ctr,
                None if allS is None else allS[: g.n], None if allr is None else allr[: g.n])


def textbook_topk(g, k, threads: int = 0) -> TopK:
    """Textbook algorithm: BFS from every vertex, then the exact top-k."""
    S, r = bfs_sums(g, threads=threads)
    ids, tied = topk(S, r, k)
    return TopK(ids, S[ids], r[ids], tied)


NB_FRAC = 46          # fixed-point bits of the neighbourhood-bound order key
NB_DEFAULT_LEVELS = 256


@dataclass
class NBBounds:
    S: np.ndarray       # S~ at the minimising candidate reach
    r: np.ndarray       # that reach (1: out-degree 0, closeness 0)
    key: np.ndarray     # floor(S * 2^46 / (r-1)^2); UINT64_MAX when r = 1
    levels: int         # sweeps run
    counts: np.ndarray | None = None  # counts[k][v] = N~_k(v)
    h_ub: np.ndarray | None = None    # harmonic-centrality upper bound


def nb_bounds(g, max_levels=NB_DEFAULT_LEVELS, counts_levels=0, alpha=None, omega=None) -> NBBounds:
    """computeBoundsNB (Algorithm 3; Eq. 3 for directed graphs; Eq. 6 with the
    Algorithm 6 reach bounds).  alpha/omega default to this oracle's own."""
    off, col = _csr(g)
    if alpha is None or omega is None:
        alpha, omega = alpha_omega(g)
    a = np.ascontiguousarray(alpha, dtype=np.uint32)
    o = np.ascontiguousarray(omega, dtype=np.uint32)
    n1 = max(g.n, 1)
    S = np.zeros(n1, np.uint64)
    r = np.zeros(n1, np.uint32)
    key = np.zeros(n1, np.uint64)
    counts = np.zeros((max(counts_levels, 1), n1), np.uint64) if counts_levels else None
    hub = np.zeros(n1, np.float64)
    lev = _check(_load().orc_nb_bounds(g.n, _p(off, _u32p), _p(col, _u32p), int(g.directed), _p(a, _u32p),
                                       _p(o, _u32p), max_levels, _p(S, _u64p), _p(r, _u32p), _p(key, _u64p),
                                       _p(counts, _u64p), counts_levels, _p(hub, _dp)))
    return NBBounds(S[: g.n], r[: g.n], key[: g.n], int(lev),
                    None if counts is None else counts[:, : g.n], hub[: g.n])


def nb_order(g, key):
    """Sources of out-degree >= 1 by increasing key, ties by increasing id
    (computeBoundsNB's queue Q)."""
    deg = np.diff(np.asarray(g.offsets, dtype=np.int64))
    ids = np.nonzero(deg > 0)[0].astype(np.uint32)
    key = np.asarray(key, dtype=np.uint64)[ids]
    return ids[np.lexsort((ids, key))]


def nb_full_order(g, key):
    """nb_order followed by the vertices of out-degree 0 (never searched): a
    permutation of all n vertices, as bfscut's `order` must be."""
    return np.concatenate([nb_order(g, key), np.nonzero(g.outdeg() == 0)[0].astype(np.uint32)])


# ---------------------------------------------------------------- harmonic centrality

def harmonic_sums(g, sources=None, threads: int = 0):
    """Textbook h(v) = sum over w != v of 1/d(v,w) (per-level FP64 sums) and r(v)."""
    off, col = _csr(g)
    srcs = None if sources is None else np.ascontiguousarray(sources, dtype=np.uint32)
    cnt = g.n if srcs is None else len(srcs)
    H = np.zeros(max(cnt, 1), np.float64)
    r = np.zeros(max(cnt, 1), np.uint32)
    _check(_load().orc_harmonic_sums(g.n, _p(off, _u32p), _p(col, _u32p), cnt, _p(srcs, _u32p), _p(H, _dp),
                                     _p(r, _u32p), threads))
    return H[:cnt], r[:cnt]


def harmonic_topk(H, k):
    n = len(H)
    H = np.ascontiguousarray(H, dtype=np.float64)
    ids = np.zeros(max(min(k, n), 1), np.uint32)
    tied = ctypes.c_uint32(0)
    cnt = _check(_load().orc_harmonic_topk(n, _p(H, _dp), k, _p(ids, _u32p), ctypes.byref(tied)))
    return ids[:cnt], int(tied.value)


@dataclass
class HarmonicTopK:
    ids: np.ndarray
    H: np.ndarray
    r: np.ndarray
    n_tied: int
    counters: Counters | None = None
    all_H: np.ndarray | None = None
    all_r: np.ndarray | None = None


def textbook_harmonic_topk(g, k, threads: int = 0) -> HarmonicTopK:
    H, r = harmonic_sums(g, threads=threads)
    ids, tied = harmonic_topk(H, k)
    return HarmonicTopK(ids, H[ids], r[ids], tied)


def bfscut_harmonic(g, k, order=None, ub=None, want_all=False, max_sources=0) -> HarmonicTopK:
    """Algorithm 1 + BFSCut for harmonic centrality (degree order or `order`);
    ub with `order` sorted by decreasing ub gives the NBCut stop."""
    off, col = _csr(g)
    kk = min(k, g.n)
    ids = np.zeros(max(kk, 1), np.uint32)
    H = np.zeros(max(kk, 1), np.float64)
    r = np.zeros(max(kk, 1), np.uint32)
    tied = ctypes.c_uint32(0)
    ctr = Counters()
    order_a = _full_order(g, order)
    ub_a = None if ub is None else np.ascontiguousarray(ub, dtype=np.float64)
    allH = np.zeros(max(g.n, 1), np.float64) if want_all else None
    allr = np.zeros(max(g.n, 1), np.uint32) if want_all else None
    cnt = _check(_load().orc_bfscut_harmonic(g.n, _p(off, _u32p), _p(col, _u32p), int(g.directed), k,
                                             _p(order_a, _u32p), _p(ub_a, _dp), _p(ids, _u32p), _p(H, _dp),
                                             _p(r, _u32p), ctypes.byref(tied), ctypes.byref(ctr), _p(allH, _dp),
                                             _p(allr, _u32p), max_sources))
    return HarmonicTopK(ids[:cnt], H[:cnt], r[:cnt], int(tied.value), ctr,
                        None if allH is None else allH[: g.n], None if allr is None else allr[: g.n])


H_MARGIN = 1.0 + 2.0 ** -20   # a search is abandoned only when bound * H_MARGIN < x


def harmonic_cut_bounds(g, v, omega_v, maxlev=256):
    """U_0, U_1, ...: BFSCut's upper bounds on h(v) after each level, at reach omega_v."""
    off, col = _csr(g)
    U = np.zeros(maxlev, np.float64)
    cnt = _check(_load().orc_harmonic_cut_bounds(g.n, _p(off, _u32p), _p(col, _u32p), int(g.directed), v,
                                                 omega_v, _p(U, _dp), maxlev))
    return U[:cnt]


def nb_harmonic_order(g, h_ub):
    """Sources of out-degree >= 1 by decreasing harmonic upper bound, ties by id."""
    deg = np.diff(np.asarray(g.offsets, dtype=np.int64))
    ids = np.nonzero(deg > 0)[0].astype(np.uint32)
    h = np.asarray(h_ub, dtype=np.float64)[ids]
    return ids[np.lexsort((ids, -h))]


# ---------------------------------------------------------------- updateBoundsLB (DegBound / NBBound)

def lb_level_bounds(g, s):
    """BFS from s: (level per vertex, UINT32_MAX if unreachable; level bound L(i) per level)."""
    off, col = _csr(g)
    level = np.zeros(max(g.n, 1), np.uint32)
    L = np.zeros(max(g.n, 1) + 1, np.uint64)
    nl = _check(_load().orc_lb_level_bounds(g.n, _p(off, _u32p), _p(col, _u32p), int(g.directed), s,
                                            _p(level, _u32p), _p(L, _u64p)))
    return level[: g.n], L[:nl]


def bfsbound(g, k, order=None, nb=None, max_sources=0) -> TopK:
    """Algorithm 1 with updateBoundsLB: DegBound (nb None, degree order unless
    `order`) or NBBound (nb = nb_bounds(g), order = its NB order)."""
    off, col = _csr(g)
    kk = min(k, g.n)
    ids = np.zeros(max(kk, 1), np.uint32)
    S = np.zeros(max(kk, 1), np.uint64)
    r = np.zeros(max(kk, 1), np.uint32)
    tied = ctypes.c_uint32(0)
    ctr = Counters()
    order_a = _full_order(g, order)
    iS = None if nb is None else np.ascontiguousarray(nb.S, dtype=np.uint64)
    ir = None if nb is None else np.ascontiguousarray(nb.r, dtype=np.uint32)
    cnt = _check(_load().orc_bfsbound(g.n, _p(off, _u32p), _p(col, _u32p), int(g.directed), k, _p(order_a, _u32p),
                                      _p(iS, _u64p), _p(ir, _u32p), _p(ids, _u32p), _p(S, _u64p), _p(r, _u32p),
                                      ctypes.byref(tied), ctypes.byref(ctr), max_sources))
    return TopK(ids[:cnt], S[:cnt], r[:cnt], int(tied.value), ctr)
