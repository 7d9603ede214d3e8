"""Pins for the oracle's harmonic centrality (Section 9: h(v) = sum over w != v
of 1/d(v,w), the same method with f(d) = 1/d): textbook values against exact
rationals from Floyd-Warshall distances within the rounding bound, against
networkx and closed forms; the per-level FP64 definition against level counts
taken from Floyd-Warshall; BFSCut's bound sequence; the neighbourhood upper
bound; and BFSCut / NBCut top-k equal to the textbook top-k."""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1704_01077_gb300 import graphgen as gg

U = 2.0 ** -53


def _fw_dist(g):
    n = g.n
    INF = 1 << 30
    D = [[0 if i == j else INF for j in range(n)] for i in range(n)]
    off = np.asarray(g.offsets, dtype=np.int64)
    col = np.asarray(g.cols, dtype=np.int64)
    for u in range(n):
        for e in range(off[u], off[u + 1]):
            D[u][col[e]] = 1
    for m in range(n):
        Dm = D[m]
        for i in range(n):
            dim = D[i][m]
            if dim == INF:
                continue
            Di = D[i]
            for j in range(n):
                if dim + Dm[j] < Di[j]:
                    Di[j] = dim + Dm[j]
    return D, INF


def _exact_and_levels(g):
    D, INF = _fw_dist(g)
    out = []
    for i in range(g.n):
        ds = [d for j, d in enumerate(D[i]) if j != i and d < INF]
        exact = sum((Fraction(1, d) for d in ds), Fraction(0))
        levels = {}
        for d in ds:
            levels[d] = levels.get(d, 0) + 1
        out.append((exact, levels, max(ds, default=0)))
    return out


def test_textbook_within_rounding_of_exact_and_per_level_definition():
    for seed in range(200):
        n = 3 + seed % 14
        g = gg.random_graph(n, [0.1, 0.2, 0.35][seed % 3], 40_000 + seed, bool(seed % 2))
        H, r = oracle.harmonic_sums(g)
        for v, (exact, levels, ecc) in enumerate(_exact_and_levels(g)):
            assert r[v] == 1 + sum(levels.values())
            assert abs(Fraction(float(H[v])) - exact) <= exact * (ecc + 2) * U, (seed, v)
            # the FP64 definition: level counts over level, added in increasing level
            h = 0.0
            for d in sorted(levels):
                h = h + levels[d] / d
            assert H[v] == h, (seed, v)


def test_against_networkx():
    nx = pytest.importorskip("networkx")
    for seed in range(20):
        g = gg.random_graph(40, 0.08, 77 + seed, bool(seed % 2))
        G = nx.DiGraph() if g.directed else nx.Graph()
        G.add_nodes_from(range(g.n))
        off = np.asarray(g.offsets)
        for u in range(g.n):
            for w in g.cols[off[u]:off[u + 1]]:
                G.add_edge(u, int(w))
        # networkx sums distances towards each vertex; h(v) here uses d(v, w)
        ref = nx.harmonic_centrality(G.reverse() if g.directed else G)
        H, _ = oracle.harmonic_sums(g)
        for v in range(g.n):
            assert math.isclose(H[v], ref[v], rel_tol=1e-13, abs_tol=0.0), (seed, v)


def test_closed_forms():
    n = 11
    H, _ = oracle.harmonic_sums(gg.complete(n))
    assert set(H.tolist()) == {float(n - 1)}
    H, _ = oracle.harmonic_sums(gg.star(n))
    assert H[0] == n - 1 and set(H[1:].tolist()) == {1.0 + (n - 2) / 2}
    # path end: the harmonic number H_{n-1}; middle of an odd path: 2 H_{(n-1)/2}
    H, _ = oracle.harmonic_sums(gg.path(n))
    hn = sum(Fraction(1, d) for d in range(1, n))
    assert abs(Fraction(float(H[0])) - hn) <= hn * n * U
    hm = 2 * sum(Fraction(1, d) for d in range(1, (n - 1) // 2 + 1))
    assert abs(Fraction(float(H[(n - 1) // 2])) - hm) <= hm * n * U
    # hypercube Q_d: C(d, i) vertices at distance i
    for d in (3, 5):
        H, _ = oracle.harmonic_sums(gg.hypercube(d))
        want = sum(Fraction(math.comb(d, i), i) for i in range(1, d + 1))
        assert all(abs(Fraction(float(x)) - want) <= want * (d + 2) * U for x in H)
    # directed path: h(i) = H_{n-1-i}; last vertex 0
    H, _ = oracle.harmonic_sums(gg.path(6, directed=True))
    assert H[5] == 0.0 and H[4] == 1.0 and H[3] == 1.5


def test_topk_order_and_ties():
    rng = np.random.default_rng(5)
    for _ in range(200):
        n = int(rng.integers(1, 30))
        H = rng.integers(0, 6, n).astype(np.float64) / 2
        k = int(rng.integers(1, n + 2))
        ids, tied = oracle.harmonic_topk(H, k)
        want = sorted(range(n), key=lambda v: (-H[v], v))[: min(k, n)]
        assert list(ids) == want
        assert tied == int(np.sum(H == H[want[-1]]))


def test_cut_bounds_hold_and_tighten():
    for seed in range(60):
        n = 5 + seed % 20
        directed = bool(seed % 2)
        g = gg.random_graph(n, [0.1, 0.2, 0.3][seed % 3], 51_000 + seed, directed)
        H, r = oracle.harmonic_sums(g)
        _, omega = oracle.alpha_omega(g)
        for v in range(g.n):
            for om in {int(omega[v]), int(r[v])}:
                Us = oracle.harmonic_cut_bounds(g, v, om)
                assert all(u * oracle.H_MARGIN >= H[v] for u in Us), (seed, v)
                assert all(Us[i + 1] <= Us[i] * (1 + 4 * n * U) for i in range(len(Us) - 1))
                if om == r[v]:
                    assert Us[-1] == H[v]


def _check_cut(g, k, order=None, ub=None):
    ref = oracle.textbook_harmonic_topk(g, k)
    got = oracle.bfscut_harmonic(g, k, order, ub)
    assert list(got.ids) == list(ref.ids), (g.name, k)
    assert np.array_equal(got.H, ref.H) and np.array_equal(got.r, ref.r)
    assert got.n_tied == ref.n_tied, (g.name, k)
    return got


def test_bfscut_equals_textbook_small_random():
    for seed in range(1000):
        n = 2 + seed % 23
        g = gg.random_graph(n, [0.05, 0.1, 0.2, 0.4][seed % 4], 60_000 + seed, seed % 3 == 0)
        for k in {1, 2, 3, n // 2 + 1, n, n + 2}:
            _check_cut(g, k)


TIED = [lambda: gg.cycle(12), lambda: gg.cycle(9, directed=True), lambda: gg.hypercube(4),
        lambda: gg.complete_bipartite(4, 4), lambda: gg.random_tree(50, 1), lambda: gg.star(8),
        lambda: gg.disjoint_union(gg.cycle(6), gg.cycle(6)), lambda: gg.path(15),
        lambda: gg.reduction_graph(3, [{0}, {1, 2}, {0, 2}])[0]]


@pytest.mark.parametrize("gi", range(len(TIED)))
def test_bfscut_and_nbcut_on_tied_families(gi):
    g = TIED[gi]()
    nb = oracle.nb_bounds(g)
    order = oracle.nb_harmonic_order(g, nb.h_ub)
    full = np.concatenate([order, np.nonzero(g.outdeg() == 0)[0].astype(np.uint32)])
    for k in (1, 2, 5, g.n):
        _check_cut(g, k)
        _check_cut(g, k, full, nb.h_ub)


def test_nb_upper_bound_holds():
    for seed in range(300):
        n = 2 + seed % 25
        g = gg.random_graph(n, [0.05, 0.1, 0.2, 0.35][seed % 4], 70_000 + seed, seed % 3 != 0)
        H, _ = oracle.harmonic_sums(g)
        for lev in (1, 2, 64):
            nb = oracle.nb_bounds(g, max_levels=lev)
            assert all(nb.h_ub[v] * oracle.H_MARGIN >= H[v] for v in range(g.n)), (seed, lev)
            assert all((nb.h_ub[v] == 0.0) == (g.outdeg()[v] == 0) for v in range(g.n))


@pytest.mark.parametrize("seed", range(6))
def test_nb_upper_bound_exact_on_trees(seed):
    g = gg.random_tree(60 + 31 * seed, seed)
    H, _ = oracle.harmonic_sums(g)
    nb = oracle.nb_bounds(g, max_levels=g.n + 1)
    assert np.array_equal(nb.h_ub, H)


def test_nbcut_equals_textbook_random_and_stops_early():
    for seed in range(600):
        n = 2 + seed % 23
        g = gg.random_graph(n, [0.05, 0.1, 0.2, 0.4][seed % 4], 80_000 + seed, seed % 3 == 0)
        nb = oracle.nb_bounds(g)
        order = oracle.nb_harmonic_order(g, nb.h_ub)
        full = np.concatenate([order, np.nonzero(g.outdeg() == 0)[0].astype(np.uint32)])
        for k in {1, 3, n}:
            _check_cut(g, k, full, nb.h_ub)
    g = gg.barabasi_albert(2000, 4, gg.workload_seed(0))
    nb = oracle.nb_bounds(g)
    got = _check_cut(g, 10, oracle.nb_harmonic_order(g, nb.h_ub), nb.h_ub)
    assert got.counters.bfs_started < g.n // 2
