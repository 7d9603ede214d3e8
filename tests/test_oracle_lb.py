"""Pins for the oracle's updateBoundsLB (Section 7, Algorithm 5, Eq. 4 and Eq. 5)
and Algorithm 1 with it (DegBound, NBBound): the level bound against its
per-vertex form and the Section 7 difference lemma, the resulting vertex
bounds against the textbook S on the reach class, and the top-k against the
textbook on random graphs, grids and tied families."""
import numpy as np
import pytest

import oracle
from paper_1704_01077_gb300 import graphgen as gg

UNREACHED = np.iinfo(np.uint32).max


def _per_vertex_level_bound(level, i, directed):
    """Eq. 4 / Eq. 5 summed vertex by vertex over R(s): 2 for every x within one
    level (above, if directed), the level difference otherwise, minus 2."""
    tot = 0
    for lx in level:
        if lx == UNREACHED:
            continue
        diff = int(lx) - i
        near = diff <= 1 if directed else abs(diff) <= 1
        tot += 2 if near else (diff if directed else abs(diff))
    return tot - 2


def test_level_bound_definition_and_difference_lemma():
    for seed in range(80):
        n = 4 + seed % 20
        directed = bool(seed % 2)
        g = gg.random_graph(n, [0.1, 0.2, 0.3][seed % 3], 90_000 + seed, directed)
        for s in range(0, g.n, 3):
            level, L = oracle.lb_level_bounds(g, s)
            D = len(L) - 1
            for i in range(D + 1):
                assert int(L[i]) == _per_vertex_level_bound(level, i, directed), (seed, s, i)
            if not directed:
                # Section 7: L(i) - L(i-1) = sum_{j < i-2} g_j - sum_{j > i+1} g_j
                gcnt = np.bincount(level[level != UNREACHED].astype(np.int64), minlength=D + 1)
                for i in range(1, D + 1):
                    want = int(gcnt[: max(i - 2, 0)].sum()) - int(gcnt[i + 2:].sum())
                    assert int(L[i]) - int(L[i - 1]) == want, (seed, s, i)


def test_vertex_bounds_below_distance_sums():
    for seed in range(120):
        n = 4 + seed % 25
        directed = seed % 3 != 0
        g = gg.random_graph(n, [0.08, 0.15, 0.3][seed % 3], 91_000 + seed, directed)
        S, r = oracle.bfs_sums(g)
        comp, _ = oracle.scc(g)
        deg = g.outdeg()
        for s in range(g.n):
            level, L = oracle.lb_level_bounds(g, s)
            for w in range(g.n):
                if level[w] == UNREACHED or comp[w] != comp[s]:
                    continue
                lb = int(L[level[w]]) - int(deg[w])
                assert 0 <= lb <= int(S[w]), (seed, s, w)
                assert r[w] == r[s]


def test_grid_level_bound_by_hand():
    # 1 x 5 path as a grid, source at an end: levels 0..4 one vertex each;
    # L(0) = 2(1+1) + 2 + 3 + 4 - 2 = 11, the middle vertex (level 2, deg 2):
    # L(2) - 2 = (2 + 2 + 2 + 2 + 2) - 2 - 2 = 6 = S(middle) (1+1+2+2)
    g = gg.grid(1, 5)
    level, L = oracle.lb_level_bounds(g, 0)
    assert list(level) == [0, 1, 2, 3, 4]
    assert int(L[0]) == 11 and int(L[2]) - 2 == 6
    S, _ = oracle.bfs_sums(g)
    assert S[2] == 6


def _check(g, k, nb):
    ref = oracle.textbook_topk(g, k)
    if nb:
        b = oracle.nb_bounds(g)
        got = oracle.bfsbound(g, k, oracle.nb_order(g, b.key).tolist()
                              + np.nonzero(g.outdeg() == 0)[0].tolist(), b)
    else:
        got = oracle.bfsbound(g, k)
    assert list(got.ids) == list(ref.ids), (g.name, k, nb)
    assert np.array_equal(got.S, ref.S) and np.array_equal(got.r, ref.r)
    assert got.n_tied == ref.n_tied, (g.name, k, nb)
    return got


@pytest.mark.parametrize("nb", [False, True])
def test_bfsbound_equals_textbook_random(nb):
    for seed in range(500):
        n = 2 + seed % 23
        g = gg.random_graph(n, [0.05, 0.1, 0.2, 0.4][seed % 4], 92_000 + seed, seed % 3 == 0)
        for k in {1, 2, 3, n // 2 + 1, n, n + 2}:
            _check(g, k, nb)


FAMILIES = [lambda: gg.grid(7, 9), lambda: gg.grid(6, 6, directed=True, seed=3, drop=0.3),
            lambda: gg.grid(10, 10, seed=4, drop=0.2), lambda: gg.cycle(12), lambda: gg.hypercube(4),
            lambda: gg.random_tree(60, 2), lambda: gg.star(9), lambda: gg.complete_bipartite(3, 5),
            lambda: gg.disjoint_union(gg.cycle(6), gg.path(5), gg.path(1)), lambda: gg.path(9, directed=True),
            lambda: gg.reduction_graph(3, [{0}, {1, 2}, {0, 2}])[0]]


@pytest.mark.parametrize("nb", [False, True])
@pytest.mark.parametrize("fi", range(len(FAMILIES)))
def test_bfsbound_equals_textbook_families(fi, nb):
    g = FAMILIES[fi]()
    for k in (1, 3, 10, g.n):
        _check(g, k, nb)


def test_bfsbound_bounds_only_the_reach_class():
    # s -> w and s -> p1 -> ... -> p20; w -> 10 leaves; u -> 5 leaves (apart).
    # From s the level bound of w (different SCC) would be 205 / 31^2 = 0.213,
    # above u's exact 5 / 5^2 = 0.2 but w's own ratio is 10 / 10^2 = 0.1:
    # applying it would stop the search before w, the true top-1.
    s, w, u = 0, 1, 2
    path = list(range(3, 23))
    leaves_w = list(range(23, 33))
    leaves_u = list(range(33, 38))
    src = [s, s] + path[:-1] + [w] * 10 + [u] * 5
    dst = [w, path[0]] + path[1:] + leaves_w + leaves_u
    g = gg.from_arcs(38, src, dst, True, "reach_class")
    order = [s, u, w] + [v for v in range(38) if v not in (s, u, w)]
    ref = oracle.textbook_topk(g, 1)
    assert list(ref.ids) == [w]
    got = oracle.bfsbound(g, 1, order)
    assert list(got.ids) == [w]


def test_bfsbound_prunes_on_grids():
    g = gg.grid(40, 40)
    got = _check(g, 10, False)
    cut = oracle.bfscut(g, 10)
    assert got.counters.bfs_started * 5 < g.n
    assert got.counters.edges_visited < cut.counters.edges_visited
    got = _check(g, 10, True)
    assert got.counters.bfs_started * 5 < g.n
