"""Pins for the oracle's neighbourhood-based bound (computeBoundsNB, Section 5,
Algorithm 3; Eq. 3 for directed graphs; Eq. 6 for unknown reach) and for
Algorithm 1's stop under that bound (NBCut).  Each check comes from outside
the oracle: brute-force walk enumeration, the exact distance sums of the
textbook BFS, hand-computed hypercube values, or a brute-force minimum over
every reach in [alpha, omega] with exact rationals."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1704_01077_gb300 import graphgen as gg

CAP = 1 << 32


def _adj(g):
    off = np.asarray(g.offsets, dtype=np.int64)
    col = np.asarray(g.cols, dtype=np.int64)
    return [list(col[off[v]:off[v + 1]]) for v in range(g.n)]


def _walks(adj, s, k, non_backtracking):
    """Number of walks of length k from s (non-backtracking: no step returns
    along the arc just used), by explicit enumeration."""
    count = 0
    stack = [(s, -1, 0)]
    while stack:
        v, prev, d = stack.pop()
        if d == k:
            count += 1
            continue
        for w in adj[v]:
            if non_backtracking and w == prev:
                continue
            stack.append((w, v, d + 1))
    return count


@pytest.mark.parametrize("directed", [False, True])
def test_counts_equal_enumerated_walks(directed):
    for seed in range(60):
        n = 3 + seed % 6
        g = gg.random_graph(n, 0.35 + 0.05 * (seed % 4), 500 + seed, directed)
        adj = _adj(g)
        nb = oracle.nb_bounds(g, max_levels=64, counts_levels=7)
        for k in range(7):
            for s in range(g.n):
                want = _walks(adj, s, k, not directed)
                assert int(nb.counts[k][s]) == min(want, CAP), (seed, k, s)


def test_counts_bound_level_sizes():
    # N~_k(s) >= number of vertices at distance exactly k (walks reach them all)
    for seed in range(40):
        g = gg.random_graph(12, 0.2, 900 + seed, bool(seed & 1))
        nb = oracle.nb_bounds(g, max_levels=64, counts_levels=12)
        for s in range(g.n):
            dist = _bfs_dist(_adj(g), s)
            for k in range(12):
                assert int(nb.counts[k][s]) >= sum(1 for d in dist if d == k)


def _bfs_dist(adj, s):
    dist = [-1] * len(adj)
    dist[s] = 0
    q = [s]
    for v in q:
        for w in adj[v]:
            if dist[w] < 0:
                dist[w] = dist[v] + 1
                q.append(w)
    return dist


@pytest.mark.parametrize("seed", range(8))
def test_exact_on_trees(seed):
    # on a tree the non-backtracking walks are the BFS levels (Algorithm 2)
    g = gg.random_tree(40 + 17 * seed, seed)
    S, r = oracle.bfs_sums(g)
    nb = oracle.nb_bounds(g, max_levels=g.n + 1)
    assert np.array_equal(nb.S, S) and np.array_equal(nb.r, r)


def test_exact_on_cycles_paths_stars_complete_bipartite():
    for g in (gg.cycle(9), gg.cycle(10), gg.path(12), gg.star(7), gg.complete(6),
              gg.complete_bipartite(3, 5), gg.cycle(7, directed=True), gg.path(9, directed=True)):
        S, r = oracle.bfs_sums(g)
        nb = oracle.nb_bounds(g, max_levels=64)
        assert np.array_equal(nb.S, S), g.name
        assert np.array_equal(nb.r, r), g.name


def test_hypercube_by_hand():
    # Q3: 3 neighbours, 6 non-backtracking 2-walks but only 4 vertices left:
    # S~ = 1*3 + 2*4 = 11 (true S = 3 + 2*3 + 3 = 12).
    # Q4: 4 neighbours, 12 2-walks, 11 vertices left: S~ = 4 + 2*11 = 26 (true 32).
    for d, want in ((3, 11), (4, 26)):
        nb = oracle.nb_bounds(gg.hypercube(d))
        assert set(nb.S.tolist()) == {want}
        assert set(nb.r.tolist()) == {1 << d}


def test_out_degree_zero_has_closeness_zero():
    g = gg.from_arcs(4, [0, 1], [1, 2], True)
    nb = oracle.nb_bounds(g)
    assert nb.r[2] == 1 and nb.r[3] == 1 and nb.S[2] == 0
    assert nb.key[2] == np.iinfo(np.uint64).max


def _lower_bound_ok(g, nb):
    S, r = oracle.bfs_sums(g)
    for v in range(g.n):
        if r[v] <= 1:
            assert nb.r[v] == 1
            continue
        assert nb.r[v] >= 2
        lb = Fraction(int(nb.S[v]), (int(nb.r[v]) - 1) ** 2)
        f = Fraction(int(S[v]), (int(r[v]) - 1) ** 2)
        assert lb <= f, (g.name, v)
        assert Fraction(int(nb.key[v]), 1 << oracle.NB_FRAC) <= lb
        assert int(nb.key[v]) == (int(nb.S[v]) << oracle.NB_FRAC) // (int(nb.r[v]) - 1) ** 2


def test_bound_below_farness_random():
    for seed in range(300):
        n = 2 + seed % 25
        directed = seed % 3 != 0
        g = gg.random_graph(n, [0.05, 0.1, 0.2, 0.35][seed % 4], 2000 + seed, directed)
        for lev in (1, 2, 64):
            _lower_bound_ok(g, oracle.nb_bounds(g, max_levels=lev))


def test_bound_below_farness_families():
    for g in (gg.reduction_graph(3, [{0}, {1, 2}, {0, 2}])[0], gg.barabasi_albert(300, 3, 5),
              gg.rmat(8, 8, seed=3), gg.disjoint_union(gg.cycle(5), gg.path(6), gg.path(1))):
        _lower_bound_ok(g, oracle.nb_bounds(g))


def _sum_bound(counts, r, K):
    """Section 5's proposition: S~(r) = sum_k k min(N~_k, max(r - c_{k-1}, 0)),
    with N~_{K+1} unbounded."""
    total, c = 0, 1
    for k in range(1, K + 1):
        take = min(counts[k], max(r - c, 0))
        total += k * take
        c += counts[k]
    return total + (K + 1) * max(r - c, 0), c


@pytest.mark.parametrize("K", [1, 2, 3, 40])
def test_candidate_minimum_equals_minimum_over_every_reach(K):
    checked = 0
    for seed in range(250):
        n = 3 + seed % 12
        directed = seed % 4 != 0
        g = gg.random_graph(n, [0.08, 0.15, 0.3][seed % 3], 7000 + seed, directed)
        alpha, omega = oracle.alpha_omega(g)
        nb = oracle.nb_bounds(g, max_levels=K, counts_levels=K + 2)
        for v in range(g.n):
            cnt = [int(nb.counts[k][v]) for k in range(K + 2)]
            if cnt[1] == 0:
                continue
            hi = int(omega[v])
            # walks that stop before level K+1 bound the reach: r <= c at that point
            c = 1
            for k in range(1, K + 1):
                if cnt[k] == 0:
                    hi = min(hi, c)
                    break
                c += cnt[k]
            vals = []
            for r in range(max(int(alpha[v]), 2), hi + 1):
                s, _ = _sum_bound(cnt, r, K)
                vals.append(Fraction(s, (r - 1) ** 2))
            assert Fraction(int(nb.S[v]), (int(nb.r[v]) - 1) ** 2) == min(vals), (seed, v, K)
            s_at, _ = _sum_bound(cnt, int(nb.r[v]), K)
            assert s_at == int(nb.S[v])
            checked += 1
    assert checked > 500


def test_walks_that_stop_bound_the_reach():
    # vertex 0 (the biggest SCC by the smallest-id tie) points to T leaves; a
    # chain X_L -> ... -> X_1 -> 0; isolated vertices keep omega below n.
    # Algorithm 6 adds omega(0) again at every chain step, so omega(X_j) grows
    # like j (T + 1) while r(X_j) = j + T + 1.  The walks from X_j stop after
    # level j + 1, so r <= (their count) = r(X_j): with alpha exact the bound
    # is S itself; without that cap the omega candidate (tail slope K+1)
    # would win at K = 8.
    T, L, iso = 20, 5, 200
    src = [0] * T + [T + 1] + [T + j for j in range(2, L + 1)]
    dst = list(range(1, T + 1)) + [0] + [T + j - 1 for j in range(2, L + 1)]
    g = gg.from_arcs(T + L + 1 + iso, src, dst, True)
    alpha, omega = oracle.alpha_omega(g)
    S, r = oracle.bfs_sums(g)
    x = T + L
    assert omega[x] > 3 * r[x] and alpha[x] == r[x]
    for K in (L + 2, 8, 64):
        nb = oracle.nb_bounds(g, max_levels=K)
        assert nb.S[x] == S[x] and nb.r[x] == r[x], K


def test_order_is_key_then_id():
    g = gg.barabasi_albert(500, 2, 9)
    nb = oracle.nb_bounds(g)
    order = oracle.nb_order(g, nb.key)
    want = sorted((int(nb.key[v]), v) for v in range(g.n) if g.outdeg()[v] > 0)
    assert [v for _, v in want] == order.tolist()


# ---------------------------------------------------------------- NBCut

def _check_nbcut(g, k):
    ref = oracle.textbook_topk(g, k)
    nb = oracle.nb_bounds(g)
    order = oracle.nb_order(g, nb.key)
    full = np.concatenate([order, np.nonzero(g.outdeg() == 0)[0].astype(np.uint32)])
    got = oracle.bfscut(g, k, full, lb_key=nb.key)
    assert list(got.ids) == list(ref.ids), (g.name, k)
    assert np.array_equal(got.S, ref.S) and np.array_equal(got.r, ref.r)
    assert got.n_tied == ref.n_tied, (g.name, k)
    return got


def test_nbcut_equals_textbook_small_random():
    for seed in range(800):
        n = 2 + seed % 23
        directed = bool(seed % 3 == 0)
        g = gg.random_graph(n, [0.05, 0.1, 0.2, 0.4][seed % 4], 30_000 + seed, directed)
        for k in {1, 2, 3, n // 2 + 1, n, n + 2}:
            _check_nbcut(g, k)


def test_nbcut_equals_textbook_with_ties():
    # every vertex of a cycle or hypercube ties; on trees and cycles the bound is
    # exact, so a non-strict stop would drop tied vertices
    for g in (gg.cycle(12), gg.cycle(9, directed=True), gg.hypercube(4), gg.random_tree(50, 1), gg.star(8),
              gg.complete_bipartite(4, 4), gg.disjoint_union(gg.cycle(6), gg.cycle(6))):
        for k in (1, 2, 5, g.n):
            _check_nbcut(g, k)


def test_nbcut_stops_early():
    g = gg.barabasi_albert(2000, 4, gg.workload_seed(0))
    got = _check_nbcut(g, 10)
    assert got.counters.bfs_started < g.n // 2
    g = gg.rmat(11, 16, seed=gg.workload_seed(1))
    got = _check_nbcut(g, 10)
    assert got.counters.bfs_started < int((g.outdeg() > 0).sum())
