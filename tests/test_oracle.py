"""Pins for the CPU oracle: each check comes from outside the oracle itself --
a second algorithm (Floyd-Warshall, Algorithm 2 on trees), a closed form, the
paper's own closeness formulas for the reduction graph (Section 3), a library
routine (networkx, numpy), or brute force with exact rationals."""
import itertools
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1704_01077_gb300 import graphgen as gg


def _all_graphs(n, directed):
    pairs = [(a, b) for a in range(n) for b in range(n) if a != b and (directed or a < b)]
    for mask in range(1 << len(pairs)):
        src = [pairs[i][0] for i in range(len(pairs)) if mask >> i & 1]
        dst = [pairs[i][1] for i in range(len(pairs)) if mask >> i & 1]
        yield gg.from_arcs(n, src, dst, directed)


# ---------------------------------------------------------------- distances

@pytest.mark.parametrize("n,directed", [(1, False), (2, False), (3, False), (4, False), (5, False),
                                        (2, True), (3, True), (4, True)])
def test_bfs_equals_floyd_warshall_exhaustive(n, directed):
    for g in _all_graphs(n, directed):
        S1, r1 = oracle.bfs_sums(g)
        S2, r2 = oracle.floyd_warshall(g)
        assert np.array_equal(S1, S2) and np.array_equal(r1, r2)


def test_bfs_equals_floyd_warshall_random():
    for seed in range(300):
        n = 6 + seed % 7
        directed = bool(seed & 1)
        g = gg.random_graph(n, 0.15 + 0.05 * (seed % 5), seed, directed)
        S1, r1 = oracle.bfs_sums(g)
        S2, r2 = oracle.floyd_warshall(g)
        assert np.array_equal(S1, S2) and np.array_equal(r1, r2), seed


def test_bfs_subset_of_sources_matches_all():
    g = gg.barabasi_albert(300, 3, 7)
    S, r = oracle.bfs_sums(g)
    src = np.array([5, 0, 299, 17], np.uint32)
    S2, r2 = oracle.bfs_sums(g, src)
    assert np.array_equal(S[src], S2) and np.array_equal(r[src], r2)


def test_closeness_against_networkx():
    nx = pytest.importorskip("networkx")
    for seed in range(12):
        directed = bool(seed & 1)
        g = gg.random_graph(40, 0.06, 100 + seed, directed)
        S, r = oracle.bfs_sums(g)
        G = nx.DiGraph() if directed else nx.Graph()
        G.add_nodes_from(range(g.n))
        deg = g.outdeg()
        G.add_edges_from(zip(np.repeat(np.arange(g.n), deg).tolist(), g.cols.tolist()))
        # networkx measures incoming distance on digraphs; reverse for outgoing
        ref = nx.closeness_centrality(G.reverse() if directed else G, wf_improved=True)
        for v in range(g.n):
            f, c = oracle.farness(g.n, S[v], r[v])
            assert c == pytest.approx(ref[v], rel=1e-12, abs=0.0), (seed, v)


# ------------------------------------------------------------- closed forms

@pytest.mark.parametrize("n", [1, 2, 3, 10, 57])
def test_path_undirected(n):
    S, r = oracle.bfs_sums(gg.path(n))
    for i in range(n):
        assert S[i] == i * (i + 1) // 2 + (n - 1 - i) * (n - i) // 2
        assert r[i] == n


@pytest.mark.parametrize("n", [2, 9, 40])
def test_path_directed(n):
    S, r = oracle.bfs_sums(gg.path(n, directed=True))
    for i in range(n):
        assert S[i] == (n - 1 - i) * (n - i) // 2
        assert r[i] == n - i


@pytest.mark.parametrize("n", [3, 4, 11, 30])
def test_cycles(n):
    S, r = oracle.bfs_sums(gg.cycle(n))
    assert (S == n * n // 4).all() and (r == n).all()
    S, r = oracle.bfs_sums(gg.cycle(n, directed=True))
    assert (S == n * (n - 1) // 2).all() and (r == n).all()


@pytest.mark.parametrize("n", [2, 5, 33])
def test_star_and_complete(n):
    S, r = oracle.bfs_sums(gg.star(n))
    assert S[0] == n - 1 and all(S[i] == 2 * n - 3 for i in range(1, n))
    S, r = oracle.bfs_sums(gg.complete(n))
    assert (S == n - 1).all() and (r == n).all()


@pytest.mark.parametrize("a,b", [(1, 1), (2, 3), (5, 7)])
def test_complete_bipartite(a, b):
    S, _ = oracle.bfs_sums(gg.complete_bipartite(a, b))
    assert all(S[i] == b + 2 * (a - 1) for i in range(a))
    assert all(S[a + j] == a + 2 * (b - 1) for j in range(b))


@pytest.mark.parametrize("d", [1, 2, 3, 6])
def test_hypercube(d):
    S, _ = oracle.bfs_sums(gg.hypercube(d))
    assert (S == d * 2 ** (d - 1)).all()


def test_disjoint_union_reach_is_component_size():
    g = gg.disjoint_union(gg.path(4), gg.complete(3), gg.star(6), gg.path(1))
    S, r = oracle.bfs_sums(g)
    assert list(r) == [4] * 4 + [3] * 3 + [6] * 6 + [1]
    a, o = oracle.alpha_omega(g)
    assert np.array_equal(a, r) and np.array_equal(o, r)


# ------------------------------------------------------- trees (Algorithm 2)

@pytest.mark.parametrize("seed", range(20))
def test_tree_algorithm_matches_bfs(seed):
    g = gg.random_tree(5 + 13 * seed, seed)
    S_bfs, _ = oracle.bfs_sums(g)
    assert np.array_equal(oracle.tree_sums(g), S_bfs)


def test_tree_algorithm_on_path_and_star():
    for g in (gg.path(30), gg.star(12)):
        assert np.array_equal(oracle.tree_sums(g), oracle.bfs_sums(g)[0])


# ---------------------------------------------- reduction graph (Section 3)

def _reduction_case(X, sets, p=7, q=36):
    g, ids = gg.reduction_graph(X, sets, p, q)
    S, r = oracle.bfs_sums(g)
    nc = len(sets)
    n = g.n
    assert n == q * nc + q + nc + 2 * X + p * nc
    gp = (p + 1) * (p + 2) // 2 - 1
    c0 = ids["C0"][0]
    for ci, C in enumerate(sets):
        Rc = sum(1 for D in sets if C & D)
        # closeness of C_0 is (q(1+|C|)+|X|+pR)^2 / ((q(1+2|C|)+|X|+g(p)R)(n-1))
        assert r[c0 + ci] - 1 == q * (1 + nc) + X + p * Rc
        assert S[c0 + ci] == q * (1 + 2 * nc) + X + gp * Rc
    y0 = ids["Y"][0]
    for j in range(q):  # Y: |C| vertices at distance 1
        assert r[y0 + j] - 1 == nc and S[y0 + j] == nc
    for i in range(1, p + 1):  # C_i: p-i vertices at distances 1..p-i
        for ci in range(nc):
            v = ids[f"C{i}"][0] + ci
            assert r[v] - 1 == p - i and S[v] == (p - i) * (p - i + 1) // 2
    x1 = ids["X1"][0]
    for x in range(X):  # X_1: N_x vertices in each of C_1..C_p
        Nx = sum(1 for C in sets if x in C)
        assert r[x1 + x] - 1 == p * Nx and S[x1 + x] == Nx * p * (p + 1) // 2
    # the most central vertex is in C_0 and minimises R_C
    ids_top, _ = oracle.topk(S, r, 1)
    assert ids["C0"][0] <= ids_top[0] < ids["C0"][1]
    best = min(range(nc), key=lambda ci: sum(1 for D in sets if sets[ci] & D))
    bestR = sum(1 for D in sets if sets[best] & D)
    assert sum(1 for D in sets if sets[ids_top[0] - c0] & D) == bestR
    return g


def test_reduction_graph_closed_forms():
    _reduction_case(3, [{0}, {1, 2}, {0, 2}])
    _reduction_case(4, [{0, 1}, {2}, {3}, {0, 3}, {1, 2, 3}])
    _reduction_case(5, [{0, 1, 2, 3, 4}, {0}, {1}, {2, 3}])


# ------------------------------------------------------------- ordering/top-k

def _key(S, r):
    return Fraction(10 ** 30) if r <= 1 else Fraction(int(S), (int(r) - 1) ** 2)


def test_topk_against_fraction_brute_force():
    rng = np.random.default_rng(5)
    for trial in range(200):
        n = int(rng.integers(1, 40))
        S = rng.integers(0, 60, n).astype(np.uint64)
        r = rng.integers(1, 9, n).astype(np.uint32)
        k = int(rng.integers(1, n + 3))
        ids, tied = oracle.topk(S, r, k)
        ref = sorted(range(n), key=lambda v: (_key(S[v], r[v]), v))[:k]
        assert list(ids) == ref
        kth = _key(S[ref[-1]], r[ref[-1]])
        assert tied == sum(1 for v in range(n) if _key(S[v], r[v]) == kth)


def test_cmp_farness_large_values_exact():
    # values whose cross products exceed 64 bits
    Sa, ra = 2 ** 43 + 1, 2 ** 22
    Sb, rb = 2 ** 43, 2 ** 22
    assert oracle.cmp_farness(Sa, ra, Sb, rb) == 1
    assert oracle.cmp_farness(Sb, rb, Sa, ra) == -1
    assert oracle.cmp_farness(3 * 4, 3, 3 * 9, 4) == 0  # 12/4 == 27/9
    assert oracle.cmp_farness(5, 1, 10 ** 12, 2) == 1  # r = 1 is +infinity


def test_farness_doubles_are_single_rounded():
    for n, S, r in [(2000, 5555, 1999), (65536, 123456789, 40000), (7, 9, 3), (10 ** 6, 3 * 10 ** 6, 10 ** 6)]:
        f, c = oracle.farness(n, S, r)
        num = float(n - 1) * float(S)
        den = float((r - 1) * (r - 1))
        assert f == num / den and c == den / num
    f, c = oracle.farness(10, 0, 1)
    assert f == float("inf") and c == 0.0


def test_degree_order_matches_lexsort():
    for g in (gg.barabasi_albert(500, 3, 1), gg.rmat(10, 8, seed=3), gg.path(1), gg.star(7)):
        deg = g.outdeg()
        ref = np.lexsort((np.arange(g.n), -deg))
        assert np.array_equal(oracle.degree_order(g), ref)


# ---------------------------------------------------------------- SCC, alpha/omega

def _reach_sets(g):
    S, r = oracle.floyd_warshall(g) if g.n <= 64 else oracle.bfs_sums(g)
    n = g.n
    reach = np.zeros((n, n), bool)
    deg = g.outdeg()
    adj = [g.cols[g.offsets[v]:g.offsets[v + 1]] for v in range(n)]
    for v in range(n):
        seen = {v}
        st = [v]
        while st:
            u = st.pop()
            for w in adj[u]:
                if int(w) not in seen:
                    seen.add(int(w))
                    st.append(int(w))
        reach[v, list(seen)] = True
    return reach, r


def test_scc_by_mutual_reachability():
    for seed in range(60):
        g = gg.random_graph(12 + seed % 9, 0.12, 500 + seed, True)
        comp, nc = oracle.scc(g)
        reach, _ = _reach_sets(g)
        mutual = reach & reach.T
        assert np.array_equal(mutual, comp[:, None] == comp[None, :])
        assert nc == len(set(comp.tolist()))


def test_alpha_omega_bracket_reach_and_exact_on_biggest_scc():
    for seed in range(80):
        g = gg.random_graph(10 + seed % 25, 0.06 + 0.01 * (seed % 6), 900 + seed, True)
        a, o = oracle.alpha_omega(g)
        reach, r = _reach_sets(g)
        assert (a <= r).all() and (r <= o).all(), seed
        assert (o <= g.n).all()
        comp, nc = oracle.scc(g)
        sizes = np.bincount(comp, minlength=nc)
        best = max(range(nc), key=lambda c: (sizes[c], -int(np.flatnonzero(comp == c).min())))
        members = np.flatnonzero(comp == best)
        assert (a[members] == r[members]).all() and (o[members] == r[members]).all()


def test_alpha_omega_hand_built_dag():
    # SCCs: A={0,1} -> B={2} -> D={4,5,6}; A -> C={3} -> D; E={7} -> C
    src = [0, 1, 0, 2, 1, 3, 4, 5, 6, 7]
    dst = [1, 0, 2, 4, 3, 4, 5, 6, 4, 3]
    g = gg.from_arcs(8, src, dst, True)
    a, o = oracle.alpha_omega(g)
    # biggest SCC is D (size 3): exact reach 3
    assert a[4] == o[4] == 3
    # B and C reach D: omega = w + omega(D) (D is the biggest), alpha = w + 3
    assert a[2] == o[2] == 4 and a[3] == o[3] == 4
    # A: alpha = 2 + max(4, 4) = 6; A reaches D, successors B, C not reachable from D:
    # omega = 2 + omega(D) + omega(B) + omega(C) = 2 + 3 + 4 + 4 = 13 -> clamp to n = 8
    assert a[0] == a[1] == 6 and o[0] == o[1] == 8
    # E: alpha = 1 + 4 = 5, omega = 1 + 3 + 4 = 8
    assert a[7] == 5 and o[7] == 8


# ------------------------------------------------------ BFSCut (Algorithm 4)

def test_cut_bound_invariants():
    for seed in range(150):
        directed = bool(seed & 1)
        g = gg.random_graph(8 + seed % 12, 0.2, 2000 + seed, directed)
        S, r = oracle.bfs_sums(g)
        for v in range(g.n):
            L = oracle.cut_bounds(g, v)
            assert (L <= S[v]).all(), (seed, v)
            assert (np.diff(L.astype(np.int64)) >= 0).all(), (seed, v, L)
            assert L[-1] == S[v]


def test_cut_min_is_minimum_over_whole_interval():
    """Section 8's lemma: the bound's minimum over [alpha', omega] is at a candidate point;
    brute force over every integer r with exact rationals."""
    rng = np.random.default_rng(17)
    for _ in range(3000):
        nd = int(rng.integers(1, 40))
        d = int(rng.integers(0, 6))
        Sd = int(rng.integers(nd - 1, 8 * nd + 2)) if d > 0 else 0
        g = int(rng.integers(0, 60))
        lo = int(rng.integers(1, nd + 30))
        hi = lo + int(rng.integers(0, 120))
        L, r = oracle.cut_min(Sd, d, nd, g, lo, hi)

        def bound(rr):
            rem = rr - nd
            return Sd + (d + 1) * rem + max(0, rem - g)

        lo2 = max(lo, nd)
        vals = [Fraction(bound(rr), (rr - 1) ** 2) for rr in range(max(lo2, 2), max(hi, lo2) + 1)]
        if not vals:
            continue
        assert L == bound(r) and r >= 2
        assert Fraction(L, (r - 1) ** 2) == min(vals), (Sd, d, nd, g, lo, hi)


def _check_bfscut(g, k, order=None):
    ref = oracle.textbook_topk(g, k)
    got = oracle.bfscut(g, k, order)
    assert list(got.ids) == list(ref.ids), (g.name, k)
    assert np.array_equal(got.S, ref.S) and np.array_equal(got.r, ref.r)
    assert got.n_tied == ref.n_tied
    return got


def test_bfscut_equals_textbook_small_random():
    for seed in range(1500):
        n = 2 + seed % 23
        directed = bool(seed % 3 == 0)
        p = [0.05, 0.1, 0.2, 0.4][seed % 4]
        g = gg.random_graph(n, p, 10_000 + seed, directed)
        for k in {1, 2, 3, n // 2 + 1, n, n + 2}:
            _check_bfscut(g, k)


def test_bfscut_equals_textbook_families():
    for g in (gg.path(20), gg.cycle(15, True), gg.star(9), gg.complete_bipartite(3, 5), gg.hypercube(4),
              gg.random_tree(60, 3), gg.disjoint_union(gg.cycle(5), gg.path(7), gg.path(1)),
              gg.reduction_graph(3, [{0}, {1, 2}, {0, 2}])[0]):
        for k in (1, 3, 10, g.n):
            _check_bfscut(g, k)


def test_bfscut_any_order_same_result():
    g = gg.barabasi_albert(400, 3, 11)
    rng = np.random.default_rng(1)
    base = _check_bfscut(g, 10)
    for _ in range(5):
        got = _check_bfscut(g, 10, rng.permutation(g.n))
        assert list(got.ids) == list(base.ids)
    rev = _check_bfscut(g, 10, oracle.degree_order(g)[::-1].copy())
    assert rev.counters.edges_visited >= base.counters.edges_visited


def test_bfscut_prunes_on_ba_and_rmat():
    g = gg.barabasi_albert(2000, 4, gg.workload_seed(0))
    got = _check_bfscut(g, 10)
    assert got.counters.edges_visited * 5 < g.arcs * g.n
    g = gg.rmat(11, 16, seed=gg.workload_seed(1))
    got = _check_bfscut(g, 10)
    assert got.counters.bfs_cut > 0


def test_bfscut_degenerate():
    empty = gg.from_arcs(5, [], [], True)
    got = oracle.bfscut(empty, 3)
    assert list(got.ids) == [0, 1, 2] and got.n_tied == 5 and list(got.r) == [1, 1, 1]
    one = gg.from_arcs(1, [], [], False)
    assert list(oracle.bfscut(one, 4).ids) == [0]
    assert len(oracle.bfscut(gg.path(3), 0).ids) == 0
