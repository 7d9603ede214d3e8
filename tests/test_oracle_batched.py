"""Pins for the oracle's batched schedule (oracle.bfscut_batched): Algorithm 1
with updateBoundsBFSCut where B searches advance one BFS level per step and
the k-th threshold changes only between steps.

What pins it, from outside the function itself:
- with B = 1 the schedule is Algorithm 1 run one source at a time, so every
  counter equals the sequential oracle's (itself pinned against the textbook);
- at every B the top-k (ids, S, r, ties) equals the textbook all-sources
  result, since any valid threshold gives the exact answer (Section 4);
- a star counted by hand at B = 1 and B = 2 fixes when the threshold is read:
  after a step's finished searches are merged, before its survivors' cut test.
"""
import numpy as np
import pytest

import oracle
from paper_1704_01077_gb300 import graphgen as gg


def _same_counters(a, b):
    for f in ("edges_visited", "bfs_started", "bfs_cut", "bfs_finished"):
        assert getattr(a, f) == getattr(b, f), f


def _nb(g):
    nb = oracle.nb_bounds(g)
    return oracle.nb_full_order(g, nb.key), nb.key


def test_b1_equals_sequential_bfscut():
    graphs = [gg.random_graph(2 + s % 20, [0.1, 0.2, 0.4][s % 3], 500 + s, bool(s % 2)) for s in range(120)]
    graphs += [gg.barabasi_albert(600, 3, 5), gg.rmat(10, 8, seed=7), gg.star(12), gg.path(9, True),
               gg.disjoint_union(gg.cycle(6), gg.path(4), gg.path(1))]
    for g in graphs:
        for k in (1, 3, 10):
            seq = oracle.bfscut(g, k)
            bat = oracle.bfscut_batched(g, k, 1)
            assert list(bat.ids) == list(seq.ids) and bat.n_tied == seq.n_tied
            _same_counters(bat.counters, seq.counters)
        order, key = _nb(g)
        seq = oracle.bfscut(g, 5, order=order, lb_key=key)
        bat = oracle.bfscut_batched(g, 5, 1, order=order, lb_key=key)
        assert list(bat.ids) == list(seq.ids)
        _same_counters(bat.counters, seq.counters)


@pytest.mark.parametrize("B", [2, 3, 64, 128])
def test_every_width_equals_textbook(B):
    for s in range(150):
        n = 2 + s % 25
        g = gg.random_graph(n, [0.05, 0.15, 0.3][s % 3], 900 + s, s % 3 == 0)
        for k in (1, 2, n // 2 + 1):
            ref = oracle.textbook_topk(g, k)
            got = oracle.bfscut_batched(g, k, B)
            assert list(got.ids) == list(ref.ids), (s, k)
            assert np.array_equal(got.S, ref.S) and np.array_equal(got.r, ref.r) and got.n_tied == ref.n_tied
            order, key = _nb(g)
            got = oracle.bfscut_batched(g, k, B, order=order, lb_key=key)
            assert list(got.ids) == list(ref.ids) and got.n_tied == ref.n_tied


def test_families_and_seeding_prefix_equal_textbook():
    for g in (gg.hypercube(4), gg.complete_bipartite(3, 5), gg.cycle(15, True), gg.random_tree(80, 4),
              gg.reduction_graph(3, [{0}, {1, 2}, {0, 2}])[0], gg.barabasi_albert(500, 2, 8)):
        for k in (1, 4, 10):
            ref = oracle.textbook_topk(g, k)
            for B, prefix in ((5, 0), (64, 0), (7, 9), (64, 30)):
                got = oracle.bfscut_batched(g, k, B, nocut_prefix=prefix)
                assert list(got.ids) == list(ref.ids) and got.n_tied == ref.n_tied, (g.name, k, B, prefix)
                assert got.counters.bfs_started == got.counters.bfs_cut + got.counters.bfs_finished


@pytest.mark.parametrize("m", [2, 5, 40])
def test_star_counted_by_hand(m):
    # Star: centre 0 with m leaves, k = 1; degree order = centre, then leaves.
    # B = 1: the centre's search expands its level 0 (m arcs) and level 1 (the
    #   m leaves, one arc each) and finishes: x = (S, r) = (m, m + 1).  Each
    #   leaf's level-0 bound is (n - 1) + (n - 2) = 2m - 1 > m: cut before any
    #   arc.  Arcs 2m, started m + 1, cut m, steps 2.
    # B = 2: the centre and leaf 1 are seeded together (no x yet): m + 1 arcs.
    #   Step 1: neither finishes (no x), both continue: m + m arcs.  Step 2: the
    #   centre finishes; x = (m, m + 1) is set BEFORE leaf 1 is tested; leaf 1
    #   has found every vertex (S_2 = 1 + 2(m - 1) = 2m - 1 > m) and is cut.
    #   The other leaves are cut at level 0.  Arcs 3m + 1, steps 2.
    g = gg.star(m + 1)
    one = oracle.bfscut_batched(g, 1, 1)
    assert list(one.ids) == [0] and list(one.S) == [m] and list(one.r) == [m + 1]
    c = one.counters
    assert (c.edges_visited, c.bfs_started, c.bfs_cut, c.bfs_finished, c.levels) == (2 * m, m + 1, m, 1, 2)
    two = oracle.bfscut_batched(g, 1, 2)
    assert list(two.ids) == [0]
    c = two.counters
    assert (c.edges_visited, c.bfs_started, c.bfs_cut, c.bfs_finished, c.levels) == (3 * m + 1, m + 1, m, 1, 2)


def test_directed_path_counted_by_hand():
    # Directed path 0 -> 1 -> ... -> 5, k = 1.  Sources of out-degree >= 1:
    # 0..4 (5 has r = 1).  r(v) = 6 - v, S(v) = (5 - v)(6 - v)/2, so
    # S/(r - 1)^2 = (6 - v)/(2(5 - v)): 1, 3/4, 2/3, 5/8, 3/5 for v = 4..0;
    # vertex 0 is the top-1.  B = 8: one batch of all five searches (5 arcs at
    # seeding).  The search from v finds one vertex per step and finishes at
    # step 6 - v, so x takes the values 1, 3/4, 2/3, 5/8 after steps 2..5.  At
    # every test the surviving search's bound is at most its true
    # S/(r - 1)^2 (for example after step 2, search 0: S_2 = 3, n_2 = 3,
    # gamma = 1, at r = 6: (3 + 3*3 + 2)/25 = 14/25 < 1) and every true value
    # below x is smaller than x, so nothing is cut whatever alpha and omega are.
    # Arcs: each step, every continuing search expands one vertex of
    # out-degree 1 except the one whose newest vertex is 5:
    # 5 (seeding) + 4 + 3 + 2 + 1 + 0 = 15; steps 6.
    g = gg.path(6, directed=True)
    got = oracle.bfscut_batched(g, 1, 8)
    assert list(got.ids) == [0] and list(got.S) == [15] and list(got.r) == [6]
    c = got.counters
    assert (c.edges_visited, c.bfs_started, c.bfs_cut, c.bfs_finished, c.levels) == (15, 5, 0, 5, 6)
