"""Pins of the feature oracle's core numbers (oracle/features.py): networkx's
core_number on undirected graphs and on digraphs (whose degree networkx takes
as in-degree + out-degree, both neighbour lists, as the feature does), closed
forms, and the h-index fixed point the GPU iteration stops at (Lu et al.
2016: the core numbers are the fixed point reached from the degrees)."""
import networkx as nx
import numpy as np
import pytest

from oracle import features
from paper_1704_01077_gb300 import graphgen as gg


def _nx(g):
    G = nx.DiGraph() if g.directed else nx.Graph()
    G.add_nodes_from(range(g.n))
    off = g.offsets.astype(np.int64)
    for v in range(g.n):
        for w in g.cols[off[v]:off[v + 1]]:
            G.add_edge(v, int(w))
    return G


CASES = [lambda s=s: gg.random_graph(30 + s % 17, [0.05, 0.12, 0.3][s % 3], 70 + s, s % 2 == 1) for s in range(30)]
CASES += [lambda: gg.barabasi_albert(400, 3, 2), lambda: gg.rmat(10, 8, seed=3), lambda: gg.rmat(9, 16, seed=4),
          lambda: gg.erdos_renyi(300, 1500, 5, directed=True)]


@pytest.mark.parametrize("ci", range(len(CASES)))
def test_core_numbers_equal_networkx(ci):
    g = CASES[ci]()
    want = nx.core_number(_nx(g))
    got = features.core_numbers(g)
    assert [int(got[v]) for v in range(g.n)] == [want[v] for v in range(g.n)]


def test_closed_forms():
    assert set(features.core_numbers(gg.complete(7)).tolist()) == {6}
    assert set(features.core_numbers(gg.complete(5, directed=True)).tolist()) == {8}  # both arcs: 2 (n - 1)
    assert set(features.core_numbers(gg.cycle(11)).tolist()) == {2}
    assert set(features.core_numbers(gg.random_tree(50, 3)).tolist()) == {1}
    assert set(features.core_numbers(gg.star(9)).tolist()) == {1}
    assert features.core_numbers(gg.from_arcs(4, [], [], True)).tolist() == [0, 0, 0, 0]


def test_h_index_fixed_point():
    for ci in (0, 5, 31, 32):
        g = CASES[ci]()
        c = features.core_numbers(g)
        off = g.offsets.astype(np.int64)
        nbrs = [list(g.cols[off[v]:off[v + 1]]) for v in range(g.n)]
        if g.directed:
            for v in range(g.n):
                for w in g.cols[off[v]:off[v + 1]]:
                    nbrs[int(w)].append(v)
        for v in range(g.n):
            vals = sorted((int(c[w]) for w in nbrs[v]), reverse=True)
            h = max([i + 1 for i, x in enumerate(vals) if x >= i + 1], default=0)
            assert h == c[v], (ci, v)
