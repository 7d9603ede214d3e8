"""The seeded input generators, on the CPU: splitmix64 against its published
outputs, the CSR contract every generator promises (sorted rows, no self-loops
or duplicates, symmetric when undirected), the recipe facts quoted for the
workloads (BA n = 2 000 has 7 990 edges and is connected; grid edge counts),
determinism in the seed and independence from the thread count."""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1704_01077_gb300 import graphgen as gg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_splitmix64_published_outputs():
    # the first outputs of splitmix64 from state 0 (Steele, Lea, Flood 2014;
    # the values every reference implementation prints)
    golden = 0x9E3779B97F4A7C15
    want = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    state = 0
    for w in want:
        assert gg.splitmix64(state) == w
        state = (state + golden) & 0xFFFFFFFFFFFFFFFF


def _csr_ok(g):
    off = np.asarray(g.offsets, dtype=np.int64)
    col = np.asarray(g.cols, dtype=np.int64)
    assert off[0] == 0 and np.all(np.diff(off) >= 0) and off[-1] == len(col)
    assert col.size == 0 or (col.min() >= 0 and col.max() < g.n)
    rows = np.repeat(np.arange(g.n), np.diff(off))
    assert not np.any(rows == col), "self-loop"
    # strictly increasing inside each row: sorted and duplicate-free
    same_row = rows[1:] == rows[:-1]
    assert np.all(col[1:][same_row] > col[:-1][same_row])
    if not g.directed:
        fwd = set(zip(rows.tolist(), col.tolist()))
        assert all((b, a) in fwd for a, b in fwd), "asymmetric"


@pytest.mark.parametrize("make", [
    lambda: gg.barabasi_albert(2000, 4, gg.workload_seed(0)),
    lambda: gg.rmat(12, 16, seed=3),
    lambda: gg.rmat(10, 8, seed=4, directed=False),
    lambda: gg.erdos_renyi(3000, 24000, 5, directed=True),
    lambda: gg.erdos_renyi(1000, 4000, 6, directed=False),
    lambda: gg.grid(13, 17, seed=7, drop=0.2),
    lambda: gg.grid(9, 11, directed=True, seed=8, drop=0.25),
    lambda: gg.random_tree(300, 9),
    lambda: gg.random_graph(200, 0.03, 10, True),
    lambda: gg.hypercube(6),
])
def test_csr_contract(make):
    _csr_ok(make())


def test_ba2000_recipe():
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import connected_components

    g = gg.barabasi_albert(2000, 4, gg.workload_seed(0))
    assert g.arcs == 2 * 7990
    assert int(g.outdeg().min()) >= 4
    m = csr_matrix((np.ones(g.arcs), np.asarray(g.cols), np.asarray(g.offsets)), shape=(g.n, g.n))
    assert connected_components(m, directed=False)[0] == 1


def test_rmat_recipe():
    g = gg.rmat(12, 16, seed=gg.workload_seed(1))
    assert g.n == 4096 and 0 < g.arcs <= 16 * 4096
    # skewed: the top 1% of vertices by out-degree hold far more than 1% of the arcs
    d = np.sort(g.outdeg())[::-1]
    assert d[: g.n // 100].sum() > 0.1 * g.arcs


def test_grid_edge_counts():
    for r, c in ((1, 1), (1, 5), (4, 4), (7, 3)):
        g = gg.grid(r, c)
        assert g.arcs == 2 * (r * (c - 1) + c * (r - 1))
        gd = gg.grid(r, c, directed=True)
        assert gd.arcs == g.arcs
    assert gg.grid(30, 30, seed=1, drop=0.1).arcs < gg.grid(30, 30).arcs


def test_deterministic_in_the_seed():
    a, b, c = gg.rmat(11, 8, seed=5), gg.rmat(11, 8, seed=5), gg.rmat(11, 8, seed=6)
    assert np.array_equal(a.offsets, b.offsets) and np.array_equal(a.cols, b.cols)
    assert not (np.array_equal(a.offsets, c.offsets) and np.array_equal(a.cols, c.cols))
    s = gg.log_uniform_sizes(64, 1000, 200000, 11)
    assert s == gg.log_uniform_sizes(64, 1000, 200000, 11)
    assert all(1000 <= x < 200000 for x in s)


def test_independent_of_thread_count():
    code = ("import hashlib, sys; sys.path.insert(0, %r); from paper_1704_01077_gb300 import graphgen as gg; "
            "h = hashlib.sha256(); "
            "[h.update(x.offsets.tobytes() + x.cols.tobytes()) for x in "
            "(gg.rmat(14, 16, seed=2), gg.barabasi_albert(20000, 5, 3), gg.erdos_renyi(20000, 160000, 4))]; "
            "print(h.hexdigest())") % ROOT
    out = []
    for threads in ("1", "4"):
        env = dict(os.environ, OMP_NUM_THREADS=threads)
        out.append(subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                                  check=True).stdout.strip())
    assert out[0] == out[1] and len(out[0]) == 64
