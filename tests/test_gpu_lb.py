"""DegBound / NBBound (Algorithm 1 with updateBoundsLB) on the GPU against the
CPU oracle, through the C ABI.  Results must equal the textbook top-k; one
source per round the device takes the oracle's sources in the oracle's order,
so the counters (searches, arcs visited) must match exactly."""
import numpy as np
import pytest

import oracle
from paper_1704_01077_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(gpu_lib):
    c = gpu_lib.tkc_create(gpu_lib.Options())
    yield c
    gpu_lib.tkc_destroy(c)


def _run(tkc, ctx, g, k, bits, nb):
    tkc.tkc_set_options(ctx, tkc.Options(batch_bits=bits, order=tkc.TKC_ORDER_NB if nb else tkc.TKC_ORDER_DEG))
    h = tkc.tkc_load_csr(ctx, g.n, g.offsets, g.cols, g.directed)
    try:
        return tkc.tkc_topk_closeness_bound(h, k)
    finally:
        tkc.tkc_free_graph(h)
        tkc.tkc_set_options(ctx, tkc.Options())


def _expect_equal(got, ref, g, k):
    assert list(got.ids) == list(ref.ids), (g.name, k)
    assert np.array_equal(got.dist_sum, ref.S) and np.array_equal(got.reach, ref.r)
    assert got.n_tied_at_kth == ref.n_tied, (g.name, k, got.n_tied_at_kth, ref.n_tied)
    for i in range(len(ref.ids)):
        f, c = oracle.farness(g.n, ref.S[i], ref.r[i])
        assert got.farness[i].tobytes() == np.float64(f).tobytes()


def _oracle(g, k, nb):
    if not nb:
        return oracle.bfsbound(g, k)
    b = oracle.nb_bounds(g)
    order = oracle.nb_order(g, b.key).tolist() + np.nonzero(g.outdeg() == 0)[0].tolist()
    return oracle.bfsbound(g, k, order, b)


GRAPHS = [lambda: gg.grid(12, 15), lambda: gg.grid(9, 9, directed=True, seed=3, drop=0.25),
          lambda: gg.grid(14, 14, seed=4, drop=0.15), lambda: gg.cycle(20), lambda: gg.hypercube(5),
          lambda: gg.random_tree(120, 2), lambda: gg.star(12), lambda: gg.complete_bipartite(3, 7),
          lambda: gg.disjoint_union(gg.cycle(6), gg.path(9), gg.path(1)), lambda: gg.path(11, directed=True),
          lambda: gg.reduction_graph(3, [{0}, {1, 2}, {0, 2}])[0], lambda: gg.from_arcs(6, [], [], True, "empty6"),
          lambda: gg.barabasi_albert(500, 3, 7)]


@pytest.mark.parametrize("nb", [False, True])
@pytest.mark.parametrize("gi", range(len(GRAPHS)))
def test_plain_rounds_match_oracle(gpu_lib, ctx, gi, nb):
    g = GRAPHS[gi]()
    for k in sorted({1, 3, 10, g.n}):
        ref = _oracle(g, k, nb)
        got = _run(gpu_lib, ctx, g, k, 1, nb)
        _expect_equal(got, oracle.textbook_topk(g, k), g, k)
        c = ref.counters
        assert (got.bfs_started, got.edges_visited) == (c.bfs_started, c.edges_visited), (g.name, k, nb)


@pytest.mark.parametrize("bits", [64, 128, 512])
def test_batched_rounds_equal_textbook(gpu_lib, ctx, bits):
    for gi in range(len(GRAPHS)):
        g = GRAPHS[gi]()
        for k in (1, 10):
            for nb in (False, True):
                _expect_equal(_run(gpu_lib, ctx, g, k, bits, nb), oracle.textbook_topk(g, k), g, k)


def test_random_graphs(gpu_lib, ctx):
    for seed in range(40):
        n = 20 + 17 * (seed % 9)
        g = gg.random_graph(n, 2.5 / n, 13_000 + seed, seed % 2 == 0)
        k = [1, 5, 10, n][seed % 4]
        nb = seed % 3 == 0
        _expect_equal(_run(gpu_lib, ctx, g, k, [1, 64, 128][seed % 3], nb), oracle.textbook_topk(g, k), g, k)


def test_road_like_grid_prunes(gpu_lib, ctx):
    g = gg.grid(60, 60, seed=11, drop=0.1)
    ref = oracle.textbook_topk(g, 10, threads=0)
    for nb in (False, True):
        got = _run(gpu_lib, ctx, g, 10, 64, nb)
        _expect_equal(got, ref, g, 10)
        assert got.bfs_started * 4 < g.n


def test_bound_rejects_other_orders(gpu_lib, ctx):
    tkc = gpu_lib
    g = gg.grid(4, 4)
    tkc.tkc_set_options(ctx, tkc.Options(order=tkc.TKC_ORDER_GIVEN))
    h = tkc.tkc_load_csr(ctx, g.n, g.offsets, g.cols, g.directed)
    try:
        with pytest.raises(tkc.TkcError):
            tkc.tkc_topk_closeness_bound(h, 3)
    finally:
        tkc.tkc_free_graph(h)
        tkc.tkc_set_options(ctx, tkc.Options())


def test_several_teams_per_round(gpu_lib, ctx):
    """Rounds where several teams each run one batch: the same top-k."""
    tkc = gpu_lib
    for g in (gg.grid(30, 40, seed=5, drop=0.1), gg.grid(12, 12, directed=True, seed=6, drop=0.2),
              gg.barabasi_albert(700, 3, 8), gg.random_tree(400, 9)):
        ref = oracle.textbook_topk(g, 10)
        for bits, teams, nb in ((64, 2, False), (64, 3, True), (128, 4, False), (256, 2, True)):
            tkc.tkc_set_options(ctx, tkc.Options(batch_bits=bits, teams=teams,
                                                 order=tkc.TKC_ORDER_NB if nb else tkc.TKC_ORDER_DEG))
            h = tkc.tkc_load_csr(ctx, g.n, g.offsets, g.cols, g.directed)
            try:
                got = tkc.tkc_topk_closeness_bound(h, 10)
            finally:
                tkc.tkc_free_graph(h)
                tkc.tkc_set_options(ctx, tkc.Options())
            _expect_equal(got, ref, g, 10)
