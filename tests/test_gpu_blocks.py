"""Both block sizes of the search kernel against the CPU oracle, on graphs small
enough for the textbook top-k.  By default the larger blocks (1024 threads for
64-bit batches, 768 for 128-bit) run only on graphs of 2^20 vertices or more;
options.large_blocks = 1 forces them here, 2 forces 512 threads, so every
variant of the kernel is checked bit for bit on every path: closeness with
the degree and NB orders, several teams, harmonic centrality, updateBoundsLB
rounds and many graphs in one launch."""
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


def _expect_equal(got, ref, g, k):
    assert list(got.ids) == list(ref.ids), (g.name, k)
    assert np.array_equal(got.dist_sum, ref.S) and np.array_equal(got.reach, ref.r), (g.name, k)
    assert got.n_tied_at_kth == ref.n_tied, (g.name, k, got.n_tied_at_kth, ref.n_tied)
    for i in range(len(ref.ids)):
        f, c = oracle.farness(g.n, ref.S[i], ref.r[i])
        assert got.farness[i].tobytes() == np.float64(f).tobytes()


def _one(tkc, ctx, g, opts, fn):
    tkc.tkc_set_options(ctx, opts)
    h = tkc.tkc_load_csr(ctx, g.n, g.offsets, g.cols, g.directed)
    try:
        return fn(h)
    finally:
        tkc.tkc_free_graph(h)
        tkc.tkc_set_options(ctx, tkc.Options())


GRAPHS = [lambda: gg.path(17), lambda: gg.cycle(8, True), lambda: gg.star(30), lambda: gg.hypercube(5),
          lambda: gg.complete_bipartite(3, 9), lambda: gg.random_tree(150, 4),
          lambda: gg.disjoint_union(gg.cycle(5), gg.path(7), gg.path(1), gg.star(4)),
          lambda: gg.reduction_graph(4, [{0, 1}, {2}, {3}, {0, 3}, {1, 2, 3}])[0],
          lambda: gg.from_arcs(7, [], [], True, "empty7"), lambda: gg.barabasi_albert(2000, 4, gg.workload_seed(0)),
          lambda: gg.rmat(12, 16, seed=5), lambda: gg.grid(20, 30, seed=3, drop=0.1)]


@pytest.mark.parametrize("large", [1, 2])
@pytest.mark.parametrize("bits", [64, 128])
@pytest.mark.parametrize("gi", range(len(GRAPHS)))
def test_closeness_both_orders(gpu_lib, ctx, gi, bits, large):
    t = gpu_lib
    g = GRAPHS[gi]()
    for k in sorted({1, 10, min(g.n, 300)}):
        ref = oracle.textbook_topk(g, k)
        for order in (t.TKC_ORDER_DEG, t.TKC_ORDER_NB):
            got = _one(t, ctx, g, t.Options(batch_bits=bits, order=order, large_blocks=large),
                       lambda h: t.tkc_topk_closeness(h, k))
            _expect_equal(got, ref, g, k)


@pytest.mark.parametrize("large", [1, 2])
def test_random_graphs(gpu_lib, ctx, large):
    t = gpu_lib
    for seed in range(30):
        n = 20 + 37 * (seed % 7)
        g = gg.random_graph(n, 2.5 / n, 9100 + seed, seed % 2 == 0)
        k = [1, 5, 10, n][seed % 4]
        bits = [64, 128][seed % 2]
        order = [t.TKC_ORDER_DEG, t.TKC_ORDER_NB][(seed // 2) % 2]
        got = _one(t, ctx, g, t.Options(batch_bits=bits, order=order, large_blocks=large),
                   lambda h: t.tkc_topk_closeness(h, k))
        _expect_equal(got, oracle.textbook_topk(g, k), g, k)


@pytest.mark.parametrize("teams,bits", [(2, 64), (4, 128), (8, 64)])
def test_teams_large_blocks(gpu_lib, ctx, teams, bits):
    t = gpu_lib
    for g in (gg.rmat(13, 16, seed=gg.workload_seed(1) + teams), gg.barabasi_albert(6000, 4, teams),
              gg.random_graph(400, 0.01, 31 + teams, True)):
        ref = oracle.textbook_topk(g, 10, threads=0)
        for order in (t.TKC_ORDER_DEG, t.TKC_ORDER_NB):
            got = _one(t, ctx, g, t.Options(batch_bits=bits, teams=teams, order=order, large_blocks=1),
                       lambda h: t.tkc_topk_closeness(h, 10))
            _expect_equal(got, ref, g, 10)


@pytest.mark.parametrize("large", [1, 2])
def test_harmonic(gpu_lib, ctx, large):
    t = gpu_lib
    for gi in (0, 1, 3, 6, 9, 10, 11):
        g = GRAPHS[gi]()
        ref = oracle.textbook_harmonic_topk(g, 10)
        for bits, order in ((64, t.TKC_ORDER_DEG), (128, t.TKC_ORDER_NB)):
            got = _one(t, ctx, g, t.Options(batch_bits=bits, order=order, large_blocks=large),
                       lambda h: t.tkc_topk_harmonic(h, 10))
            assert list(got.ids) == list(ref.ids), g.name
            assert got.closeness.tobytes() == np.asarray(ref.H, dtype=np.float64).tobytes(), g.name
            assert np.array_equal(got.reach, ref.r) and got.n_tied_at_kth == ref.n_tied, g.name


@pytest.mark.parametrize("large", [1, 2])
def test_update_bounds_lb(gpu_lib, ctx, large):
    t = gpu_lib
    for g in (gg.grid(30, 40, seed=5, drop=0.1), gg.grid(12, 12, directed=True, seed=6, drop=0.2),
              gg.barabasi_albert(700, 3, 8)):
        ref = oracle.textbook_topk(g, 10)
        for bits, teams, order in ((64, 2, t.TKC_ORDER_DEG), (128, 3, t.TKC_ORDER_NB), (1, 0, t.TKC_ORDER_DEG)):
            got = _one(t, ctx, g, t.Options(batch_bits=bits, teams=teams, order=order, large_blocks=large),
                       lambda h: t.tkc_topk_closeness_bound(h, 10))
            _expect_equal(got, ref, g, 10)


@pytest.mark.parametrize("large", [1, 2])
def test_many_graphs_one_launch(gpu_lib, ctx, large):
    t = gpu_lib
    graphs = [gg.barabasi_albert(900, 3, 41), gg.rmat(11, 16, seed=42), gg.cycle(30), gg.path(12, directed=True),
              gg.erdos_renyi(1500, 12000, 43, directed=True), gg.from_arcs(4, [], [], True, "isolated4"),
              gg.grid(15, 15, seed=44, drop=0.1)]
    for bits, order in ((64, t.TKC_ORDER_DEG), (128, t.TKC_ORDER_NB)):
        t.tkc_set_options(ctx, t.Options(batch_bits=bits, order=order, large_blocks=large))
        hs = [t.tkc_load_csr(ctx, g.n, g.offsets, g.cols, g.directed) for g in graphs]
        try:
            res = t.tkc_topk_closeness_multi(ctx, hs, 10)
        finally:
            for h in hs:
                t.tkc_free_graph(h)
            t.tkc_set_options(ctx, t.Options())
        for g, r in zip(graphs, res):
            _expect_equal(r, oracle.textbook_topk(g, 10), g, 10)


def test_option_is_validated(gpu_lib):
    t = gpu_lib
    with pytest.raises(t.TkcError):
        t.tkc_create(t.Options(large_blocks=3))
