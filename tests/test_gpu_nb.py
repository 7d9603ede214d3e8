"""computeBoundsNB and NBCut on the GPU against the CPU oracle, through the C ABI.

The neighbourhood bounds (S~, r per vertex), their order keys, the NBCut order
and the number of sweeps are integers and must be bit-exact.  Top-k results
under NBCut must equal the textbook (or the oracle's BFSCut at sizes the
textbook cannot reach); one source at a time the device schedule is the
oracle's, so the counters must match too."""
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


def _nb_gpu(tkc, ctx, g, levels):
    h = tkc.tkc_load_csr(ctx, g.n, g.offsets, g.cols, g.directed)
    try:
        return tkc.tkc_nb_bounds(h, g.n, levels)
    finally:
        tkc.tkc_free_graph(h)


def _star_heavy(n, directed):
    # one row of n-1 arcs: far above the warp-per-row limit, so the gather
    # takes the segment path; leaves chained so that levels go deeper
    src = [0] * (n - 1) + list(range(1, n - 1))
    dst = list(range(1, n)) + list(range(2, n))
    return gg.from_arcs(n, src, dst, directed, f"star_chain{n}")


CASES = [
    lambda: gg.path(40), lambda: gg.path(25, directed=True), lambda: gg.cycle(17), lambda: gg.cycle(12, True),
    lambda: gg.star(40), lambda: gg.complete(9), lambda: gg.complete_bipartite(4, 11), lambda: gg.hypercube(6),
    lambda: gg.random_tree(300, 2), lambda: gg.disjoint_union(gg.cycle(5), gg.path(7), gg.path(1), gg.star(4)),
    lambda: gg.reduction_graph(4, [{0, 1}, {2}, {3}, {0, 3}, {1, 2, 3}])[0],
    lambda: gg.from_arcs(7, [], [], True, "empty7"),
    lambda: gg.barabasi_albert(2000, 4, gg.workload_seed(0)),
    lambda: gg.rmat(12, 16, seed=5), lambda: gg.rmat(14, 16, seed=gg.workload_seed(1)),
    lambda: gg.erdos_renyi(5000, 40000, 21, directed=True),
    lambda: _star_heavy(5000, False), lambda: _star_heavy(7000, True),
]


@pytest.mark.parametrize("levels", [0, 1, 2, 3])
@pytest.mark.parametrize("ci", range(len(CASES)))
def test_bounds_equal_oracle(gpu_lib, ctx, ci, levels):
    g = CASES[ci]()
    K = levels or oracle.NB_DEFAULT_LEVELS
    ref = oracle.nb_bounds(g, max_levels=K)
    got = _nb_gpu(gpu_lib, ctx, g, levels)
    assert np.array_equal(got.S, ref.S), g.name
    assert np.array_equal(got.r, ref.r), g.name
    assert np.array_equal(got.key, ref.key), g.name
    assert np.array_equal(got.order, oracle.nb_order(g, ref.key)), g.name
    assert got.levels == ref.levels, (g.name, got.levels, ref.levels)


def test_random_graphs_bounds(gpu_lib, ctx):
    for seed in range(60):
        directed = seed % 3 != 0
        n = 10 + 53 * (seed % 9)
        g = gg.random_graph(n, [1.5, 3.0, 6.0][seed % 3] / n, 11_000 + seed, directed)
        lev = [0, 1, 4][seed % 3]
        ref = oracle.nb_bounds(g, max_levels=lev or oracle.NB_DEFAULT_LEVELS)
        got = _nb_gpu(gpu_lib, ctx, g, lev)
        assert np.array_equal(got.S, ref.S) and np.array_equal(got.r, ref.r), seed
        assert np.array_equal(got.order, oracle.nb_order(g, ref.key)), seed


def _run_nb(tkc, ctx, g, k, bits, teams=0, levels=0):
    tkc.tkc_set_options(ctx, tkc.Options(batch_bits=bits, order=tkc.TKC_ORDER_NB, teams=teams, nb_levels=levels))
    h = tkc.tkc_load_csr(ctx, g.n, g.offsets, g.cols, g.directed)
    try:
        return tkc.tkc_topk_closeness(h, k)
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
        assert got.closeness[i].tobytes() == np.float64(c).tobytes()


def _oracle_nbcut(g, k, levels=oracle.NB_DEFAULT_LEVELS):
    nb = oracle.nb_bounds(g, max_levels=levels)
    order = oracle.nb_order(g, nb.key)
    full = np.concatenate([order, np.nonzero(g.outdeg() == 0)[0].astype(np.uint32)])
    return oracle.bfscut(g, k, full, lb_key=nb.key)


@pytest.mark.parametrize("bits", [1, 64, 512])
@pytest.mark.parametrize("ci", range(12))
def test_nbcut_small_families(gpu_lib, ctx, ci, bits):
    g = CASES[ci]()
    for k in sorted({1, 3, 10, g.n}):
        _expect_equal(_run_nb(gpu_lib, ctx, g, k, bits), oracle.textbook_topk(g, k), g, k)


@pytest.mark.parametrize("bits", [64, 128, 256])
def test_nbcut_random_graphs(gpu_lib, ctx, bits):
    for seed in range(30):
        directed = seed % 2 == 0
        n = 20 + 41 * (seed % 7)
        g = gg.random_graph(n, 2.5 / n, 8100 + seed, directed)
        k = [1, 5, 10, n][seed % 4]
        _expect_equal(_run_nb(gpu_lib, ctx, g, k, bits), oracle.textbook_topk(g, k), g, k)


def test_nbcut_plain_counters_match_oracle(gpu_lib, ctx):
    """One source at a time: the stop and every cut fall where the oracle's do."""
    for seed in range(12):
        directed = seed % 2 == 1
        n = 60 + 10 * seed
        g = gg.random_graph(n, 3.0 / n, 300 + seed, directed)
        ref = _oracle_nbcut(g, 5)
        got = _run_nb(gpu_lib, ctx, g, 5, 1)
        _expect_equal(got, ref, g, 5)
        c = ref.counters
        assert (got.edges_visited, got.bfs_started, got.bfs_cut, got.bfs_finished) == \
            (c.edges_visited, c.bfs_started, c.bfs_cut, c.bfs_finished), seed


def test_nbcut_ba2000_and_rmat16(gpu_lib, ctx):
    g = gg.barabasi_albert(2000, 4, gg.workload_seed(0))
    ref = _oracle_nbcut(g, 10)
    got = _run_nb(gpu_lib, ctx, g, 10, 1)
    _expect_equal(got, ref, g, 10)
    assert got.bfs_started == ref.counters.bfs_started < g.n // 2
    assert got.edges_visited == ref.counters.edges_visited
    _expect_equal(_run_nb(gpu_lib, ctx, g, 10, 64), ref, g, 10)
    g = gg.rmat(16, 16, seed=gg.workload_seed(1))
    ref = _oracle_nbcut(g, 10)
    assert list(ref.ids) == list(oracle.bfscut(g, 10).ids)
    got = _run_nb(gpu_lib, ctx, g, 10, 1)
    _expect_equal(got, ref, g, 10)
    assert got.edges_visited == ref.counters.edges_visited
    for bits, teams in ((64, 0), (512, 1), (64, 4)):
        got = _run_nb(gpu_lib, ctx, g, 10, bits, teams)
        _expect_equal(got, ref, g, 10)
        assert got.bfs_started < int((g.outdeg() > 0).sum())


def test_nbcut_level_cap_and_teams(gpu_lib, ctx):
    g = gg.rmat(13, 16, seed=17)
    ref = oracle.bfscut(g, 20)
    for levels in (1, 2, 5):
        for teams in (1, 3):
            _expect_equal(_run_nb(gpu_lib, ctx, g, 20, 64, teams, levels), ref, g, 20)


def test_nb_degenerate_and_options(gpu_lib, ctx):
    tkc = gpu_lib
    g0 = gg.from_arcs(0, [], [], False)
    got = _nb_gpu(tkc, ctx, g0, 0)
    assert got.levels == 0 and got.order.size == 0
    g1 = gg.from_arcs(1, [], [], True)
    got = _nb_gpu(tkc, ctx, g1, 0)
    assert list(got.r) == [1] and got.order.size == 0
    r = _run_nb(tkc, ctx, gg.path(5), 9, 64)
    assert len(r.ids) == 5 and list(r.ids) == list(oracle.textbook_topk(gg.path(5), 9).ids)
    with pytest.raises(tkc.TkcError):
        tkc.tkc_set_options(ctx, tkc.Options(order=tkc.TKC_ORDER_NB, nb_levels=70000))
    with pytest.raises(tkc.TkcError):
        tkc.tkc_set_options(ctx, tkc.Options(order=5))
    h = tkc.tkc_load_csr(ctx, 5, gg.path(5).offsets, gg.path(5).cols, False)
    try:
        with pytest.raises(tkc.TkcError):
            tkc.tkc_nb_bounds(h, 5, 70000)
    finally:
        tkc.tkc_free_graph(h)


def test_nbcut_many_graphs_in_one_launch(gpu_lib, ctx):
    """Several graphs, NBCut order over their union: each graph stops on its own."""
    tkc = gpu_lib
    gs = [gg.barabasi_albert(900, 3, 41), gg.rmat(11, 16, seed=42), gg.cycle(30), gg.path(12, directed=True),
          gg.erdos_renyi(1500, 12000, 43, directed=True), gg.from_arcs(5, [], [], True, "empty5"),
          gg.random_tree(400, 44), gg.hypercube(5)]
    for bits, teams in ((1, 1), (64, 0), (256, 3)):
        tkc.tkc_set_options(ctx, tkc.Options(batch_bits=bits, order=tkc.TKC_ORDER_NB, teams=teams))
        hs = [tkc.tkc_load_csr(ctx, g.n, g.offsets, g.cols, g.directed) for g in gs]
        try:
            res = tkc.tkc_topk_closeness_multi(ctx, hs, 7)
        finally:
            for h in hs:
                tkc.tkc_free_graph(h)
            tkc.tkc_set_options(ctx, tkc.Options())
        for g, got in zip(gs, res):
            _expect_equal(got, oracle.textbook_topk(g, 7), g, 7)
        big = res[1]
        assert big.bfs_started < int((gs[1].outdeg() > 0).sum())
