"""Top-k harmonic centrality on the GPU against the CPU oracle, through the C ABI.

h(v) is an FP64 value formed the same way on both sides (per-level counts over
level, added in increasing level), so ids, h bits, reach and tie counts must be
identical; 1/h is one correctly rounded quotient on both sides.  One source at a
time the device schedule is the oracle's, so the counters must match too."""
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


def _run(tkc, ctx, g, k, bits, order, teams=0, levels=0):
    tkc.tkc_set_options(ctx, tkc.Options(batch_bits=bits, order=order, teams=teams, nb_levels=levels))
    h = tkc.tkc_load_csr(ctx, g.n, g.offsets, g.cols, g.directed)
    try:
        return tkc.tkc_topk_harmonic(h, k)
    finally:
        tkc.tkc_free_graph(h)
        tkc.tkc_set_options(ctx, tkc.Options())


def _expect_equal(got, ref, g, k):
    assert list(got.ids) == list(ref.ids), (g.name, k)
    assert got.closeness.tobytes() == np.asarray(ref.H, dtype=np.float64).tobytes(), g.name
    assert np.array_equal(got.reach, ref.r), g.name
    assert got.n_tied_at_kth == ref.n_tied, (g.name, k, got.n_tied_at_kth, ref.n_tied)
    for i, hv in enumerate(ref.H):
        want = np.float64(1.0 / hv) if hv > 0 else np.float64(np.inf)
        assert got.farness[i].tobytes() == want.tobytes()
    assert not np.any(got.dist_sum)


SMALL = [
    lambda: gg.path(17), lambda: gg.path(12, directed=True), lambda: gg.cycle(9), lambda: gg.cycle(8, True),
    lambda: gg.star(30), lambda: gg.complete(6), lambda: gg.complete_bipartite(3, 9), lambda: gg.hypercube(5),
    lambda: gg.random_tree(150, 4), lambda: gg.disjoint_union(gg.cycle(5), gg.path(7), gg.path(1), gg.star(4)),
    lambda: gg.reduction_graph(4, [{0, 1}, {2}, {3}, {0, 3}, {1, 2, 3}])[0],
    lambda: gg.from_arcs(7, [], [], True, "empty7"),
]


@pytest.mark.parametrize("nb", [False, True])
@pytest.mark.parametrize("bits", [1, 64, 512])
@pytest.mark.parametrize("gi", range(len(SMALL)))
def test_small_families(gpu_lib, ctx, gi, bits, nb):
    g = SMALL[gi]()
    order = gpu_lib.TKC_ORDER_NB if nb else gpu_lib.TKC_ORDER_DEG
    for k in sorted({1, 3, 10, g.n}):
        _expect_equal(_run(gpu_lib, ctx, g, k, bits, order), oracle.textbook_harmonic_topk(g, k), g, k)


@pytest.mark.parametrize("bits", [64, 128, 256])
def test_random_graphs(gpu_lib, ctx, bits):
    for seed in range(40):
        directed = seed % 2 == 0
        n = 20 + 37 * (seed % 7)
        g = gg.random_graph(n, 2.5 / n, 9100 + seed, directed)
        k = [1, 5, 10, n][seed % 4]
        order = gpu_lib.TKC_ORDER_NB if seed % 3 else gpu_lib.TKC_ORDER_DEG
        _expect_equal(_run(gpu_lib, ctx, g, k, bits, order), oracle.textbook_harmonic_topk(g, k), g, k)


def _oracle_nb(g, k, levels=oracle.NB_DEFAULT_LEVELS):
    nb = oracle.nb_bounds(g, max_levels=levels)
    order = oracle.nb_harmonic_order(g, nb.h_ub)
    full = np.concatenate([order, np.nonzero(g.outdeg() == 0)[0].astype(np.uint32)])
    return oracle.bfscut_harmonic(g, k, full, nb.h_ub)


def test_plain_counters_match_oracle(gpu_lib, ctx):
    tkc = gpu_lib
    for seed in range(12):
        directed = seed % 2 == 1
        n = 60 + 10 * seed
        g = gg.random_graph(n, 3.0 / n, 500 + seed, directed)
        for nb in (False, True):
            ref = _oracle_nb(g, 5) if nb else oracle.bfscut_harmonic(g, 5)
            got = _run(tkc, ctx, g, 5, 1, tkc.TKC_ORDER_NB if nb else tkc.TKC_ORDER_DEG)
            _expect_equal(got, ref, g, 5)
            c = ref.counters
            assert (got.edges_visited, got.bfs_started, got.bfs_cut, got.bfs_finished) == \
                (c.edges_visited, c.bfs_started, c.bfs_cut, c.bfs_finished), (seed, nb)


NB_CASES = [lambda: gg.path(40), lambda: gg.cycle(12, True), lambda: gg.hypercube(6), lambda: gg.random_tree(300, 2),
            lambda: gg.barabasi_albert(2000, 4, gg.workload_seed(0)), lambda: gg.rmat(12, 16, seed=5),
            lambda: gg.erdos_renyi(5000, 40000, 21, directed=True),
            lambda: gg.reduction_graph(4, [{0, 1}, {2}, {3}, {0, 3}, {1, 2, 3}])[0]]


@pytest.mark.parametrize("levels", [0, 2])
@pytest.mark.parametrize("ci", range(len(NB_CASES)))
def test_nb_harmonic_bounds_equal_oracle(gpu_lib, ctx, ci, levels):
    g = NB_CASES[ci]()
    ref = oracle.nb_bounds(g, max_levels=levels or oracle.NB_DEFAULT_LEVELS)
    h = gpu_lib.tkc_load_csr(ctx, g.n, g.offsets, g.cols, g.directed)
    try:
        hub, order = gpu_lib.tkc_nb_harmonic_bounds(h, g.n, levels)
    finally:
        gpu_lib.tkc_free_graph(h)
    assert hub.tobytes() == ref.h_ub.tobytes(), g.name
    assert np.array_equal(order, oracle.nb_harmonic_order(g, ref.h_ub)), g.name


def test_ba2000_and_rmat16(gpu_lib, ctx):
    tkc = gpu_lib
    g = gg.barabasi_albert(2000, 4, gg.workload_seed(0))
    ref = oracle.textbook_harmonic_topk(g, 10)
    for bits, order in ((1, tkc.TKC_ORDER_DEG), (1, tkc.TKC_ORDER_NB), (64, tkc.TKC_ORDER_NB)):
        _expect_equal(_run(tkc, ctx, g, 10, bits, order), ref, g, 10)
    g = gg.rmat(16, 16, seed=gg.workload_seed(1))
    ref = oracle.bfscut_harmonic(g, 10)
    got = _run(tkc, ctx, g, 10, 1, tkc.TKC_ORDER_DEG)
    _expect_equal(got, ref, g, 10)
    assert got.edges_visited == ref.counters.edges_visited
    for bits, order, teams in ((64, tkc.TKC_ORDER_DEG, 0), (64, tkc.TKC_ORDER_NB, 0), (512, tkc.TKC_ORDER_NB, 1),
                               (128, tkc.TKC_ORDER_NB, 4)):
        _expect_equal(_run(tkc, ctx, g, 10, bits, order, teams), ref, g, 10)


def test_many_graphs_in_one_launch(gpu_lib, ctx):
    tkc = gpu_lib
    gs = [gg.barabasi_albert(900, 3, 41), gg.rmat(11, 16, seed=42), gg.cycle(30), gg.path(12, directed=True),
          gg.erdos_renyi(1500, 12000, 43, directed=True), gg.from_arcs(5, [], [], True, "empty5"),
          gg.random_tree(400, 44), gg.hypercube(5)]
    for bits, order, teams in ((1, tkc.TKC_ORDER_DEG, 1), (64, tkc.TKC_ORDER_NB, 0), (256, tkc.TKC_ORDER_DEG, 3)):
        tkc.tkc_set_options(ctx, tkc.Options(batch_bits=bits, order=order, teams=teams))
        hs = [tkc.tkc_load_csr(ctx, g.n, g.offsets, g.cols, g.directed) for g in gs]
        try:
            res = tkc.tkc_topk_harmonic_multi(ctx, hs, 7)
        finally:
            for h in hs:
                tkc.tkc_free_graph(h)
            tkc.tkc_set_options(ctx, tkc.Options())
        for g, got in zip(gs, res):
            _expect_equal(got, oracle.textbook_harmonic_topk(g, 7), g, 7)
