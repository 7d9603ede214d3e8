"""The search kernel's in-degree labelling (options.relabel = 1), forced on for
graphs the oracle can check, through the C ABI.

With relabel on, the search walks a copy of the graph whose vertices are
numbered by in-degree; sources, slots, list entries and ties keep the graph's
own ids.  So every result must equal the oracle's exactly, as without it: the
top-k ids, S, r, tie counts and farness bits against the textbook; and, under
the deterministic schedule, every counter against the oracle's simulation of
the batched Algorithm 1 (the counters do not depend on vertex labels).  Also
covered: harmonic centrality, the multi-graph launch, updateBoundsLB (whose
level records are written by id), complete distance sums, and a graph whose
in-degree order is far from its id order (a reversed star and a directed
path)."""
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


GRAPHS = {
    "ba2000": lambda: gg.barabasi_albert(2000, 4, gg.workload_seed(0)),
    "rmat12": lambda: gg.rmat(12, 16, seed=gg.workload_seed(1)),
    "rmat14": lambda: gg.rmat(14, 16, seed=gg.workload_seed(1) ^ 14),
    "er3000": lambda: gg.erdos_renyi(3000, 24000, seed=77),
    "in_star": lambda: gg.from_arcs(40, np.arange(1, 40), np.zeros(39, np.int64), True, "in_star"),
    "dpath": lambda: gg.path(300, directed=True),
    "union": lambda: gg.disjoint_union(gg.cycle(7), gg.path(9), gg.path(1), gg.star(5)),
}
_cache = {}


def _graph(name):
    if name not in _cache:
        _cache[name] = GRAPHS[name]()
    return _cache[name]


def _opts(t, **kw):
    return t.Options(relabel=1, **kw)


def _load(t, ctx, g):
    return t.tkc_load_csr(ctx, g.n, g.offsets, g.cols, g.directed)


def _expect_topk(got, ref, g, what):
    assert list(got.ids) == list(ref.ids), what
    assert np.array_equal(got.dist_sum, ref.S) and np.array_equal(got.reach, ref.r), what
    assert got.n_tied_at_kth == ref.n_tied, what
    for i in range(len(ref.ids)):
        f, _ = oracle.farness(g.n, ref.S[i], ref.r[i])
        assert got.farness[i].tobytes() == np.float64(f).tobytes(), what


@pytest.mark.parametrize("bits", [64, 128, 256, 512])
@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_topk_equals_textbook(gpu_lib, ctx, name, bits):
    t = gpu_lib
    g = _graph(name)
    for order in (t.TKC_ORDER_DEG, t.TKC_ORDER_NB):
        t.tkc_set_options(ctx, _opts(t, batch_bits=bits, order=order))
        h = _load(t, ctx, g)
        try:
            for k in sorted({1, 10, min(100, g.n)}):
                _expect_topk(t.tkc_topk_closeness(h, k), oracle.textbook_topk(g, k), g, (name, bits, order, k))
        finally:
            t.tkc_free_graph(h)
            t.tkc_set_options(ctx, t.Options())


@pytest.mark.parametrize("bits", [64, 128, 512])
@pytest.mark.parametrize("name", ["ba2000", "rmat12", "rmat14"])
def test_deterministic_counters_equal_oracle_schedule(gpu_lib, ctx, name, bits):
    t = gpu_lib
    g = _graph(name)
    nb = oracle.nb_bounds(g)
    nb_order = oracle.nb_full_order(g, nb.key)
    for order, ref in ((t.TKC_ORDER_DEG, oracle.bfscut_batched(g, 10, bits)),
                       (t.TKC_ORDER_NB, oracle.bfscut_batched(g, 10, bits, order=nb_order, lb_key=nb.key))):
        t.tkc_set_options(ctx, _opts(t, batch_bits=bits, order=order, deterministic=1))
        h = _load(t, ctx, g)
        try:
            got = t.tkc_topk_closeness(h, 10)
        finally:
            t.tkc_free_graph(h)
            t.tkc_set_options(ctx, t.Options())
        _expect_topk(got, ref, g, (name, bits, order))
        c = ref.counters
        assert (got.edges_visited, got.bfs_started, got.bfs_cut, got.bfs_finished, got.levels) == \
            (c.edges_visited, c.bfs_started, c.bfs_cut, c.bfs_finished, c.levels), (name, bits, order)


def test_same_results_and_counters_with_and_without_labels(gpu_lib, ctx):
    """One graph, both labellings, deterministic schedule: identical results and
    identical label-free counters; only edges_scanned may differ."""
    t = gpu_lib
    g = _graph("rmat14")
    out = {}
    for relabel in (1, 2):
        t.tkc_set_options(ctx, t.Options(batch_bits=128, order=t.TKC_ORDER_NB, deterministic=1, relabel=relabel))
        h = _load(t, ctx, g)
        try:
            out[relabel] = t.tkc_topk_closeness(h, 10)
        finally:
            t.tkc_free_graph(h)
            t.tkc_set_options(ctx, t.Options())
    a, b = out[1], out[2]
    assert list(a.ids) == list(b.ids) and np.array_equal(a.dist_sum, b.dist_sum)
    assert (a.edges_visited, a.bfs_started, a.bfs_cut, a.levels) == (b.edges_visited, b.bfs_started, b.bfs_cut,
                                                                     b.levels)


@pytest.mark.parametrize("name", ["ba2000", "rmat12", "union", "dpath"])
def test_harmonic_equals_textbook(gpu_lib, ctx, name):
    t = gpu_lib
    g = _graph(name)
    for order in (t.TKC_ORDER_DEG, t.TKC_ORDER_NB):
        t.tkc_set_options(ctx, _opts(t, batch_bits=128, order=order))
        h = _load(t, ctx, g)
        try:
            got = t.tkc_topk_harmonic(h, 10)
        finally:
            t.tkc_free_graph(h)
            t.tkc_set_options(ctx, t.Options())
        ref = oracle.textbook_harmonic_topk(g, 10)
        assert list(got.ids) == list(ref.ids), (name, order)
        assert got.closeness.tobytes() == np.asarray(ref.H, dtype=np.float64).tobytes(), (name, order)
        assert np.array_equal(got.reach, ref.r) and got.n_tied_at_kth == ref.n_tied, (name, order)


def test_multi_graph_launch(gpu_lib, ctx):
    t = gpu_lib
    gs = [gg.barabasi_albert(300 + 50 * i, 4, 100 + i) if i % 2 == 0 else
          gg.erdos_renyi(300 + 50 * i, 8 * (300 + 50 * i), seed=200 + i) for i in range(8)]
    for order in (t.TKC_ORDER_DEG, t.TKC_ORDER_NB):
        t.tkc_set_options(ctx, _opts(t, batch_bits=128, order=order))
        hs = [_load(t, ctx, g) for g in gs]
        try:
            res = t.tkc_topk_closeness_multi(ctx, hs, 10)
        finally:
            for h in hs:
                t.tkc_free_graph(h)
            t.tkc_set_options(ctx, t.Options())
        for g, got in zip(gs, res):
            _expect_topk(got, oracle.textbook_topk(g, 10), g, (g.name, order))


@pytest.mark.parametrize("nb", [False, True])
def test_update_bounds_lb(gpu_lib, ctx, nb):
    """updateBoundsLB records each vertex's discovery level by vertex id."""
    t = gpu_lib
    for g in (gg.grid(14, 14, seed=4, drop=0.15), gg.grid(9, 9, directed=True, seed=3, drop=0.25),
              _graph("in_star"), gg.barabasi_albert(500, 3, 7)):
        t.tkc_set_options(ctx, _opts(t, batch_bits=64, order=t.TKC_ORDER_NB if nb else t.TKC_ORDER_DEG))
        h = _load(t, ctx, g)
        try:
            got = t.tkc_topk_closeness_bound(h, 5)
        finally:
            t.tkc_free_graph(h)
            t.tkc_set_options(ctx, t.Options())
        _expect_topk(got, oracle.textbook_topk(g, 5), g, (g.name, nb))


@pytest.mark.parametrize("name", ["rmat12", "ba2000", "dpath"])
def test_distance_sums(gpu_lib, ctx, name):
    t = gpu_lib
    g = _graph(name)
    src = np.arange(0, g.n, 7, dtype=np.uint32)
    t.tkc_set_options(ctx, _opts(t, batch_bits=128))
    h = _load(t, ctx, g)
    try:
        S, r = t.tkc_distance_sums(h, src)
    finally:
        t.tkc_free_graph(h)
        t.tkc_set_options(ctx, t.Options())
    S0, r0 = oracle.bfs_sums(g, src)
    assert np.array_equal(S, S0) and np.array_equal(r, r0)


def test_one_handle_switching_labellings(gpu_lib, ctx):
    """One graph handle searched with the labelling, without it, and with it
    again (the copy is built alongside the preprocessing, dropped, rebuilt),
    then freed right after a call: every result equals the textbook."""
    t = gpu_lib
    g = _graph("rmat14")
    ref = oracle.textbook_topk(g, 10)
    h = _load(t, ctx, g)
    try:
        for relabel in (1, 2, 1, 0):
            t.tkc_set_options(ctx, t.Options(batch_bits=128, order=t.TKC_ORDER_NB, relabel=relabel))
            _expect_topk(t.tkc_topk_closeness(h, 10), ref, g, relabel)
            S, r = t.tkc_distance_sums(h, np.asarray(ref.ids, np.uint32))
            assert np.array_equal(S, ref.S) and np.array_equal(r, ref.r), relabel
    finally:
        t.tkc_free_graph(h)
        t.tkc_set_options(ctx, t.Options())
    h = _load(t, ctx, g)
    t.tkc_set_options(ctx, t.Options(batch_bits=128, relabel=1))
    try:
        _expect_topk(t.tkc_topk_closeness(h, 10), oracle.textbook_topk(g, 10), g, "fresh")
    finally:
        t.tkc_free_graph(h)
        t.tkc_set_options(ctx, t.Options())
