"""Arcs visited under batching, pinned: with options.deterministic = 1 the GPU
runs the batched schedule of Algorithm 1 with Algorithm 4 (B searches advance
one BFS level per step; a step's finished searches enter the top list before
its survivors' cut test) and every counter must equal the CPU oracle's
simulation of that schedule (oracle.bfscut_batched), bit for bit: arcs visited
(the paper's m_vis), searches started, cut and finished, and level steps --
besides the exact top-k itself."""
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
    "rmat16": lambda: gg.rmat(16, 16, seed=gg.workload_seed(1)),
}
_cache = {}


def _graph(name):
    if name not in _cache:
        g = GRAPHS[name]()
        nb = oracle.nb_bounds(g)
        _cache[name] = (g, oracle.nb_full_order(g, nb.key), nb.key)
    return _cache[name]


def _gpu(t, ctx, g, k, bits, order, **extra):
    t.tkc_set_options(ctx, t.Options(batch_bits=bits, order=order, deterministic=1, **extra))
    h = t.tkc_load_csr(ctx, g.n, g.offsets, g.cols, g.directed)
    try:
        return t.tkc_topk_closeness(h, k)
    finally:
        t.tkc_free_graph(h)
        t.tkc_set_options(ctx, t.Options())


def _expect(got, ref, what):
    assert list(got.ids) == list(ref.ids), what
    assert np.array_equal(got.dist_sum, ref.S) and np.array_equal(got.reach, ref.r), what
    assert got.n_tied_at_kth == ref.n_tied, what
    c = ref.counters
    assert (got.edges_visited, got.bfs_started, got.bfs_cut, got.bfs_finished, got.levels) == \
        (c.edges_visited, c.bfs_started, c.bfs_cut, c.bfs_finished, c.levels), what


@pytest.mark.parametrize("bits", [64, 128, 256, 512])
@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_batched_counters_equal_oracle_schedule(gpu_lib, ctx, name, bits):
    t = gpu_lib
    g, nb_order, nb_key = _graph(name)
    for k in (1, 10):
        ref = oracle.bfscut_batched(g, k, bits)
        _expect(_gpu(t, ctx, g, k, bits, t.TKC_ORDER_DEG), ref, (name, "DegCut", bits, k))
        ref = oracle.bfscut_batched(g, k, bits, order=nb_order, lb_key=nb_key)
        _expect(_gpu(t, ctx, g, k, bits, t.TKC_ORDER_NB), ref, (name, "NBCut", bits, k))


def test_plain_and_seeding_prefix(gpu_lib, ctx):
    """B = 1 (the sequential oracle's schedule) and a prefix of searches that
    are never cut (seed_factor * k positions of the order)."""
    t = gpu_lib
    g, nb_order, nb_key = _graph("rmat12")
    ref = oracle.bfscut_batched(g, 10, 1, order=nb_order, lb_key=nb_key)
    _expect(_gpu(t, ctx, g, 10, 1, t.TKC_ORDER_NB), ref, "plain NBCut")
    for bits in (64, 256):
        ref = oracle.bfscut_batched(g, 10, bits, order=nb_order, lb_key=nb_key, nocut_prefix=30)
        _expect(_gpu(t, ctx, g, 10, bits, t.TKC_ORDER_NB, seed_factor=3), ref, ("NB seeded", bits))


def test_deterministic_repeats_and_ignores_teams(gpu_lib, ctx):
    t = gpu_lib
    g, _, _ = _graph("rmat16")
    a = _gpu(t, ctx, g, 10, 128, t.TKC_ORDER_NB)
    b = _gpu(t, ctx, g, 10, 128, t.TKC_ORDER_NB, teams=8)
    assert list(a.ids) == list(b.ids)
    assert (a.edges_visited, a.bfs_cut, a.levels) == (b.edges_visited, b.bfs_cut, b.levels)
