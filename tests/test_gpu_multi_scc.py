"""Many directed graphs with many strongly connected components each, in one
multi-graph launch, through the C ABI.

The union's reach bounds start with one forward-backward search from a pivot
in every graph at once; the rest of each graph's SCCs come from trimming and
colouring.  Whatever the pivots, every result must equal the textbook top-k of
each graph on its own (ids, S, r, ties, farness bits), under both orders and
several batch widths, including graphs whose lists end with vertices of
out-degree 0."""
import numpy as np
import pytest

import oracle
from paper_1704_01077_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu


def _graphs():
    gs = []
    for i in range(6):
        gs.append(gg.rmat(10 + (i % 3), 8, seed=3000 + i))
    gs.append(gg.path(40, directed=True))
    gs.append(gg.cycle(25, True))
    gs.append(gg.reduction_graph(4, [{0, 1}, {2}, {3}, {0, 3}, {1, 2, 3}])[0])
    # a chain of directed cycles: every cycle an SCC, each reaching the next
    src, dst = [], []
    for c in range(8):
        b = 6 * c
        for j in range(6):
            src.append(b + j)
            dst.append(b + (j + 1) % 6)
        if c < 7:
            src.append(b)
            dst.append(b + 6)
    gs.append(gg.from_arcs(48, src, dst, True, "cycle_chain"))
    # fewer than k vertices that reach another: the lists end with out-degree-0 vertices in id order
    gs.append(gg.from_arcs(7, [], [], True, "empty7"))
    gs.append(gg.from_arcs(6, [3, 4], [4, 0], True, "tiny"))
    gs.append(gg.from_arcs(1, [], [], True, "single"))
    gs.append(gg.erdos_renyi(800, 2400, seed=91))
    gs.append(gg.barabasi_albert(600, 3, 92))
    return gs


@pytest.fixture(scope="module")
def ctx(gpu_lib):
    c = gpu_lib.tkc_create(gpu_lib.Options())
    yield c
    gpu_lib.tkc_destroy(c)


@pytest.mark.parametrize("bits", [64, 256])
@pytest.mark.parametrize("nb", [False, True])
def test_union_of_many_scc_graphs(gpu_lib, ctx, nb, bits):
    t = gpu_lib
    gs = _graphs()
    t.tkc_set_options(ctx, t.Options(batch_bits=bits, order=t.TKC_ORDER_NB if nb else t.TKC_ORDER_DEG))
    hs = [t.tkc_load_csr(ctx, g.n, g.offsets, g.cols, g.directed) for g in gs]
    try:
        res = t.tkc_topk_closeness_multi(ctx, hs, 5)
    finally:
        for h in hs:
            t.tkc_free_graph(h)
        t.tkc_set_options(ctx, t.Options())
    for g, got in zip(gs, res):
        ref = oracle.textbook_topk(g, 5)
        assert list(got.ids) == list(ref.ids), g.name
        assert np.array_equal(got.dist_sum, ref.S) and np.array_equal(got.reach, ref.r), g.name
        assert got.n_tied_at_kth == ref.n_tied, g.name
        for i in range(len(ref.ids)):
            f, _ = oracle.farness(g.n, ref.S[i], ref.r[i])
            assert got.farness[i].tobytes() == np.float64(f).tobytes(), g.name


def _expect_all(gs, res, k):
    for g, got in zip(gs, res):
        ref = oracle.textbook_topk(g, k)
        assert list(got.ids) == list(ref.ids), g.name
        assert np.array_equal(got.dist_sum, ref.S) and np.array_equal(got.reach, ref.r), g.name
        assert got.n_tied_at_kth == ref.n_tied, g.name


@pytest.mark.parametrize("on_device", [False, True])
def test_load_many_then_one_launch(gpu_lib, ctx, on_device):
    """tkc_load_csr_many: every graph validated with one host wait, then one
    multi-graph launch; results equal the textbook per graph."""
    import torch

    t = gpu_lib
    gs = _graphs()
    if on_device:
        spec = [(g.n, torch.from_numpy(g.offsets.astype(np.int32)).cuda(),
                 torch.from_numpy(g.cols.astype(np.int32)).cuda(), g.directed) for g in gs]
    else:
        spec = [(g.n, g.offsets, g.cols, g.directed) for g in gs]
    t.tkc_set_options(ctx, t.Options(batch_bits=64, order=t.TKC_ORDER_NB))
    hs = t.tkc_load_csr_many(ctx, spec)
    try:
        res = t.tkc_topk_closeness_multi(ctx, hs, 5)
    finally:
        for h in hs:
            t.tkc_free_graph(h)
        t.tkc_set_options(ctx, t.Options())
    _expect_all(gs, res, 5)


def test_load_many_reports_the_first_malformed_graph(gpu_lib, ctx):
    t = gpu_lib
    gs = _graphs()[:6]
    for bad_at, bad in ((3, (3, np.array([0, 1, 1, 1], np.uint32), np.array([7], np.uint32), True)),
                        (5, (3, np.array([0, 1, 1, 1], np.uint32), np.array([1], np.uint32), False)),
                        (0, (3, np.array([0, 1, 1, 2], np.uint32), np.array([1], np.uint32), True))):
        spec = [(g.n, g.offsets, g.cols, g.directed) for g in gs]
        spec.insert(bad_at, bad)
        with pytest.raises(t.TkcError) as e:
            t.tkc_load_csr_many(ctx, spec)
        assert e.value.code == t.TKC_EGRAPH and e.value.first_bad == bad_at
    # the context still loads and searches
    hs = t.tkc_load_csr_many(ctx, [(g.n, g.offsets, g.cols, g.directed) for g in gs])
    try:
        res = t.tkc_topk_closeness_multi(ctx, hs, 5)
    finally:
        for h in hs:
            t.tkc_free_graph(h)
    _expect_all(gs, res, 5)
