"""Checkpoint and resume through the library (tkc_topk_closeness_shard from a
position, tkc_count_tied) on the GPU: runs in segments, and runs interrupted,
saved as JSON and resumed on a fresh context and graph copy, must return the
oracle's exact top-k and tie count -- the textbook result on BA n = 2 000, the
CPU BFSCut on R-MAT 16, the stored complete oracle run on R-MAT 22."""
import json
import os

import pytest

import oracle
from paper_1704_01077_gb300 import checkpoint as cp
from paper_1704_01077_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _segments(t, g, k, order, segment, resume=None, stop_after=None):
    ctx = t.tkc_create(t.Options(order=order))
    h = t.tkc_load_csr(ctx, g.n, g.offsets, g.cols, g.directed)
    try:
        return cp.run(cp.LibrarySegments(t, h, k), min(k, g.n), segment, resume=resume, stop_after=stop_after)
    finally:
        t.tkc_free_graph(h)
        t.tkc_destroy(ctx)


def _expect(entries, tied, ids, S, r, n_tied, what):
    assert [e[2] for e in entries] == [int(x) for x in ids], what
    assert [e[0] for e in entries] == [int(x) for x in S], what
    assert [e[1] for e in entries] == [int(x) for x in r], what
    assert tied == n_tied, what


def test_ba2000_segments(gpu_lib):
    t = gpu_lib
    g = gg.barabasi_albert(2000, 4, gg.workload_seed(0))
    for k in (1, 10):
        ref = oracle.textbook_topk(g, k)
        for order, segment in ((t.TKC_ORDER_DEG, 100), (t.TKC_ORDER_DEG, 700), (t.TKC_ORDER_NB, 64)):
            entries, tied, ck = _segments(t, g, k, order, segment)
            assert ck.done
            _expect(entries, tied, ref.ids, ref.S, ref.r, ref.n_tied, (k, order, segment))


def test_rmat16_interrupted_and_resumed(gpu_lib):
    t = gpu_lib
    g = gg.rmat(16, 16, seed=gg.workload_seed(1))
    ref = oracle.bfscut(g, 10)
    for order in (t.TKC_ORDER_NB, t.TKC_ORDER_DEG):
        _, _, ck = _segments(t, g, 10, order, 256, stop_after=2)
        assert not ck.done and ck.position == 512
        back = cp.Checkpoint.loads(ck.dumps())
        entries, tied, ck2 = _segments(t, g, 10, order, 256, resume=back)  # new context and graph copy
        assert ck2.done
        _expect(entries, tied, ref.ids, ref.S, ref.r, ref.n_tied, order)


def test_rmat22_segments_against_stored_oracle_run(gpu_lib):
    t = gpu_lib
    with open(os.path.join(GOLDEN, "fullsize_rmat22.json")) as f:
        want = json.load(f)["graphs"][0]["results"][0]
    g = gg.rmat(22, 16, seed=gg.workload_seed(4))
    entries, tied, ck = _segments(t, g, 10, t.TKC_ORDER_NB, 4096)
    assert ck.done
    _expect(entries, tied, want["ids"], want["S"], want["r"], want["n_tied"], "rmat22")
