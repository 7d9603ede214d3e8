"""The library's shard entry points (tkc_topk_closeness_shard, tkc_count_tied)
under the sharded driver (paper_1704_01077_gb300.shard), on one GPU: each
rank is a host thread with its own context and graph copy, the exchange is a
host barrier between library calls (calls are serialised, so no kernel ever
waits on another), and the merged result must equal the oracle's: the
textbook top-k on BA n = 2 000, the CPU BFSCut on R-MAT 16, and the stored
complete oracle run on R-MAT 22 (ids, S, r and the tie count)."""
import json
import os
import threading

import numpy as np
import pytest

import oracle
from paper_1704_01077_gb300 import graphgen as gg
from paper_1704_01077_gb300 import shard

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _sharded(t, g, k, world, order, opening):
    kk = min(k, g.n)
    ctxs = [t.tkc_create(t.Options(order=order)) for _ in range(world)]
    hs = [t.tkc_load_csr(c, g.n, g.offsets, g.cols, g.directed) for c in ctxs]
    lock = threading.Lock()
    barrier = threading.Barrier(world, timeout=300)
    slots = [None] * world

    class Locked(shard.LibraryShard):
        def search(self, max_sources, seed):
            with lock:
                return super().search(max_sources, seed)

        def count_tied(self, entry):
            with lock:
                return super().count_tied(entry)

    def exchange(rank):
        def allgather(x):
            slots[rank] = x
            barrier.wait()
            out = list(slots)
            barrier.wait()
            return out

        def allreduce(x):
            return sum(allgather(x))

        return allgather, allreduce

    results, errors = [None] * world, []

    def worker(rank):
        try:
            results[rank] = shard.topk_sharded(Locked(t, hs[rank], k, rank, world), kk, opening, *exchange(rank))
        except BaseException as e:  # noqa: BLE001 -- reported below, after every thread ends
            errors.append(e)
            barrier.abort()

    threads = [threading.Thread(target=worker, args=(r,)) for r in range(world)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    for h in hs:
        t.tkc_free_graph(h)
    for c in ctxs:
        t.tkc_destroy(c)
    if errors:
        raise errors[0]
    for r in results[1:]:
        assert r == results[0]
    return results[0]


def _expect(res, ids, S, r, tied, what):
    assert [e[2] for e in res.entries] == [int(x) for x in ids], what
    assert [e[0] for e in res.entries] == [int(x) for x in S], what
    assert [e[1] for e in res.entries] == [int(x) for x in r], what
    assert res.n_tied_at_kth == tied, what


@pytest.mark.parametrize("world", [2, 3])
def test_shards_ba2000_against_textbook(gpu_lib, world):
    t = gpu_lib
    g = gg.barabasi_albert(2000, 4, gg.workload_seed(0))
    for k in (1, 10, 50):
        ref = oracle.textbook_topk(g, k)
        for order in (t.TKC_ORDER_DEG, t.TKC_ORDER_NB):
            res = _sharded(t, g, k, world, order, 64)
            _expect(res, ref.ids, ref.S, ref.r, ref.n_tied, (k, order, world))


def test_shards_rmat16_against_cpu_bfscut(gpu_lib):
    t = gpu_lib
    g = gg.rmat(16, 16, seed=gg.workload_seed(1))
    ref = oracle.bfscut(g, 10)
    for world, order, opening in ((2, t.TKC_ORDER_NB, 128), (4, t.TKC_ORDER_DEG, 64), (3, t.TKC_ORDER_NB, 0)):
        _expect(_sharded(t, g, 10, world, order, opening), ref.ids, ref.S, ref.r, ref.n_tied, (world, order))


def test_shards_rmat22_against_stored_oracle_run(gpu_lib):
    t = gpu_lib
    with open(os.path.join(GOLDEN, "fullsize_rmat22.json")) as f:
        want = json.load(f)["graphs"][0]["results"][0]
    g = gg.rmat(22, 16, seed=gg.workload_seed(4))
    res = _sharded(t, g, 10, 2, t.TKC_ORDER_NB, 128)
    _expect(res, want["ids"], want["S"], want["r"], want["n_tied"], "rmat22")


def test_shard_arguments(gpu_lib):
    t = gpu_lib
    ctx = t.tkc_create(t.Options(order=t.TKC_ORDER_NB))
    g = gg.path(8)
    h = t.tkc_load_csr(ctx, g.n, g.offsets, g.cols, False)
    try:
        with pytest.raises(t.TkcError):
            t.tkc_topk_closeness_shard(h, 3, 2, 2)  # shard >= nshards
        with pytest.raises(t.TkcError):  # seed not best first
            t.tkc_topk_closeness_shard(h, 3, 0, 2, 0, (np.array([20, 10], np.uint64), np.array([8, 8], np.uint32),
                                                       np.array([0, 1], np.uint32)))
        with pytest.raises(t.TkcError):  # tie count before any shard run of this graph
            t.tkc_count_tied(h, 16, 8)
        r = t.tkc_topk_closeness_shard(h, 3, 1, 2)
        assert len(r.ids) == 3
        assert t.tkc_count_tied(h, int(r.dist_sum[0]), int(r.reach[0])) >= 1
    finally:
        t.tkc_free_graph(h)
        t.tkc_destroy(ctx)
