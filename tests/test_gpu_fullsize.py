"""The full-size workloads (directed R-MAT scale 22, Barabasi-Albert 10^6 with
k = 1, 10, 100, and the 512 graphs of one multi-graph launch), in the launch
configuration bench.py times (library defaults), against the CPU oracle's
complete run of Algorithm 1 on the same graphs.

The expected values are stored in tests/golden/fullsize_*.json, written by
tests/golden/make_fullsize_fixtures.py, which calls only the oracle (NBCut
order and stop, one source at a time, run to the end).  Each fixture holds
the SHA-256 of its graph's CSR, checked here first, so a different generator
build cannot pass silently.  Ids, S, r, the tie count and the farness doubles
must be identical, for DegCut and NBCut and both block sizes of the search
kernel; harmonic centrality compares the FP64 h bit for bit."""
import hashlib
import json
import os

import numpy as np
import pytest

from paper_1704_01077_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _fixture(name):
    with open(os.path.join(GOLDEN, f"fullsize_{name}.json")) as f:
        return json.load(f)


def _sha(g):
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(g.offsets, dtype="<u4").tobytes())
    h.update(np.ascontiguousarray(g.cols, dtype="<u4").tobytes())
    return h.hexdigest()


@pytest.fixture(scope="module")
def ctx(gpu_lib):
    c = gpu_lib.tkc_create(gpu_lib.Options())
    yield c
    gpu_lib.tkc_destroy(c)


@pytest.fixture(scope="module")
def rmat22():
    g = gg.rmat(22, 16, seed=gg.workload_seed(4))
    assert _sha(g) == _fixture("rmat22")["graphs"][0]["csr_sha256"]
    return g


@pytest.fixture(scope="module")
def ba1m():
    g = gg.barabasi_albert(1_000_000, 5, gg.workload_seed(2))
    assert _sha(g) == _fixture("ba1m")["graphs"][0]["csr_sha256"]
    return g


def _run(t, ctx, g, k, fn, **opts):
    t.tkc_set_options(ctx, t.Options(**opts))
    h = t.tkc_load_csr(ctx, g.n, g.offsets, g.cols, g.directed)
    try:
        return fn(h, k)
    finally:
        t.tkc_free_graph(h)
        t.tkc_set_options(ctx, t.Options())


def _expect(res, want, what):
    assert [int(x) for x in res.ids] == want["ids"], what
    assert [int(x) for x in res.dist_sum] == want["S"], what
    assert [int(x) for x in res.reach] == want["r"], what
    assert res.n_tied_at_kth == want["n_tied"], what
    assert [float(f).hex() for f in res.farness] == want["farness_hex"], what


def _want(name, k, index=0):
    for r in _fixture(name)["graphs"][index]["results"]:
        if r["k"] == k:
            return r
    raise KeyError((name, k))


def test_rmat22_closeness(gpu_lib, ctx, rmat22):
    t = gpu_lib
    want = _want("rmat22", 10)
    nb = _run(t, ctx, rmat22, 10, t.tkc_topk_closeness, order=t.TKC_ORDER_NB)
    assert nb.batch_bits == 128
    _expect(nb, want, "NBCut")
    _expect(_run(t, ctx, rmat22, 10, t.tkc_topk_closeness, order=t.TKC_ORDER_DEG), want, "DegCut")
    _expect(_run(t, ctx, rmat22, 10, t.tkc_topk_closeness, order=t.TKC_ORDER_NB, large_blocks=2), want,
            "NBCut, 512-thread blocks")


def test_rmat22_harmonic(gpu_lib, ctx, rmat22):
    t = gpu_lib
    fx = _fixture("rmat22_harmonic")
    assert fx["graphs"][0]["csr_sha256"] == _sha(rmat22)
    want = fx["graphs"][0]["results"][0]
    res = _run(t, ctx, rmat22, 10, t.tkc_topk_harmonic, order=t.TKC_ORDER_NB)
    assert [int(x) for x in res.ids] == want["ids"]
    assert [float(h).hex() for h in res.closeness] == want["h_hex"]
    assert [int(x) for x in res.reach] == want["r"] and res.n_tied_at_kth == want["n_tied"]


@pytest.mark.parametrize("k", [1, 10, 100])
def test_ba1m_closeness(gpu_lib, ctx, ba1m, k):
    t = gpu_lib
    want = _want("ba1m", k)
    _expect(_run(t, ctx, ba1m, k, t.tkc_topk_closeness, order=t.TKC_ORDER_NB), want, ("NBCut", k))
    _expect(_run(t, ctx, ba1m, k, t.tkc_topk_closeness, order=t.TKC_ORDER_NB, large_blocks=1), want,
            ("NBCut, larger blocks", k))
    if k == 10:
        _expect(_run(t, ctx, ba1m, k, t.tkc_topk_closeness, order=t.TKC_ORDER_DEG), want, ("DegCut", k))


def test_multi512_one_launch(gpu_lib, ctx):
    t = gpu_lib
    fx = _fixture("multi512")
    rc = fx["recipe"]
    seed = gg.workload_seed(rc["seed_index"])
    sizes = gg.log_uniform_sizes(rc["count"], rc["lo"], rc["hi"], seed)
    graphs = [gg.barabasi_albert(n, 4, gg.splitmix64(seed + i)) if i % 2 == 0
              else gg.erdos_renyi(n, 8 * n, gg.splitmix64(seed + i), directed=True) for i, n in enumerate(sizes)]
    for g, e in zip(graphs, fx["graphs"]):
        assert _sha(g) == e["csr_sha256"], e["index"]
    for order in (t.TKC_ORDER_NB, t.TKC_ORDER_DEG):
        t.tkc_set_options(ctx, t.Options(order=order))
        hs = [t.tkc_load_csr(ctx, g.n, g.offsets, g.cols, g.directed) for g in graphs]
        try:
            res = t.tkc_topk_closeness_multi(ctx, hs, 10)
        finally:
            for h in hs:
                t.tkc_free_graph(h)
            t.tkc_set_options(ctx, t.Options())
        for i, (r, e) in enumerate(zip(res, fx["graphs"])):
            _expect(r, e["results"][0], (order, i, e["name"]))
