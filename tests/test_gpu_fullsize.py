"""The bench workloads at full size (R-MAT scale 22, Barabasi-Albert 10^6), in
the launch configuration bench.py times (library defaults: 128-bit NBCut
batches with 768-thread blocks on R-MAT 22, 512-thread blocks on BA 10^6),
checked against the CPU oracle vertex by vertex, since the textbook top-k is
out of reach at these sizes:
- every returned vertex's S and r (h for harmonic) equal the oracle's BFS from
  it, and its farness the oracle's IEEE value;
- the list is ordered by (farness, id);
- no vertex of a sample (the highest out-degrees and uniform random sources)
  beats the k-th;
- DegCut, NBCut and both block sizes return the same list."""
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


@pytest.fixture(scope="module")
def rmat22():
    return gg.rmat(22, 16, seed=gg.workload_seed(4))


@pytest.fixture(scope="module")
def ba1m():
    return gg.barabasi_albert(1_000_000, 5, gg.workload_seed(2))


def _sample(g, ids, seed, count=40):
    outd = g.outdeg()
    top = np.argsort(-outd, kind="stable")[:count]
    rng = np.random.default_rng(seed)
    rnd = rng.choice(np.nonzero(outd > 0)[0], size=count, replace=False)
    return np.setdiff1d(np.concatenate([top, rnd]), np.asarray(ids, dtype=np.int64)).astype(np.uint32)


def _run(t, ctx, g, k, fn, **opts):
    t.tkc_set_options(ctx, t.Options(**opts))
    h = t.tkc_load_csr(ctx, g.n, g.offsets, g.cols, g.directed)
    try:
        return fn(h, k)
    finally:
        t.tkc_free_graph(h)
        t.tkc_set_options(ctx, t.Options())


def _check_closeness(g, res, k, seed):
    ids = np.asarray(res.ids)
    assert len(ids) == k
    S, r = oracle.bfs_sums(g, ids)
    assert np.array_equal(S, res.dist_sum) and np.array_equal(r, res.reach)
    for i in range(k):
        f, _ = oracle.farness(g.n, S[i], r[i])
        assert res.farness[i].tobytes() == np.float64(f).tobytes()
    for i in range(k - 1):
        c = oracle.cmp_farness(int(S[i]), int(r[i]), int(S[i + 1]), int(r[i + 1]))
        assert c < 0 or (c == 0 and ids[i] < ids[i + 1]), i
    smp = _sample(g, ids, seed)
    Ss, rs = oracle.bfs_sums(g, smp)
    for v, s_, r_ in zip(smp, Ss, rs):
        c = oracle.cmp_farness(int(s_), int(r_), int(S[-1]), int(r[-1]))
        assert c > 0 or (c == 0 and v > ids[-1]), int(v)


def _same(a, b):
    assert list(a.ids) == list(b.ids)
    assert np.array_equal(a.dist_sum, b.dist_sum) and np.array_equal(a.reach, b.reach)
    assert a.n_tied_at_kth == b.n_tied_at_kth


def test_rmat22_closeness(gpu_lib, ctx, rmat22):
    t = gpu_lib
    g = rmat22
    nb = _run(t, ctx, g, 10, t.tkc_topk_closeness, order=t.TKC_ORDER_NB)
    assert nb.batch_bits == 128
    _check_closeness(g, nb, 10, 1)
    _same(_run(t, ctx, g, 10, t.tkc_topk_closeness, order=t.TKC_ORDER_DEG), nb)
    _same(_run(t, ctx, g, 10, t.tkc_topk_closeness, order=t.TKC_ORDER_NB, large_blocks=2), nb)


def test_rmat22_harmonic(gpu_lib, ctx, rmat22):
    t = gpu_lib
    g = rmat22
    res = _run(t, ctx, g, 10, t.tkc_topk_harmonic, order=t.TKC_ORDER_NB)
    ids = np.asarray(res.ids)
    H, r = oracle.harmonic_sums(g, ids)
    assert H.tobytes() == res.closeness.tobytes() and np.array_equal(r, res.reach)
    assert all(H[i] > H[i + 1] or (H[i] == H[i + 1] and ids[i] < ids[i + 1]) for i in range(len(ids) - 1))
    smp = _sample(g, ids, 2)
    Hs, _ = oracle.harmonic_sums(g, smp)
    assert all(h < H[-1] or (h == H[-1] and v > ids[-1]) for v, h in zip(smp, Hs))


@pytest.mark.parametrize("k", [1, 10, 100])
def test_ba1m_closeness(gpu_lib, ctx, ba1m, k):
    t = gpu_lib
    g = ba1m
    nb = _run(t, ctx, g, k, t.tkc_topk_closeness, order=t.TKC_ORDER_NB)
    _check_closeness(g, nb, k, 3 + k)
    _same(_run(t, ctx, g, k, t.tkc_topk_closeness, order=t.TKC_ORDER_NB, large_blocks=1), nb)
    if k == 10:
        _same(_run(t, ctx, g, k, t.tkc_topk_closeness, order=t.TKC_ORDER_DEG), nb)
