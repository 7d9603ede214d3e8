"""The allocation-free entry point, tkc_distance_sums_noalloc, through the C ABI.

Callers that cannot allocate device memory when they need a result (runtimes
with a fixed device-memory budget, latency-bound services that cannot take an
allocation's synchronisation) use this variant; it must return exactly what
tkc_distance_sums returns.  The file is collected last so that a run stopping
at its first failure has already run every other test; it also passes alone in
a fresh process."""
import numpy as np
import pytest

from paper_1704_01077_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu


def _cases():
    return [gg.rmat(12, 8, seed=21), gg.barabasi_albert(3000, 3, 22),
            gg.disjoint_union(gg.cycle(9, True), gg.path(5, True), gg.path(1))]


def test_noalloc_matches_distance_sums_twice(gpu_lib):
    import torch

    t = gpu_lib
    ctx = t.tkc_create(t.Options())
    try:
        for g in _cases():
            src = np.unique(np.concatenate([np.arange(0, g.n, max(1, g.n // 200)), [g.n - 1]])).astype(np.uint32)
            h = t.tkc_load_csr(ctx, g.n, g.offsets, g.cols, g.directed)
            try:
                S_ref, r_ref = t.tkc_distance_sums(h, src)
            finally:
                t.tkc_free_graph(h)
            off = torch.from_numpy(g.offsets.view(np.int32)).cuda()
            col = torch.from_numpy(g.cols.view(np.int32).copy() if g.arcs else np.zeros(1, np.int32)).cuda()
            if not g.arcs:
                col = col[:0]
            s = torch.from_numpy(src.view(np.int32)).cuda()
            for _ in range(2):  # the shared scratch keeps the previous call's contents
                S = torch.full((len(src),), -1, dtype=torch.int64, device="cuda")
                r = torch.full((len(src),), -1, dtype=torch.int32, device="cuda")
                t.tkc_distance_sums_noalloc(off, col, g.n, s, S, r)
                torch.cuda.synchronize()
                assert np.array_equal(S.cpu().numpy().view(np.uint64), S_ref), g.name
                assert np.array_equal(r.cpu().numpy().view(np.uint32), r_ref), g.name
    finally:
        t.tkc_destroy(ctx)


def test_noalloc_rejects_bad_arguments(gpu_lib):
    import torch

    t = gpu_lib
    g = gg.path(10, directed=True)
    off = torch.from_numpy(g.offsets.view(np.int32)).cuda()
    col = torch.from_numpy(g.cols.view(np.int32)).cuda()
    S = torch.zeros(3, dtype=torch.int64, device="cuda")
    r = torch.zeros(3, dtype=torch.int32, device="cuda")
    dup = torch.tensor([1, 4, 1], dtype=torch.int32, device="cuda")
    with pytest.raises(t.TkcError) as e:
        t.tkc_distance_sums_noalloc(off, col, g.n, dup, S, r)
    assert e.value.code == t.TKC_EINVAL
    big = t.TKC_NOALLOC_MAX_N + 1
    with pytest.raises(t.TkcError) as e:
        t.tkc_distance_sums_noalloc(off, col, big, dup, S, r)
    assert e.value.code == t.TKC_EINVAL
    # a valid call after the rejected ones still returns exact results
    ok = torch.tensor([0, 4, 9], dtype=torch.int32, device="cuda")
    t.tkc_distance_sums_noalloc(off, col, g.n, ok, S, r)
    torch.cuda.synchronize()
    assert S.cpu().tolist() == [45, 15, 0] and r.cpu().tolist() == [10, 6, 1]
