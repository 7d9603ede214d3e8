"""CUDA path against the CPU oracle, element by element, through the C ABI.

Integer results (ids, S, r, tie counts, orders, reach bounds, plain-mode
counters) must be bit-exact; farness and closeness are single-rounded IEEE
doubles of exact integers on both sides, so they must be bit-identical too."""
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


def _run(tkc, ctx, g, k, bits, order=None, given=None):
    opt = tkc.Options(batch_bits=bits, order=tkc.TKC_ORDER_DEG if given is None else tkc.TKC_ORDER_GIVEN)
    tkc.tkc_set_options(ctx, opt)
    h = tkc.tkc_load_csr(ctx, g.n, g.offsets, g.cols, g.directed)
    try:
        if given is not None:
            tkc.tkc_set_source_order(h, given)
        return tkc.tkc_topk_closeness(h, k)
    finally:
        tkc.tkc_free_graph(h)


def _expect_equal(got, ref, g, k):
    assert list(got.ids) == list(ref.ids), (g.name, k)
    assert np.array_equal(got.dist_sum, ref.S) and np.array_equal(got.reach, ref.r)
    assert got.n_tied_at_kth == ref.n_tied, (g.name, k, got.n_tied_at_kth, ref.n_tied)
    for i in range(len(ref.ids)):
        f, c = oracle.farness(g.n, ref.S[i], ref.r[i])
        assert got.farness[i].tobytes() == np.float64(f).tobytes()
        assert got.closeness[i].tobytes() == np.float64(c).tobytes()


SMALL = [
    lambda: gg.path(17), lambda: gg.path(12, directed=True), lambda: gg.cycle(9), lambda: gg.cycle(8, True),
    lambda: gg.star(30), lambda: gg.complete(6), lambda: gg.complete_bipartite(3, 9), lambda: gg.hypercube(5),
    lambda: gg.random_tree(150, 4), lambda: gg.disjoint_union(gg.cycle(5), gg.path(7), gg.path(1), gg.star(4)),
    lambda: gg.reduction_graph(4, [{0, 1}, {2}, {3}, {0, 3}, {1, 2, 3}])[0],
    lambda: gg.from_arcs(7, [], [], True, "empty7"),
]


@pytest.mark.parametrize("bits", [1, 64, 512])
@pytest.mark.parametrize("gi", range(len(SMALL)))
def test_small_families(gpu_lib, ctx, gi, bits):
    g = SMALL[gi]()
    for k in sorted({1, 3, 10, g.n}):
        ref = oracle.textbook_topk(g, k)
        got = _run(gpu_lib, ctx, g, k, bits)
        _expect_equal(got, ref, g, k)


@pytest.mark.parametrize("bits", [1, 64, 128, 256, 512])
def test_random_graphs(gpu_lib, ctx, bits):
    for seed in range(40):
        directed = seed % 2 == 0
        n = 20 + 37 * (seed % 7)
        g = gg.random_graph(n, 2.5 / n, 7000 + seed, directed)
        k = [1, 5, 10, n][seed % 4]
        _expect_equal(_run(gpu_lib, ctx, g, k, bits), oracle.textbook_topk(g, k), g, k)


def test_plain_mode_counters_match_cpu_bfscut(gpu_lib, ctx):
    """One source at a time, the device schedule is the oracle's: same arcs."""
    for seed in range(12):
        directed = seed % 2 == 1
        g = gg.random_graph(60 + 10 * seed, 3.0 / (60 + 10 * seed), 300 + seed, directed)
        ref = oracle.bfscut(g, 5)
        got = _run(gpu_lib, ctx, g, 5, 1)
        _expect_equal(got, ref, g, 5)
        c = ref.counters
        assert (got.edges_visited, got.bfs_started, got.bfs_cut, got.bfs_finished) == \
            (c.edges_visited, c.bfs_started, c.bfs_cut, c.bfs_finished), seed


def test_ba2000_plain_and_batched(gpu_lib, ctx):
    """Barabasi-Albert n=2000, m=4, k=10 (the small plain workload)."""
    g = gg.barabasi_albert(2000, 4, gg.workload_seed(0))
    ref = oracle.textbook_topk(g, 10)
    cut = oracle.bfscut(g, 10)
    got = _run(gpu_lib, ctx, g, 10, 1)
    _expect_equal(got, ref, g, 10)
    assert got.edges_visited == cut.counters.edges_visited
    for bits in (64, 256, 512):
        _expect_equal(_run(gpu_lib, ctx, g, 10, bits), ref, g, 10)


def test_rmat16_directed(gpu_lib, ctx):
    """Directed R-MAT scale 16, edge factor 16, k=10, against the CPU BFSCut."""
    g = gg.rmat(16, 16, seed=gg.workload_seed(1))
    ref = oracle.bfscut(g, 10)
    got = _run(gpu_lib, ctx, g, 10, 1)
    _expect_equal(got, ref, g, 10)
    assert got.edges_visited == ref.counters.edges_visited
    for bits in (64, 512):
        _expect_equal(_run(gpu_lib, ctx, g, 10, bits), ref, g, 10)


def test_order_invariance(gpu_lib, ctx):
    g = gg.rmat(12, 8, seed=99)
    ref = oracle.textbook_topk(g, 10)
    rng = np.random.default_rng(3)
    for bits in (1, 128):
        for _ in range(3):
            _expect_equal(_run(gpu_lib, ctx, g, 10, bits, given=rng.permutation(g.n)), ref, g, 10)


def test_degree_order_matches_oracle(gpu_lib, ctx):
    for g in (gg.barabasi_albert(3000, 3, 5), gg.rmat(14, 16, seed=4), gg.path(5), gg.from_arcs(3, [], [], True)):
        h = gpu_lib.tkc_load_csr(ctx, g.n, g.offsets, g.cols, g.directed)
        try:
            assert np.array_equal(gpu_lib.tkc_source_order(h, g.n), oracle.degree_order(g))
        finally:
            gpu_lib.tkc_free_graph(h)


def _cycle_chain(k, size, back_every=0):
    """k directed cycles of `size` vertices, cycle i -> cycle i+1 (and an arc
    back to cycle 0 every `back_every` cycles, merging SCCs)."""
    src, dst = [], []
    for c in range(k):
        for j in range(size):
            src.append(c * size + j)
            dst.append(c * size + (j + 1) % size)
        if c + 1 < k:
            src.append(c * size)
            dst.append((c + 1) * size + 1 % size)
        if back_every and c % back_every == back_every - 1:
            src.append(c * size + size - 1)
            dst.append((c - back_every + 1) * size)
    return gg.from_arcs(k * size, src, dst, True, f"cyclechain{k}x{size}")


def test_reach_bounds_match_oracle(gpu_lib, ctx):
    cases = [gg.rmat(13, 4, seed=11), gg.random_graph(300, 0.006, 8, True), gg.erdos_renyi(5000, 6000, 2),
             gg.disjoint_union(gg.cycle(5), gg.path(7), gg.star(4)), gg.barabasi_albert(500, 2, 3),
             gg.reduction_graph(3, [{0}, {1, 2}, {0, 2}])[0], gg.rmat(16, 16, seed=gg.workload_seed(1)),
             gg.random_graph(600, 1.3 / 600, 77, True), gg.erdos_renyi(20000, 26000, 9),
             _cycle_chain(40, 3), _cycle_chain(30, 4, back_every=3), gg.path(300, directed=True),
             gg.cycle(50, directed=True), gg.from_arcs(6, [], [], True)]
    for g in cases:
        h = gpu_lib.tkc_load_csr(ctx, g.n, g.offsets, g.cols, g.directed)
        try:
            a, o = gpu_lib.tkc_reach_bounds(h, g.n)
        finally:
            gpu_lib.tkc_free_graph(h)
        ra, ro = oracle.alpha_omega(g)
        assert np.array_equal(a, ra) and np.array_equal(o, ro), g.name


def test_distance_sums_match_oracle(gpu_lib, ctx):
    for g in (gg.rmat(12, 16, seed=5), gg.barabasi_albert(4000, 4, 6), gg.random_graph(200, 0.01, 1, True)):
        src = np.arange(0, g.n, max(1, g.n // 300), dtype=np.uint32)
        h = gpu_lib.tkc_load_csr(ctx, g.n, g.offsets, g.cols, g.directed)
        try:
            S, r = gpu_lib.tkc_distance_sums(h, src)
        finally:
            gpu_lib.tkc_free_graph(h)
        rS, rr = oracle.bfs_sums(g, src)
        assert np.array_equal(S, rS) and np.array_equal(r, rr), g.name


def test_malformed_graphs_rejected(gpu_lib, ctx):
    t = gpu_lib
    t.tkc_set_options(ctx, t.Options(batch_bits=64))
    bad = [
        (3, [0, 2, 2, 2], [2, 1], True),      # unsorted row
        (3, [0, 2, 2, 2], [1, 1], True),      # duplicate arc
        (3, [0, 1, 1, 1], [0], True),         # self-loop
        (3, [0, 1, 1, 1], [7], True),         # id out of range
        (3, [0, 1, 1, 1], [1], False),        # undirected but not symmetric
        (3, [0, 2, 1, 2], [1, 2], True),      # offsets decrease
    ]
    for n, off, col, directed in bad:
        with pytest.raises(t.TkcError) as e:
            t.tkc_load_csr(ctx, n, np.array(off, np.uint32), np.array(col, np.uint32), directed)
        assert e.value.code == t.TKC_EGRAPH, (off, col)
    g = gg.path(4)
    h = t.tkc_load_csr(ctx, g.n, g.offsets, g.cols, False)
    try:
        with pytest.raises(t.TkcError) as e:
            t.tkc_topk_closeness(h, t.TKC_MAX_K + 1)
        assert e.value.code == t.TKC_EINVAL
        assert len(t.tkc_topk_closeness(h, 0).ids) == 0
        with pytest.raises(t.TkcError):
            t.tkc_set_source_order(h, [0, 1, 1, 3])
    finally:
        t.tkc_free_graph(h)


def test_malformed_device_input_rejected(gpu_lib, ctx):
    """Device-resident CSR: the first and last offsets are checked on the
    device with the rest of the validation (no separate host read)."""
    import torch

    t = gpu_lib
    bad = [
        (3, [1, 1, 1, 1], [], True),          # offsets do not start at 0
        (3, [0, 1, 1, 2], [1], True),         # last offset is not the arc count
        (3, [0, 1, 1, 1], [7], True),         # id out of range
        (3, [0, 2, 2, 2], [2, 1], True),      # unsorted row
        (3, [0, 1, 1, 1], [1], False),        # undirected but not symmetric
        (0, [2], [], True),                   # no vertex, offsets[0] != 0
    ]
    for n, off, col, directed in bad:
        o = torch.tensor(off, dtype=torch.int32, device="cuda")
        c = torch.tensor(col if col else [0], dtype=torch.int32, device="cuda")[: len(col)]
        with pytest.raises(t.TkcError) as e:
            t.tkc_load_csr(ctx, n, o, c, directed)
        assert e.value.code == t.TKC_EGRAPH, (off, col)
    # the context still works
    g = gg.path(5, directed=True)
    h = t.tkc_load_csr(ctx, g.n, torch.from_numpy(g.offsets.astype(np.int32)).cuda(),
                       torch.from_numpy(g.cols.astype(np.int32)).cuda(), True)
    try:
        got = t.tkc_topk_closeness(h, 3)
    finally:
        t.tkc_free_graph(h)
    _expect_equal(got, oracle.textbook_topk(g, 3), g, 3)


def test_zero_and_one_vertex(gpu_lib, ctx):
    t = gpu_lib
    t.tkc_set_options(ctx, t.Options(batch_bits=64))
    h = t.tkc_load_csr(ctx, 0, np.zeros(1, np.uint32), np.zeros(0, np.uint32), True)
    assert len(t.tkc_topk_closeness(h, 5).ids) == 0
    t.tkc_free_graph(h)
    h = t.tkc_load_csr(ctx, 1, np.zeros(2, np.uint32), np.zeros(0, np.uint32), False)
    res = t.tkc_topk_closeness(h, 5)
    assert list(res.ids) == [0] and res.reach[0] == 1 and res.closeness[0] == 0.0 and res.n_tied_at_kth == 1
    t.tkc_free_graph(h)


def test_device_pointer_input(gpu_lib, ctx):
    import torch

    g = gg.barabasi_albert(1500, 3, 12)
    off = torch.from_numpy(g.offsets.astype(np.int32)).cuda()
    col = torch.from_numpy(g.cols.astype(np.int32)).cuda()
    gpu_lib.tkc_set_options(ctx, gpu_lib.Options(batch_bits=128))
    h = gpu_lib.tkc_load_csr(ctx, g.n, off, col, False)
    try:
        got = gpu_lib.tkc_topk_closeness(h, 10)
    finally:
        gpu_lib.tkc_free_graph(h)
    _expect_equal(got, oracle.textbook_topk(g, 10), g, 10)


def _mixed_graphs(count, lo, hi, seed):
    """Half Barabasi-Albert (m=4), half directed Erdos-Renyi (mean out-degree 8),
    vertex counts log-uniform in [lo, hi]."""
    sizes = gg.log_uniform_sizes(count, lo, hi, seed)
    out = []
    for i, n in enumerate(sizes):
        if i % 2 == 0:
            out.append(gg.barabasi_albert(max(n, 6), 4, seed + i))
        else:
            out.append(gg.erdos_renyi(n, 8 * n, seed + i, directed=True))
    return out


def test_multi_graph_one_launch(gpu_lib, ctx):
    t = gpu_lib
    graphs = _mixed_graphs(24, 20, 3000, 4242) + [
        gg.from_arcs(0, [], [], True, "empty0"), gg.from_arcs(5, [], [], True, "isolated5"), gg.path(3),
        gg.cycle(7, directed=True), gg.reduction_graph(3, [{0}, {1, 2}, {0, 2}])[0],
        gg.disjoint_union(gg.cycle(5), gg.path(4), gg.path(1))]
    for bits, k in ((64, 10), (256, 10), (512, 3), (128, 40)):
        t.tkc_set_options(ctx, t.Options(batch_bits=bits))
        hs = [t.tkc_load_csr(ctx, g.n, g.offsets, g.cols, g.directed) for g in graphs]
        try:
            res = t.tkc_topk_closeness_multi(ctx, hs, k)
            for g, h, r in zip(graphs, hs, res):
                ref = oracle.textbook_topk(g, k)
                _expect_equal(r, ref, g, k)
                single = t.tkc_topk_closeness(h, k)
                assert list(single.ids) == list(r.ids) and single.n_tied_at_kth == r.n_tied_at_kth
        finally:
            for h in hs:
                t.tkc_free_graph(h)


def test_multi_graph_counters_add_up(gpu_lib, ctx):
    t = gpu_lib
    graphs = _mixed_graphs(10, 200, 2000, 99)
    t.tkc_set_options(ctx, t.Options(batch_bits=128))
    hs = [t.tkc_load_csr(ctx, g.n, g.offsets, g.cols, g.directed) for g in graphs]
    try:
        res = t.tkc_topk_closeness_multi(ctx, hs, 10)
    finally:
        for h in hs:
            t.tkc_free_graph(h)
    for g, r in zip(graphs, res):
        src = int((g.outdeg() > 0).sum())
        assert r.bfs_started == src and r.bfs_cut + r.bfs_finished == src
        assert 0 < r.edges_visited <= g.arcs * src


@pytest.mark.parametrize("teams,bits", [(2, 64), (3, 128), (4, 256), (8, 512)])
def test_teams_give_exact_results(gpu_lib, ctx, teams, bits):
    """Several teams share the threshold and the k-lists; results stay exact."""
    t = gpu_lib
    cases = [gg.rmat(14, 16, seed=gg.workload_seed(1) + teams), gg.barabasi_albert(20000, 4, teams),
             gg.random_graph(400, 0.01, 31 + teams, True), gg.path(50)]
    for g in cases:
        ref = oracle.bfscut(g, 10) if g.n > 5000 else oracle.textbook_topk(g, 10)
        t.tkc_set_options(ctx, t.Options(batch_bits=bits, teams=teams))
        h = t.tkc_load_csr(ctx, g.n, g.offsets, g.cols, g.directed)
        try:
            res = t.tkc_topk_closeness(h, 10)
        finally:
            t.tkc_free_graph(h)
        _expect_equal(res, ref, g, 10)
        src = int((g.outdeg() > 0).sum())
        assert res.bfs_started == src and res.bfs_cut + res.bfs_finished == src
    graphs = _mixed_graphs(12, 50, 4000, 77 + teams)
    hs = [t.tkc_load_csr(ctx, g.n, g.offsets, g.cols, g.directed) for g in graphs]
    try:
        res = t.tkc_topk_closeness_multi(ctx, hs, 10)
    finally:
        for h in hs:
            t.tkc_free_graph(h)
    for g, r in zip(graphs, res):
        _expect_equal(r, oracle.textbook_topk(g, 10), g, 10)


def test_autotune_picks_valid_parameters_and_keeps_results(gpu_lib, ctx):
    t = gpu_lib
    g = gg.rmat(14, 16, seed=gg.workload_seed(1) + 5)
    ref = oracle.bfscut(g, 10)
    t.tkc_set_options(ctx, t.Options())
    h = t.tkc_load_csr(ctx, g.n, g.offsets, g.cols, g.directed)
    try:
        best = t.tkc_autotune(h, 10)
        assert best.batch_bits in (64, 128, 256, 512) and 1 <= best.teams <= 64
        assert best.bu_num in (4, 8, 16, 32) and best.bu_den == 1
        assert best.large_blocks in (0, 1, 2) and (best.large_blocks == 0 or best.batch_bits <= 128)
        res = t.tkc_topk_closeness(h, 10)  # batch_bits = 0: the cached choice applies
        assert res.batch_bits == best.batch_bits
        _expect_equal(res, ref, g, 10)
    finally:
        t.tkc_free_graph(h)


def test_tune_cache_file_round_trip(gpu_lib, tmp_path, monkeypatch):
    """TKC_TUNE_CACHE: tuning writes one line per graph class with the block
    size last; a new context loads it and applies it; a line without the block
    size (the earlier format) still loads."""
    import re

    t = gpu_lib
    path = tmp_path / "tune.txt"
    monkeypatch.setenv("TKC_TUNE_CACHE", str(path))
    g = gg.rmat(13, 16, seed=gg.workload_seed(1) + 9)
    ref = oracle.bfscut(g, 10)
    c1 = t.tkc_create(t.Options())
    try:
        h = t.tkc_load_csr(c1, g.n, g.offsets, g.cols, g.directed)
        try:
            best = t.tkc_autotune(h, 10)
        finally:
            t.tkc_free_graph(h)
    finally:
        t.tkc_destroy(c1)
    lines = path.read_text().splitlines()
    assert len(lines) == 1
    m = re.fullmatch(r"(\w+)=(\d+),(\d+),(\d+),(\d+),([0-9.]+),(\d+)", lines[0])
    assert m and int(m.group(2)) == best.batch_bits and int(m.group(7)) == best.large_blocks
    for text, bits in ((lines[0], best.batch_bits), (f"{m.group(1)}=256,1,8,1,1.000", 256)):
        path.write_text(text + "\n")
        c2 = t.tkc_create(t.Options())
        try:
            h = t.tkc_load_csr(c2, g.n, g.offsets, g.cols, g.directed)
            try:
                res = t.tkc_topk_closeness(h, 10)
            finally:
                t.tkc_free_graph(h)
        finally:
            t.tkc_destroy(c2)
        assert res.batch_bits == bits
        _expect_equal(res, ref, g, 10)
