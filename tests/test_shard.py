"""Sharding the sources of one graph over ranks (paper_1704_01077_gb300.shard),
on the CPU: real gloo process groups of 2 and 3 ranks drive the exchange and
the merge, with each rank's search stood in by the oracle (exact S and r of
every source of its shard, the k-list seeded as Algorithm 1's would be).  The
merged top-k, its (S, r) and the tie count must equal the textbook result
(Section 4), for several graphs, k and opening sizes."""
import os
import socket
from fractions import Fraction

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from paper_1704_01077_gb300 import graphgen as gg
from paper_1704_01077_gb300 import shard


class OracleShard:
    """Shard `rank` of `world` over the degree order's sources of out-degree >= 1."""

    def __init__(self, g, kk, rank, world):
        order = oracle.degree_order(g)
        srcs = [int(v) for v in order if g.outdeg()[v] > 0]
        self.mine = srcs[rank::world]
        self.g, self.kk = g, kk
        S, r = oracle.bfs_sums(g, np.array(self.mine, np.uint32)) if self.mine else ([], [])
        self.exact = {v: (int(s), int(x)) for v, s, x in zip(self.mine, S, r)}
        self.finished = []

    def search(self, max_sources, seed):
        # the library's contract: a seed holds no vertex of this shard
        assert not {e[2] for e in seed} & set(self.mine), "seed repeats a vertex of this shard"
        part = self.mine[:max_sources] if max_sources else self.mine
        self.finished = part
        lst = shard.merge([seed, [(self.exact[v][0], self.exact[v][1], v) for v in part]], self.kk)
        zeros = [v for v in range(self.g.n) if self.g.outdeg()[v] == 0]
        lst += [(0, 1, v) for v in zeros[: self.kk - len(lst)]]
        return lst

    def count_tied(self, entry):
        return sum(shard.same_farness((self.exact[v][0], self.exact[v][1], v), entry) for v in self.finished)

    def closeness_zero_ties(self):
        return int((self.g.outdeg() == 0).sum())


GRAPHS = {
    "ba": lambda: gg.barabasi_albert(300, 3, 4),
    "rmat": lambda: gg.rmat(9, 8, seed=5),
    "cycle": lambda: gg.cycle(12),
    "union": lambda: gg.disjoint_union(gg.cycle(6), gg.path(5, True), gg.path(1)),
    "sparse": lambda: gg.random_graph(40, 0.03, 8, True),
}


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        allgather, allreduce = shard.torch_exchange(dist)
        res = {}
        for name, make in GRAPHS.items():
            g = make()
            for k in (1, 3, 10, g.n + 2):
                kk = min(k, g.n)
                for opening in (0, 2):
                    r = shard.topk_sharded(OracleShard(g, kk, rank, world), kk, opening, allgather, allreduce)
                    res[(name, k, opening)] = (r.entries, r.n_tied_at_kth)
        out.put((rank, res))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_topk_equals_textbook_over_gloo(world):
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    got = dict(out.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for (name, k, opening), (entries, tied) in got[0].items():
        for r in range(1, world):
            assert got[r][(name, k, opening)] == (entries, tied)  # every rank ends with the same answer
        g = GRAPHS[name]()
        ref = oracle.textbook_topk(g, k)
        assert [e[2] for e in entries] == [int(x) for x in ref.ids], (name, k, opening)
        assert [e[0] for e in entries if e[1] >= 2] == [int(s) for s, r in zip(ref.S, ref.r) if r >= 2]
        assert [e[1] for e in entries] == [max(int(x), 1) for x in ref.r]
        assert tied == ref.n_tied, (name, k, opening)


def test_merge_orders_by_exact_farness():
    rng = np.random.default_rng(3)
    entries = [(int(rng.integers(1, 50)), int(rng.integers(1, 9)), i) for i in range(200)]
    want = sorted(entries, key=lambda e: (e[1] <= 1, Fraction(e[0], (e[1] - 1) ** 2) if e[1] > 1 else 0, e[2]))
    got = shard.merge([entries[:120], entries[80:], entries[50:60]], 37)
    assert got == want[:37]
