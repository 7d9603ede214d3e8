"""Exact top-k closeness with the sources of one graph sharded over ranks.

Algorithm 1 (Section 4) returns the exact top-k for any threshold x that is
the k-th best of exactly known farness values; only the pruning depends on
how tight x is.  So the source order can be split round-robin over ranks, each
holding a copy of the graph, with only the k best (S, r, id) entries
exchanged:

  1. opening: every rank searches the first `opening` sources of its shard;
     the ranks all-gather their k-lists and merge them into a seed (without
     the rank's own entries, which its next search finds again);
  2. every rank searches its whole shard starting from the seed (its x is then
     the k-th of the best entries found anywhere so far);
  3. the ranks all-gather their final k-lists and merge them: the best
     min(k, n) entries of the union (a vertex appears once: ids repeat when a
     seed entry is handed back) are the exact top-k;
  4. every vertex tied with the k-th was finished on its own rank (its bound
     never exceeds a threshold that is at least its farness), so the tie count
     is the all-reduced sum of each rank's finished searches tied with it.

The per-rank search is anything with the interface of `ShardSearch` (the
CUDA library's shard entry points in production; a CPU stand-in in tests), and
the exchange is two callables, so this module holds no device or transport
code.  Farness is compared exactly: S_a (r_b-1)^2 against S_b (r_a-1)^2 in
Python integers, ties by id.
"""
from __future__ import annotations

from dataclasses import dataclass
from functools import cmp_to_key
from typing import Callable, Protocol, Sequence

Entry = tuple[int, int, int]  # (S, r, id); r <= 1 marks a closeness-0 vertex


def compare(a: Entry, b: Entry) -> int:
    """Order of two entries by farness (n-1) S/(r-1)^2, then id; r <= 1 last."""
    (Sa, ra, ia), (Sb, rb, ib) = a, b
    inf_a, inf_b = ra <= 1, rb <= 1
    if inf_a != inf_b:
        return 1 if inf_a else -1
    if not inf_a:
        lhs, rhs = Sa * (rb - 1) ** 2, Sb * (ra - 1) ** 2
        if lhs != rhs:
            return -1 if lhs < rhs else 1
    return (ia > ib) - (ia < ib)


def same_farness(a: Entry, b: Entry) -> bool:
    (Sa, ra, _), (Sb, rb, _) = a, b
    if ra <= 1 or rb <= 1:
        return ra <= 1 and rb <= 1
    return Sa * (rb - 1) ** 2 == Sb * (ra - 1) ** 2


def merge(lists: Sequence[Sequence[Entry]], kk: int) -> list[Entry]:
    """The best kk entries of the union of several k-lists, one per vertex."""
    seen: dict[int, Entry] = {}
    for lst in lists:
        for e in lst:
            seen.setdefault(int(e[2]), (int(e[0]), int(e[1]), int(e[2])))
    return sorted(seen.values(), key=cmp_to_key(compare))[:kk]


class ShardSearch(Protocol):
    def search(self, max_sources: int, seed: list[Entry]) -> list[Entry]:
        """Algorithm 1 over this rank's shard (at most max_sources sources, 0 =
        all) from the seeded k-list; the resulting list, best first."""

    def count_tied(self, entry: Entry) -> int:
        """This rank's finished searches (of the latest `search`) with the
        same farness as `entry` (r >= 2)."""

    def closeness_zero_ties(self) -> int:
        """Vertices of out-degree 0 in the graph (all tied when the k-th has
        closeness 0)."""


@dataclass
class ShardedResult:
    entries: list[Entry]
    n_tied_at_kth: int


def topk_sharded(search: ShardSearch, kk: int, opening: int, allgather: Callable[[list[Entry]], list[list[Entry]]],
                 allreduce_sum: Callable[[int], int]) -> ShardedResult:
    """Steps 1-4 above on one rank; every rank calls it with the same kk and
    opening, and gets the same exact top-kk and tie count."""
    if kk == 0:
        return ShardedResult([], 0)
    seed: list[Entry] = []
    if opening > 0:
        mine = [e for e in search.search(opening, []) if e[1] >= 2]
        # this rank searches its own vertices again from the start: they stay
        # out of its seed (a k-list holds each vertex once)
        own = {e[2] for e in mine}
        seed = [e for e in merge(allgather(mine), kk) if e[2] not in own]
    final = merge(allgather(search.search(0, seed)), kk)
    kth = final[-1]
    if kth[1] >= 2:
        tied = allreduce_sum(search.count_tied(kth))
    else:
        tied = search.closeness_zero_ties()
    return ShardedResult(final, tied)


class LibraryShard:
    """ShardSearch over the CUDA library (tkc_topk_closeness_shard and
    tkc_count_tied) for one graph handle on this rank's context."""

    def __init__(self, tkc, graph, k: int, rank: int, world: int):
        self.tkc, self.g, self.k, self.rank, self.world = tkc, graph, k, rank, world
        self.last = None

    def search(self, max_sources: int, seed: list[Entry]) -> list[Entry]:
        import numpy as np

        sd = None
        if seed:
            sd = (np.array([e[0] for e in seed], np.uint64), np.array([e[1] for e in seed], np.uint32),
                  np.array([e[2] for e in seed], np.uint32))
        self.last = self.tkc.tkc_topk_closeness_shard(self.g, self.k, self.rank, self.world, max_sources, sd, first=0)
        return [(int(S), int(r), int(i)) for S, r, i in zip(self.last.dist_sum, self.last.reach, self.last.ids)]

    def count_tied(self, entry: Entry) -> int:
        return self.tkc.tkc_count_tied(self.g, entry[0], entry[1])

    def closeness_zero_ties(self) -> int:
        return int(self.last.n_tied_at_kth)


def torch_exchange(dist):
    """all-gather and sum over a torch.distributed process group (gloo or nccl)."""

    def allgather(entries: list[Entry]) -> list[list[Entry]]:
        out: list = [None] * dist.get_world_size()
        dist.all_gather_object(out, entries)
        return out

    def allreduce_sum(x: int) -> int:
        out: list = [None] * dist.get_world_size()
        dist.all_gather_object(out, int(x))
        return sum(out)

    return allgather, allreduce_sum
