"""Checkpoint and resume of one exact top-k closeness run (Algorithm 1).

Algorithm 1 (Section 4) stays exact for any threshold x that is the k-th best
of exactly known farness values, so a run can stop after any prefix of its
source order and continue later from the k-list reached so far.  A checkpoint
after positions [0, p) holds:

  position  p;
  entries   the best min(k, n) finished searches so far, (S, r, id), best first;
  tied_kth  how many searches finished so far tie with entries[-1] (a full
            list), since Section 4 asks for every vertex tied with the k-th.

That is enough for an exact tie count at the end: a vertex finished before p
that ties with the final k-th has farness at most the checkpoint's k-th (the
threshold only falls), so it is either strictly better than the checkpoint's
k-th -- and then in its list -- or tied with it, and then counted in tied_kth.

The run goes in segments of `segment` positions: each segment is one call of
the library's part-of-the-order search (tkc_topk_closeness_shard with shard 0
of 1 from position p, seeded with the checkpoint's list), followed by a new
checkpoint.  A segment that examines fewer sources than it was given reached
the end of the order or Algorithm 1's stop (NBCut): the run is complete.
"""
from __future__ import annotations

import json
from dataclasses import asdict, dataclass, field
from typing import Callable, Optional, Protocol

from .shard import Entry, compare, same_farness


@dataclass
class Checkpoint:
    position: int = 0
    entries: list = field(default_factory=list)
    tied_kth: int = 0
    done: bool = False

    def dumps(self) -> str:
        return json.dumps(asdict(self))

    @staticmethod
    def loads(text: str) -> "Checkpoint":
        d = json.loads(text)
        return Checkpoint(int(d["position"]), [tuple(int(x) for x in e) for e in d["entries"]], int(d["tied_kth"]),
                          bool(d["done"]))


class Segments(Protocol):
    def search(self, first: int, count: int, seed: list[Entry]) -> tuple[list[Entry], int]:
        """Algorithm 1 over positions [first, first + count) of the order from
        the seeded k-list: (the resulting list best first, sources examined)."""

    def count_tied(self, entry: Entry) -> int:
        """Searches finished by the latest `search` tied with `entry`."""

    def closeness_zero_ties(self) -> int:
        """Vertices of out-degree 0 (all tied when the k-th has closeness 0)."""


def ties_before(ck: Checkpoint, kk: int, key: Entry) -> int:
    """Searches finished before the checkpoint that tie with `key`, a k-th
    reached after it (no worse than the checkpoint's k-th)."""
    if len(ck.entries) < kk:
        return sum(same_farness(e, key) for e in ck.entries)  # a short list holds every finished search
    kth = ck.entries[-1]
    if same_farness(kth, key):
        return ck.tied_kth
    assert compare(key, kth) < 0, "the threshold cannot rise"
    return sum(same_farness(e, key) for e in ck.entries)


def run(seg: Segments, kk: int, segment: int, resume: Optional[Checkpoint] = None,
        save: Optional[Callable[[Checkpoint], None]] = None,
        stop_after: Optional[int] = None) -> tuple[list[Entry], int, Checkpoint]:
    """Runs (or resumes) the search segment by segment; save(checkpoint) after
    each.  stop_after = n: return after n segments (an interrupted run).
    Returns (entries, n_tied_at_kth, last checkpoint); entries and the tie
    count are final only when the checkpoint is done."""
    if segment <= 0:
        raise ValueError("segment must be positive")
    ck = resume or Checkpoint()
    last: list[Entry] = []
    steps = 0
    while not ck.done and (stop_after is None or steps < stop_after):
        lst, examined = seg.search(ck.position, segment, list(ck.entries))
        last = lst
        entries = [e for e in lst if e[1] >= 2][:kk]
        tied = 0
        if len(entries) == kk:
            tied = ties_before(ck, kk, entries[-1]) + seg.count_tied(entries[-1])
        ck = Checkpoint(ck.position + segment, entries, tied, examined < segment)
        steps += 1
        if save:
            save(ck)
    if not ck.done:
        return list(ck.entries), ck.tied_kth, ck
    out = list(ck.entries)
    fill = sorted((e for e in last if e[1] <= 1), key=lambda e: e[2])
    out += fill[: kk - len(out)]
    tied = ck.tied_kth if len(ck.entries) == kk else seg.closeness_zero_ties()
    return out, tied, ck


class LibrarySegments:
    """Segments over the CUDA library for one graph handle (options.order
    DEG or NB on its context)."""

    def __init__(self, tkc, graph, k: int):
        self.tkc, self.g, self.k = tkc, graph, k
        self.last = None

    def search(self, first: int, count: int, seed: list[Entry]) -> tuple[list[Entry], int]:
        import numpy as np

        sd = None
        if seed:
            sd = (np.array([e[0] for e in seed], np.uint64), np.array([e[1] for e in seed], np.uint32),
                  np.array([e[2] for e in seed], np.uint32))
        self.last = self.tkc.tkc_topk_closeness_shard(self.g, self.k, 0, 1, count, sd, first=first)
        lst = [(int(S), int(r), int(i)) for S, r, i in zip(self.last.dist_sum, self.last.reach, self.last.ids)]
        return lst, int(self.last.bfs_started)

    def count_tied(self, entry: Entry) -> int:
        return self.tkc.tkc_count_tied(self.g, entry[0], entry[1])

    def closeness_zero_ties(self) -> int:
        return int(self.last.n_tied_at_kth)
