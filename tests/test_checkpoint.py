"""Checkpoint and resume (paper_1704_01077_gb300.checkpoint) on the CPU: the
search of each segment is stood in by the oracle (exact S and r of the
segment's sources, merged with the seeded k-list as Algorithm 1's list would
be), so what is tested is the driver: its checkpoints, the tie count carried
across them, the JSON round trip and the resume.  Results must equal the
textbook top-k (Section 4), ties included, on families where many vertices
tie (cycles, hypercube, complete bipartite, stars) and on random graphs."""
import pytest

import oracle
from paper_1704_01077_gb300 import checkpoint as cp
from paper_1704_01077_gb300 import graphgen as gg
from paper_1704_01077_gb300 import shard


class OracleSegments:
    def __init__(self, g, kk):
        order = oracle.degree_order(g)
        self.order = [int(v) for v in order if g.outdeg()[v] > 0]
        S, r = oracle.bfs_sums(g) if g.n else ([], [])
        self.exact = {v: (int(S[v]), int(r[v])) for v in range(g.n)}
        self.g, self.kk = g, kk
        self.finished = []
        self.searched = set()

    def search(self, first, count, seed):
        part = self.order[first:first + count]
        assert not {e[2] for e in seed} & set(part)  # a k-list holds each vertex once
        assert not self.searched & set(part)  # a resumed run never searches a position twice
        self.searched |= set(part)
        self.finished = part
        lst = shard.merge([seed, [(self.exact[v][0], self.exact[v][1], v) for v in part]], self.kk)
        zeros = [v for v in range(self.g.n) if self.g.outdeg()[v] == 0]
        return lst + [(0, 1, v) for v in zeros[: self.kk - len(lst)]], len(part)

    def count_tied(self, entry):
        return sum(shard.same_farness((*self.exact[v], v), entry) for v in self.finished)

    def closeness_zero_ties(self):
        return int((self.g.outdeg() == 0).sum())


GRAPHS = [lambda: gg.cycle(12), lambda: gg.cycle(9, True), lambda: gg.hypercube(4), lambda: gg.complete_bipartite(3, 6),
          lambda: gg.star(10), lambda: gg.disjoint_union(gg.cycle(6), gg.path(5, True), gg.path(1)),
          lambda: gg.from_arcs(6, [], [], True)]
GRAPHS += [lambda s=s: gg.random_graph(14 + s % 9, [0.1, 0.25][s % 2], 400 + s, s % 3 == 0) for s in range(40)]


def _expect(entries, tied, ref, what):
    assert [e[2] for e in entries] == [int(x) for x in ref.ids], what
    assert [e[1] for e in entries] == [max(int(x), 1) for x in ref.r], what
    assert [e[0] for e in entries if e[1] >= 2] == [int(s) for s, r in zip(ref.S, ref.r) if r >= 2], what
    assert tied == ref.n_tied, what


@pytest.mark.parametrize("gi", range(len(GRAPHS)))
def test_segments_equal_textbook(gi):
    g = GRAPHS[gi]()
    for k in (1, 3, 5, g.n):
        ref = oracle.textbook_topk(g, k)
        kk = min(k, g.n)
        for segment in (1, 2, 3, 7, 1000):
            entries, tied, ck = cp.run(OracleSegments(g, kk), kk, segment)
            assert ck.done
            _expect(entries, tied, ref, (gi, k, segment))


@pytest.mark.parametrize("gi", [0, 2, 3, 5, 10, 20])
def test_interrupt_serialise_resume(gi):
    g = GRAPHS[gi]()
    for k in (2, 4):
        kk = min(k, g.n)
        ref = oracle.textbook_topk(g, k)
        seg = OracleSegments(g, kk)
        saved = []
        _, _, ck = cp.run(seg, kk, 2, save=lambda c: saved.append(c.dumps()), stop_after=2)
        if ck.done:
            continue
        back = cp.Checkpoint.loads(saved[-1])
        assert back == ck
        entries, tied, ck2 = cp.run(seg, kk, 2, resume=back)  # the same stand-in: no position searched twice
        assert ck2.done
        _expect(entries, tied, ref, (gi, k))


def test_tie_rule_cases():
    ck = cp.Checkpoint(4, [(3, 4, 1), (4, 4, 2), (4, 4, 5)], 3)
    assert cp.ties_before(ck, 3, (4, 4, 9)) == 3  # the checkpoint's own k-th value: its count
    assert cp.ties_before(ck, 3, (3, 4, 7)) == 1  # strictly better: the list holds all of them
    assert cp.ties_before(cp.Checkpoint(4, [(3, 4, 1)], 0), 3, (3, 4, 2)) == 1  # a short list holds all
    with pytest.raises(AssertionError):
        cp.ties_before(ck, 3, (9, 4, 8))


def test_planted_mistake_dropping_earlier_ties_is_caught(monkeypatch):
    monkeypatch.setattr(cp, "ties_before", lambda ck, kk, key: 0)
    with pytest.raises(AssertionError):
        test_segments_equal_textbook(0)  # a 12-cycle: every vertex ties
