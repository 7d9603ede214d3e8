"""Stored values from the paper, checked against the oracle on the CPU.

tests/golden/reduction_section3.json instantiates, for one small
TwoDisjointSet instance, the reach and distance-sum counts that Section 3
prints for every vertex role of its reduction graph (each entry cites the
passage; the numbers were written by hand from those formulas, not computed by
any code of this repository)."""
import json
import os

import oracle
from paper_1704_01077_gb300 import graphgen as gg

HERE = os.path.dirname(os.path.abspath(__file__))


def test_reduction_graph_values_of_section3():
    d = json.load(open(os.path.join(HERE, "golden", "reduction_section3.json")))
    inst = d["instance"]
    g, ids = gg.reduction_graph(inst["X"], [set(s) for s in inst["sets"]], inst["p"], inst["q"])
    assert g.n == d["n"]
    assert {k: list(v) for k, v in ids.items()} == d["ranges"]
    S, r = oracle.bfs_sums(g)
    for e in d["expected"]:
        v = d["ranges"][e["role"]][0] + e["index"]
        assert (int(S[v]), int(r[v])) == (e["S"], e["r"]), e
    top, _ = oracle.topk(S, r, 1)
    m = d["most_central"]
    assert int(top[0]) == d["ranges"][m["role"]][0] + m["index"]
