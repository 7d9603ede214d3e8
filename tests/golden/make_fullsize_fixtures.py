"""Writes tests/golden/fullsize_<workload>.json: the exact top-k of the full-size
benchmark workloads, computed by the CPU oracle alone.

The oracle used is Algorithm 1 with computeBoundsNB's order and stop (Section
5) and updateBoundsBFSCut (Section 6, Algorithm 4), reach bounds by Algorithm 6
(Section 8), one source at a time, run to completion: `oracle.bfscut` with the
`oracle.nb_bounds` key.  Its top-k (ids by farness then id, S, r, the count of
vertices tied with the k-th) equals the textbook all-sources result, which is
pinned on thousands of small graphs by the oracle's own tests; at these sizes
it is the only feasible oracle.  Nothing here calls the CUDA library.

Each fixture records how its graph was generated and a SHA-256 of its CSR, so
a test on another machine can check that it rebuilt the same graph.

    python tests/golden/make_fullsize_fixtures.py [--only rmat22,ba1m,multi512,rmat22_harmonic] [--jobs 8]

Run time on an 8-core x86 host: R-MAT scale 22 dominates (see the `seconds`
field of each entry).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import platform
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)



def out_path(name: str) -> str:
    return os.path.join(HERE, f"fullsize_{name}.json")

# Workload recipes: the same generators and seeds as the benchmark's.
RECIPES = {
    "rmat22": {"gen": "rmat", "scale": 22, "edge_factor": 16, "seed_index": 4, "k": [10]},
    "ba1m": {"gen": "ba", "n": 1_000_000, "m": 5, "seed_index": 2, "k": [1, 10, 100]},
    "multi512": {"gen": "multi", "count": 512, "lo": 1_000, "hi": 200_000, "seed_index": 3, "k": [10]},
    "rmat22_harmonic": {"gen": "rmat", "scale": 22, "edge_factor": 16, "seed_index": 4, "k": [10],
                        "measure": "harmonic"},
}


def csr_sha256(g) -> str:
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(g.offsets, dtype="<u4").tobytes())
    h.update(np.ascontiguousarray(g.cols, dtype="<u4").tobytes())
    return h.hexdigest()


def build_graphs(name):
    """The workload's graph(s), in the benchmark's order."""
    from paper_1704_01077_gb300 import graphgen as gg

    rc = RECIPES[name]
    seed = gg.workload_seed(rc["seed_index"])
    if rc["gen"] == "rmat":
        return [gg.rmat(rc["scale"], rc["edge_factor"], seed=seed)]
    if rc["gen"] == "ba":
        return [gg.barabasi_albert(rc["n"], rc["m"], seed)]
    sizes = gg.log_uniform_sizes(rc["count"], rc["lo"], rc["hi"], seed)
    return [gg.barabasi_albert(n, 4, gg.splitmix64(seed + i)) if i % 2 == 0
            else gg.erdos_renyi(n, 8 * n, gg.splitmix64(seed + i), directed=True) for i, n in enumerate(sizes)]


def solve_closeness(g, ks):
    """Oracle NBCut, run to completion, for every k in ks."""
    import oracle

    nb = oracle.nb_bounds(g)
    order = oracle.nb_full_order(g, nb.key)
    out = []
    for k in ks:
        t0 = time.perf_counter()
        res = oracle.bfscut(g, k, order=order, lb_key=nb.key)
        dt = time.perf_counter() - t0
        far = [oracle.farness(g.n, int(s), int(r))[0] for s, r in zip(res.S, res.r)]
        out.append({"k": k, "ids": [int(x) for x in res.ids], "S": [int(x) for x in res.S],
                    "r": [int(x) for x in res.r], "n_tied": res.n_tied,
                    "farness_hex": [float(f).hex() for f in far],
                    "oracle_counters": {"edges_visited": res.counters.edges_visited,
                                        "bfs_started": res.counters.bfs_started,
                                        "bfs_cut": res.counters.bfs_cut,
                                        "bfs_finished": res.counters.bfs_finished},
                    "seconds": round(dt, 2)})
    return out


def solve_harmonic(g, ks):
    import oracle

    nb = oracle.nb_bounds(g)
    order = np.concatenate([oracle.nb_harmonic_order(g, nb.h_ub), np.nonzero(g.outdeg() == 0)[0].astype(np.uint32)])
    out = []
    for k in ks:
        t0 = time.perf_counter()
        res = oracle.bfscut_harmonic(g, k, order=order, ub=nb.h_ub)
        dt = time.perf_counter() - t0
        out.append({"k": k, "ids": [int(x) for x in res.ids], "h_hex": [float(h).hex() for h in res.H],
                    "r": [int(x) for x in res.r], "n_tied": res.n_tied,
                    "oracle_counters": {"edges_visited": res.counters.edges_visited,
                                        "bfs_started": res.counters.bfs_started,
                                        "bfs_cut": res.counters.bfs_cut,
                                        "bfs_finished": res.counters.bfs_finished},
                    "seconds": round(dt, 2)})
    return out


def _one_graph(args):
    name, index = args
    g = build_graphs(name)[index]
    rc = RECIPES[name]
    t0 = time.perf_counter()
    res = solve_harmonic(g, rc["k"]) if rc.get("measure") == "harmonic" else solve_closeness(g, rc["k"])
    return {"index": index, "n": g.n, "arcs": g.arcs, "directed": bool(g.directed), "name": g.name,
            "csr_sha256": csr_sha256(g), "results": res, "seconds_total": round(time.perf_counter() - t0, 2)}


def make(name, jobs):
    from paper_1704_01077_gb300 import graphgen as gg

    rc = RECIPES[name]
    count = rc.get("count", 1)
    t0 = time.perf_counter()
    work = [(name, i) for i in range(count)]
    if count == 1:
        graphs = [_one_graph(work[0])]
    else:
        # the biggest graphs first so that the pool ends together
        sizes = gg.log_uniform_sizes(rc["count"], rc["lo"], rc["hi"], gg.workload_seed(rc["seed_index"]))
        work.sort(key=lambda w: -sizes[w[1]])
        with mp.get_context("spawn").Pool(jobs) as pool:
            graphs = sorted(pool.map(_one_graph, work, chunksize=1), key=lambda e: e["index"])
    return {"recipe": rc, "seed": gg.workload_seed(rc["seed_index"]), "graphs": graphs,
            "method": ("oracle.bfscut_harmonic with the nb_bounds upper bound on h (NBCut order and stop)"
                       if rc.get("measure") == "harmonic" else
                       "oracle.bfscut with the nb_bounds key (NBCut order and stop), one source at a time"),
            "host": {"machine": platform.machine(), "cpus": os.cpu_count()},
            "seconds": round(time.perf_counter() - t0, 1)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--only", default=",".join(RECIPES))
    ap.add_argument("--jobs", type=int, default=os.cpu_count() or 1)
    args = ap.parse_args()
    for name in args.only.split(","):
        print(f"[fixtures] {name} ...", flush=True)
        entry = make(name, args.jobs)
        entry["about"] = ("Exact top-k by the CPU oracle, written by tests/golden/make_fullsize_fixtures.py; "
                          "no value comes from the CUDA library.")
        print(f"[fixtures] {name} done in {entry['seconds']} s", flush=True)
        tmp = out_path(name) + ".tmp"
        with open(tmp, "w") as f:
            json.dump(entry, f, separators=(",", ":"))
            f.write("\n")
        os.replace(tmp, out_path(name))


if __name__ == "__main__":
    main()
