"""Benchmark: exact top-k closeness (batched BFSCut) on a directed R-MAT graph.

One step = one full pass of the method through the C ABI: load the CSR
(validate, in-arc CSR), degree order, reach bounds (SCC / Algorithm 6), the
source order (by default computeBoundsNB: NBCut; --order degree: DegCut), the
persistent batched BFSCut kernel, and the output.

The metric is throughput at a fixed amount of work: the arcs that the paper's
own procedure (plain one-source-at-a-time NBCut, Algorithm 1) visits on the
workload -- its m_vis, counted once by the CPU oracle and stored with the
workload's exact top-k in tests/golden/fullsize_<workload>.json -- divided by
the step's wall time.  Work the batched search adds (more arcs under a
threshold that lags behind) therefore cannot raise the figure; only a shorter
wall time does.  The batched searches' own arcs visited are reported as
detail.  Alongside, the same process times the plain one-source BFSCut (NBCut,
and DegCut where it finishes in reasonable time) and the learned-seed order on
the same GPU (vs_plain), and checks every returned top-k against the stored
oracle result.

Prints ONE JSON line on rank 0.  `--impl reference` times the CPU oracle (the
sequential BFSCut of oracle/) on a bounded prefix of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (builder, k, description)
    "ba2000": (lambda gg: gg.barabasi_albert(2000, 4, gg.workload_seed(0)), 10,
               "undirected Barabasi-Albert n=2,000, m=4 (7,990 edges), k=10"),
    "rmat22": (lambda gg: gg.rmat(22, 16, seed=gg.workload_seed(4)), 10,
               "directed R-MAT scale 22 (4,194,304 vertices), edge factor 16, a/b/c/d=0.57/0.19/0.19/0.05, "
               "self-loops and duplicates removed, k=10"),
    "rmat16": (lambda gg: gg.rmat(16, 16, seed=gg.workload_seed(1)), 10,
               "directed R-MAT scale 16, edge factor 16, k=10"),
    "rmat20": (lambda gg: gg.rmat(20, 16, seed=gg.workload_seed(1)), 10,
               "directed R-MAT scale 20, edge factor 16, k=10 (profiling size: inputs above L2, a few GB)"),
    "ba1m": (lambda gg: gg.barabasi_albert(1_000_000, 5, gg.workload_seed(2)), 10,
             "undirected Barabasi-Albert n=1,000,000, m=5, k=10"),
    "grid1k": (lambda gg: gg.grid(1000, 1000, seed=gg.workload_seed(5), drop=0.1), 10,
               "undirected 1000 x 1000 grid, 10% of edges dropped (street-network stand-in), k=10"),
    "multi512": (lambda gg: multi_graphs(gg, 512, 1_000, 200_000, gg.workload_seed(3)), 10,
                 "512 graphs in one launch, n log-uniform in [1k, 200k]; even: undirected Barabasi-Albert m=4, "
                 "odd: directed Erdos-Renyi with 8n uniform arcs; top-10 of each"),
}


def multi_graphs(gg, count, lo, hi, seed):
    sizes = gg.log_uniform_sizes(count, lo, hi, seed)
    return [gg.barabasi_albert(n, 4, gg.splitmix64(seed + i)) if i % 2 == 0
            else gg.erdos_renyi(n, 8 * n, gg.splitmix64(seed + i), directed=True) for i, n in enumerate(sizes)]

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "bfscut_traffic.json")
KERNEL_SRC = os.path.join(ROOT, "paper_1704_01077_gb300", "csrc", "tkc_bfscut.cu")


def kernel_hash() -> str:
    return hashlib.sha256(open(KERNEL_SRC, "rb").read()).hexdigest()[:16]


def hbm_peak():
    try:
        with open(PEAKS_FILE) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def ncu_traffic(workload: str, order: str, bits: int):
    """DRAM bytes per step (all launches) of the search kernel from a committed
    ncu summary, only if it was taken on the current kernel source."""
    try:
        with open(TRAFFIC_FILE) as f:
            d = json.load(f)
        e = d.get(f"{workload}_{order}_b{bits}")
        if e and e.get("kernel_sha") == kernel_hash():
            return e["dram_bytes_per_step"], e
    except Exception:
        pass
    return None, None


class ClockSampler:
    """nvidia-smi samples during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", f"tkc_clocks_{os.getpid()}.csv")

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_over_ranks(ms_total, edges, dist, device, shared=False):
    """Whole-job figures over the ranks: the slowest rank's time, and the work
    of all ranks -- summed when each rank ran its own replica, taken once when
    the ranks shared one query (shared=True: sources sharded over the ranks).
    One rank (dist None): unchanged."""
    if not dist:
        return float(ms_total), float(edges)
    import torch

    t = torch.tensor([float(ms_total)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if shared:
        return float(t.item()), float(edges)
    e = torch.tensor([float(edges)], device=device, dtype=torch.float64)
    dist.all_reduce(e)
    return float(t.item()), float(e.item())


METRIC = "top-k closeness wall time & GTEPS, batched/learned vs plain BFSCut, exact top-k"
GOLDEN = os.path.join(ROOT, "tests", "golden")


def fixture_for(workload: str, measure: str = "closeness"):
    """The stored oracle result of a workload (tests/golden/fullsize_*.json), or None."""
    name = workload + ("_harmonic" if measure == "harmonic" else "")
    path = os.path.join(GOLDEN, f"fullsize_{name}.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        return json.load(f)


def fixture_results(fx, k):
    """Per graph, the stored result for this k (None where k was not stored)."""
    out = []
    for g in fx["graphs"]:
        out.append(next((r for r in g["results"] if r["k"] == k), None))
    return out


def plain_work(fx, k):
    """Arcs visited by the oracle's plain one-source NBCut over the workload's
    graphs (the fixed work of the metric), or None."""
    if fx is None:
        return None
    rs = fixture_results(fx, k)
    if any(r is None for r in rs):
        return None
    return sum(int(r["oracle_counters"]["edges_visited"]) for r in rs)


def csr_sha256(g) -> str:
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(g.offsets, dtype="<u4").tobytes())
    h.update(np.ascontiguousarray(g.cols, dtype="<u4").tobytes())
    return h.hexdigest()


def matches_fixture(results, fx, k, graphs, measure="closeness"):
    """Every graph's top-k (ids, S, r, tie count, farness bits; harmonic: ids,
    h bits, r, ties) equals the stored oracle result on the same graph."""
    if fx is None:
        return None
    want = fixture_results(fx, k)
    if len(want) != len(results) or any(w is None for w in want):
        return False
    for g, e, res, w in zip(graphs, fx["graphs"], results, want):
        if csr_sha256(g) != e["csr_sha256"]:
            return False
        if [int(x) for x in res.ids] != w["ids"] or [int(x) for x in res.reach] != w["r"]:
            return False
        if res.n_tied_at_kth != w["n_tied"]:
            return False
        if measure == "harmonic":
            if [float(h).hex() for h in res.closeness] != w["h_hex"]:
                return False
        elif [int(x) for x in res.dist_sum] != w["S"] or [float(f).hex() for f in res.farness] != w["farness_hex"]:
            return False
    return True


def survey_level_bytes(st) -> float:
    """Bytes of the level kernels by the per-level formula of the design plan
    (B-bit rows of B/8 bytes), reported beside the kernel's own count: it
    charges three row sweeps of all n vertices at every level, which this
    kernel does not perform (it touches only listed vertices), so on runs of
    many short levels it exceeds what any memory could move in the time:
      top-down : sum over frontier u of (8 + 4 outdeg(u) + B/8)
                 + 2 (B/8) sum over frontier u of outdeg(u) + 3 (B/8) n
      bottom-up: sum over scanned w of (8 + (4 + B/8) scanned_in(w)) + 3 (B/8) n
    from the run's per-level totals (tkc_last_run_stats)."""
    rb = st["batch_bits"] / 8.0 if st["batch_bits"] >= 8 else st["row_bytes"]
    n = st["n"]
    td = (st["td_frontier"] * (8 + rb) + 4 * st["td_frontier_arcs"] + 2 * rb * st["td_frontier_arcs"]
          + 3 * rb * n * st["td_levels"])
    bu = 8 * st["bu_scanned_vertices"] + (4 + rb) * st["bu_scanned_arcs"] + 3 * rb * n * st["bu_levels"]
    return float(td + bu)


def host_cpu():
    """Core count and model of the host the CPU figures were taken on."""
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    import platform

    return {"nproc": os.cpu_count(), "machine": platform.machine(), "model": model}


def cpu_oracle_sample(g, k, sample_sources):
    """Sequential CPU BFSCut (the oracle as it stands) on a prefix of the
    degree order; returns (GTEPS, seconds, edges_visited)."""
    import oracle

    t0 = time.perf_counter()
    res = oracle.bfscut(g, k, max_sources=sample_sources)
    dt = time.perf_counter() - t0
    ev = res.counters.edges_visited
    return ev / dt / 1e9, dt, ev


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    from paper_1704_01077_gb300 import graphgen as gg

    build, k, desc = WORKLOADS[args.workload]
    g = build(gg)
    if isinstance(g, list):  # several graphs: the sample is taken from the largest
        g = max(g, key=lambda x: x.arcs)
    for _ in range(args.warmup):
        cpu_oracle_sample(g, k, args.ref_sample)
    vals, times, evs = [], [], []
    for _ in range(args.steps):
        v, dt, ev = cpu_oracle_sample(g, k, args.ref_sample)
        vals.append(v)
        times.append(dt)
        evs.append(ev)
    value = sum(evs) / sum(times) / 1e9
    sample = (f"first {args.ref_sample} sources of the degree order of {g.name} (sequential CPU BFSCut, incl. its "
              f"preprocessing), per step; rate = arcs the plain one-source BFSCut visits per second")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GTEPS",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * statistics.mean(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": args.workload, "description": desc, "k": k},
            "cpu_baseline": {"value": value, "unit": "GTEPS", "cores": 1, "kind": "oracle", "sample": sample,
                             "host": host_cpu()},
            "e2e": {"value": value, "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="tkc", choices=["tkc", "reference"])
    ap.add_argument("--workload", default="rmat22", choices=sorted(WORKLOADS))
    ap.add_argument("--bits", type=int, default=0, help="source batch width (0 = library default)")
    ap.add_argument("--no-plain", action="store_true",
                    help="skip the plain one-source runs and the learned-seed arm (vs_plain)")
    ap.add_argument("--plain-degcut", default="auto", choices=["auto", "yes", "no"],
                    help="also time plain one-source DegCut (auto: on graphs below 2^22 vertices)")
    ap.add_argument("--sample", type=int, default=96, help="CPU oracle sample: number of sources")
    ap.add_argument("--ref-sample", type=int, default=32,
                    help="--impl reference: sources per step (about 4 s of CPU work each on R-MAT 22)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-check", action="store_true")
    ap.add_argument("--k", type=int, default=0, help="top-k (0 = the workload's k)")
    ap.add_argument("--order", default="nb", choices=["degree", "nb", "learned", "learned-seed", "learned-nb"],
                    help="source order: degree bound (DegCut), neighbourhood bound with its stop (NBCut), "
                         "learned model, learned seeding prefix + degree, or learned seeding prefix + NBCut")
    ap.add_argument("--nb-levels", type=int, default=0, help="NBCut: most sweeps of the bound (0 = 256)")
    ap.add_argument("--measure", default="closeness", choices=["closeness", "harmonic"],
                    help="rank by closeness (the paper's main measure) or harmonic centrality")
    ap.add_argument("--bound", default="cut", choices=["cut", "lb"],
                    help="updateBounds: BFSCut (cut) or updateBoundsLB (lb: DegBound / NBBound)")
    ap.add_argument("--teams", type=int, default=0, help="teams of SMs (0 = library default)")
    ap.add_argument("--bu-num", type=int, default=0,
                    help="a level runs bottom-up when its frontier arcs exceed arcs / BU_NUM (0 = library default)")
    ap.add_argument("--deterministic", type=int, default=0, help="1: one team, reproducible counters")
    ap.add_argument("--relabel", type=int, default=0, choices=[0, 1, 2],
                    help="search on the in-degree labelling: 0 = library choice, 1 = always, 2 = never")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "tkc":
        args.warmup = 3
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch

    from paper_1704_01077_gb300 import graphgen as gg
    from paper_1704_01077_gb300 import tkc

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    build, k, desc = WORKLOADS[args.workload]
    k = args.k or k
    built = build(gg)
    multi = isinstance(built, list)
    graphs = built if multi else [built]
    g = graphs[0]
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    dev_csr = [(torch.from_numpy(x.offsets.view(np.int32)).to(dev), torch.from_numpy(x.cols.view(np.int32)).to(dev))
               for x in graphs]
    host_csr = [(torch.from_numpy(x.offsets.view(np.int32)).pin_memory(),
                 torch.from_numpy(x.cols.view(np.int32)).pin_memory()) for x in graphs]
    orders = {"degree": tkc.TKC_ORDER_DEG, "nb": tkc.TKC_ORDER_NB, "learned": tkc.TKC_ORDER_LEARNED,
              "learned-seed": tkc.TKC_ORDER_LEARNED, "learned-nb": tkc.TKC_ORDER_LEARNED_NB}
    base_opt = dict(device=local, stream=stream.cuda_stream, batch_bits=args.bits, order=orders[args.order],
                    teams=args.teams, seed_factor=5 if args.order in ("learned-seed", "learned-nb") else 0,
                    nb_levels=args.nb_levels, deterministic=args.deterministic, bu_num=args.bu_num, bu_den=1,
                    relabel=args.relabel)
    ctx = tkc.tkc_create(tkc.Options(**base_opt))
    weights = None
    if args.order.startswith("learned") or (not args.no_plain and not multi and args.measure == "closeness"):
        from paper_1704_01077_gb300.train_order import load_weights

        weights = load_weights()
        if weights is not None:
            tkc.tkc_set_source_model(ctx, weights)
    fx = fixture_for(args.workload, args.measure) if args.bound == "cut" or args.measure == "closeness" else None
    work_fixed = plain_work(fx, k)

    class Step:
        """One step's results summed over the graphs it ran."""

        def __init__(self, results):
            self.results = results
            r0 = results[0]
            self.edges_visited = sum(r.edges_visited for r in results)
            self.bfs_started = sum(r.bfs_started for r in results)
            self.bfs_cut = sum(r.bfs_cut for r in results)
            self.bfs_finished = sum(r.bfs_finished for r in results)
            for name in ("edges_scanned", "levels", "ms_pre", "ms_bfs", "ms_kernel", "alg_bytes", "batch_bits",
                         "ids", "dist_sum", "reach", "closeness"):
                setattr(self, name, getattr(r0, name))

    # several GPUs on one graph: the sources are sharded over the ranks (the
    # k best entries exchanged after an opening batch and at the end)
    sharded = world > 1 and not multi and args.measure == "closeness" and args.bound == "cut" and \
        args.order in ("nb", "degree")
    if sharded:
        from types import SimpleNamespace

        from paper_1704_01077_gb300 import shard

        allgather, allreduce = shard.torch_exchange(dist)
        opening = args.bits or (128 if args.order == "nb" and g.n >= (1 << 16) else 64)

    def run_sharded(h):
        ls = shard.LibraryShard(tkc, h, k, rank, world)
        kk = min(k, g.n)
        res = shard.topk_sharded(ls, kk, opening, allgather, allreduce)
        mine = ls.last
        S = np.array([e[0] for e in res.entries], np.uint64)
        r = np.array([e[1] for e in res.entries], np.uint32)
        far = np.array([float(g.n - 1) * float(a) / float((int(b) - 1) ** 2) if b > 1 else float("inf")
                        for a, b in zip(S, r)])
        view = SimpleNamespace(ids=np.array([e[2] for e in res.entries], np.uint32), dist_sum=S, reach=r,
                               farness=far, closeness=np.where(far > 0, 1.0 / far, 0.0),
                               n_tied_at_kth=res.n_tied_at_kth)
        for name in ("edges_visited", "bfs_started", "bfs_cut", "bfs_finished", "edges_scanned", "levels", "ms_pre",
                     "ms_bfs", "ms_kernel", "alg_bytes", "batch_bits"):
            setattr(view, name, getattr(mine, name))
        return Step([view])

    def run_step(csr):
        if multi:  # many graphs: validated with one host wait for all
            hs = tkc.tkc_load_csr_many(ctx, [(x.n, o, c, x.directed) for x, (o, c) in zip(graphs, csr)])
        else:
            hs = [tkc.tkc_load_csr(ctx, x.n, o, c, x.directed) for x, (o, c) in zip(graphs, csr)]
        try:
            if sharded:
                return run_sharded(hs[0])
            if args.bound == "lb":
                if multi or args.measure != "closeness":
                    raise SystemExit("--bound lb runs closeness on one graph")
                return Step([tkc.tkc_topk_closeness_bound(hs[0], k)])
            if args.measure == "harmonic":
                if multi:
                    return Step(tkc.tkc_topk_harmonic_multi(ctx, hs, k))
                return Step([tkc.tkc_topk_harmonic(hs[0], k)])
            if multi:
                return Step(tkc.tkc_topk_closeness_multi(ctx, hs, k))
            return Step([tkc.tkc_topk_closeness(hs[0], k)])
        finally:
            for h in hs:
                tkc.tkc_free_graph(h)

    def step_device():
        return run_step(dev_csr)

    def step_host():
        return run_step(host_csr)

    def timed_arm(opts, repeats):
        """Median device time (ms) of `repeats` steps under other options, and the last result."""
        tkc.tkc_set_options(ctx, tkc.Options(**dict(base_opt, **opts)))
        try:
            times, res = [], None
            for _ in range(repeats):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record(stream)
                res = step_device()
                e1.record(stream)
                torch.cuda.synchronize()
                times.append(e0.elapsed_time(e1))
            return statistics.median(times), res
        finally:
            tkc.tkc_set_options(ctx, tkc.Options(**base_opt))

    for _ in range(args.warmup):
        res = step_device()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches0 = tkc.tkc_kernel_launches()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    results = []
    stats = []
    with ClockSampler(torch.cuda.current_device()) as clk:
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            results.append(step_device())
            stats.append(tkc.tkc_last_run_stats(ctx))
        ev1.record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches = tkc.tkc_kernel_launches() - launches0
    own_edges = sum(r.edges_visited for r in results)
    # fixed work per step: the plain one-source NBCut's arcs (oracle-counted);
    # without a stored oracle result, the batched search's own arcs
    work = work_fixed if work_fixed is not None else statistics.mean(r.edges_visited for r in results)
    ms_total, total_work = reduce_over_ranks(ev0.elapsed_time(ev1), work * args.steps, dist, dev, shared=sharded)
    value = total_work / (ms_total / 1e3) / 1e9
    ms_step = ms_total / args.steps

    # end to end: host (pinned) CSR in, results out, copies inside the timed region
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    # one untimed step first: the first transfer out of the pinned buffers
    # maps them for the copy engines (a few ms, once), as warm-up did for the
    # device-resident steps
    step_host()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    e2e_steps = max(1, min(args.steps, 10))
    t0 = time.perf_counter()
    e2e_res = [step_host() for _ in range(e2e_steps)]
    torch.cuda.synchronize()
    e2e_ms, e2e_work = reduce_over_ranks((time.perf_counter() - t0) * 1e3, work * e2e_steps, dist, dev,
                                         shared=sharded)
    e2e_value = e2e_work / (e2e_ms / 1e3) / 1e9
    h2d = sum(4 * (x.n + 1) + 4 * x.arcs for x in graphs)
    d2h = len(graphs) * k * (4 + 8 + 4 + 8 + 8)

    # roofline of the dominant kernel (the persistent search kernel)
    peak, peak_src = hbm_peak()
    kern_ms = statistics.mean(st["ms_kernel"] for st in stats)
    kern_bytes = statistics.mean(st["alg_bytes"] for st in stats)
    plan_bytes = statistics.mean(survey_level_bytes(st) for st in stats)
    achieved = kern_bytes / (kern_ms / 1e3) / 1e9
    achieved_plan = plan_bytes / (kern_ms / 1e3) / 1e9
    traffic, traffic_entry = (ncu_traffic(args.workload, args.order, res.batch_bits)
                              if args.measure == "closeness" and args.bound == "cut" else (None, None))
    launches_per_step = stats[-1]["launches"]
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "peak_source": peak_src,
                "bytes_model": "the level kernels' own accesses at their load sizes (top-down: per frontier vertex "
                               "its list entry, offsets, row read and clear; per frontier arc its column, the "
                               "target's seen row and next-row update; per new vertex list, seen and row writes. "
                               "Bottom-up: per swept vertex its list entry and seen row; per scanned vertex its "
                               "in-offsets; per scanned in-arc its column and frontier-bitmap word; per frontier "
                               "in-neighbour found its row; per new vertex list, seen and row writes) -- "
                               "tkc_result.alg_bytes, summed on the device",
                "alg_bytes_per_step": kern_bytes, "kernel_ms_per_step": kern_ms,
                "launches_per_step": launches_per_step, "per": "step (all launches of the search kernel)",
                "plan_formula_bytes_per_step": plan_bytes, "achieved_plan_formula": achieved_plan}
    if traffic is not None:
        roofline["traffic_frac"] = traffic / (kern_ms / 1e3) / 1e9 / peak

    last = results[-1]
    st = stats[-1]
    line = {"metric": METRIC, "value": value, "unit": "GTEPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "strong" if sharded else "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": args.workload, "description": desc, "k": k, "batch_bits": res.batch_bits,
                       "order": args.order, "measure": args.measure, "bound": args.bound,
                       "teams": args.teams or "library default", "bu_num": args.bu_num or "library default", "deterministic": args.deterministic,
                       "relabel": args.relabel or "library default",
                       "work_per_step": work,
                       "work_unit": ("arcs visited by plain one-source NBCut (Algorithm 1), counted by the CPU "
                                     "oracle on the same graph" if work_fixed is not None else
                                     "arcs visited by this batched search (no stored oracle count)"),
                       "l2": "inputs larger than L2 (CSR 280 MB + bit rows)" if args.workload in
                       ("rmat22", "multi512", "ba1m") else "small graph: may be L2-resident",
                       "parallelism": (f"sources sharded over {world} GPUs, k best entries exchanged over NCCL"
                                       if sharded else f"replicas x{world}" if world > 1 else "single")},
            "e2e": {"value": e2e_value, "unit": "GTEPS", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "ms_per_step": e2e_ms / e2e_steps},
            "roofline": roofline, "gpu_launches": launches, "clocks": clk.summary(),
            "detail": {"wall_ms_per_step": ms_step,
                       "edges_visited": last.edges_visited, "edges_scanned": last.edges_scanned,
                       "own_gteps": own_edges / (ms_total / 1e3) / 1e9 if world == 1 else None,
                       "bfs_started": last.bfs_started, "bfs_cut": last.bfs_cut,
                       "bfs_finished": last.bfs_finished, "levels": last.levels,
                       "ms_pre": last.ms_pre, "ms_bfs": last.ms_bfs, "ms_kernel": last.ms_kernel,
                       "level_stats": st,
                       "textbook_teps_equiv": sum(x.arcs * x.n for x in graphs) / (ms_step / 1e3) / 1e9,
                       "graphs": len(graphs), "vertices": sum(x.n for x in graphs),
                       "arcs": sum(x.arcs for x in graphs),
                       "top_ids": [int(x) for x in last.ids]}}
    if rank == 0 and not args.no_check:
        import oracle

        ok = True
        for x, top in zip(graphs, last.results):
            if args.measure == "harmonic":
                H, r = oracle.harmonic_sums(x, top.ids)
                ok &= bool(H.tobytes() == top.closeness.tobytes() and np.array_equal(r, top.reach))
            else:
                S, r = oracle.bfs_sums(x, top.ids)
                ok &= bool(np.array_equal(S, top.dist_sum) and np.array_equal(r, top.reach))
        key = "top_k_h_r_match_oracle_bfs" if args.measure == "harmonic" else "top_k_S_r_match_oracle_bfs"
        line["check"] = {key: ok}
        if args.bound == "cut" or args.measure == "closeness":
            line["check"]["top_k_matches_oracle_fixture"] = matches_fixture(last.results, fx, k, graphs,
                                                                            args.measure)
    if rank == 0 and world == 1 and not args.no_plain and not multi and args.measure == "closeness" and \
            args.bound == "cut":
        arms = {}

        def arm(name, opts, repeats):
            ms, r = timed_arm(opts, repeats)
            arms[name] = {"ms": ms, "edges_visited": r.edges_visited, "bfs_started": r.bfs_started,
                          "bfs_cut": r.bfs_cut, "batch_bits": r.batch_bits,
                          "matches_oracle_fixture": matches_fixture(r.results, fx, k, graphs)}
            return ms

        plain_nb = arm("plain_nbcut", dict(order=tkc.TKC_ORDER_NB, batch_bits=1, seed_factor=0), 1)
        do_deg = args.plain_degcut == "yes" or (args.plain_degcut == "auto" and g.n < (1 << 22))
        plain_deg = arm("plain_degcut", dict(order=tkc.TKC_ORDER_DEG, batch_bits=1, seed_factor=0), 1) \
            if do_deg else None
        arm("batched_degcut", dict(order=tkc.TKC_ORDER_DEG, batch_bits=0, seed_factor=0), 3)
        arms["batched_nbcut"] = {"ms": ms_step, "edges_visited": last.edges_visited, "bfs_started": last.bfs_started,
                                 "bfs_cut": last.bfs_cut, "batch_bits": last.batch_bits,
                                 "matches_oracle_fixture": line.get("check", {}).get("top_k_matches_oracle_fixture")}
        if weights is not None:
            arm("batched_learned_seed_nbcut", dict(order=tkc.TKC_ORDER_LEARNED_NB, batch_bits=0, seed_factor=5), 3)
        vp = {"arms": arms, "plain_ms": plain_nb, "batched_ms": ms_step, "speedup": plain_nb / ms_step,
              "plain": "one source per search (B = 1), one team, NBCut order and stop, same GPU",
              "target": 5.0}
        if plain_deg is not None:
            vp["speedup_vs_plain_degcut"] = plain_deg / ms_step
        if "batched_learned_seed_nbcut" in arms:
            lm = arms["batched_learned_seed_nbcut"]["ms"]
            vp["learned_seed_speedup_vs_plain"] = plain_nb / lm
            vp["learned_seed_vs_nbcut_time_ratio"] = lm / ms_step
        line["vs_plain"] = vp
    if rank == 0 and world == 1 and not args.no_cpu and not multi:
        v, dt, ev = cpu_oracle_sample(g, k, args.sample)
        line["cpu_baseline"] = {"value": v, "unit": "GTEPS", "cores": 1, "kind": "oracle", "host": host_cpu(),
                                "sample": f"first {args.sample} sources of the degree order, sequential CPU "
                                          f"BFSCut incl. its preprocessing ({dt:.1f} s, {ev} edges); rate = arcs "
                                          f"of the plain one-source BFSCut per second"}
        if fx is not None:
            secs = sum(r["seconds"] for r in fixture_results(fx, k) if r)
            line["cpu_baseline"]["full_run"] = {
                "seconds": secs, "host": fx.get("host"),
                "what": "the oracle's complete plain NBCut on this workload, when the stored result was written "
                        "(another host: context only)"}
    tkc.tkc_destroy(ctx)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
