"""Python binding of the CUDA library ``libtkc.so`` (C ABI in include/tkc.h).

Argument marshalling only: every function here converts Python/numpy/torch
arguments to the C call of the same name and converts results back.  All
computation happens in the library's CUDA kernels; if the library is missing
the import fails (there is no CPU fallback).

Host inputs are numpy arrays; device inputs may be torch CUDA tensors (their
data pointers are passed with ``ptr_on_device=1``).  PyTorch is used only for
streams and device memory.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtkc.so")

TKC_OK = 0
TKC_EINVAL = -1
TKC_EGRAPH = -2
TKC_ENOMEM = -3
TKC_ECUDA = -4
TKC_ETIMEOUT = -5
TKC_EOVERFLOW = -6

TKC_ORDER_DEG = 0
TKC_ORDER_GIVEN = 1
TKC_ORDER_LEARNED = 2
TKC_ORDER_NB = 3
TKC_ORDER_LEARNED_NB = 4
TKC_MAX_K = 1024
TKC_NOALLOC_MAX_N = 65536
TKC_MLP_FEATURES = 5
TKC_MLP_HIDDEN = 64
TKC_MLP_PARAMS = 4609


class TkcError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {tkc_strerror(code)} ({code})")


class tkc_options(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("stream", ctypes.c_void_p), ("order", ctypes.c_uint32),
                ("batch_bits", ctypes.c_uint32), ("bu_num", ctypes.c_uint32), ("bu_den", ctypes.c_uint32),
                ("blocks", ctypes.c_uint32), ("seed_factor", ctypes.c_uint32),
                ("timeout_cycles", ctypes.c_uint64), ("teams", ctypes.c_uint32), ("nb_levels", ctypes.c_uint32),
                ("large_blocks", ctypes.c_uint32), ("deterministic", ctypes.c_uint32), ("relabel", ctypes.c_uint32)]


class tkc_result(ctypes.Structure):
    _fields_ = [("ids", ctypes.POINTER(ctypes.c_uint32)), ("dist_sum", ctypes.POINTER(ctypes.c_uint64)),
                ("reach", ctypes.POINTER(ctypes.c_uint32)), ("farness", ctypes.POINTER(ctypes.c_double)),
                ("closeness", ctypes.POINTER(ctypes.c_double)), ("capacity", ctypes.c_uint32),
                ("n_returned", ctypes.c_uint32), ("n_tied_at_kth", ctypes.c_uint32),
                ("edges_visited", ctypes.c_uint64), ("edges_scanned", ctypes.c_uint64),
                ("bfs_started", ctypes.c_uint64), ("bfs_cut", ctypes.c_uint64), ("bfs_finished", ctypes.c_uint64),
                ("levels", ctypes.c_uint64), ("batch_bits", ctypes.c_uint32), ("pad", ctypes.c_uint32),
                ("ms_pre", ctypes.c_double), ("ms_bfs", ctypes.c_double), ("ms_kernel", ctypes.c_double),
                ("alg_bytes", ctypes.c_uint64)]


class tkc_run_stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint32), ("batch_bits", ctypes.c_uint32), ("row_bytes", ctypes.c_uint32),
                ("teams", ctypes.c_uint32), ("launches", ctypes.c_uint32), ("pad", ctypes.c_uint32),
                ("arcs", ctypes.c_uint64), ("td_levels", ctypes.c_uint64), ("td_frontier", ctypes.c_uint64),
                ("td_frontier_arcs", ctypes.c_uint64), ("td_new", ctypes.c_uint64), ("bu_levels", ctypes.c_uint64),
                ("bu_scanned_vertices", ctypes.c_uint64), ("bu_scanned_arcs", ctypes.c_uint64),
                ("bu_new", ctypes.c_uint64), ("bu_frontier", ctypes.c_uint64), ("bu_rows_read", ctypes.c_uint64),
                ("bu_swept", ctypes.c_uint64), ("seeded", ctypes.c_uint64),
                ("cleared", ctypes.c_uint64), ("compactions", ctypes.c_uint64), ("compacted_away", ctypes.c_uint64),
                ("alg_bytes", ctypes.c_uint64), ("ms_kernel", ctypes.c_double)]


EXPORTED = ["tkc_create", "tkc_set_options", "tkc_destroy", "tkc_load_csr", "tkc_load_csr_many", "tkc_free_graph",
            "tkc_topk_closeness", "tkc_topk_closeness_multi", "tkc_source_order", "tkc_set_source_order",
            "tkc_reach_bounds", "tkc_distance_sums", "tkc_distance_sums_noalloc", "tkc_kernel_launches",
            "tkc_strerror", "tkc_vertex_features", "tkc_mlp_init", "tkc_set_source_model", "tkc_get_source_model",
            "tkc_mlp_forward", "tkc_mlp_gradient", "tkc_mlp_train_step", "tkc_autotune", "tkc_nb_bounds",
            "tkc_topk_harmonic", "tkc_topk_harmonic_multi", "tkc_nb_harmonic_bounds", "tkc_topk_closeness_bound", "tkc_last_run_stats", "tkc_topk_closeness_shard",
            "tkc_count_tied"]


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"CUDA library {path} is not built; run __graft_entry__.build() first")
    lib = ctypes.CDLL(path)
    vp = ctypes.c_void_p
    u32p = ctypes.POINTER(ctypes.c_uint32)
    u64p = ctypes.POINTER(ctypes.c_uint64)
    lib.tkc_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(tkc_options)]
    lib.tkc_set_options.argtypes = [vp, ctypes.POINTER(tkc_options)]
    lib.tkc_destroy.argtypes = [vp]
    lib.tkc_destroy.restype = None
    lib.tkc_load_csr.argtypes = [vp, ctypes.c_uint32, ctypes.c_uint64, vp, vp, ctypes.c_int, ctypes.c_int,
                                 ctypes.POINTER(vp)]
    lib.tkc_load_csr_many.argtypes = [vp, ctypes.c_uint32, u32p, u64p, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                      ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.POINTER(vp), u32p]
    lib.tkc_free_graph.argtypes = [vp]
    lib.tkc_free_graph.restype = None
    lib.tkc_topk_closeness.argtypes = [vp, ctypes.c_uint32, ctypes.POINTER(tkc_result)]
    lib.tkc_topk_closeness_multi.argtypes = [vp, ctypes.POINTER(vp), ctypes.c_uint32, ctypes.c_uint32,
                                             ctypes.POINTER(tkc_result)]
    lib.tkc_source_order.argtypes = [vp, u32p]
    lib.tkc_set_source_order.argtypes = [vp, u32p]
    lib.tkc_reach_bounds.argtypes = [vp, u32p, u32p]
    lib.tkc_distance_sums.argtypes = [vp, ctypes.c_uint32, u32p, u64p, u32p]
    lib.tkc_distance_sums_noalloc.argtypes = [vp, vp, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint32, vp, vp, vp,
                                              vp]
    fp = ctypes.POINTER(ctypes.c_float)
    lib.tkc_vertex_features.argtypes = [vp, vp]
    lib.tkc_mlp_init.argtypes = [vp, ctypes.c_uint64]
    lib.tkc_set_source_model.argtypes = [vp, fp, ctypes.c_uint32]
    lib.tkc_get_source_model.argtypes = [vp, fp, ctypes.c_uint32]
    lib.tkc_mlp_forward.argtypes = [vp, vp, ctypes.c_uint32, vp]
    lib.tkc_mlp_gradient.argtypes = [vp, vp, vp, ctypes.c_uint32, vp, fp]
    lib.tkc_mlp_train_step.argtypes = [vp, vp, vp, ctypes.c_uint32, ctypes.c_float, fp]
    lib.tkc_autotune.argtypes = [vp, ctypes.c_uint32, ctypes.POINTER(tkc_options)]
    lib.tkc_nb_bounds.argtypes = [vp, ctypes.c_uint32, u64p, u32p, u64p, u32p, u32p, u32p]
    lib.tkc_topk_harmonic.argtypes = [vp, ctypes.c_uint32, ctypes.POINTER(tkc_result)]
    lib.tkc_topk_closeness_bound.argtypes = [vp, ctypes.c_uint32, ctypes.POINTER(tkc_result)]
    lib.tkc_topk_harmonic_multi.argtypes = [vp, ctypes.POINTER(vp), ctypes.c_uint32, ctypes.c_uint32,
                                            ctypes.POINTER(tkc_result)]
    lib.tkc_nb_harmonic_bounds.argtypes = [vp, ctypes.c_uint32, ctypes.POINTER(ctypes.c_double), u32p, u32p]
    lib.tkc_last_run_stats.argtypes = [vp, ctypes.POINTER(tkc_run_stats)]
    lib.tkc_topk_closeness_shard.argtypes = [vp, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                             ctypes.c_uint32, u64p, u32p, u32p, ctypes.c_uint32,
                                             ctypes.POINTER(tkc_result)]
    lib.tkc_count_tied.argtypes = [vp, ctypes.c_uint64, ctypes.c_uint32, u32p]
    lib.tkc_kernel_launches.argtypes = []
    lib.tkc_kernel_launches.restype = ctypes.c_uint64
    lib.tkc_strerror.argtypes = [ctypes.c_int]
    lib.tkc_strerror.restype = ctypes.c_char_p
    return lib


_lib = load_library()


def tkc_kernel_launches() -> int:
    return int(_lib.tkc_kernel_launches())


def tkc_last_run_stats(ctx) -> dict:
    """Per-level totals of ctx's latest search-kernel run, as a dict."""
    st = tkc_run_stats()
    _check(_lib.tkc_last_run_stats(ctx, ctypes.byref(st)), "tkc_last_run_stats")
    return {name: getattr(st, name) for name, _ in st._fields_ if name != "pad"}


def tkc_strerror(code: int) -> str:
    return _lib.tkc_strerror(int(code)).decode()


def _check(rc: int, where: str):
    if rc != TKC_OK:
        raise TkcError(rc, where)


def _u32p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def _u64p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def _f64p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def current_stream_handle(device: int = 0) -> int | None:
    try:
        import torch

        if torch.cuda.is_available():
            return torch.cuda.current_stream(device).cuda_stream
    except Exception:  # torch missing or CUDA unavailable
        pass
    return None


@dataclass
class Options:
    device: int = 0
    stream: int | None = None
    order: int = TKC_ORDER_DEG
    batch_bits: int = 0
    bu_num: int = 0
    bu_den: int = 0
    blocks: int = 0
    seed_factor: int = 0
    timeout_cycles: int = 0
    teams: int = 0
    nb_levels: int = 0
    large_blocks: int = 0
    deterministic: int = 0
    relabel: int = 0

    def to_c(self) -> tkc_options:
        return tkc_options(self.device, self.stream, self.order, self.batch_bits, self.bu_num, self.bu_den,
                           self.blocks, self.seed_factor, self.timeout_cycles, self.teams, self.nb_levels,
                           self.large_blocks, self.deterministic, self.relabel)


@dataclass
class Result:
    ids: np.ndarray
    dist_sum: np.ndarray
    reach: np.ndarray
    farness: np.ndarray
    closeness: np.ndarray
    n_tied_at_kth: int
    edges_visited: int
    edges_scanned: int
    bfs_started: int
    bfs_cut: int
    bfs_finished: int
    levels: int
    batch_bits: int
    ms_pre: float
    ms_bfs: float
    ms_kernel: float
    alg_bytes: int
    extra: dict = field(default_factory=dict)


def tkc_create(options: Options | None = None) -> ctypes.c_void_p:
    opt = options or Options()
    if opt.stream is None:
        opt.stream = current_stream_handle(opt.device)
    ctx = ctypes.c_void_p()
    c = opt.to_c()
    _check(_lib.tkc_create(ctypes.byref(ctx), ctypes.byref(c)), "tkc_create")
    return ctx


def tkc_set_options(ctx, options: Options) -> None:
    if options.stream is None:
        options.stream = current_stream_handle(options.device)
    c = options.to_c()
    _check(_lib.tkc_set_options(ctx, ctypes.byref(c)), "tkc_set_options")


def tkc_destroy(ctx) -> None:
    _lib.tkc_destroy(ctx)


def tkc_load_csr(ctx, n: int, offsets, cols, directed: bool) -> ctypes.c_void_p:
    """offsets/cols: numpy uint32 arrays or torch int32/uint32 tensors.  CUDA
    tensors are passed as device pointers, CPU tensors (e.g. pinned) as host
    pointers; both must be contiguous."""
    g = ctypes.c_void_p()
    if hasattr(offsets, "data_ptr"):
        if not (offsets.is_contiguous() and cols.is_contiguous()) or offsets.element_size() != 4:
            raise ValueError("CSR tensors must be contiguous 32-bit")
        arcs = int(cols.numel())
        rc = _lib.tkc_load_csr(ctx, n, arcs, ctypes.c_void_p(offsets.data_ptr()),
                               ctypes.c_void_p(cols.data_ptr() if arcs else 0), int(directed),
                               1 if offsets.is_cuda else 0, ctypes.byref(g))
    else:
        off = np.ascontiguousarray(offsets, dtype=np.uint32)
        col = np.ascontiguousarray(cols, dtype=np.uint32)
        arcs = int(col.size)
        rc = _lib.tkc_load_csr(ctx, n, arcs, off.ctypes.data_as(ctypes.c_void_p),
                               col.ctypes.data_as(ctypes.c_void_p) if arcs else None, int(directed), 0,
                               ctypes.byref(g))
    _check(rc, "tkc_load_csr")
    return g


def tkc_load_csr_many(ctx, graphs) -> list:
    """graphs: (n, offsets, cols, directed) tuples, arrays as for tkc_load_csr
    (all CUDA tensors, or all host arrays).  Returns the handles.  On a
    malformed graph raises TkcError with .first_bad = its index."""
    ng = len(graphs)
    if ng == 0:
        return []
    keep, offp, colp = [], [], []
    dev = [hasattr(o, "data_ptr") and o.is_cuda for _, o, _, _ in graphs]
    if any(dev) and not all(dev):
        raise ValueError("tkc_load_csr_many: all CSRs on the device or all on the host")
    nn = np.array([int(x[0]) for x in graphs], np.uint32)
    arcs = np.zeros(ng, np.uint64)
    for i, (n, offsets, cols, _) in enumerate(graphs):
        if hasattr(offsets, "data_ptr"):
            if not (offsets.is_contiguous() and cols.is_contiguous()) or offsets.element_size() != 4:
                raise ValueError("CSR tensors must be contiguous 32-bit")
            arcs[i] = int(cols.numel())
            offp.append(offsets.data_ptr())
            colp.append(cols.data_ptr() if arcs[i] else 0)
        else:
            off = np.ascontiguousarray(offsets, dtype=np.uint32)
            col = np.ascontiguousarray(cols, dtype=np.uint32)
            keep += [off, col]
            arcs[i] = col.size
            offp.append(off.ctypes.data)
            colp.append(col.ctypes.data if col.size else 0)
    VP = ctypes.c_void_p * ng
    dirs = (ctypes.c_int * ng)(*[int(bool(x[3])) for x in graphs])
    out = VP()
    bad = ctypes.c_uint32(ng)
    rc = _lib.tkc_load_csr_many(ctx, ng, _u32p(nn), arcs.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                VP(*offp), VP(*colp), dirs, 1 if all(dev) else 0, out, ctypes.byref(bad))
    if rc != TKC_OK:
        err = TkcError(rc, "tkc_load_csr_many")
        err.first_bad = int(bad.value)
        raise err
    return [ctypes.c_void_p(out[i]) for i in range(ng)]


def tkc_free_graph(g) -> None:
    _lib.tkc_free_graph(g)


def _new_result(cap: int):
    ids = np.zeros(max(cap, 1), np.uint32)
    S = np.zeros(max(cap, 1), np.uint64)
    r = np.zeros(max(cap, 1), np.uint32)
    f = np.zeros(max(cap, 1), np.float64)
    c = np.zeros(max(cap, 1), np.float64)
    res = tkc_result()
    res.ids, res.dist_sum, res.reach, res.farness, res.closeness = _u32p(ids), _u64p(S), _u32p(r), _f64p(f), _f64p(c)
    res.capacity = cap
    return res, (ids, S, r, f, c)


def _to_result(res: tkc_result, arrays) -> Result:
    m = res.n_returned
    ids, S, r, f, c = arrays
    return Result(ids[:m].copy(), S[:m].copy(), r[:m].copy(), f[:m].copy(), c[:m].copy(), res.n_tied_at_kth,
                  res.edges_visited, res.edges_scanned, res.bfs_started, res.bfs_cut, res.bfs_finished, res.levels,
                  res.batch_bits, res.ms_pre, res.ms_bfs, res.ms_kernel, res.alg_bytes)


def tkc_topk_closeness(g, k: int, capacity: int | None = None) -> Result:
    cap = k if capacity is None else capacity
    res, arrays = _new_result(cap)
    _check(_lib.tkc_topk_closeness(g, k, ctypes.byref(res)), "tkc_topk_closeness")
    return _to_result(res, arrays)


def tkc_topk_closeness_shard(g, k: int, shard: int, nshards: int, max_sources: int = 0, seed=None,
                             capacity: int | None = None, first: int = 0) -> Result:
    """Part of the source order (see include/tkc.h): positions first + shard,
    first + shard + nshards, ...; seed = (S, r, ids) host arrays, best first,
    or None."""
    cap = k if capacity is None else capacity
    res, arrays = _new_result(cap)
    if seed is None or len(seed[2]) == 0:
        sS = sr = si = None
        ns = 0
    else:
        sS = np.ascontiguousarray(seed[0], dtype=np.uint64)
        sr = np.ascontiguousarray(seed[1], dtype=np.uint32)
        si = np.ascontiguousarray(seed[2], dtype=np.uint32)
        ns = len(si)
    _check(_lib.tkc_topk_closeness_shard(g, k, first, shard, nshards, max_sources, None if sS is None else _u64p(sS),
                                         None if sr is None else _u32p(sr), None if si is None else _u32p(si), ns,
                                         ctypes.byref(res)), "tkc_topk_closeness_shard")
    return _to_result(res, arrays)


def tkc_count_tied(g, S: int, r: int) -> int:
    cnt = ctypes.c_uint32(0)
    _check(_lib.tkc_count_tied(g, int(S), int(r), ctypes.byref(cnt)), "tkc_count_tied")
    return int(cnt.value)


def tkc_topk_closeness_multi(ctx, graphs, k: int) -> list[Result]:
    ng = len(graphs)
    arr = (ctypes.c_void_p * max(ng, 1))(*[g.value if isinstance(g, ctypes.c_void_p) else g for g in graphs])
    results = (tkc_result * max(ng, 1))()
    keep = []
    for i in range(ng):
        res, arrays = _new_result(k)
        results[i] = res
        keep.append(arrays)
    _check(_lib.tkc_topk_closeness_multi(ctx, arr, ng, k, results), "tkc_topk_closeness_multi")
    return [_to_result(results[i], keep[i]) for i in range(ng)]


def tkc_topk_harmonic(g, k: int, capacity: int | None = None) -> Result:
    """Top-k harmonic centrality: closeness[] holds h(v), farness[] 1/h(v)."""
    cap = k if capacity is None else capacity
    res, arrays = _new_result(cap)
    _check(_lib.tkc_topk_harmonic(g, k, ctypes.byref(res)), "tkc_topk_harmonic")
    return _to_result(res, arrays)


def tkc_topk_closeness_bound(g, k: int, capacity: int | None = None) -> Result:
    """Top-k closeness by DegBound / NBBound (Algorithm 1 with updateBoundsLB)."""
    cap = k if capacity is None else capacity
    res, arrays = _new_result(cap)
    _check(_lib.tkc_topk_closeness_bound(g, k, ctypes.byref(res)), "tkc_topk_closeness_bound")
    return _to_result(res, arrays)


def tkc_topk_harmonic_multi(ctx, graphs, k: int) -> list[Result]:
    ng = len(graphs)
    arr = (ctypes.c_void_p * max(ng, 1))(*[g.value if isinstance(g, ctypes.c_void_p) else g for g in graphs])
    results = (tkc_result * max(ng, 1))()
    keep = []
    for i in range(ng):
        res, arrays = _new_result(k)
        results[i] = res
        keep.append(arrays)
    _check(_lib.tkc_topk_harmonic_multi(ctx, arr, ng, k, results), "tkc_topk_harmonic_multi")
    return [_to_result(results[i], keep[i]) for i in range(ng)]


def tkc_nb_harmonic_bounds(g, n: int, max_levels: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """(h_ub, order): the upper bound on h per vertex and the sources by decreasing bound."""
    h = np.zeros(max(n, 1), np.float64)
    order = np.zeros(max(n, 1), np.uint32)
    cnt = ctypes.c_uint32(0)
    _check(_lib.tkc_nb_harmonic_bounds(g, max_levels, h.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                       _u32p(order), ctypes.byref(cnt)), "tkc_nb_harmonic_bounds")
    return h[:n], order[: cnt.value]


def tkc_source_order(g, n: int) -> np.ndarray:
    order = np.zeros(max(n, 1), np.uint32)
    _check(_lib.tkc_source_order(g, _u32p(order)), "tkc_source_order")
    return order[:n]


def tkc_set_source_order(g, order) -> None:
    o = np.ascontiguousarray(order, dtype=np.uint32)
    _check(_lib.tkc_set_source_order(g, _u32p(o) if o.size else None), "tkc_set_source_order")


def tkc_reach_bounds(g, n: int) -> tuple[np.ndarray, np.ndarray]:
    a = np.zeros(max(n, 1), np.uint32)
    o = np.zeros(max(n, 1), np.uint32)
    _check(_lib.tkc_reach_bounds(g, _u32p(a), _u32p(o)), "tkc_reach_bounds")
    return a[:n], o[:n]


@dataclass
class NBBounds:
    S: np.ndarray       # S~ at the minimising reach
    r: np.ndarray       # that reach (1: out-degree 0)
    key: np.ndarray     # floor(S * 2^46 / (r-1)^2)
    order: np.ndarray   # out-degree >= 1 vertices by (key, id)
    levels: int


def tkc_nb_bounds(g, n: int, max_levels: int = 0) -> NBBounds:
    S = np.zeros(max(n, 1), np.uint64)
    r = np.zeros(max(n, 1), np.uint32)
    key = np.zeros(max(n, 1), np.uint64)
    order = np.zeros(max(n, 1), np.uint32)
    cnt = ctypes.c_uint32(0)
    lev = ctypes.c_uint32(0)
    _check(_lib.tkc_nb_bounds(g, max_levels, _u64p(S), _u32p(r), _u64p(key), _u32p(order), ctypes.byref(cnt),
                              ctypes.byref(lev)), "tkc_nb_bounds")
    return NBBounds(S[:n], r[:n], key[:n], order[: cnt.value], int(lev.value))


def tkc_distance_sums(g, sources) -> tuple[np.ndarray, np.ndarray]:
    src = np.ascontiguousarray(sources, dtype=np.uint32)
    S = np.zeros(max(src.size, 1), np.uint64)
    r = np.zeros(max(src.size, 1), np.uint32)
    _check(_lib.tkc_distance_sums(g, src.size, _u32p(src), _u64p(S), _u32p(r)), "tkc_distance_sums")
    return S[: src.size], r[: src.size]


def tkc_distance_sums_noalloc(offsets, cols, n: int, sources, S, r, stream=None) -> None:
    """Allocation-free distance sums: every argument is a torch CUDA tensor on
    the current device (offsets/cols/sources 32-bit, S 64-bit, r 32-bit); the
    library allocates nothing.  stream defaults to torch's current stream."""
    for t in (offsets, cols, sources, S, r):
        if not (t.is_cuda and t.is_contiguous()):
            raise ValueError("tkc_distance_sums_noalloc takes contiguous CUDA tensors")
    if stream is None:
        stream = current_stream_handle(offsets.device.index)
    rc = _lib.tkc_distance_sums_noalloc(ctypes.c_void_p(offsets.data_ptr()),
                                        ctypes.c_void_p(cols.data_ptr() if cols.numel() else 0), n, int(cols.numel()),
                                        int(sources.numel()), ctypes.c_void_p(sources.data_ptr()),
                                        ctypes.c_void_p(S.data_ptr()), ctypes.c_void_p(r.data_ptr()),
                                        ctypes.c_void_p(stream))
    _check(rc, "tkc_distance_sums_noalloc")


def tkc_autotune(g, k: int) -> Options:
    """Tunes the launch parameters on g; returns them as Options (stream left to the caller)."""
    o = tkc_options()
    _check(_lib.tkc_autotune(g, k, ctypes.byref(o)), "tkc_autotune")
    return Options(device=o.device, stream=o.stream, order=o.order, batch_bits=o.batch_bits, bu_num=o.bu_num,
                   bu_den=o.bu_den, blocks=o.blocks, seed_factor=o.seed_factor, timeout_cycles=o.timeout_cycles,
                   teams=o.teams, nb_levels=o.nb_levels, large_blocks=o.large_blocks)


def _dev(t):
    if not (t.is_cuda and t.is_contiguous()):
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def tkc_vertex_features(g, n: int, device: int = 0):
    """Standardized vertex features as a float32 CUDA tensor of shape (n, 5)."""
    import torch

    x = torch.empty((max(n, 1), TKC_MLP_FEATURES), dtype=torch.float32, device=f"cuda:{device}")
    _check(_lib.tkc_vertex_features(g, _dev(x)), "tkc_vertex_features")
    return x[:n]


def tkc_mlp_init(ctx, seed: int) -> None:
    _check(_lib.tkc_mlp_init(ctx, seed), "tkc_mlp_init")


def tkc_set_source_model(ctx, params) -> None:
    w = np.ascontiguousarray(params, dtype=np.float32)
    _check(_lib.tkc_set_source_model(ctx, w.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), w.size),
           "tkc_set_source_model")


def tkc_get_source_model(ctx) -> np.ndarray:
    w = np.zeros(TKC_MLP_PARAMS, np.float32)
    _check(_lib.tkc_get_source_model(ctx, w.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), w.size),
           "tkc_get_source_model")
    return w


def tkc_mlp_forward(ctx, x, y) -> None:
    _check(_lib.tkc_mlp_forward(ctx, _dev(x), x.shape[0], _dev(y)), "tkc_mlp_forward")


def tkc_mlp_gradient(ctx, x, t, grad) -> float:
    loss = ctypes.c_float()
    _check(_lib.tkc_mlp_gradient(ctx, _dev(x), _dev(t), x.shape[0], _dev(grad), ctypes.byref(loss)),
           "tkc_mlp_gradient")
    return loss.value


def tkc_mlp_train_step(ctx, x, t, lr: float) -> float:
    loss = ctypes.c_float()
    _check(_lib.tkc_mlp_train_step(ctx, _dev(x), _dev(t), x.shape[0], lr, ctypes.byref(loss)),
           "tkc_mlp_train_step")
    return loss.value


class Graph:
    """Owns a loaded graph handle; frees it on close()."""

    def __init__(self, ctx, graph, directed: bool = False):
        self.ctx = ctx
        self.n = graph.n
        self.directed = graph.directed
        self.handle = tkc_load_csr(ctx, graph.n, graph.offsets, graph.cols, graph.directed)

    def close(self):
        if self.handle:
            tkc_free_graph(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
