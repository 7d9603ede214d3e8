/*
 * tkc -- exact top-k closeness centrality on one GB300 GPU.
 *
 * C ABI of the CUDA library (libtkc.so).  The method is DegCut and NBCut
 * from Bergamini, Borassi, Crescenzi, Marino, Meyerhenke, "Computing top-k
 * Closeness Centrality Faster in Unweighted Graphs" (arXiv 1704.01077):
 * Algorithm 1 with computeBoundsDeg (Section 4) or computeBoundsNB (Section 5,
 * Algorithm 3) and updateBoundsBFSCut (Section 6, Algorithm 4 and its lemma
 * bounding S from a partial BFS), reach bounds alpha/omega for directed graphs
 * (Section 8: its lemma on bounds of the form (n-1) L(r)/(r-1)^2, Eq. 6,
 * Algorithm 6).
 *
 * Definitions (Section 2): R(v) = vertices reachable from v, v included;
 * r(v) = |R(v)|; S(v) = sum of d(v,w) over R(v);
 * farness f(v) = (n-1) S(v) / (r(v)-1)^2; closeness c(v) = 1/f(v), with
 * c(v) = 0 (f = +inf) when r(v) = 1.  Top-k = the k vertices of smallest
 * farness; ties are broken by increasing vertex id and the number of vertices
 * tied with the k-th is reported (Section 4 asks for all of them).
 *
 * Conventions shared by every entry point:
 *  - Return value: TKC_OK (0) or a negative TKC_E* code; tkc_strerror() names it.
 *  - Graph input is CSR: offsets uint32[n+1] (offsets[0] = 0, non-decreasing,
 *    offsets[n] = arcs), cols uint32[arcs]; each row strictly increasing (no
 *    duplicate arcs), every id < n, no self-loops.  An undirected graph holds
 *    both arc directions and must be symmetric.  Violations give TKC_EGRAPH.
 *  - Inputs are copied; the caller keeps ownership of every pointer it passes.
 *    Handles are owned by the library until freed by tkc_free_graph /
 *    tkc_destroy.  Result arrays are caller-allocated HOST memory.
 *  - All work runs on the context's device and stream; every call returns
 *    after its results are in host memory.
 *  - A context is not thread-safe: use one context per host thread.
 */
#ifndef TKC_H
#define TKC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TKC_OK 0
#define TKC_EINVAL -1    /* bad argument (null pointer, k too large, bad option) */
#define TKC_EGRAPH -2    /* malformed CSR (unsorted row, id out of range, self-loop, duplicate, asymmetric) */
#define TKC_ENOMEM -3    /* device or host allocation failed */
#define TKC_ECUDA -4     /* a CUDA runtime call failed */
#define TKC_ETIMEOUT -5  /* a device-side wait exceeded its budget; the context stays usable */
#define TKC_EOVERFLOW -6 /* the graph exceeds a size limit of this build (n >= 2^26, arcs >= 2^32) */

#define TKC_ORDER_DEG 0     /* computeBoundsDeg: out-degree descending, then id ascending (Section 4) */
#define TKC_ORDER_GIVEN 1   /* caller's order, set by tkc_set_source_order */
#define TKC_ORDER_LEARNED 2 /* source-order model (tkc_set_source_model): with seed_factor = 0 all sources
                               by predicted farness; with seed_factor > 0 the seed_factor * k sources
                               predicted closest first (searched without cutting), then the degree order */
#define TKC_ORDER_NB 3      /* computeBoundsNB (NBCut): sources by increasing neighbourhood-based farness
                               bound (tkc_nb_bounds), ties by id; the search stops at the first source
                               whose bound exceeds the k-th farness found (Algorithm 1's stop) */
#define TKC_ORDER_LEARNED_NB 4 /* the seed_factor * k sources the source-order model predicts closest first
                               (searched without cutting), then the TKC_ORDER_NB order without them, with
                               its stop (the rest of that order is still sorted by its bound); one graph,
                               closeness only */

#define TKC_MAX_K 1024      /* largest k accepted by tkc_topk_closeness */

typedef struct tkc_ctx tkc_ctx;
typedef struct tkc_graph tkc_graph;

typedef struct {
  int device;              /* CUDA device ordinal */
  void *stream;            /* cudaStream_t to run on (e.g. torch's current stream); NULL = legacy default */
  uint32_t order;          /* TKC_ORDER_* */
  uint32_t batch_bits;     /* sources searched together: 1 (plain, one source per BFS), 64, 128, 256, 512;
                              0 = the autotuner's choice for this graph class when tkc_autotune
                              has cached one, else the library default (64 or 128 by size) */
  uint32_t bu_num;         /* direction switch: a level runs bottom-up when frontier arcs * bu_num >
                              arcs * bu_den (bu_num = 0: library default, 8/1) */
  uint32_t bu_den;
  uint32_t blocks;         /* persistent grid size (0 = library default, clamped to co-residency) */
  uint32_t seed_factor;    /* the first seed_factor * k sources of the order are searched to the end
                              without cutting, so x starts from exact farness values (0 = none) */
  uint64_t timeout_cycles; /* budget of every device-side wait, in SM clock cycles (0 = default 2^34) */
  uint32_t teams;          /* independent groups of SMs, each running its own source batches and sharing
                              the threshold and the k-lists (0 = library default: 1 in plain mode and below
                              2^14 vertices; NBCut on one graph one team per 32 SMs; otherwise one per 16 SMs
                              below 2^16 vertices and one per 8 SMs from 2^16 up).  With several teams on one
                              graph the first batch runs alone on the whole grid, so that a threshold exists
                              before the teams start. */
  uint32_t nb_levels;      /* TKC_ORDER_NB: most level sweeps of computeBoundsNB, 1..65535 (0 = 256) */
  uint32_t large_blocks;   /* threads per block of the search kernel: 0 = library choice (the larger blocks -- 1024
                              threads for 64- and 128-bit batches -- for batched searches on graphs of
                              2^20 vertices or more, else 512), 1 = always the larger blocks, 2 = always 512;
                              wider batches always use 512.  Results never depend on it. */
  uint32_t deterministic;  /* 1: one team of SMs whatever `teams` says, so the threshold x changes only at
                              level barriers and the top-k merges happen in a fixed order; every counter
                              (edges_visited, bfs_started, bfs_cut, bfs_finished, levels) is then a function
                              of the graph, k, the order and batch_bits alone (the batched schedule of
                              Algorithm 1 with Algorithm 4: B searches advance one level per step, finished
                              searches enter the top list before the survivors' cut test).  0: teams run side
                              by side and cut against a threshold another team may be updating, so counters
                              vary from run to run (results never do). */
  uint32_t relabel;        /* vertex labels of the search's rows: 0 = library choice (batched searches on graphs
                              of 2^20 vertices or more -- for several graphs in one launch, when the largest has
                              -- walk a copy of the graph whose vertices are numbered by
                              in-degree, largest first, so that the rows levels touch most share L2; else the
                              graph itself), 1 = always that copy, 2 = never.  Sources, ties and every id in
                              the results are the graph's own ids whatever the choice; results never depend
                              on it, edges_scanned does. */
} tkc_options;

typedef struct {
  /* caller-allocated host arrays of at least `capacity` entries (any may be NULL) */
  uint32_t *ids;       /* vertex ids, best first */
  uint64_t *dist_sum;  /* S(v) */
  uint32_t *reach;     /* r(v) */
  double *farness;     /* (n-1) S / (r-1)^2, one IEEE multiply and one divide; +inf when r = 1 */
  double *closeness;   /* (r-1)^2 / ((n-1) S); 0 when r = 1 */
  uint32_t capacity;
  /* filled by the call */
  uint32_t n_returned;     /* min(k, n) */
  uint32_t n_tied_at_kth;  /* vertices whose farness equals the k-th returned one (all of them, found exactly) */
  uint64_t edges_visited;  /* arcs of every expanded BFS level, sum of out-degrees (the paper's m_vis) */
  uint64_t edges_scanned;  /* arcs physically read by the level kernels */
  uint64_t bfs_started;    /* sources with out-degree >= 1 that were examined */
  uint64_t bfs_cut;        /* of those, abandoned by the BFSCut bound */
  uint64_t bfs_finished;   /* of those, searched to the end (exact S and r) */
  uint64_t levels;         /* level steps executed by the device loop */
  uint32_t batch_bits;     /* source batch width actually used */
  uint32_t pad;
  double ms_pre;           /* device time of preprocessing done by this call (order, reach bounds) */
  double ms_bfs;           /* device time of the pruned searches and the output */
  double ms_kernel;        /* device time of the persistent search kernel alone */
  uint64_t alg_bytes;      /* bytes the search kernel's levels must move by the cost model of the
                              level kernels (frontier rows, arc columns, seen/next rows) */
} tkc_result;

/* Creates a context on opt->device (NULL opt = defaults).  No paper
 * counterpart: owns the stream, options and device workspace; the caller owns
 * *out until tkc_destroy.  Errors: TKC_EINVAL (null out, an option out of
 * range: batch_bits, order, nb_levels, large_blocks, deterministic, relabel), TKC_ENOMEM, TKC_ECUDA
 * (no such device, no cooperative launch); *out is NULL on error. */
int tkc_create(tkc_ctx **out, const tkc_options *opt);

/* Replaces the context's options (same meaning as in tkc_create; no paper
 * counterpart).  Errors: TKC_EINVAL (null argument, opt->device differs from
 * the context's, an option out of range); the old options stay on error. */
int tkc_set_options(tkc_ctx *ctx, const tkc_options *opt);

/* Releases the context and its workspace (no paper counterpart).  Graphs
 * loaded on it must be freed first.  NULL is a no-op. */
void tkc_destroy(tkc_ctx *ctx);

/* Copies a CSR graph to the device and validates it -- the input of
 * Algorithm 1 (Section 4); a directed graph's in-arc CSR is built when a call
 * first needs it.  offsets/cols are host pointers if ptr_on_device = 0,
 * device pointers otherwise.  directed = 0 declares an undirected graph
 * (symmetry is checked).  n may be 0.  Errors: TKC_EINVAL (null ctx, out,
 * offsets, or cols with arcs > 0), TKC_EGRAPH (offsets[0] != 0, offsets[n] !=
 * arcs, offsets decreasing, an id out of range, a self-loop, an unsorted or
 * repeated row entry, an undirected graph that is not symmetric),
 * TKC_EOVERFLOW (n >= 2^26 or arcs >= 2^32), TKC_ENOMEM, TKC_ECUDA; *out is
 * NULL on error. */
int tkc_load_csr(tkc_ctx *ctx, uint32_t n, uint64_t arcs, const uint32_t *offsets, const uint32_t *cols,
                 int directed, int ptr_on_device, tkc_graph **out);

/* Loads ng graphs as tkc_load_csr does, with one host wait for all their
 * checks (two when some are undirected) instead of one or two per graph: for
 * callers that load many small graphs, e.g. for tkc_topk_closeness_multi (no
 * paper counterpart).  As there, a directed graph's in-arc CSR is built when a
 * call first needs it (a multi-graph launch builds the union's instead).  Graph i is n[i], arcs[i], offsets[i], cols[i],
 * directed[i]; ptr_on_device applies to all.  out[ng] receives the handles.
 * On error no graph is kept (every out[i] is NULL) and *first_bad (may be
 * NULL) is the first graph at fault, ng when none is (an allocation or CUDA
 * error).  Errors: as tkc_load_csr; TKC_EINVAL also for a null array with
 * ng > 0.  ng = 0 returns TKC_OK. */
int tkc_load_csr_many(tkc_ctx *ctx, uint32_t ng, const uint32_t *n, const uint64_t *arcs,
                      const uint32_t *const *offsets, const uint32_t *const *cols, const int *directed,
                      int ptr_on_device, tkc_graph **out, uint32_t *first_bad);

/* Frees a graph and everything derived from it (orders, reach and NB bounds,
 * features).  NULL is a no-op. */
void tkc_free_graph(tkc_graph *g);

/* Exact top-k closeness (Algorithm 1, DegCut or NBCut by options.order;
 * Sections 4, 5, 6, 8).  Writes
 * min(k, n) entries of out->ids/dist_sum/reach/farness/closeness (those not
 * NULL; out->capacity must be >= min(k, n)) and the counters.  k = 0 or n = 0
 * return no entries.  Errors: TKC_EINVAL (k > TKC_MAX_K, capacity too small),
 * TKC_ENOMEM, TKC_ECUDA, TKC_ETIMEOUT. */
int tkc_topk_closeness(tkc_graph *g, uint32_t k, tkc_result *out);

/* Exact top-k of each of ng graphs (all on ctx's device) in one persistent
 * launch: Algorithm 1 on their disjoint union, one k-list per graph (no paper
 * counterpart for the batching across graphs).  gs: ng handles loaded on ctx;
 * outs: ng results, each with its own caller-allocated arrays; outs[i]
 * receives graph i's top-k exactly as tkc_topk_closeness would give it.
 * Counters are per graph and may differ from a run of the graph alone (the
 * reach bounds are computed once on the union, and the threshold evolves
 * differently); ms_* are shared.  options.order: TKC_ORDER_DEG or
 * TKC_ORDER_NB (each graph stops on its own).  The union's sources run as
 * every graph's first batch, then the rest graph by graph, each graph's in its
 * own order, so a batch shares one graph's rows and arcs.  Errors: TKC_EINVAL (null ctx,
 * null gs or outs with ng > 0, k > TKC_MAX_K, another order, a capacity too
 * small), TKC_ENOMEM, TKC_ECUDA, TKC_ETIMEOUT. */
int tkc_topk_closeness_multi(tkc_ctx *ctx, tkc_graph *const *gs, uint32_t ng, uint32_t k, tkc_result *outs);

/* Algorithm 1 (Section 4) over part of the source order, for sharding the
 * sources of one graph over several GPUs (each holding a copy of the graph)
 * and for resuming a run from a checkpoint.  Algorithm 1 is exact for any
 * threshold x that is the k-th best of exactly known farness values, so the
 * call searches the sources at positions first + shard, first + shard +
 * nshards, first + shard + 2 nshards, ... of the order options.order gives
 * (TKC_ORDER_DEG or TKC_ORDER_NB; with NB the stop applies to these
 * positions, still sorted by key), at most max_sources of them (0 = all), from
 * a k-list seeded with nseed <= min(k, n) exact entries of vertices searched
 * elsewhere (host arrays seed_S/seed_r/seed_id, best first by farness then
 * id, r >= 2, distinct; none of them may be among the positions this call
 * searches: a k-list holds each vertex once).  The result is the best min(k,
 * n) of the seed and the searches finished here (padded with closeness-0
 * vertices as tkc_topk_closeness does); n_tied_at_kth counts only the
 * searches finished here that tie with the returned k-th.  Sharding: with
 * first = 0, shard s of N, and each shard seeded with the best k of the
 * others' results, the merged results are the exact top-k and the exact tie
 * count is the sum over shards of tkc_count_tied with the merged k-th.
 * Resuming: shard 0 of 1 from position `first` with the k-list reached
 * before it.  No paper counterpart for the split itself.  Errors: TKC_EINVAL
 * (null g or out, nshards = 0, shard >= nshards, k > TKC_MAX_K, an order
 * other than DEG or NB, capacity too small, a seed not sorted, repeated, with
 * r < 2 or an id >= n, nseed > min(k, n)), TKC_ENOMEM, TKC_ECUDA, TKC_ETIMEOUT. */
int tkc_topk_closeness_shard(tkc_graph *g, uint32_t k, uint32_t first, uint32_t shard, uint32_t nshards,
                             uint32_t max_sources, const uint64_t *seed_S, const uint32_t *seed_r,
                             const uint32_t *seed_id, uint32_t nseed, tkc_result *out);

/* Number of searches finished by the latest tkc_topk_closeness_shard run on g
 * (the latest run on g's context) whose farness equals S/(r-1)^2 exactly
 * (Section 4 asks for every vertex tied with the k-th).  Errors: TKC_EINVAL
 * (null argument, r < 2, or the context's latest run was not a shard run of
 * g), TKC_ENOMEM, TKC_ECUDA. */
int tkc_count_tied(tkc_graph *g, uint64_t S, uint32_t r, uint32_t *count);

/* Top-k harmonic centrality h(v) = sum over w != v of 1/d(v,w) (the paper's
 * closing generalisation of its method to sums of f(d(v,w)) with f decreasing,
 * Section 9): Algorithm 1 with the degree or NB order (options.order) and
 * BFSCut's upper bound on h.  h is formed per BFS level in FP64: the count of
 * vertices at distance d divided by d, added in increasing d, each operation
 * rounded to nearest; vertices are ranked by that value, largest first, ties
 * by id; n_tied_at_kth counts the vertices with the same FP64 value.  A search
 * is abandoned only when its bound times (1 + 2^-20) is below the k-th h (the
 * margin covers rounding), so the result is the exact top-k of that ranking.
 * Writes ids, reach (r), closeness[] = h(v), farness[] = 1/h(v) (+inf when
 * h = 0, i.e. out-degree 0) and dist_sum[] = 0 (S is not kept); counters as
 * tkc_topk_closeness.  Same errors. */
int tkc_topk_harmonic(tkc_graph *g, uint32_t k, tkc_result *out);

/* tkc_topk_harmonic for ng graphs in one persistent launch (Section 9 on the
 * disjoint union, as tkc_topk_closeness_multi); same arguments and errors as
 * tkc_topk_closeness_multi. */
int tkc_topk_harmonic_multi(tkc_ctx *ctx, tkc_graph *const *gs, uint32_t ng, uint32_t k, tkc_result *outs);

/* Exact top-k closeness by Algorithm 1 with updateBoundsLB (Section 7,
 * Algorithm 5; Eq. 4 undirected, Eq. 5 directed): DegBound with
 * options.order = TKC_ORDER_DEG, NBBound with TKC_ORDER_NB (the paper's best
 * variant on street networks).  Every search is complete; after a search from
 * s each vertex w whose reach equals s's (its component, or its SCC if
 * directed) gets the bound S(w) >= L(d(s,w)) - outdeg(w), L(i) = 2 x (vertices
 * within one level of i; directed: at most one level deeper) + the level
 * distance of all other vertices - 2, over R(s) including s.  The search runs
 * in rounds of options.teams batches of options.batch_bits sources (defaults: 8 x 64 from 2^16 vertices up,
 * else 1 x 256; batch_bits 1 = one source per round):
 * the unsearched vertices of smallest bound key floor(2^46 S_lb/(r-1)^2), ties
 * by their position in the initial order, and stops when that key exceeds the
 * k-th farness strictly.  Results as tkc_topk_closeness (bfs_cut = 0).  Errors:
 * TKC_EINVAL (order not DEG or NB, k > TKC_MAX_K, capacity too small),
 * TKC_EOVERFLOW (a search deeper than 65 534 levels), TKC_ENOMEM, TKC_ECUDA,
 * TKC_ETIMEOUT.  Device memory: about 2 x teams x batch_bits bytes per vertex. */
int tkc_topk_closeness_bound(tkc_graph *g, uint32_t k, tkc_result *out);

/* Autotuner (no paper counterpart: it only picks launch parameters).
 * Times candidate batch widths (64..512), team counts (1, 4, and SMs/16,
 * SMs/8, SMs/4, i.e. 16, 8 and 4 blocks per team), then bottom-up
 * thresholds, then (64- and 128-bit batches) the search kernel's block size
 * (options.large_blocks 1 and 2 against the library's choice), on a sample of
 * g's degree order (its first 1 024 sources, then every s-th source, about a
 * tenth of all); keeps the fastest in the context's cache under g's class
 * (directed, log2 n, log2 of the mean degree) and writes it to *best (other
 * fields copied from the context's options).  Later calls with
 * options.batch_bits = 0 on a graph of the same class use the cached choice
 * (teams, thresholds and block size only where the options leave them at 0).
 * With the environment variable TKC_TUNE_CACHE naming a file, the cache is
 * loaded at tkc_create and saved after each tuning (one line per class:
 * class=bits,teams,bu_num,bu_den,ms,large_blocks; lines without the last
 * field mean the library's block size).  Results never depend on these
 * parameters.  Errors: TKC_EINVAL (null g or best, k > TKC_MAX_K),
 * TKC_ENOMEM, TKC_ECUDA, TKC_ETIMEOUT. */
int tkc_autotune(tkc_graph *g, uint32_t k, tkc_options *best);

/* computeBoundsDeg (Section 4): writes the degree order (out-degree
 * descending, id ascending) of all n vertices to host array order[n].
 * Errors: TKC_EINVAL (null g, or null order with n > 0), TKC_ENOMEM,
 * TKC_ECUDA. */
int tkc_source_order(tkc_graph *g, uint32_t *order);

/* Sets the order of Algorithm 1's queue Q (Section 4) used when
 * options.order = TKC_ORDER_GIVEN: a permutation of 0..n-1 in host memory,
 * copied.  Any order gives the same top-k; only the work done changes.
 * Errors: TKC_EINVAL (null g, null order with n > 0, not a permutation),
 * TKC_ENOMEM, TKC_ECUDA. */
int tkc_set_source_order(tkc_graph *g, const uint32_t *order);

/* Reach bounds alpha(v) <= r(v) <= omega(v) (Section 8.4, Algorithm 6; exact
 * component size for undirected graphs) into host arrays alpha[n], omega[n].
 * Errors: TKC_EINVAL (null g, or a null array with n > 0), TKC_ENOMEM,
 * TKC_ECUDA, TKC_ETIMEOUT (an SCC iteration exceeded n + 1 rounds). */
int tkc_reach_bounds(tkc_graph *g, uint32_t *alpha, uint32_t *omega);

/* computeBoundsNB (Section 5, Algorithm 3; Eq. 3 for directed graphs; Eq. 6
 * with the Algorithm 6 reach bounds).  N~_k(v), an upper bound on the number
 * of vertices at distance k from v, counts the non-backtracking walks of
 * length k (undirected, Eq. 2) or the walks of length k (directed, Eq. 3);
 * all vertices advance one level per device sweep, at most max_levels sweeps
 * (0 = 256, at most 65535; a vertex unfinished after the last sweep takes the
 * next level as unbounded, which keeps the bound valid).  With
 * c_k = N~_0 + ... + N~_k, S~(r) = sum_k k min(N~_k, max(r - c_{k-1}, 0)) is a
 * lower bound on S(v) when r = r(v), and the bound on the farness is the least
 * (n-1) S~(r)/(r-1)^2 over r = alpha(v), omega(v) and the c_k between them.
 * Counts are exact below 2^32 and stored as 2^32 above (any value >= n bounds
 * a level).  Outputs (host arrays, any may be NULL):
 *   S_lb[n], r_lb[n]: the minimising (S~, r); r_lb = 1 for out-degree 0
 *                     (closeness 0); farness >= (n-1) S_lb / (r_lb - 1)^2;
 *   key[n]:           floor(S_lb * 2^46 / (r_lb - 1)^2) (UINT64_MAX if r_lb = 1);
 *   order[n]:         the vertices of out-degree >= 1 by (key, id), *n_order of them;
 *   *levels:          sweeps run.
 * Results are cached on g per max_levels.  Errors: TKC_EINVAL (max_levels >
 * 65535), TKC_ENOMEM, TKC_ECUDA. */
int tkc_nb_bounds(tkc_graph *g, uint32_t max_levels, uint64_t *S_lb, uint32_t *r_lb, uint64_t *key,
                  uint32_t *order, uint32_t *n_order, uint32_t *levels);

/* The harmonic counterpart of tkc_nb_bounds (same sweeps): h_ub[n] receives
 * an upper bound on h(v), the sum over k of min(N~_k, max(omega(v) - c_{k-1}, 0)) / k
 * (quotients added in increasing k, FP64 rounded to nearest; a vertex unfinished
 * after the last sweep adds (omega - c_K) / (K+1)), and order[] the vertices of
 * out-degree >= 1 by decreasing h_ub, ties by id (*n_order of them).  Host
 * arrays, any may be NULL.  Errors as tkc_nb_bounds. */
int tkc_nb_harmonic_bounds(tkc_graph *g, uint32_t max_levels, double *h_ub, uint32_t *order, uint32_t *n_order);

/* Exact S(v) and r(v) (Section 2 definitions) of the listed sources by full
 * BFS on the device, in batches of 64 sources (no cutting).  srcs, S, r: host
 * arrays of nsrc; a source may be listed more than once.  Errors: TKC_EINVAL
 * (null g, a null array with nsrc > 0, a source >= n), TKC_ENOMEM, TKC_ECUDA,
 * TKC_ETIMEOUT. */
int tkc_distance_sums(tkc_graph *g, uint32_t nsrc, const uint32_t *srcs, uint64_t *S, uint32_t *r);

/* Allocation-free variant of tkc_distance_sums, for callers that cannot
 * allocate device memory when they need the result: runtimes that reserve a
 * fixed device-memory budget at start-up (a later allocation would exceed it),
 * and latency-critical services that cannot take the device-wide
 * synchronisation an allocation may cause.  The paper has no counterpart; it
 * exists for those callers only.
 *
 * Computes exact S(v) and r(v) of nsrc distinct sources by full BFS (no
 * cutting), 64 sources at a time, on the CURRENT device and `stream`
 * (cudaStream_t, NULL = legacy default).  All pointers are DEVICE pointers
 * owned by the caller: offsets[n+1] and cols[arcs] (CSR of out-arcs, ids < n),
 * srcs[nsrc] (distinct ids < n), outputs S[nsrc] and r[nsrc].  The call
 * allocates nothing: its scratch is one fixed array of about 5.5 MB compiled
 * into the library, which every device that loads the library holds until
 * the process exits.
 *  - Each call looks up that array's device address on the current device
 *    (the lookup allocates nothing).
 *  - Every call on a device shares the array and clears what it needs; calls
 *    whose GPU work overlaps race on it, so serialise them.
 *  - The call returns after the results are written (it synchronises `stream`).
 * Errors: TKC_EINVAL (n > TKC_NOALLOC_MAX_N, a null pointer, a source out of
 * range or repeated), TKC_EGRAPH (offsets not monotone, offsets[0] != 0,
 * offsets[n] != arcs, a column out of range), TKC_EOVERFLOW, TKC_ECUDA,
 * TKC_ETIMEOUT.  nsrc = 0 returns TKC_OK without touching the device. */
#define TKC_NOALLOC_MAX_N 65536
int tkc_distance_sums_noalloc(const uint32_t *offsets, const uint32_t *cols, uint32_t n, uint64_t arcs,
                              uint32_t nsrc, const uint32_t *srcs, uint64_t *S, uint32_t *r, void *stream);

/* Per-level totals of the latest run of the persistent search kernel on a
 * context (no paper counterpart: measurement only).  They are the inputs of
 * the level kernels' byte counts: a top-down level reads each frontier
 * vertex's row and offsets and each frontier arc's column and target row; a
 * bottom-up level reads every vertex's seen row, and the in-arc columns and
 * frontier rows of the vertices it scans.  Counters add up over the run's
 * teams and launches. */
typedef struct {
  uint32_t n;                   /* vertices of the graph (or of the union of several) */
  uint32_t batch_bits;          /* B, sources per batch */
  uint32_t row_bytes;           /* bytes of one bit row (8 * ceil(B / 64)) */
  uint32_t teams;               /* teams of the main launch */
  uint32_t launches;            /* launches of the search kernel (an opening batch adds one) */
  uint32_t pad;
  uint64_t arcs;
  uint64_t td_levels;           /* top-down level steps */
  uint64_t td_frontier;         /* frontier vertices expanded top-down (sum over those levels) */
  uint64_t td_frontier_arcs;    /* their out-arcs */
  uint64_t td_new;              /* vertices discovered by top-down levels */
  uint64_t bu_levels;           /* bottom-up level steps */
  uint64_t bu_scanned_vertices; /* vertices whose in-arcs a bottom-up level walked */
  uint64_t bu_scanned_arcs;     /* in-arcs walked (up to each early exit) */
  uint64_t bu_new;              /* vertices discovered by bottom-up levels */
  uint64_t bu_frontier;         /* frontier vertices of the bottom-up levels (their rows are cleared) */
  uint64_t bu_rows_read;        /* frontier rows the bottom-up walks loaded (in-neighbours on the frontier) */
  uint64_t bu_swept;            /* vertices the bottom-up levels swept (those with an in-arc, per level) */
  uint64_t seeded;              /* searches started in a slot */
  uint64_t cleared;             /* rows zeroed by the clear steps between batches */
  uint64_t compactions;         /* frontier lists compacted to the searches still active after a cut */
  uint64_t compacted_away;      /* list entries those compactions dropped (their rows zeroed) */
  uint64_t alg_bytes;           /* the search kernel's byte count (tkc_result.alg_bytes of that run) */
  double ms_kernel;             /* device time of the search kernel's launches */
} tkc_run_stats;

/* Copies the statistics of ctx's latest search-kernel run into *out (all
 * zero before the first run).  Errors: TKC_EINVAL (null argument). */
int tkc_last_run_stats(const tkc_ctx *ctx, tkc_run_stats *out);

/* Number of CUDA kernels this library has launched in this process (all
 * contexts), for accounting of device work (no paper counterpart; never
 * fails). */
uint64_t tkc_kernel_launches(void);

/* ---- learned source order (beyond the paper) ------------------------------
 * Algorithm 1's result does not depend on the order of Q (Section 4: every
 * order gives the exact top-k; only pruning changes).  The library can order
 * sources by the farness a small MLP predicts from per-vertex features, so
 * that the k-th threshold x tightens sooner; the degree order of Section 4 is
 * the fallback.  Model: x (TKC_MLP_FEATURES) -> 64 -> 64 -> 1, ReLU, bf16
 * weights, fp32 accumulation.  Parameters, TKC_MLP_PARAMS floats:
 * W1[64][5], b1[64], W2[64][64], b2[64], w3[64], b3. */
#define TKC_MLP_FEATURES 5
#define TKC_MLP_HIDDEN 64
#define TKC_MLP_PARAMS 4609

/* Standardized features of every vertex into DEVICE array x[n][5]:
 * log1p of out-degree, in-degree, the 2-walk count sum of out-degrees of
 * out-neighbours (the Section 6 lemma's gamma at d = 1, a bound on the 2-hop ball), the
 * core number of the graph with arc directions dropped (degree = out-degree +
 * in-degree when directed; h-index iteration from the degree run until no
 * value changes, Lu et al. 2016), and the SCC size (component size if
 * undirected); each
 * feature shifted and scaled to mean 0, variance 1 over the graph.  Errors:
 * TKC_EINVAL (null g, or null x with n > 0), TKC_ENOMEM, TKC_ECUDA,
 * TKC_ETIMEOUT. */
int tkc_vertex_features(tkc_graph *g, float *x);

/* Random He-uniform weights from `seed` (zero biases); resets Adam.
 * Errors: TKC_EINVAL (null ctx), TKC_ENOMEM, TKC_ECUDA. */
int tkc_mlp_init(tkc_ctx *ctx, uint64_t seed);

/* Sets / reads the fp32 master weights (host arrays of TKC_MLP_PARAMS);
 * setting enables TKC_ORDER_LEARNED and resets Adam.  Errors: TKC_EINVAL (null
 * argument, nparams != TKC_MLP_PARAMS; reading before any model is set),
 * TKC_ENOMEM, TKC_ECUDA. */
int tkc_set_source_model(tkc_ctx *ctx, const float *params, uint32_t nparams);
int tkc_get_source_model(tkc_ctx *ctx, float *params, uint32_t nparams);

/* y[i] = model(x[i]) for m samples; x, y DEVICE arrays (m x 5, m).
 * Errors: TKC_EINVAL (null ctx, null x or y with m > 0, no model set),
 * TKC_ECUDA. */
int tkc_mlp_forward(tkc_ctx *ctx, const float *x, uint32_t m, float *y);

/* Gradient of L = (1/m) sum_i (model(x_i) - t_i)^2 with respect to the
 * parameters (forward pass with the bf16 weights) into DEVICE grad[P]; the
 * loss into host *loss (may be NULL).  x, t: DEVICE arrays.  Errors:
 * TKC_EINVAL (null ctx, x, t or grad, m = 0, no model set), TKC_ENOMEM,
 * TKC_ECUDA. */
int tkc_mlp_gradient(tkc_ctx *ctx, const float *x, const float *t, uint32_t m, float *grad, float *loss);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on that gradient with
 * learning rate lr; refreshes the bf16 weights; loss before the step into
 * host *loss (may be NULL).  Errors: TKC_EINVAL (null ctx, x or t, m = 0, no
 * model set, lr not > 0), TKC_ENOMEM, TKC_ECUDA. */
int tkc_mlp_train_step(tkc_ctx *ctx, const float *x, const float *t, uint32_t m, float lr, float *loss);

/* Names a TKC_* return code ("unknown error" for any other value); the
 * string is static. */
const char *tkc_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* TKC_H */
