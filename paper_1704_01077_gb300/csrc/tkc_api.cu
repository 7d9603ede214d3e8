// The C ABI of include/tkc.h: contexts, graph upload, and the top-k driver
// that runs preprocessing, the persistent BFSCut kernel and the output step.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <vector>

#include "tkc_internal.cuh"

#include <atomic>

static thread_local char g_last_err[512] = {0};
static std::atomic<unsigned long long> g_launches{0};

void tkc::note_launches(unsigned count) { g_launches.fetch_add(count, std::memory_order_relaxed); }

void tkc_set_last_cuda_error(cudaError_t e, const char *what, const char *file, int line) {
  snprintf(g_last_err, sizeof(g_last_err), "%s: %s (%s:%d)", cudaGetErrorString(e), what, file, line);
}

namespace tkc {

typedef uint32_t u32;
typedef unsigned long long u64;

static constexpr uint64_t kDefaultTimeout = 1ull << 34;

template <typename T>
static int dalloc(T **p, size_t count, cudaStream_t st) {
  if (*p) {
    TKC_TRY(cudaFreeAsync(*p, st));
    *p = nullptr;
  }
  TKC_TRY(cudaMallocAsync((void **)p, std::max<size_t>(count, 1) * sizeof(T), st));
  return TKC_OK;
}

int ensure_workspace(tkc_ctx *ctx, u32 n, int words, u32 top_entries, u32 ng, u32 teams) {
  Workspace &w = ctx->ws;
  cudaStream_t st = ctx->stream;
  if (!w.sh) {
    TKC_RC(dalloc(&w.sh, 1, st));
  }
  if (teams > w.teams_cap) {
    TKC_RC(dalloc(&w.ctl, teams, st));
    TKC_RC(dalloc(&w.slots, (size_t)teams * 64 * kMaxWords, st));
    TKC_RC(dalloc(&w.cnt, (size_t)teams * 64 * kMaxWords, st));
    TKC_RC(dalloc(&w.wsum, (size_t)teams * 64 * kMaxWords, st));
    TKC_TRY(cudaMemsetAsync(w.cnt, 0, (size_t)teams * 64 * kMaxWords * sizeof(unsigned), st));
    TKC_TRY(cudaMemsetAsync(w.wsum, 0, (size_t)teams * 64 * kMaxWords * sizeof(u64), st));
    w.teams_cap = teams;
    w.n_cap = 0;  // per-team vertex buffers are reallocated for the new team count
  }
  if (top_entries > w.top_cap) {
    u32 cap = std::max<u32>(top_entries, TKC_MAX_K);
    TKC_RC(dalloc(&w.top_S, cap, st));
    TKC_RC(dalloc(&w.top_r, cap, st));
    TKC_RC(dalloc(&w.top_id, cap, st));
    TKC_RC(dalloc(&w.out_S, cap, st));
    TKC_RC(dalloc(&w.out_r, cap, st));
    TKC_RC(dalloc(&w.out_id, cap, st));
    TKC_RC(dalloc(&w.out_f, cap, st));
    TKC_RC(dalloc(&w.out_c, cap, st));
    w.top_cap = cap;
  }
  if (ng > w.ng_cap) {
    u32 cap = std::max<u32>(ng, 16);
    TKC_RC(dalloc(&w.tied, cap, st));
    TKC_RC(dalloc(&w.g_ntop, cap, st));
    TKC_RC(dalloc(&w.g_stop, cap, st));
    TKC_RC(dalloc(&w.g_ctr, 4 * (size_t)cap, st));
    TKC_RC(dalloc(&w.x_seq, cap, st));
    TKC_RC(dalloc(&w.x_S, cap, st));
    TKC_RC(dalloc(&w.x_r, cap, st));
    TKC_RC(dalloc(&w.x_id, cap, st));
    w.ng_cap = cap;
  }
  const u32 T = w.teams_cap;
  if (n > w.n_cap) {
    u32 cap = std::max<u32>(n, 1024);
    size_t tv = (size_t)T * cap, tfb = (size_t)T * (cap / 32 + 1);
    TKC_RC(dalloc(&w.L0, tv, st));
    TKC_RC(dalloc(&w.L1, tv, st));
    TKC_RC(dalloc(&w.Loff0, tv, st));
    TKC_RC(dalloc(&w.Loff1, tv, st));
    TKC_RC(dalloc(&w.VL, tv, st));
    TKC_RC(dalloc(&w.stamp, tv, st));
    TKC_RC(dalloc(&w.res_S, cap, st));
    TKC_RC(dalloc(&w.res_r, cap, st));
    TKC_RC(dalloc(&w.FB0, tfb, st));
    TKC_RC(dalloc(&w.FB1, tfb, st));
    TKC_TRY(cudaMemsetAsync(w.FB0, 0, tfb * sizeof(u32), st));
    TKC_TRY(cudaMemsetAsync(w.FB1, 0, tfb * sizeof(u32), st));
    TKC_TRY(cudaMemsetAsync(w.stamp, 0xff, tv * sizeof(u32), st));
    w.level_base = 0;
    w.n_cap = cap;
    w.words_cap = 0;  // rows must be reallocated for the new n
  }
  if (words > w.words_cap) {
    size_t rows = (size_t)T * w.n_cap * words;
    TKC_RC(dalloc(&w.seen, rows, st));
    TKC_RC(dalloc(&w.F0, rows, st));
    TKC_RC(dalloc(&w.F1, rows, st));
    TKC_RC(dalloc(&w.N, rows, st));
    TKC_TRY(cudaMemsetAsync(w.seen, 0, rows * sizeof(u64), st));
    TKC_TRY(cudaMemsetAsync(w.F0, 0, rows * sizeof(u64), st));
    TKC_TRY(cudaMemsetAsync(w.F1, 0, rows * sizeof(u64), st));
    TKC_TRY(cudaMemsetAsync(w.N, 0, rows * sizeof(u64), st));
    w.words_cap = words;
  }
  return TKC_OK;
}

static void free_workspace(tkc_ctx *ctx) {
  Workspace &w = ctx->ws;
  void *ptrs[] = {w.seen, w.F0, w.F1, w.N, w.FB0, w.FB1, w.L0, w.L1, w.Loff0, w.Loff1, w.VL, w.stamp, w.res_S, w.res_r,
                  w.slots, w.cnt, w.wsum, w.top_S, w.top_r, w.top_id, w.ctl, w.out_S, w.out_r, w.out_id,
                  w.out_f, w.out_c, w.tied, w.g_ntop, w.g_stop, w.g_ctr, w.sh, w.x_seq, w.x_S, w.x_r, w.x_id};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  w = Workspace();
}

// Row buffers hold only the current run's bits; the kernel leaves them zero
// when it ends normally.  After an error they are cleared here.
static int reset_rows(tkc_ctx *ctx) {
  Workspace &w = ctx->ws;
  const size_t T = w.teams_cap;
  size_t rows = T * w.n_cap * w.words_cap;
  cudaStream_t st = ctx->stream;
  TKC_TRY(cudaMemsetAsync(w.seen, 0, rows * sizeof(u64), st));
  TKC_TRY(cudaMemsetAsync(w.F0, 0, rows * sizeof(u64), st));
  TKC_TRY(cudaMemsetAsync(w.F1, 0, rows * sizeof(u64), st));
  TKC_TRY(cudaMemsetAsync(w.N, 0, rows * sizeof(u64), st));
  TKC_TRY(cudaMemsetAsync(w.FB0, 0, T * ((size_t)w.n_cap / 32 + 1) * sizeof(u32), st));
  TKC_TRY(cudaMemsetAsync(w.FB1, 0, T * ((size_t)w.n_cap / 32 + 1) * sizeof(u32), st));
  TKC_TRY(cudaMemsetAsync(w.cnt, 0, T * 64 * kMaxWords * sizeof(unsigned), st));
  TKC_TRY(cudaMemsetAsync(w.wsum, 0, T * 64 * kMaxWords * sizeof(u64), st));
  return TKC_OK;
}

// ------------------------------------------------------------------ output

// What the output step needs of each graph of a run.
struct GraphOut {
  u32 n;          // vertices of the graph
  u32 base;       // first id of the graph in the run's (union) numbering
  u32 kk;         // min(k, n)
  u32 nzero;      // vertices of out-degree 0 (closeness 0)
  const u32 *zero_ids;  // those vertices in increasing id order (graph-local ids)
};

// Ties with each graph's k-th entry among finished searches (exact key
// equality).  A graph whose k-th entry is a closeness-0 vertex is counted on
// the host (every closeness-0 vertex ties with it).
__global__ void k_count_ties(const u64 *res_S, const u32 *res_r, const u32 *gid, u32 nv, const u64 *top_S,
                             const u32 *top_r, const unsigned *g_ntop, u32 kk, const GraphOut *go, int harmonic,
                             unsigned *tied) {
  for (u32 v = blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += gridDim.x * blockDim.x) {
    u32 r = res_r[v];
    if (r < 2) continue;
    u32 g = gid ? gid[v] : 0;
    u32 kg = go[g].kk;
    if (g_ntop[g] < kg) continue;
    size_t x = (size_t)g * kk + kg - 1;
    if (harmonic) {
      // the same FP64 h, bit for bit
      if (res_S[v] == top_S[x]) atomicAdd(&tied[g], 1u);
      continue;
    }
    u64 rx = top_r[x];
    unsigned __int128 a = (unsigned __int128)res_S[v] * (unsigned __int128)((rx - 1) * (rx - 1));
    unsigned __int128 b = (unsigned __int128)top_S[x] * (unsigned __int128)((u64)(r - 1) * (u64)(r - 1));
    if (a == b) atomicAdd(&tied[g], 1u);
  }
}

// Final list of graph blockIdx.x: its top entries, then (if fewer than k of
// its vertices reach another vertex) closeness-0 vertices in id order.  f and
// c are one IEEE product and one quotient of exact integers.  Harmonic runs:
// c = h (the list key's FP64 value), f = 1/h, S not kept (0).
__global__ void k_output(const u64 *top_S, const u32 *top_r, const u32 *top_id, const unsigned *g_ntop, u32 kk,
                         const GraphOut *go, int harmonic, u64 *oS, u32 *or_, u32 *oid, double *of, double *oc) {
  const u32 g = blockIdx.x;
  const GraphOut G = go[g];
  const u32 ntop = g_ntop[g];
  for (u32 i = threadIdx.x; i < G.kk; i += blockDim.x) {
    size_t src = (size_t)g * kk + i;
    u64 S;
    u32 r, id;
    if (i < ntop) {
      S = top_S[src];
      r = top_r[src];
      id = top_id[src] - G.base;
    } else {
      S = 0;
      r = 1;
      id = G.zero_ids[i - ntop];
    }
    oS[src] = harmonic ? 0 : S;
    or_[src] = r;
    oid[src] = id;
    if (harmonic) {
      const double h = r <= 1 ? 0.0 : __longlong_as_double((long long)S);
      oc[src] = h;
      of[src] = h > 0.0 ? __ddiv_rn(1.0, h) : __longlong_as_double(0x7ff0000000000000ll);
    } else if (r <= 1) {
      of[src] = __longlong_as_double(0x7ff0000000000000ll);
      oc[src] = 0.0;
    } else {
      double num = __dmul_rn((double)(G.n - 1), (double)S);
      double den = (double)((u64)(r - 1) * (u64)(r - 1));
      of[src] = __ddiv_rn(num, den);
      oc[src] = __ddiv_rn(den, num);
    }
  }
}

static int words_for(u32 bits) {
  if (bits <= 64) return 1;
  if (bits <= 128) return 2;
  if (bits <= 256) return 4;
  return 8;
}

// Batch width used when the options leave it to the library.
static u32 default_batch_bits(u32 n, bool nb = false) {
  if (n < 4096) return 64;
  if (n >= (1u << 16)) return nb ? 128 : 64;
  return 128;
}

// One run of the persistent kernel: a graph, or the union of several.
struct RunSetup {
  const tkc_graph *g;       // the graph (or the union's stand-in graph)
  const u32 *order;
  u32 norder;
  u32 B;
  int W;
  int nocut;
  int harmonic;             // rank by harmonic centrality instead of closeness
  u32 nocut_prefix;
  const u64 *lb_key;        // NBCut order keys (nullptr: no stop test)
  u32 kk;                   // list length per graph
  u32 ng;
  const u32 *gid;           // nullptr for one graph
  const uint8_t *g_directed;
  // updateBoundsLB rounds: level recording, one team, lists kept across rounds
  uint16_t *lvl;
  u32 *hist;
  u32 *lvl_src;
  u32 hist_cap;
  u32 lvl_stride;
  int keep_lists;
  u32 force_teams;
  // a starting k-list (one graph; host arrays, best first): exact entries of
  // vertices searched elsewhere, so that x is tight from the start
  const u64 *seed_S;
  const u32 *seed_r, *seed_id;
  u32 nseed;
  // size that decides the library's labelling choice: the largest graph of a
  // multi-graph union (0: g->n)
  u32 size_n;
  // several graphs, sources graph by graph after every graph's opening batch:
  // one past each graph's last position in `order` (nullptr: graphs
  // interleaved), and the first position after the openings
  const u32 *g_end;
  u32 g_rest;
};

// Teams used when the options leave it to the library: one team for small
// graphs (a level is short and the whole GPU serves it), more for large ones
// so that the latency of one team's level steps overlaps with the others.
// NBCut on one graph examines few sources, each batch deeper: fewer, larger
// teams (measured on R-MAT 22: 4 teams 357 ms, 9 teams 372 ms, 19 teams 411 ms).
static u32 default_teams(u32 n, u32 B, u32 maxb, bool nb) {
  if (B <= 1 || n < (1u << 14)) return 1;
  if (nb) return std::max<u32>(1, maxb / 32);
  if (n < (1u << 16)) return std::max<u32>(1, maxb / 16);
  return std::max<u32>(1, maxb / 8);  // eight blocks (SMs) per team, every SM used
}

// Whether the search walks the in-degree labelling: batched searches of
// large graphs (its hot rows stay in L2); one-source searches and small
// graphs (of a union: when no graph is large, each one's rows fit L2 anyway)
// the graph itself.
static bool labelled_search(const tkc_options &o, u32 B, u32 size_n) {
  return o.relabel == 1 || (o.relabel == 0 && B > 1 && size_n >= (1u << 20));
}

static int run_search(tkc_ctx *ctx, const RunSetup &rs, Ctl *hctl) {
  const tkc_graph *g = rs.g;
  Workspace &w = ctx->ws;
  cudaStream_t st = ctx->stream;
  const tkc_options &o = ctx->opt;
  int maxb = max_coresident_blocks(ctx, rs.W);
  if (maxb <= 0) return TKC_ECUDA;
  const bool nb_one = rs.lb_key != nullptr && rs.ng == 1;
  u32 T = rs.B <= 1 ? 1u : (o.teams ? o.teams : default_teams(g->n, rs.B, (u32)maxb, nb_one));
  if (rs.force_teams) T = rs.force_teams;
  // deterministic schedule: one team, so x moves only at its level barriers
  // (updateBoundsLB rounds fix their own team count: no cuts, already exact)
  if (o.deterministic && !rs.force_teams) T = 1;
  T = std::max<u32>(1, std::min<u32>(T, (u32)maxb));
  TKC_RC(ensure_workspace(ctx, g->n, rs.W, rs.kk * rs.ng, rs.ng, T));
  if (w.level_base > 0xF0000000u) {
    TKC_TRY(cudaMemsetAsync(w.stamp, 0xff, (size_t)w.teams_cap * w.n_cap * sizeof(u32), st));
    w.level_base = 0;
  }
  ctx->last_shard = nullptr;  // this run replaces the finished searches' (S, r)
  if (!rs.keep_lists) {
    TKC_TRY(cudaMemsetAsync(w.res_r, 0, (size_t)g->n * sizeof(u32), st));
    TKC_TRY(cudaMemsetAsync(w.res_S, 0, (size_t)g->n * sizeof(u64), st));
    TKC_TRY(cudaMemsetAsync(w.g_ntop, 0, (size_t)rs.ng * sizeof(unsigned), st));
    TKC_TRY(cudaMemsetAsync(w.g_stop, 0, (size_t)rs.ng * sizeof(unsigned), st));
    TKC_TRY(cudaMemsetAsync(w.g_ctr, 0, (size_t)rs.ng * 4 * sizeof(u64), st));
    TKC_TRY(cudaMemsetAsync(w.x_seq, 0, (size_t)rs.ng * sizeof(unsigned), st));
    TKC_TRY(cudaMemsetAsync(w.x_r, 0, (size_t)rs.ng * sizeof(u32), st));
  }
  if (rs.nseed) {
    const unsigned ns = rs.nseed;
    TKC_TRY(cudaMemcpyAsync(w.g_ntop, &ns, sizeof(unsigned), cudaMemcpyHostToDevice, st));
    TKC_TRY(cudaMemcpyAsync(w.top_S, rs.seed_S, ns * sizeof(u64), cudaMemcpyHostToDevice, st));
    TKC_TRY(cudaMemcpyAsync(w.top_r, rs.seed_r, ns * sizeof(u32), cudaMemcpyHostToDevice, st));
    TKC_TRY(cudaMemcpyAsync(w.top_id, rs.seed_id, ns * sizeof(u32), cudaMemcpyHostToDevice, st));
    if (ns == rs.kk) {  // a full list: its k-th entry is the published threshold
      TKC_TRY(cudaMemcpyAsync(w.x_S, rs.seed_S + ns - 1, sizeof(u64), cudaMemcpyHostToDevice, st));
      TKC_TRY(cudaMemcpyAsync(w.x_r, rs.seed_r + ns - 1, sizeof(u32), cudaMemcpyHostToDevice, st));
      TKC_TRY(cudaMemcpyAsync(w.x_id, rs.seed_id + ns - 1, sizeof(u32), cudaMemcpyHostToDevice, st));
    }
    TKC_TRY(cudaStreamSynchronize(st));  // the seed arrays are the caller's pageable memory
  }
  RunParams p;
  memset(&p, 0, sizeof(p));
  p.n = g->n;
  p.directed = g->directed;
  p.arcs = g->arcs;
  const bool relabel = labelled_search(o, rs.B, rs.size_n ? rs.size_n : g->n);
  TKC_RC(ensure_search_csr(g, relabel));
  const bool lab = g->s_mode == 1;
  p.off = lab ? g->s_off : g->off;
  p.col = lab ? g->s_col : g->col;
  p.ioff = lab ? g->s_ioff : g->ioff;
  p.icol = lab ? g->s_icol : g->icol;
  p.lab = lab ? g->s_lab : nullptr;
  p.unlab = lab ? g->s_unlab : nullptr;
  p.bu_list = g->bu_list;
  p.n_bu = g->n_bu;
  p.n_bu_heavy = g->n_bu_heavy;
  p.heavy_in = g->heavy_in ? g->heavy_in : kHeavyIn;
  p.large_blocks = o.large_blocks;
  p.alpha = g->alpha;
  p.omega = g->omega;
  p.order = rs.order;
  p.norder = rs.norder;
  p.ng = rs.ng;
  p.gid = rs.gid;
  p.g_end = rs.g_end;
  p.g_rest = rs.g_rest;
  p.g_directed = rs.g_directed;
  p.g_ntop = w.g_ntop;
  p.g_ctr = rs.ng > 1 ? w.g_ctr : nullptr;
  p.kk = rs.kk;
  p.B = rs.B;
  p.nocut = rs.nocut;
  p.nocut_prefix = rs.nocut_prefix;
  p.lb_key = rs.lb_key;
  p.g_stop = w.g_stop;
  p.harmonic = rs.harmonic;
  p.lvl = rs.lvl;
  p.hist = rs.hist;
  p.lvl_src = rs.lvl_src;
  p.hist_cap = rs.hist_cap;
  p.lvl_stride = rs.lvl_stride;
  p.teams = T;
  p.row_stride = (u64)w.n_cap * w.words_cap;
  p.vtx_stride = w.n_cap;
  p.fb_stride = w.n_cap / 32 + 1;
  p.sh = w.sh;
  p.x_seq = w.x_seq;
  p.x_S = w.x_S;
  p.x_r = w.x_r;
  p.x_id = w.x_id;
  // default: a level runs bottom-up when its frontier's arcs exceed 1/8 of all arcs
  p.bu_num = o.bu_num ? o.bu_num : 8;
  p.bu_den = o.bu_num ? std::max<u32>(o.bu_den, 1) : 1;
  p.timeout = o.timeout_cycles ? o.timeout_cycles : kDefaultTimeout;
  p.seen = w.seen;
  p.F0 = w.F0;
  p.F1 = w.F1;
  p.N = w.N;
  p.FB0 = w.FB0;
  p.FB1 = w.FB1;
  p.L0 = w.L0;
  p.L1 = w.L1;
  p.Loff0 = w.Loff0;
  p.Loff1 = w.Loff1;
  p.VL = w.VL;
  p.stamp = w.stamp;
  p.slots = w.slots;
  p.cnt = w.cnt;
  p.wsum = w.wsum;
  p.top_S = w.top_S;
  p.top_r = w.top_r;
  p.top_id = w.top_id;
  p.res_S = w.res_S;
  p.res_r = w.res_r;
  p.ctl = w.ctl;
  int blocks = o.blocks ? (int)o.blocks : (int)std::max<u64>(8, ((u64)g->n + 511) / 512);
  blocks = std::min(blocks, maxb);
  blocks = std::max<int>(T, blocks / (int)T * (int)T);  // a multiple of the team count
  // optional per-step trace for profiling: TKC_TRACE=<csv path>
  const char *trace_path = getenv("TKC_TRACE");
  const uint32_t trace_cap = 1u << 20;
  if (trace_path) {
    TKC_TRY(cudaMallocAsync(&p.trace, (size_t)trace_cap * 16 * sizeof(u64), st));
    TKC_TRY(cudaMemsetAsync(p.trace, 0, (size_t)trace_cap * 16 * sizeof(u64), st));
    p.trace_cap = trace_cap;
  }
  // Opening: with several teams on one graph, the first batch runs alone on
  // the whole grid (one team), so that a threshold exists before the teams
  // start and the batch that sets it gets every SM; the teams then take the
  // rest of the order.  The k-lists and thresholds carry over.
  const bool opening = T > 1 && rs.ng == 1 && !rs.nocut && rs.norder > rs.B;
  struct Phase {
    u32 teams, begin, count;
  };
  std::vector<Phase> phases;
  if (opening) {
    phases.push_back({1u, 0u, rs.B});
    phases.push_back({T, rs.B, rs.norder - rs.B});
  } else {
    phases.push_back({T, 0u, rs.norder});
  }
  memset(hctl, 0, sizeof(Ctl));
  std::vector<Ctl> cs(T);
  TKC_TRY(cudaEventRecord(ctx->ev[4], st));
  for (const Phase &ph : phases) {
    for (u32 t = 0; t < ph.teams; ++t) {
      memset(&cs[t], 0, sizeof(Ctl));
      cs[t].step = 1;  // start with an (empty) clear step whose epilogue seeds the first batch
      cs[t].level_id = w.level_base;
    }
    TKC_TRY(cudaMemcpyAsync(w.ctl, cs.data(), ph.teams * sizeof(Ctl), cudaMemcpyHostToDevice, st));
    TKC_TRY(cudaMemsetAsync(w.sh, 0, sizeof(Shared), st));
    p.teams = ph.teams;
    p.order = rs.order + ph.begin;
    p.norder = ph.count;
    p.nocut_prefix = rs.nocut_prefix > ph.begin ? rs.nocut_prefix - ph.begin : 0;
    const int pblocks = std::max<int>((int)ph.teams, blocks / (int)ph.teams * (int)ph.teams);
    TKC_RC(run_bfscut(ctx, p, rs.W, pblocks));
    TKC_TRY(cudaMemcpyAsync(cs.data(), w.ctl, ph.teams * sizeof(Ctl), cudaMemcpyDeviceToHost, st));
    Shared hsh;
    TKC_TRY(cudaMemcpyAsync(&hsh, w.sh, sizeof(Shared), cudaMemcpyDeviceToHost, st));
    TKC_TRY(cudaStreamSynchronize(st));
    // the teams' counters add up; levels and batches too (they ran side by side)
    for (u32 t = 0; t < ph.teams; ++t) {
      const Ctl &x = cs[t];
      hctl->edges_visited += x.edges_visited;
      hctl->edges_scanned += x.edges_scanned;
      hctl->bfs_started += x.bfs_started;
      hctl->bfs_cut += x.bfs_cut;
      hctl->bfs_finished += x.bfs_finished;
      hctl->levels += x.levels;
      hctl->batches += x.batches;
      hctl->alg_bytes += x.alg_bytes;
      hctl->st_td_levels += x.st_td_levels;
      hctl->st_td_frontier += x.st_td_frontier;
      hctl->st_td_arcs += x.st_td_arcs;
      hctl->st_td_new += x.st_td_new;
      hctl->st_bu_levels += x.st_bu_levels;
      hctl->st_bu_scan_v += x.st_bu_scan_v;
      hctl->st_bu_scan_a += x.st_bu_scan_a;
      hctl->st_bu_new += x.st_bu_new;
      hctl->st_bu_frontier += x.st_bu_frontier;
      hctl->st_bu_rows += x.st_bu_rows;
      hctl->st_seeded += x.st_seeded;
      hctl->st_cleared += x.st_cleared;
      hctl->st_compactions += x.st_compactions;
      hctl->st_compact_dropped += x.st_compact_dropped;
      hctl->trace_n += x.trace_n;
      hctl->level_id = std::max(hctl->level_id, x.level_id);
      if (!hctl->err) hctl->err = x.err;
    }
    if (!hctl->err) hctl->err = hsh.err;
    w.level_base = hctl->level_id + 1;
    if (p.trace) {
      std::vector<u64> tr((size_t)trace_cap * 16);
      TKC_TRY(cudaMemcpy(tr.data(), p.trace, tr.size() * sizeof(u64), cudaMemcpyDeviceToHost));
      TKC_TRY(cudaMemset(p.trace, 0, tr.size() * sizeof(u64)));
      FILE *f = fopen(trace_path, "a");
      if (f) {
        fprintf(f, "# n=%u arcs=%llu B=%u blocks=%d graphs=%u teams=%u\n", g->n, (unsigned long long)g->arcs, rs.B,
                pblocks, rs.ng, ph.teams);
        fprintf(f, "t_ns,kind,a,b,c,d,e,f,t_top,t_a_end,t_a_sync,t_b_end,t_flush,t_epi,team,y\n");
        const u64 per = trace_cap / ph.teams;
        for (u32 t = 0; t < ph.teams; ++t)
          for (u64 i = 0; i < std::min<u64>(cs[t].trace_n, per); ++i) {
            u64 *r = &tr[((size_t)t * per + i) * 16];
            r[14] = t;
            for (int j = 0; j < 16; ++j) fprintf(f, j ? ",%llu" : "%llu", r[j]);
            fprintf(f, "\n");
          }
        fclose(f);
      }
      for (u32 t = 0; t < ph.teams; ++t) cs[t].trace_n = 0;
    }
    if (hctl->err) break;
  }
  TKC_TRY(cudaEventRecord(ctx->ev[5], st));
  if (p.trace) TKC_TRY(cudaFree(p.trace));
  {
    tkc_run_stats &rs_out = ctx->last_stats;
    rs_out.n = g->n;
    rs_out.arcs = g->arcs;
    rs_out.batch_bits = rs.B;
    rs_out.row_bytes = 8u * (u32)rs.W;
    rs_out.teams = T;
    rs_out.launches = (u32)phases.size();
    rs_out.td_levels = hctl->st_td_levels;
    rs_out.td_frontier = hctl->st_td_frontier;
    rs_out.td_frontier_arcs = hctl->st_td_arcs;
    rs_out.td_new = hctl->st_td_new;
    rs_out.bu_levels = hctl->st_bu_levels;
    rs_out.bu_scanned_vertices = hctl->st_bu_scan_v;
    rs_out.bu_scanned_arcs = hctl->st_bu_scan_a;
    rs_out.bu_new = hctl->st_bu_new;
    rs_out.bu_frontier = hctl->st_bu_frontier;
    rs_out.bu_rows_read = hctl->st_bu_rows;
    rs_out.bu_swept = (uint64_t)(g->bu_list ? g->n_bu : g->n) * hctl->st_bu_levels;
    rs_out.seeded = hctl->st_seeded;
    rs_out.cleared = hctl->st_cleared;
    rs_out.compactions = hctl->st_compactions;
    rs_out.compacted_away = hctl->st_compact_dropped;
    rs_out.alg_bytes = hctl->alg_bytes;
    float kms = 0;
    TKC_TRY(cudaEventSynchronize(ctx->ev[5]));
    cudaEventElapsedTime(&kms, ctx->ev[4], ctx->ev[5]);
    rs_out.ms_kernel = kms;
  }
  if (hctl->err) {
    TKC_RC(reset_rows(ctx));
    TKC_TRY(cudaStreamSynchronize(st));
    return hctl->err;
  }
  return TKC_OK;
}

// Output step of a run: ties, final lists, copies into the callers' results.
// outs[i] receives graph i.  Returns per-graph g_ntop and counters in the
// host vectors.
static int finish_run(tkc_ctx *ctx, const RunSetup &rs, const std::vector<GraphOut> &go_h, tkc_result *outs,
                      std::vector<unsigned> &ntop, std::vector<unsigned> &tied, std::vector<u64> &gctr) {
  Workspace &w = ctx->ws;
  cudaStream_t st = ctx->stream;
  const u32 ng = rs.ng;
  GraphOut *go = nullptr;
  TKC_TRY(cudaMallocAsync(&go, ng * sizeof(GraphOut), st));
  TKC_TRY(cudaMemcpyAsync(go, go_h.data(), ng * sizeof(GraphOut), cudaMemcpyHostToDevice, st));
  TKC_TRY(cudaMemsetAsync(w.tied, 0, ng * sizeof(unsigned), st));
  unsigned blocks = (unsigned)std::max<u64>(1, std::min<u64>((rs.g->n + 255) / 256, (u64)ctx->num_sms * 8));
  TKC_LAUNCH(k_count_ties<<<blocks, 256, 0, st>>>(w.res_S, w.res_r, rs.gid, rs.g->n, w.top_S, w.top_r, w.g_ntop,
                                                  rs.kk, go, rs.harmonic, w.tied));
  TKC_LAUNCH(k_output<<<ng, 256, 0, st>>>(w.top_S, w.top_r, w.top_id, w.g_ntop, rs.kk, go, rs.harmonic, w.out_S,
                                          w.out_r, w.out_id, w.out_f, w.out_c));
  TKC_TRY(cudaGetLastError());
  ntop.resize(ng);
  tied.resize(ng);
  gctr.resize(4 * (size_t)ng);
  TKC_TRY(cudaMemcpyAsync(ntop.data(), w.g_ntop, ng * sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  TKC_TRY(cudaMemcpyAsync(tied.data(), w.tied, ng * sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  if (ng > 1)
    TKC_TRY(cudaMemcpyAsync(gctr.data(), w.g_ctr, 4 * (size_t)ng * sizeof(u64), cudaMemcpyDeviceToHost, st));
  for (u32 i = 0; i < ng; ++i) {
    tkc_result *out = &outs[i];
    const u32 kg = go_h[i].kk;
    const size_t src = (size_t)i * rs.kk;
    if (!kg) continue;
    if (out->ids) TKC_TRY(cudaMemcpyAsync(out->ids, w.out_id + src, kg * sizeof(u32), cudaMemcpyDeviceToHost, st));
    if (out->dist_sum)
      TKC_TRY(cudaMemcpyAsync(out->dist_sum, w.out_S + src, kg * sizeof(u64), cudaMemcpyDeviceToHost, st));
    if (out->reach) TKC_TRY(cudaMemcpyAsync(out->reach, w.out_r + src, kg * sizeof(u32), cudaMemcpyDeviceToHost, st));
    if (out->farness)
      TKC_TRY(cudaMemcpyAsync(out->farness, w.out_f + src, kg * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (out->closeness)
      TKC_TRY(cudaMemcpyAsync(out->closeness, w.out_c + src, kg * sizeof(double), cudaMemcpyDeviceToHost, st));
  }
  TKC_TRY(cudaFreeAsync(go, st));
  TKC_TRY(cudaStreamSynchronize(st));
  for (u32 i = 0; i < ng; ++i)
    if (ntop[i] < go_h[i].kk) tied[i] = go_h[i].nzero;  // the k-th is a closeness-0 vertex
  return TKC_OK;
}

// Stand-in graph for the disjoint union of several graphs.
__global__ void k_union_offsets(const u64 *offptr, const u32 *vbase, const u64 *abase, u32 ng, u32 nv, u32 *off_u,
                                u32 *gid) {
  for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i <= nv; i += gridDim.x * blockDim.x) {
    if (i == nv) {
      off_u[nv] = (u32)abase[ng];
      continue;
    }
    u32 lo = 0, hi = ng;  // last g with vbase[g] <= i
    while (hi - lo > 1) {
      u32 mid = (lo + hi) >> 1;
      if (vbase[mid] <= i) lo = mid;
      else hi = mid;
    }
    const u32 *og = (const u32 *)offptr[lo];
    off_u[i] = og[i - vbase[lo]] + (u32)abase[lo];
    gid[i] = lo;
  }
}

__global__ void k_union_cols(const u64 *colptr, const u32 *vbase, const u64 *abase, u32 ng, u64 na, u32 *col_u) {
  for (u64 e = (u64)blockIdx.x * blockDim.x + threadIdx.x; e < na; e += (u64)gridDim.x * blockDim.x) {
    u32 lo = 0, hi = ng;
    while (hi - lo > 1) {
      u32 mid = (lo + hi) >> 1;
      if (abase[mid] <= e) lo = mid;
      else hi = mid;
    }
    col_u[e] = ((const u32 *)colptr[lo])[e - abase[lo]] + vbase[lo];
  }
}

// flag[v] = 1 for the union's vertices of out-degree 0 (flag[nv] = 0).
__global__ void k_zero_flags(const u32 *off_u, u32 nv, u32 *flag) {
  for (u32 v = blockIdx.x * blockDim.x + threadIdx.x; v <= nv; v += gridDim.x * blockDim.x)
    flag[v] = v < nv && off_u[v + 1] == off_u[v];
}

// The out-degree-0 vertices of the union in id order, as graph-local ids (pos:
// exclusive scan of k_zero_flags): graph g's are a contiguous run.
__global__ void k_zero_compact(const u32 *off_u, const u32 *pos, const u32 *gid, const u32 *vbase, u32 nv, u32 *zl) {
  for (u32 v = blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += gridDim.x * blockDim.x)
    if (off_u[v + 1] == off_u[v]) zl[pos[v]] = v - vbase[gid[v]];
}

// out[i] = a[idx[i]]
__global__ void k_gather_u32(const u32 *a, const u32 *idx, u32 m, u32 *out) {
  for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) out[i] = a[idx[i]];
}

// key[i] = graph of order[i]
__global__ void k_order_gid(const u32 *order, u32 m, const u32 *gid, u32 *key) {
  for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) key[i] = gid[order[i]];
}

// gbeg[g] / gend[g] = first / one past the last position of key g in the
// sorted keys (either may be null)
__global__ void k_segment_bounds(const u32 *key, u32 m, u32 *gbeg, u32 *gend) {
  for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    if (gbeg && (i == 0 || key[i - 1] != key[i])) gbeg[key[i]] = i;
    if (gend && (i + 1 == m || key[i + 1] != key[i])) gend[key[i]] = i + 1;
  }
}

// Graph-major keys (sorted): key += ng for every position past the first B of
// its graph, so that a second stable sort puts every graph's first B sources
// ahead of all the rest; *p1 = the first position of those rest (m if none),
// found after that sort.
__global__ void k_phase_keys(u32 *key, u32 m, const u32 *gbeg, u32 B, u32 ng) {
  for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
    if (i - gbeg[key[i]] >= B) key[i] += ng;
}

__global__ void k_phase_start(const u32 *key, u32 m, u32 ng, u32 *p1) {
  for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
    if (key[i] >= ng && (i == 0 || key[i - 1] < ng)) *p1 = i;
}

int scan_exclusive_u32(const u32 *in, u32 *out, u64 len, u32 *tmp, cudaStream_t st);
int radix_sort_u32_pairs(u32 *key, u32 *val, u32 n, int bits, cudaStream_t st);

}  // namespace tkc

using namespace tkc;

// ====================================================================== C ABI

extern "C" {

uint64_t tkc_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

int tkc_last_run_stats(const tkc_ctx *ctx, tkc_run_stats *out) {
  if (!ctx || !out) return TKC_EINVAL;
  *out = ctx->last_stats;
  return TKC_OK;
}

const char *tkc_strerror(int code) {
  switch (code) {
    case TKC_OK: return "ok";
    case TKC_EINVAL: return "invalid argument";
    case TKC_EGRAPH: return "malformed CSR graph";
    case TKC_ENOMEM: return "out of memory";
    case TKC_ECUDA: return g_last_err[0] ? g_last_err : "CUDA error";
    case TKC_ETIMEOUT: return "device-side wait exceeded its budget";
    case TKC_EOVERFLOW: return "graph exceeds a size limit of this build";
    default: return "unknown error";
  }
}

static void tune_cache_load(tkc_ctx *ctx);

static bool options_valid(const tkc_options *opt) {
  const u32 b = opt->batch_bits;
  if (!(b == 0 || b == 1 || b == 64 || b == 128 || b == 256 || b == 512)) return false;
  return opt->order <= TKC_ORDER_LEARNED_NB && opt->nb_levels <= 65535 && opt->large_blocks <= 2 && opt->deterministic <= 1 &&
         opt->relabel <= 2;
}

int tkc_create(tkc_ctx **out, const tkc_options *opt) {
  if (!out) return TKC_EINVAL;
  *out = nullptr;
  if (opt && !options_valid(opt)) return TKC_EINVAL;
  tkc_ctx *ctx = new (std::nothrow) tkc_ctx();
  if (!ctx) return TKC_ENOMEM;
  if (opt) ctx->opt = *opt;
  ctx->device = ctx->opt.device;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) {
    tkc_set_last_cuda_error(e, "cudaSetDevice", __FILE__, __LINE__);
    delete ctx;
    return TKC_ECUDA;
  }
  ctx->stream = (cudaStream_t)ctx->opt.stream;
  int coop = 0;
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, ctx->device);
  cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device);
  if (!coop || ctx->num_sms <= 0) {
    delete ctx;
    return TKC_ECUDA;
  }
  tune_cache_load(ctx);
  for (auto &ev : ctx->ev) {
    e = cudaEventCreate(&ev);
    if (e != cudaSuccess) {
      tkc_set_last_cuda_error(e, "cudaEventCreate", __FILE__, __LINE__);
      delete ctx;
      return TKC_ECUDA;
    }
  }
  *out = ctx;
  return TKC_OK;
}

int tkc_set_options(tkc_ctx *ctx, const tkc_options *opt) {
  if (!ctx || !opt) return TKC_EINVAL;
  if (opt->device != ctx->device) return TKC_EINVAL;
  if (!options_valid(opt)) return TKC_EINVAL;
  ctx->opt = *opt;
  ctx->stream = (cudaStream_t)opt->stream;
  return TKC_OK;
}

void tkc_destroy(tkc_ctx *ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  free_workspace(ctx);
  free_mlp(ctx);
  for (auto &ev : ctx->ev)
    if (ev) cudaEventDestroy(ev);
  if (ctx->aux) {
    cudaStreamSynchronize(ctx->aux);
    cudaStreamDestroy(ctx->aux);
  }
  if (ctx->aux_in) cudaEventDestroy(ctx->aux_in);
  delete ctx;
}

// A new graph handle with the CSR copied to the device (stream-ordered, no
// host wait, nothing validated yet).  Host offsets' ends are checked here;
// device ones with the validation.
static int upload_graph(tkc_ctx *ctx, uint32_t n, uint64_t arcs, const uint32_t *offsets, const uint32_t *cols,
                        int directed, int ptr_on_device, tkc_graph **out) {
  *out = nullptr;
  if (n >= kMaxN || arcs >= (1ull << 32)) return TKC_EOVERFLOW;
  if (!offsets || (arcs && !cols)) return TKC_EINVAL;
  if (!ptr_on_device && (offsets[0] != 0 || offsets[n] != arcs)) return TKC_EGRAPH;
  if (ptr_on_device && n == 0) {
    u32 end0 = 1;
    TKC_TRY(cudaMemcpy(&end0, offsets, sizeof(u32), cudaMemcpyDeviceToHost));
    if (end0 != 0 || arcs != 0) return TKC_EGRAPH;
  }
  cudaStream_t st = ctx->stream;
  tkc_graph *g = new (std::nothrow) tkc_graph();
  if (!g) return TKC_ENOMEM;
  g->ctx = ctx;
  g->n = n;
  g->arcs = arcs;
  g->directed = directed ? 1 : 0;
  ctx->graphs_alive++;
  cudaMemcpyKind kind = ptr_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  cudaError_t e = cudaMallocAsync(&g->off, ((size_t)n + 1) * sizeof(u32), st);
  if (e == cudaSuccess) e = cudaMallocAsync(&g->col, std::max<size_t>(arcs, 1) * sizeof(u32), st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(g->off, offsets, ((size_t)n + 1) * sizeof(u32), kind, st);
  if (e == cudaSuccess && arcs) e = cudaMemcpyAsync(g->col, cols, arcs * sizeof(u32), kind, st);
  if (e != cudaSuccess) {
    tkc_set_last_cuda_error(e, "graph upload", __FILE__, __LINE__);
    tkc_free_graph(g);
    return e == cudaErrorMemoryAllocation ? TKC_ENOMEM : TKC_ECUDA;
  }
  *out = g;
  return TKC_OK;
}

int tkc_load_csr(tkc_ctx *ctx, uint32_t n, uint64_t arcs, const uint32_t *offsets, const uint32_t *cols,
                 int directed, int ptr_on_device, tkc_graph **out) {
  if (!ctx || !out) return TKC_EINVAL;
  *out = nullptr;
  TKC_TRY(cudaSetDevice(ctx->device));
  tkc_graph *g = nullptr;
  TKC_RC(upload_graph(ctx, n, arcs, offsets, cols, directed, ptr_on_device, &g));
  int rc = validate_graph(g);
  if (rc == TKC_OK) {
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
      tkc_set_last_cuda_error(e, "graph upload", __FILE__, __LINE__);
      rc = TKC_ECUDA;
    }
  }
  if (rc != TKC_OK) {
    tkc_free_graph(g);
    return rc;
  }
  *out = g;
  return TKC_OK;
}

int tkc_load_csr_many(tkc_ctx *ctx, uint32_t ng, const uint32_t *n, const uint64_t *arcs,
                      const uint32_t *const *offsets, const uint32_t *const *cols, const int *directed,
                      int ptr_on_device, tkc_graph **out, uint32_t *first_bad) {
  if (!ctx || (ng && (!n || !arcs || !offsets || !cols || !directed || !out))) return TKC_EINVAL;
  if (first_bad) *first_bad = ng;
  if (ng == 0) return TKC_OK;
  TKC_TRY(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  for (u32 i = 0; i < ng; ++i) out[i] = nullptr;
  auto fail = [&](int rc, u32 bad) {
    for (u32 i = 0; i < ng; ++i) {
      tkc_free_graph(out[i]);
      out[i] = nullptr;
    }
    if (first_bad) *first_bad = bad;
    return rc;
  };
  for (u32 i = 0; i < ng; ++i) {
    const int rc = upload_graph(ctx, n[i], arcs[i], offsets[i], cols[i], directed[i], ptr_on_device, &out[i]);
    if (rc != TKC_OK) return fail(rc, i);
  }
  // every graph's checks, then one host read of all their flags; the symmetry
  // checks of the undirected ones follow (they need checked rows)
  u32 *flags = nullptr;
  std::vector<u32> hf(ng, 0);
  cudaError_t e = cudaMallocAsync(&flags, (size_t)ng * sizeof(u32), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(flags, 0, (size_t)ng * sizeof(u32), st);
  if (e != cudaSuccess) {
    tkc_set_last_cuda_error(e, "tkc_load_csr_many", __FILE__, __LINE__);
    return fail(e == cudaErrorMemoryAllocation ? TKC_ENOMEM : TKC_ECUDA, ng);
  }
  for (int pass = 0; pass < 2; ++pass) {
    bool any = false;
    for (u32 i = 0; i < ng; ++i) {
      const int rc = pass == 0 ? enqueue_validate(out[i], flags + i) : enqueue_symmetric(out[i], flags + i);
      if (rc != TKC_OK) {
        cudaFreeAsync(flags, st);
        return fail(rc, i);
      }
      any |= pass == 0 || !out[i]->directed;
    }
    if (!any) break;
    e = cudaMemcpyAsync(hf.data(), flags, (size_t)ng * sizeof(u32), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      tkc_set_last_cuda_error(e, "tkc_load_csr_many", __FILE__, __LINE__);
      cudaFreeAsync(flags, st);
      return fail(TKC_ECUDA, ng);
    }
    for (u32 i = 0; i < ng; ++i)
      if (hf[i]) {
        cudaFreeAsync(flags, st);
        return fail(TKC_EGRAPH, i);
      }
  }
  cudaFreeAsync(flags, st);
  for (u32 i = 0; i < ng; ++i)
    if (!out[i]->directed) {
      out[i]->ioff = out[i]->off;
      out[i]->icol = out[i]->col;
    }
  return TKC_OK;
}

void tkc_free_graph(tkc_graph *g) {
  if (!g) return;
  if (g->ctx->last_shard == g) g->ctx->last_shard = nullptr;
  cudaSetDevice(g->ctx->device);
  // every buffer came from the stream-ordered allocator on the context's
  // stream: freed in stream order, after the work that used it, without
  // waiting for it here
  cudaStream_t st = g->ctx->stream;
  free_search_csr(g);  // first: it orders the stream after a copy still being built from the graph
  if (g->ioff && g->ioff != g->off) cudaFreeAsync(g->ioff, st);
  if (g->icol && g->icol != g->col) cudaFreeAsync(g->icol, st);
  void *ptrs[] = {g->off, g->col, g->deg_order, g->given_order, g->alpha, g->omega, g->scc_size, g->features,
                  g->learned_order, g->seeded_order, g->nb_order, g->nb_S, g->nb_r, g->nb_key, g->nb_hkey,
                  g->nb_horder, g->comp, g->zero_ids};
  for (void *p : ptrs)
    if (p) cudaFreeAsync(p, st);
  g->ctx->graphs_alive--;
  delete g;
}

int tkc_source_order(tkc_graph *g, uint32_t *order) {
  if (!g || (!order && g->n)) return TKC_EINVAL;
  TKC_TRY(cudaSetDevice(g->ctx->device));
  TKC_RC(ensure_degree_order(g));
  if (g->n) TKC_TRY(cudaMemcpyAsync(order, g->deg_order, g->n * sizeof(u32), cudaMemcpyDeviceToHost, g->ctx->stream));
  TKC_TRY(cudaStreamSynchronize(g->ctx->stream));
  return TKC_OK;
}

int tkc_set_source_order(tkc_graph *g, const uint32_t *order) {
  if (!g || (!order && g->n)) return TKC_EINVAL;
  std::vector<uint8_t> seen(g->n, 0);
  for (u32 i = 0; i < g->n; ++i) {
    if (order[i] >= g->n || seen[order[i]]) return TKC_EINVAL;
    seen[order[i]] = 1;
  }
  TKC_TRY(cudaSetDevice(g->ctx->device));
  cudaStream_t st = g->ctx->stream;
  if (g->n == 0) return TKC_OK;
  u32 *tmp = nullptr;
  if (!g->given_order) TKC_TRY(cudaMallocAsync(&g->given_order, (size_t)g->n * sizeof(u32), st));
  TKC_TRY(cudaMallocAsync(&tmp, (size_t)g->n * sizeof(u32), st));
  TKC_TRY(cudaMemcpyAsync(tmp, order, g->n * sizeof(u32), cudaMemcpyHostToDevice, st));
  TKC_RC(filter_order(g, tmp, g->given_order, &g->n_src_given));
  TKC_TRY(cudaFreeAsync(tmp, st));
  TKC_TRY(cudaStreamSynchronize(st));
  return TKC_OK;
}

int tkc_reach_bounds(tkc_graph *g, uint32_t *alpha, uint32_t *omega) {
  if (!g || ((!alpha || !omega) && g->n)) return TKC_EINVAL;
  TKC_TRY(cudaSetDevice(g->ctx->device));
  TKC_RC(ensure_reach_bounds(g));
  cudaStream_t st = g->ctx->stream;
  if (g->n) {
    TKC_TRY(cudaMemcpyAsync(alpha, g->alpha, g->n * sizeof(u32), cudaMemcpyDeviceToHost, st));
    TKC_TRY(cudaMemcpyAsync(omega, g->omega, g->n * sizeof(u32), cudaMemcpyDeviceToHost, st));
  }
  TKC_TRY(cudaStreamSynchronize(st));
  return TKC_OK;
}

static void reset_result(tkc_result *r, u32 kk) {
  r->n_returned = kk;
  r->n_tied_at_kth = 0;
  r->edges_visited = r->edges_scanned = r->bfs_started = r->bfs_cut = r->bfs_finished = r->levels = 0;
  r->ms_pre = r->ms_bfs = r->ms_kernel = 0.0;
  r->alg_bytes = 0;
  r->batch_bits = 0;
}

static u32 nb_levels_of(const tkc_options &o) { return o.nb_levels ? o.nb_levels : 256u; }

static int source_order_of(tkc_graph *g, const tkc_options &o, u32 kk, int harmonic, const u32 **order,
                           u32 *norder, const u64 **lb_key) {
  *lb_key = nullptr;
  if (o.order == TKC_ORDER_NB) {
    TKC_RC(ensure_nb_bounds(g, nb_levels_of(o)));
    *order = harmonic ? g->nb_horder : g->nb_order;
    *norder = g->n_src_nb;
    *lb_key = harmonic ? g->nb_hkey : g->nb_key;
  } else if (o.order == TKC_ORDER_GIVEN) {
    if (!g->given_order) return TKC_EINVAL;
    *order = g->given_order;
    *norder = g->n_src_given;
  } else if (o.order == TKC_ORDER_DEG) {
    *order = g->deg_order;
    *norder = g->n_src_deg;
  } else if (o.order == TKC_ORDER_LEARNED && o.seed_factor == 0) {
    TKC_RC(ensure_learned_order(g));
    *order = g->learned_order;
    *norder = g->n_src_learned;
  } else if (o.order == TKC_ORDER_LEARNED) {
    // the model only picks the seeding prefix; the rest keeps the degree order
    TKC_RC(ensure_seeded_order(g, (u32)std::min<u64>((u64)o.seed_factor * kk, 0xffffffffull), false));
    *order = g->seeded_order;
    *norder = g->n_src_deg;
  } else if (o.order == TKC_ORDER_LEARNED_NB) {
    // the model picks the seeding prefix; the rest is the NB order with its stop
    // (still sorted by key, so the stop stays valid past the prefix)
    if (harmonic) return TKC_EINVAL;
    TKC_RC(ensure_nb_bounds(g, nb_levels_of(o)));
    TKC_RC(ensure_seeded_order(g, (u32)std::min<u64>((u64)o.seed_factor * kk, 0xffffffffull), true));
    *order = g->seeded_order;
    *norder = g->n_src_nb;
    *lb_key = g->nb_key;
  } else {
    return TKC_EINVAL;
  }
  return TKC_OK;
}

// ---------------------------------------------------------------- autotuner

static std::string graph_class(const tkc_graph *g) {
  int ln = 0;
  while (ln < 40 && (1ull << (ln + 1)) <= g->n) ++ln;
  double deg = g->n ? (double)g->arcs / g->n : 0.0;
  int ld = 0;
  while (ld < 40 && (1ull << (ld + 1)) <= (unsigned long long)(deg + 0.5)) ++ld;
  char buf[64];
  snprintf(buf, sizeof(buf), "%s_n%d_d%d", g->directed ? "dir" : "und", ln, ld);
  return buf;
}

static void tune_cache_load(tkc_ctx *ctx) {
  const char *path = getenv("TKC_TUNE_CACHE");
  if (!path) return;
  FILE *f = fopen(path, "r");
  if (!f) return;
  char line[256], key[128];
  // key=bits,teams,bu_num,bu_den,ms[,large_blocks] (files written before the
  // block size was tuned lack the last field: library choice)
  while (fgets(line, sizeof(line), f)) {
    TuneEntry e{};
    const int got = sscanf(line, " %127[^=]=%u,%u,%u,%u,%lf,%u", key, &e.batch_bits, &e.teams, &e.bu_num, &e.bu_den,
                           &e.ms, &e.large_blocks);
    if (got < 6) continue;
    if (got == 6 || e.large_blocks > 2) e.large_blocks = 0;
    ctx->tune[key] = e;
  }
  fclose(f);
}

static void tune_cache_save(tkc_ctx *ctx) {
  const char *path = getenv("TKC_TUNE_CACHE");
  if (!path) return;
  FILE *f = fopen(path, "w");
  if (!f) return;
  for (auto &kv : ctx->tune)
    fprintf(f, "%s=%u,%u,%u,%u,%.3f,%u\n", kv.first.c_str(), kv.second.batch_bits, kv.second.teams,
            kv.second.bu_num, kv.second.bu_den, kv.second.ms, kv.second.large_blocks);
  fclose(f);
}

// Sample of the degree order: its first `head` sources (they set x), then
// every stride-th of the rest.
__global__ void k_sample_order(const u32 *order, u32 norder, u32 head, u32 stride, u32 count, u32 *out) {
  for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
    out[i] = i < head ? order[i] : order[head + (u64)(i - head) * stride];
}

static int time_config(tkc_graph *g, const u32 *order, u32 norder, u32 kk, u32 bits, u32 teams, u32 bu, u32 large,
                       double *ms) {
  tkc_ctx *ctx = g->ctx;
  tkc_options saved = ctx->opt;
  ctx->opt.teams = teams;
  ctx->opt.bu_num = bu;
  ctx->opt.bu_den = 1;
  ctx->opt.large_blocks = large;
  RunSetup rs;
  memset(&rs, 0, sizeof(rs));
  rs.g = g;
  rs.order = order;
  rs.norder = norder;
  rs.B = bits;
  rs.W = words_for(bits);
  rs.kk = kk;
  rs.ng = 1;
  Ctl hc;
  int rc = run_search(ctx, rs, &hc);
  ctx->opt = saved;
  if (rc != TKC_OK) return rc;
  float t = 0;
  cudaEventElapsedTime(&t, ctx->ev[4], ctx->ev[5]);
  *ms = t;
  return TKC_OK;
}

static int topk_one(tkc_graph *g, uint32_t k, tkc_result *out, int harmonic) {
  if (!g || !out) return TKC_EINVAL;
  if (k > TKC_MAX_K) return TKC_EINVAL;
  tkc_ctx *ctx = g->ctx;
  u32 kk = std::min<u32>(k, g->n);
  if (kk > 0 && out->capacity < kk) return TKC_EINVAL;
  TKC_TRY(cudaSetDevice(ctx->device));
  tkc_result r = *out;
  reset_result(&r, kk);
  if (kk == 0) {
    *out = r;
    return TKC_OK;
  }
  cudaStream_t st = ctx->stream;
  TKC_TRY(cudaEventRecord(ctx->ev[0], st));
  const tkc_options &o = ctx->opt;
  // a labelled search's copy of the graph is built alongside the preprocessing
  if (labelled_search(o, o.batch_bits ? o.batch_bits : 64u, g->n)) TKC_RC(start_search_csr(g));
  // the degree order only where it orders the sources (the NB order has its own)
  if (o.order == TKC_ORDER_DEG || o.order == TKC_ORDER_LEARNED) TKC_RC(ensure_degree_order(g));
  TKC_RC(ensure_zero_list(g));
  TKC_RC(ensure_reach_bounds(g));
  RunSetup rs;
  memset(&rs, 0, sizeof(rs));
  TKC_RC(source_order_of(g, o, kk, harmonic, &rs.order, &rs.norder, &rs.lb_key));
  TKC_TRY(cudaEventRecord(ctx->ev[1], st));
  u32 bits = o.batch_bits ? o.batch_bits : default_batch_bits(g->n, rs.lb_key != nullptr);
  tkc_options saved = ctx->opt;
  if (!o.batch_bits) {
    auto it = ctx->tune.find(graph_class(g));
    if (it != ctx->tune.end()) {
      bits = it->second.batch_bits;
      if (!ctx->opt.teams) ctx->opt.teams = it->second.teams;
      if (!ctx->opt.bu_num) {
        ctx->opt.bu_num = it->second.bu_num;
        ctx->opt.bu_den = it->second.bu_den;
      }
      if (!ctx->opt.large_blocks) ctx->opt.large_blocks = it->second.large_blocks;
    }
  }
  rs.g = g;
  rs.B = bits;
  rs.W = words_for(bits);
  rs.nocut = 0;
  rs.harmonic = harmonic;
  rs.nocut_prefix = (u32)std::min<u64>((u64)o.seed_factor * kk, 0xffffffffull);
  rs.kk = kk;
  rs.ng = 1;
  r.batch_bits = bits;
  Ctl hc;
  int rc_run = run_search(ctx, rs, &hc);
  ctx->opt = saved;
  TKC_RC(rc_run);
  std::vector<GraphOut> go(1);
  go[0].n = g->n;
  go[0].base = 0;
  go[0].kk = kk;
  go[0].nzero = g->n_zero;
  go[0].zero_ids = g->zero_ids;
  std::vector<unsigned> ntop, tied;
  std::vector<u64> gctr;
  TKC_RC(finish_run(ctx, rs, go, &r, ntop, tied, gctr));
  TKC_TRY(cudaEventRecord(ctx->ev[2], st));
  TKC_TRY(cudaStreamSynchronize(st));
  r.n_tied_at_kth = tied[0];
  r.edges_visited = hc.edges_visited;
  r.edges_scanned = hc.edges_scanned;
  r.bfs_started = hc.bfs_started;
  r.bfs_cut = hc.bfs_cut;
  r.bfs_finished = hc.bfs_finished;
  r.levels = hc.levels;
  r.alg_bytes = hc.alg_bytes;
  float ms0 = 0, ms1 = 0, ms2 = 0;
  cudaEventElapsedTime(&ms0, ctx->ev[0], ctx->ev[1]);
  cudaEventElapsedTime(&ms1, ctx->ev[1], ctx->ev[2]);
  cudaEventElapsedTime(&ms2, ctx->ev[4], ctx->ev[5]);
  r.ms_pre = ms0;
  r.ms_bfs = ms1;
  r.ms_kernel = ms2;
  *out = r;
  return TKC_OK;
}

// The positions first, first + nshards, ... of a source order (count of them).
__global__ void k_shard_order(const u32 *order, u32 first, u32 nshards, u32 count, u32 *out) {
  for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
    out[i] = order[first + (u64)i * nshards];
}

// Finished searches of the latest run whose farness equals S/(r-1)^2 exactly.
__global__ void k_count_key(const u64 *res_S, const u32 *res_r, u32 n, u64 S, u32 r, unsigned *cnt) {
  unsigned c = 0;
  for (u32 v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const u32 rv = res_r[v];
    if (rv < 2) continue;
    const unsigned __int128 a = (unsigned __int128)res_S[v] * (unsigned __int128)((u64)(r - 1) * (u64)(r - 1));
    const unsigned __int128 b = (unsigned __int128)S * (unsigned __int128)((u64)(rv - 1) * (u64)(rv - 1));
    c += a == b;
  }
  c = __reduce_add_sync(0xffffffffu, c);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(cnt, c);
}

static bool entry_before(u64 Sa, u32 ra, u32 ia, u64 Sb, u32 rb, u32 ib) {
  const unsigned __int128 l = (unsigned __int128)Sa * (unsigned __int128)((u64)(rb - 1) * (u64)(rb - 1));
  const unsigned __int128 h = (unsigned __int128)Sb * (unsigned __int128)((u64)(ra - 1) * (u64)(ra - 1));
  return l != h ? l < h : ia < ib;
}

// Algorithm 1 over one shard of the source order (see tkc_topk_closeness_shard).
static int topk_shard(tkc_graph *g, uint32_t k, uint32_t first, uint32_t shard, uint32_t nshards, uint32_t limit,
                      const uint64_t *seed_S, const uint32_t *seed_r, const uint32_t *seed_id, uint32_t nseed,
                      tkc_result *out) {
  if (!g || !out || nshards == 0 || shard >= nshards || k > TKC_MAX_K) return TKC_EINVAL;
  if (nseed && (!seed_S || !seed_r || !seed_id)) return TKC_EINVAL;
  tkc_ctx *ctx = g->ctx;
  const tkc_options &o = ctx->opt;
  if (o.order != TKC_ORDER_DEG && o.order != TKC_ORDER_NB) return TKC_EINVAL;
  const u32 kk = std::min<u32>(k, g->n);
  if (kk > 0 && out->capacity < kk) return TKC_EINVAL;
  if (nseed > kk) return TKC_EINVAL;
  for (u32 i = 0; i < nseed; ++i) {
    if (seed_id[i] >= g->n || seed_r[i] < 2 || seed_r[i] > g->n) return TKC_EINVAL;
    if (i && !entry_before(seed_S[i - 1], seed_r[i - 1], seed_id[i - 1], seed_S[i], seed_r[i], seed_id[i]))
      return TKC_EINVAL;  // best first, no repeats
  }
  TKC_TRY(cudaSetDevice(ctx->device));
  tkc_result r = *out;
  reset_result(&r, kk);
  if (kk == 0) {
    *out = r;
    return TKC_OK;
  }
  cudaStream_t st = ctx->stream;
  TKC_TRY(cudaEventRecord(ctx->ev[0], st));
  TKC_RC(ensure_degree_order(g));
  TKC_RC(ensure_reach_bounds(g));
  RunSetup rs;
  memset(&rs, 0, sizeof(rs));
  const u32 *full = nullptr;
  u32 nfull = 0;
  TKC_RC(source_order_of(g, o, kk, 0, &full, &nfull, &rs.lb_key));
  const u64 start = (u64)first + shard;
  u32 count = nfull > start ? (u32)((nfull - start + nshards - 1) / nshards) : 0;
  if (limit && count > limit) count = limit;
  u32 *sorder = nullptr;
  TKC_TRY(cudaMallocAsync(&sorder, std::max<size_t>(count, 1) * sizeof(u32), st));
  if (count)
    TKC_LAUNCH(k_shard_order<<<(count + 255) / 256 < 4096 ? (count + 255) / 256 : 4096, 256, 0, st>>>(
        full, (u32)start, nshards, count, sorder));
  TKC_TRY(cudaEventRecord(ctx->ev[1], st));
  const u32 bits = o.batch_bits ? o.batch_bits : default_batch_bits(g->n, rs.lb_key != nullptr);
  rs.g = g;
  rs.order = sorder;
  rs.norder = count;
  rs.B = bits;
  rs.W = words_for(bits);
  rs.kk = kk;
  rs.ng = 1;
  rs.seed_S = reinterpret_cast<const u64 *>(seed_S);
  rs.seed_r = seed_r;
  rs.seed_id = seed_id;
  rs.nseed = nseed;
  r.batch_bits = bits;
  Ctl hc;
  memset(&hc, 0, sizeof(hc));
  const int rc_run = run_search(ctx, rs, &hc);  // also with no source: the list is the seed
  TKC_TRY(cudaFreeAsync(sorder, st));
  TKC_RC(rc_run);
  std::vector<GraphOut> go(1);
  go[0].n = g->n;
  go[0].base = 0;
  go[0].kk = kk;
  go[0].nzero = g->n - g->n_src_deg;
  go[0].zero_ids = g->deg_order + g->n_src_deg;
  std::vector<unsigned> ntop, tied;
  std::vector<u64> gctr;
  TKC_RC(finish_run(ctx, rs, go, &r, ntop, tied, gctr));
  TKC_TRY(cudaEventRecord(ctx->ev[2], st));
  TKC_TRY(cudaStreamSynchronize(st));
  r.n_tied_at_kth = tied[0];
  r.edges_visited = hc.edges_visited;
  r.edges_scanned = hc.edges_scanned;
  r.bfs_started = hc.bfs_started;
  r.bfs_cut = hc.bfs_cut;
  r.bfs_finished = hc.bfs_finished;
  r.levels = hc.levels;
  r.alg_bytes = hc.alg_bytes;
  float ms0 = 0, ms1 = 0;
  cudaEventElapsedTime(&ms0, ctx->ev[0], ctx->ev[1]);
  cudaEventElapsedTime(&ms1, ctx->ev[1], ctx->ev[2]);
  r.ms_pre = ms0;
  r.ms_bfs = ms1;
  float ms2 = 0;
  cudaEventElapsedTime(&ms2, ctx->ev[4], ctx->ev[5]);
  r.ms_kernel = ms2;
  ctx->last_shard = g;
  *out = r;
  return TKC_OK;
}

int tkc_autotune(tkc_graph *g, uint32_t k, tkc_options *best) {
  if (!g || !best) return TKC_EINVAL;
  if (k > TKC_MAX_K) return TKC_EINVAL;
  tkc_ctx *ctx = g->ctx;
  TKC_TRY(cudaSetDevice(ctx->device));
  *best = ctx->opt;
  u32 kk = std::min<u32>(k, g->n);
  if (kk == 0) return TKC_OK;
  TKC_RC(ensure_degree_order(g));
  TKC_RC(ensure_reach_bounds(g));
  cudaStream_t st = ctx->stream;
  const u32 ns = g->n_src_deg;
  const u32 head = std::min<u32>(ns, 1024);
  const u32 want = std::max<u32>(ns / 10, std::min<u32>(ns, 32768));
  const u32 stride = std::max<u32>(1, (ns - head) / std::max<u32>(1, want - head));
  const u32 count = head + (ns > head ? (ns - head + stride - 1) / stride : 0);
  u32 *order = nullptr;
  TKC_TRY(cudaMallocAsync(&order, std::max<u32>(count, 1) * sizeof(u32), st));
  TKC_LAUNCH(k_sample_order<<<(count + 255) / 256 > 0 ? std::min<u32>((count + 255) / 256, 4096) : 1, 256, 0, st>>>(
      g->deg_order, ns, head, stride, count, order));
  TKC_TRY(cudaGetLastError());
  const u32 bits_c[] = {64, 128, 256, 512};
  const int maxb_t = std::max(1, max_coresident_blocks(ctx, 1));
  const u32 teams_c[] = {1, 4, (u32)std::max(1, maxb_t / 16), (u32)std::max(1, maxb_t / 8),
                         (u32)std::max(1, maxb_t / 4)};
  double best_ms = 1e300;
  u32 bb = default_batch_bits(g->n), bt = 1, bu = 8, bl = 0;
  int rc = TKC_OK;
  for (u32 b : bits_c)
    for (u32 t : teams_c) {
      double ms = 0;
      rc = time_config(g, order, count, kk, b, t, 8, 0, &ms);
      if (rc != TKC_OK) break;
      if (ms < best_ms) {
        best_ms = ms;
        bb = b;
        bt = t;
      }
    }
  for (u32 u : {4u, 16u, 32u}) {
    if (rc != TKC_OK) break;
    double ms = 0;
    rc = time_config(g, order, count, kk, bb, bt, u, 0, &ms);
    if (rc == TKC_OK && ms < best_ms) {
      best_ms = ms;
      bu = u;
    }
  }
  // block shape: the larger blocks of 64- and 128-bit batches and 512 threads,
  // each against the library's choice by graph size timed above
  for (u32 l : {1u, 2u}) {
    if (rc != TKC_OK || words_for(bb) > 2) break;
    double ms = 0;
    rc = time_config(g, order, count, kk, bb, bt, bu, l, &ms);
    if (rc == TKC_OK && ms < best_ms) {
      best_ms = ms;
      bl = l;
    }
  }
  cudaFreeAsync(order, st);
  cudaStreamSynchronize(st);
  if (rc != TKC_OK) return rc;
  TuneEntry e{bb, bt, bu, 1, best_ms, bl};
  ctx->tune[graph_class(g)] = e;
  tune_cache_save(ctx);
  best->batch_bits = bb;
  best->teams = bt;
  best->bu_num = bu;
  best->bu_den = 1;
  best->large_blocks = bl;
  return TKC_OK;
}

int tkc_distance_sums(tkc_graph *g, uint32_t nsrc, const uint32_t *srcs, uint64_t *S, uint32_t *r) {
  if (!g || (nsrc && (!srcs || !S || !r))) return TKC_EINVAL;
  if (nsrc == 0) return TKC_OK;
  tkc_ctx *ctx = g->ctx;
  TKC_TRY(cudaSetDevice(ctx->device));
  for (u32 i = 0; i < nsrc; ++i)
    if (srcs[i] >= g->n) return TKC_EINVAL;
  std::vector<u32> uniq(srcs, srcs + nsrc);
  std::sort(uniq.begin(), uniq.end());
  uniq.erase(std::unique(uniq.begin(), uniq.end()), uniq.end());
  TKC_RC(ensure_degree_order(g));
  TKC_RC(ensure_reach_bounds(g));
  cudaStream_t st = ctx->stream;
  u32 *dsrc = nullptr;
  TKC_TRY(cudaMallocAsync(&dsrc, uniq.size() * sizeof(u32), st));
  TKC_TRY(cudaMemcpyAsync(dsrc, uniq.data(), uniq.size() * sizeof(u32), cudaMemcpyHostToDevice, st));
  RunSetup rs;
  memset(&rs, 0, sizeof(rs));
  rs.g = g;
  rs.order = dsrc;
  rs.norder = (u32)uniq.size();
  rs.B = 64;
  rs.W = 1;
  rs.nocut = 1;
  rs.kk = 1;
  rs.ng = 1;
  Ctl hc;
  int rc = run_search(ctx, rs, &hc);
  std::vector<u64> allS;
  std::vector<u32> allr;
  if (rc == TKC_OK) {
    allS.resize(g->n);
    allr.resize(g->n);
    cudaError_t e = cudaMemcpyAsync(allS.data(), ctx->ws.res_S, g->n * sizeof(u64), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(allr.data(), ctx->ws.res_r, g->n * sizeof(u32), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      tkc_set_last_cuda_error(e, "distance sums readback", __FILE__, __LINE__);
      rc = TKC_ECUDA;
    }
  }
  cudaFreeAsync(dsrc, st);
  cudaStreamSynchronize(st);
  if (rc != TKC_OK) return rc;
  for (u32 i = 0; i < nsrc; ++i) {
    S[i] = allS[srcs[i]];
    r[i] = allr[srcs[i]];
  }
  return TKC_OK;
}

// Algorithm 1 with updateBoundsLB (DegBound with the degree order, NBBound
// with options.order = TKC_ORDER_NB): rounds of up to B complete searches from
// the unsearched vertices of smallest bound, each round raising the bounds of
// the vertices whose reach equals a searched source's.
static int topk_bound(tkc_graph *g, uint32_t k, tkc_result *out) {
  if (!g || !out) return TKC_EINVAL;
  if (k > TKC_MAX_K) return TKC_EINVAL;
  tkc_ctx *ctx = g->ctx;
  const tkc_options &o = ctx->opt;
  if (o.order != TKC_ORDER_DEG && o.order != TKC_ORDER_NB) return TKC_EINVAL;
  u32 kk = std::min<u32>(k, g->n);
  if (kk > 0 && out->capacity < kk) return TKC_EINVAL;
  TKC_TRY(cudaSetDevice(ctx->device));
  tkc_result r = *out;
  reset_result(&r, kk);
  if (kk == 0) {
    *out = r;
    return TKC_OK;
  }
  cudaStream_t st = ctx->stream;
  const u32 n = g->n;
  TKC_TRY(cudaEventRecord(ctx->ev[0], st));
  TKC_RC(ensure_degree_order(g));
  TKC_RC(ensure_reach_bounds(g));
  const bool nb = o.order == TKC_ORDER_NB;
  if (nb) TKC_RC(ensure_nb_bounds(g, nb_levels_of(o)));
  const u32 *order0 = nb ? g->nb_order : g->deg_order;
  const u32 n0 = nb ? g->n_src_nb : g->n_src_deg;
  // defaults measured with NBBound on a 1000 x 1000 grid: 256 sources x 1 team 4.55 s, 256 x 2 4.16 s,
  // 128 x 4 4.03 s, 64 x 8 3.48 s, 64 x 16 3.99 s (more sources per round refresh the bounds less often)
  const bool large = n >= (1u << 16);
  const u32 B = o.batch_bits ? o.batch_bits : (large ? 64u : 256u);
  const u32 cap = std::min<u32>(n + 1, 65535u);  // levels per search (depth < n)
  // teams run one batch each per round (0: one team below 2^16 vertices, else 8)
  int maxb = max_coresident_blocks(ctx, words_for(B));
  if (maxb <= 0) return TKC_ECUDA;
  const u32 T = std::max<u32>(1, std::min<u32>(B <= 1 ? 1u : (o.teams ? o.teams : (large ? 8u : 1u)), (u32)maxb));
  const u32 TB = T * B;  // sources per round
  TKC_RC(ensure_workspace(ctx, n, words_for(B), kk, 1, T));
  u64 *bS = nullptr, *key = nullptr, *Ltab = nullptr, *smax = nullptr, *bkeys = nullptr;
  u32 *bR = nullptr, *cand = nullptr, *pos = nullptr, *tmp = nullptr, *lo = nullptr, *hist = nullptr, *depth = nullptr;
  u32 *srcs = nullptr;
  uint8_t *done = nullptr;
  uint16_t *lvl = nullptr;
  int rc = TKC_OK;
  auto cleanup = [&]() {
    void *ptrs[] = {bS, key, Ltab, smax, bkeys, bR, cand, pos, tmp, lo, hist, depth, done, lvl, srcs};
    for (void *q : ptrs)
      if (q) cudaFreeAsync(q, st);
    cudaStreamSynchronize(st);
  };
#define LB_TRY(expr)                                                  \
  do {                                                                \
    cudaError_t e_ = (expr);                                          \
    if (e_ != cudaSuccess) {                                          \
      tkc_set_last_cuda_error(e_, #expr, __FILE__, __LINE__);         \
      cleanup();                                                      \
      return e_ == cudaErrorMemoryAllocation ? TKC_ENOMEM : TKC_ECUDA; \
    }                                                                 \
  } while (0)
#define LB_RC(expr)     \
  do {                  \
    rc = (expr);        \
    if (rc != TKC_OK) { \
      cleanup();        \
      return rc;        \
    }                   \
  } while (0)
  const size_t n1 = std::max<size_t>(n, 1);
  LB_TRY(cudaMallocAsync(&bS, n1 * sizeof(u64), st));
  LB_TRY(cudaMallocAsync(&key, n1 * sizeof(u64), st));
  LB_TRY(cudaMallocAsync(&bR, n1 * sizeof(u32), st));
  LB_TRY(cudaMallocAsync(&done, n1, st));
  LB_TRY(cudaMallocAsync(&cand, n1 * sizeof(u32), st));
  LB_TRY(cudaMallocAsync(&pos, (n1 + 1) * sizeof(u32), st));
  LB_TRY(cudaMallocAsync(&tmp, ((n1 + 1) / 4096 + 16) * sizeof(u32), st));
  LB_TRY(cudaMallocAsync(&lo, n1 * sizeof(u32), st));
  LB_TRY(cudaMallocAsync(&smax, sizeof(u64), st));
  LB_TRY(cudaMallocAsync(&hist, (size_t)TB * cap * sizeof(u32), st));
  LB_TRY(cudaMallocAsync(&Ltab, (size_t)TB * cap * sizeof(u64), st));
  LB_TRY(cudaMallocAsync(&depth, (size_t)TB * sizeof(u32), st));
  LB_TRY(cudaMallocAsync(&bkeys, (size_t)TB * sizeof(u64), st));
  LB_TRY(cudaMallocAsync(&srcs, (size_t)TB * sizeof(u32), st));
  LB_TRY(cudaMallocAsync(&lvl, n1 * TB * sizeof(uint16_t), st));
  LB_TRY(cudaMemsetAsync(lvl, 0xff, n1 * TB * sizeof(uint16_t), st));
  LB_RC(lb_init(g, nb ? g->nb_S : nullptr, nb ? g->nb_r : nullptr, nb ? g->nb_key : nullptr, bS, bR, key, done));
  TKC_TRY(cudaEventRecord(ctx->ev[1], st));
  Ctl total;
  memset(&total, 0, sizeof(total));
  double ms_kernel = 0;
  u32 nround = 0;
  std::vector<u64> h_key(TB);
  while (true) {
    u32 m = 0;
    LB_RC(lb_sorted_candidates(g, order0, n0, done, key, cand, &m, pos, tmp, lo, smax));
    if (m == 0) break;
    const u32 take = std::min<u32>(TB, m);
    // the batch's keys and the current k-th entry decide the stop
    LB_RC(lb_gather_keys(g, take, cand, key, bkeys));
    LB_TRY(cudaMemcpyAsync(h_key.data(), bkeys, take * sizeof(u64), cudaMemcpyDeviceToHost, st));
    unsigned ntop = 0;
    u64 xS = 0;
    u32 xr = 0;
    Workspace &w = ctx->ws;
    if (nround > 0) {
      LB_TRY(cudaMemcpyAsync(&ntop, w.g_ntop, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
      LB_TRY(cudaMemcpyAsync(&xS, w.top_S + kk - 1, sizeof(u64), cudaMemcpyDeviceToHost, st));
      LB_TRY(cudaMemcpyAsync(&xr, w.top_r + kk - 1, sizeof(u32), cudaMemcpyDeviceToHost, st));
    }
    LB_TRY(cudaStreamSynchronize(st));
    // Algorithm 1: stop at the first candidate whose key exceeds x strictly
    u32 cnt = take;
    if (ntop == kk) {
      for (u32 i = 0; i < take; ++i) {
        const unsigned __int128 lhs = (unsigned __int128)h_key[i] * ((u64)(xr - 1) * (u64)(xr - 1));
        if (lhs > ((unsigned __int128)xS << 46)) {
          cnt = i;
          break;
        }
      }
    }
    if (cnt == 0) break;
    LB_TRY(cudaMemsetAsync(hist, 0, (size_t)TB * cap * sizeof(u32), st));
    LB_TRY(cudaMemsetAsync(srcs, 0xff, (size_t)TB * sizeof(u32), st));
    RunSetup rs;
    memset(&rs, 0, sizeof(rs));
    rs.g = g;
    rs.order = cand;
    rs.norder = cnt;
    rs.B = B;
    rs.W = words_for(B);
    rs.nocut = 1;
    rs.kk = kk;
    rs.ng = 1;
    rs.lvl = lvl;
    rs.hist = hist;
    rs.lvl_src = srcs;
    rs.hist_cap = cap;
    rs.lvl_stride = TB;
    rs.keep_lists = nround > 0;
    rs.force_teams = T;
    Ctl hc;
    LB_RC(run_search(ctx, rs, &hc));
    float ms = 0;
    LB_TRY(cudaEventSynchronize(ctx->ev[5]));
    LB_TRY(cudaEventElapsedTime(&ms, ctx->ev[4], ctx->ev[5]));
    ms_kernel += ms;
    total.edges_visited += hc.edges_visited;
    total.edges_scanned += hc.edges_scanned;
    total.bfs_started += hc.bfs_started;
    total.bfs_finished += hc.bfs_finished;
    total.levels += hc.levels;
    total.alg_bytes += hc.alg_bytes;
    LB_RC(lb_update(g, TB, TB, srcs, lvl, hist, cap, depth, Ltab, w.res_r, bS, bR, key, done));
    ++nround;
  }
  RunSetup rs;
  memset(&rs, 0, sizeof(rs));
  rs.g = g;
  rs.kk = kk;
  rs.ng = 1;
  r.batch_bits = B;
  if (nround == 0) {
    // nothing searched (no vertex reaches another): the list is empty
    LB_TRY(cudaMemsetAsync(ctx->ws.g_ntop, 0, sizeof(unsigned), st));
    LB_TRY(cudaMemsetAsync(ctx->ws.res_r, 0, n1 * sizeof(u32), st));
  }
  std::vector<GraphOut> go(1);
  go[0].n = n;
  go[0].base = 0;
  go[0].kk = kk;
  go[0].nzero = n - g->n_src_deg;
  go[0].zero_ids = g->deg_order + g->n_src_deg;
  std::vector<unsigned> ntop, tied;
  std::vector<u64> gctr;
  LB_RC(finish_run(ctx, rs, go, &r, ntop, tied, gctr));
  LB_TRY(cudaEventRecord(ctx->ev[2], st));
  LB_TRY(cudaStreamSynchronize(st));
  cleanup();
#undef LB_TRY
#undef LB_RC
  r.n_tied_at_kth = tied[0];
  r.edges_visited = total.edges_visited;
  r.edges_scanned = total.edges_scanned;
  r.bfs_started = total.bfs_started;
  r.bfs_cut = 0;
  r.bfs_finished = total.bfs_finished;
  r.levels = total.levels;
  r.alg_bytes = total.alg_bytes;
  float ms0 = 0, ms1 = 0;
  cudaEventElapsedTime(&ms0, ctx->ev[0], ctx->ev[1]);
  cudaEventElapsedTime(&ms1, ctx->ev[1], ctx->ev[2]);
  r.ms_pre = ms0;
  r.ms_bfs = ms1;
  r.ms_kernel = ms_kernel;
  *out = r;
  return TKC_OK;
}

static int topk_many(tkc_ctx *ctx, tkc_graph *const *gs, uint32_t ng, uint32_t k, tkc_result *outs, int harmonic) {
  if (!ctx || (ng && (!gs || !outs))) return TKC_EINVAL;
  if (k > TKC_MAX_K) return TKC_EINVAL;
  if (ng == 0) return TKC_OK;
  TKC_TRY(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  const tkc_options &o = ctx->opt;
  // the union is searched in degree order, or in NBCut order (each graph stops on its own)
  if (o.order != TKC_ORDER_DEG && o.order != TKC_ORDER_NB) return TKC_EINVAL;
  const bool nb = o.order == TKC_ORDER_NB;
  u64 nv64 = 0, na = 0;
  u32 maxn = 0;
  for (u32 i = 0; i < ng; ++i) {
    if (!gs[i] || gs[i]->ctx != ctx) return TKC_EINVAL;
    u32 kg = std::min<u32>(k, gs[i]->n);
    if (kg > 0 && outs[i].capacity < kg) return TKC_EINVAL;
    nv64 += gs[i]->n;
    na += gs[i]->arcs;
    maxn = std::max(maxn, gs[i]->n);
  }
  if (nv64 >= kMaxN || na >= (1ull << 32)) return TKC_EOVERFLOW;
  const u32 nv = (u32)nv64;
  const u32 kk = std::min<u32>(k, maxn);
  for (u32 i = 0; i < ng; ++i) reset_result(&outs[i], std::min<u32>(k, gs[i]->n));
  if (kk == 0) return TKC_OK;
  TKC_TRY(cudaEventRecord(ctx->ev[0], st));
  // per-graph preprocessing (cached in each graph), then the union
  std::vector<u32> vbase(ng + 1, 0);
  std::vector<u64> abase(ng + 1, 0), offptr(ng), colptr(ng);
  std::vector<uint8_t> gdir(ng);
  for (u32 i = 0; i < ng; ++i) {
    vbase[i + 1] = vbase[i] + gs[i]->n;
    abase[i + 1] = abase[i] + gs[i]->arcs;
    offptr[i] = (u64)gs[i]->off;
    colptr[i] = (u64)gs[i]->col;
    gdir[i] = (uint8_t)gs[i]->directed;
  }
  tkc_graph U;
  U.ctx = ctx;
  U.n = nv;
  U.arcs = na;
  U.directed = 1;
  u32 *gid = nullptr, *d_vbase = nullptr;
  u32 *zflag = nullptr, *zlist = nullptr, *zat = nullptr;  // out-degree-0 vertices of every graph
  u32 *gorder = nullptr, *gkey = nullptr, *gend = nullptr;  // the order graph by graph
  u64 *d_abase = nullptr, *d_offptr = nullptr, *d_colptr = nullptr;
  uint8_t *d_gdir = nullptr;
  int rc = TKC_OK;
  auto cleanup = [&]() {
    cudaStreamSynchronize(st);
    free_search_csr(&U);
    void *ptrs[] = {U.off, U.col, U.ioff, U.icol, U.deg_order, U.alpha, U.omega, U.scc_size, U.comp, U.nb_S, U.nb_r,
                    U.nb_key, U.nb_hkey,
                    U.nb_order, U.nb_horder, gid, d_vbase, d_abase, d_offptr, d_colptr, d_gdir, zflag, zlist,
                    zat, gorder, gkey, gend};
    for (void *q : ptrs)
      if (q) cudaFree(q);
  };
#define MULTI_TRY(expr)                                              \
  do {                                                               \
    cudaError_t e_ = (expr);                                         \
    if (e_ != cudaSuccess) {                                         \
      tkc_set_last_cuda_error(e_, #expr, __FILE__, __LINE__);        \
      cleanup();                                                     \
      return e_ == cudaErrorMemoryAllocation ? TKC_ENOMEM : TKC_ECUDA; \
    }                                                                \
  } while (0)
#define MULTI_RC(expr)  \
  do {                  \
    rc = (expr);        \
    if (rc != TKC_OK) { \
      cleanup();        \
      return rc;        \
    }                   \
  } while (0)
  MULTI_TRY(cudaMallocAsync(&U.off, ((size_t)nv + 1) * sizeof(u32), st));
  MULTI_TRY(cudaMallocAsync(&U.col, std::max<size_t>(na, 1) * sizeof(u32), st));
  MULTI_TRY(cudaMallocAsync(&gid, std::max<size_t>(nv, 1) * sizeof(u32), st));
  MULTI_TRY(cudaMallocAsync(&d_vbase, (ng + 1) * sizeof(u32), st));
  MULTI_TRY(cudaMallocAsync(&d_abase, (ng + 1) * sizeof(u64), st));
  MULTI_TRY(cudaMallocAsync(&d_offptr, ng * sizeof(u64), st));
  MULTI_TRY(cudaMallocAsync(&d_colptr, ng * sizeof(u64), st));
  MULTI_TRY(cudaMallocAsync(&d_gdir, ng, st));
  MULTI_TRY(cudaMemcpyAsync(d_vbase, vbase.data(), (ng + 1) * sizeof(u32), cudaMemcpyHostToDevice, st));
  MULTI_TRY(cudaMemcpyAsync(d_abase, abase.data(), (ng + 1) * sizeof(u64), cudaMemcpyHostToDevice, st));
  MULTI_TRY(cudaMemcpyAsync(d_offptr, offptr.data(), ng * sizeof(u64), cudaMemcpyHostToDevice, st));
  MULTI_TRY(cudaMemcpyAsync(d_colptr, colptr.data(), ng * sizeof(u64), cudaMemcpyHostToDevice, st));
  MULTI_TRY(cudaMemcpyAsync(d_gdir, gdir.data(), ng, cudaMemcpyHostToDevice, st));
  unsigned gb = (unsigned)std::max<u64>(1, std::min<u64>((nv + 256) / 256, (u64)ctx->num_sms * 16));
  TKC_LAUNCH(k_union_offsets<<<gb, 256, 0, st>>>(d_offptr, d_vbase, d_abase, ng, nv, U.off, gid));
  unsigned ga = (unsigned)std::max<u64>(1, std::min<u64>((na + 255) / 256, (u64)ctx->num_sms * 16));
  if (na) TKC_LAUNCH(k_union_cols<<<ga, 256, 0, st>>>(d_colptr, d_vbase, d_abase, ng, na, U.col));
  MULTI_TRY(cudaGetLastError());
  // each graph's vertices of out-degree 0 in id order (they fill a list that
  // fewer than k vertices with reach reach), from one pass over the union:
  // graph g's run starts at zflag's scan at vbase[g]
  std::vector<u32> zpos(ng + 1);
  {
    u32 *ztmp = nullptr;
    MULTI_TRY(cudaMallocAsync(&zflag, ((size_t)nv + 1) * sizeof(u32), st));
    MULTI_TRY(cudaMallocAsync(&zlist, std::max<size_t>(nv, 1) * sizeof(u32), st));
    MULTI_TRY(cudaMallocAsync(&zat, ((size_t)ng + 1) * sizeof(u32), st));
    MULTI_TRY(cudaMallocAsync(&ztmp, (((size_t)nv + 1) / 4096 + 2) * sizeof(u32), st));
    TKC_LAUNCH(k_zero_flags<<<gb, 256, 0, st>>>(U.off, nv, zflag));
    MULTI_RC(scan_exclusive_u32(zflag, zflag, (u64)nv + 1, ztmp, st));
    TKC_LAUNCH(k_zero_compact<<<gb, 256, 0, st>>>(U.off, zflag, gid, d_vbase, nv, zlist));
    TKC_LAUNCH(k_gather_u32<<<1, 256, 0, st>>>(zflag, d_vbase, ng + 1, zat));
    MULTI_TRY(cudaGetLastError());
    MULTI_TRY(cudaMemcpyAsync(zpos.data(), zat, ((size_t)ng + 1) * sizeof(u32), cudaMemcpyDeviceToHost, st));
    MULTI_TRY(cudaFreeAsync(ztmp, st));
  }
  MULTI_RC(build_in_csr(&U));
  // reach bounds once over the union, as a directed graph: the SCCs of the
  // union are the graphs' SCCs (an undirected graph's are its components, each
  // with alpha = omega = its size); only the biggest SCC of the union gets the
  // exact reach by BFS, so the other graphs' omega may be looser than alone,
  // which changes pruning, never results
  MULTI_RC(ensure_reach_bounds(&U, gid, ng));
  if (nb) {
    // the sweeps run once over the union (each vertex's counts involve only its
    // own graph, so they equal the per-graph values); all sources of all graphs
    // are then ordered by (key, union id)
    MULTI_RC(ensure_nb_bounds(&U, nb_levels_of(o), gid, d_gdir));
  } else {
    MULTI_RC(ensure_degree_order(&U));
  }
  TKC_TRY(cudaEventRecord(ctx->ev[1], st));
  RunSetup rs;
  memset(&rs, 0, sizeof(rs));
  u32 bits = o.batch_bits ? o.batch_bits : default_batch_bits(nv);
  rs.g = &U;
  rs.order = nb ? (harmonic ? U.nb_horder : U.nb_order) : U.deg_order;
  rs.norder = nb ? U.n_src_nb : U.n_src_deg;
  rs.lb_key = nb ? (harmonic ? U.nb_hkey : U.nb_key) : nullptr;
  rs.B = bits;
  rs.W = words_for(bits);
  rs.nocut = 0;
  rs.harmonic = harmonic;
  rs.kk = kk;
  rs.ng = ng;
  rs.gid = gid;
  rs.g_directed = d_gdir;
  rs.size_n = maxn;
  // The sources graph by graph, each graph's in its own order: first the
  // first B sources of every graph (one opening batch per graph, searched
  // before the graph has a threshold), then the rest of every graph, graph by
  // graph (stable sorts by (phase, graph)).  A batch of the second part holds
  // searches of one graph, which share its frontier rows and arcs and cut
  // against the threshold its opening batch set; a graph's NB stop there moves
  // the shared cursor past the rest of its run.  Each graph still sees its
  // sources in the order it would alone, and its threshold depends only on its
  // own searches.
  if (rs.norder > 0 && ng > 1) {
    u32 *gbeg = nullptr, *p1 = nullptr;
    MULTI_TRY(cudaMallocAsync(&gorder, (size_t)rs.norder * sizeof(u32), st));
    MULTI_TRY(cudaMallocAsync(&gkey, (size_t)rs.norder * sizeof(u32), st));
    MULTI_TRY(cudaMallocAsync(&gend, (size_t)2 * ng * sizeof(u32), st));
    MULTI_TRY(cudaMallocAsync(&gbeg, (size_t)ng * sizeof(u32), st));
    MULTI_TRY(cudaMallocAsync(&p1, sizeof(u32), st));
    MULTI_TRY(cudaMemsetAsync(gend, 0, (size_t)2 * ng * sizeof(u32), st));
    MULTI_TRY(cudaMemcpyAsync(gorder, rs.order, (size_t)rs.norder * sizeof(u32), cudaMemcpyDeviceToDevice, st));
    MULTI_TRY(cudaMemcpyAsync(p1, &rs.norder, sizeof(u32), cudaMemcpyHostToDevice, st));
    const unsigned go_grid = (unsigned)std::max<u64>(1, std::min<u64>((rs.norder + 255) / 256, (u64)ctx->num_sms * 16));
    TKC_LAUNCH(k_order_gid<<<go_grid, 256, 0, st>>>(rs.order, rs.norder, gid, gkey));
    int gbits = 0;
    while (gbits < 32 && ((2 * ng - 1) >> gbits) != 0) ++gbits;
    MULTI_RC(radix_sort_u32_pairs(gkey, gorder, rs.norder, gbits, st));  // by graph
    TKC_LAUNCH(k_segment_bounds<<<go_grid, 256, 0, st>>>(gkey, rs.norder, gbeg, nullptr));
    TKC_LAUNCH(k_phase_keys<<<go_grid, 256, 0, st>>>(gkey, rs.norder, gbeg, rs.B, ng));
    MULTI_RC(radix_sort_u32_pairs(gkey, gorder, rs.norder, gbits, st));  // openings first
    TKC_LAUNCH(k_segment_bounds<<<go_grid, 256, 0, st>>>(gkey, rs.norder, nullptr, gend));
    TKC_LAUNCH(k_phase_start<<<go_grid, 256, 0, st>>>(gkey, rs.norder, ng, p1));
    MULTI_TRY(cudaGetLastError());
    MULTI_TRY(cudaMemcpyAsync(&rs.g_rest, p1, sizeof(u32), cudaMemcpyDeviceToHost, st));
    MULTI_TRY(cudaStreamSynchronize(st));
    MULTI_TRY(cudaFreeAsync(gbeg, st));
    MULTI_TRY(cudaFreeAsync(p1, st));
    rs.order = gorder;
    rs.g_end = gend + ng;  // ends of the graphs' runs after their openings
  }
  Ctl hc;
  MULTI_RC(run_search(ctx, rs, &hc));
  std::vector<GraphOut> go(ng);
  for (u32 i = 0; i < ng; ++i) {
    go[i].n = gs[i]->n;
    go[i].base = vbase[i];
    go[i].kk = std::min<u32>(k, gs[i]->n);
    go[i].nzero = zpos[i + 1] - zpos[i];
    go[i].zero_ids = zlist + zpos[i];
  }
  std::vector<unsigned> ntop, tied;
  std::vector<u64> gctr;
  MULTI_RC(finish_run(ctx, rs, go, outs, ntop, tied, gctr));
  MULTI_TRY(cudaEventRecord(ctx->ev[2], st));
  MULTI_TRY(cudaStreamSynchronize(st));
  float ms0 = 0, ms1 = 0, ms2 = 0;
  cudaEventElapsedTime(&ms0, ctx->ev[0], ctx->ev[1]);
  cudaEventElapsedTime(&ms1, ctx->ev[1], ctx->ev[2]);
  cudaEventElapsedTime(&ms2, ctx->ev[4], ctx->ev[5]);
  for (u32 i = 0; i < ng; ++i) {
    tkc_result &r = outs[i];
    r.n_tied_at_kth = tied[i];
    r.edges_visited = gctr[4 * (size_t)i + 0];
    r.bfs_started = gctr[4 * (size_t)i + 1];
    r.bfs_cut = gctr[4 * (size_t)i + 2];
    r.bfs_finished = gctr[4 * (size_t)i + 3];
    r.edges_scanned = hc.edges_scanned;  // shared by the run
    r.levels = hc.levels;
    r.alg_bytes = hc.alg_bytes;
    r.batch_bits = bits;
    r.ms_pre = ms0;
    r.ms_bfs = ms1;
    r.ms_kernel = ms2;
  }
#undef MULTI_TRY
#undef MULTI_RC
  cleanup();
  return TKC_OK;
}

int tkc_topk_closeness(tkc_graph *g, uint32_t k, tkc_result *out) { return topk_one(g, k, out, 0); }

int tkc_topk_closeness_shard(tkc_graph *g, uint32_t k, uint32_t first, uint32_t shard, uint32_t nshards,
                             uint32_t max_sources, const uint64_t *seed_S, const uint32_t *seed_r,
                             const uint32_t *seed_id, uint32_t nseed, tkc_result *out) {
  return topk_shard(g, k, first, shard, nshards, max_sources, seed_S, seed_r, seed_id, nseed, out);
}

int tkc_count_tied(tkc_graph *g, uint64_t S, uint32_t r, uint32_t *count) {
  if (!g || !count || r < 2) return TKC_EINVAL;
  if (g->ctx->last_shard != g) return TKC_EINVAL;
  tkc_ctx *ctx = g->ctx;
  TKC_TRY(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  unsigned *d = nullptr;
  TKC_TRY(cudaMallocAsync(&d, sizeof(unsigned), st));
  TKC_TRY(cudaMemsetAsync(d, 0, sizeof(unsigned), st));
  const u32 n = g->n;
  const unsigned blocks = (unsigned)std::max<u64>(1, std::min<u64>(((u64)n + 255) / 256, (u64)ctx->num_sms * 8));
  if (n) TKC_LAUNCH(k_count_key<<<blocks, 256, 0, st>>>(ctx->ws.res_S, ctx->ws.res_r, n, S, r, d));
  TKC_TRY(cudaGetLastError());
  unsigned h = 0;
  TKC_TRY(cudaMemcpyAsync(&h, d, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  TKC_TRY(cudaFreeAsync(d, st));
  TKC_TRY(cudaStreamSynchronize(st));
  *count = h;
  return TKC_OK;
}

int tkc_topk_harmonic(tkc_graph *g, uint32_t k, tkc_result *out) { return topk_one(g, k, out, 1); }

int tkc_topk_closeness_bound(tkc_graph *g, uint32_t k, tkc_result *out) { return topk_bound(g, k, out); }

int tkc_topk_closeness_multi(tkc_ctx *ctx, tkc_graph *const *gs, uint32_t ng, uint32_t k, tkc_result *outs) {
  return topk_many(ctx, gs, ng, k, outs, 0);
}

int tkc_topk_harmonic_multi(tkc_ctx *ctx, tkc_graph *const *gs, uint32_t ng, uint32_t k, tkc_result *outs) {
  return topk_many(ctx, gs, ng, k, outs, 1);
}

}  // extern "C"
