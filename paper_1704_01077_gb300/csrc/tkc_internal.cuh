// Internal declarations of the CUDA library behind include/tkc.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <vector>

#include "../../include/tkc.h"

#define TKC_TRY(expr)                                   \
  do {                                                  \
    cudaError_t e_ = (expr);                            \
    if (e_ != cudaSuccess) {                            \
      tkc_set_last_cuda_error(e_, #expr, __FILE__, __LINE__); \
      return e_ == cudaErrorMemoryAllocation ? TKC_ENOMEM : TKC_ECUDA; \
    }                                                   \
  } while (0)

#define TKC_RC(expr)            \
  do {                          \
    int rc_ = (expr);           \
    if (rc_ != TKC_OK) return rc_; \
  } while (0)

void tkc_set_last_cuda_error(cudaError_t e, const char *what, const char *file, int line);

namespace tkc {

// Counts every kernel launch of the library (see tkc_kernel_launches).
void note_launches(unsigned count);
#define TKC_LAUNCH(...)            \
  do {                             \
    __VA_ARGS__;                   \
    ::tkc::note_launches(1);       \
  } while (0)

constexpr uint32_t kMaxN = 1u << 26; // list counters pack the count in 26 bits
constexpr int kMaxWords = 8;         // 512-bit source batches
constexpr uint32_t kBuChunkVerts = 128;  // bottom-up levels: list entries per chunk a warp takes
// bottom-up levels: in-rows longer than this are walked by the whole warp.
// In id order a warp's 32 lanes hold rows of unrelated lengths, so rows
// beyond a few steps of a lane go to the warp (kHeavyIn); in the in-degree
// labelling neighbouring rows have similar lengths and a lane may keep longer
// ones (kHeavyInLabelled; R-MAT 22, NBCut, search kernel: 24 -> 34.5 ms,
// 48 -> 33.1, 96 -> 32.4, 192 to 384 -> 32.5).
#ifndef TKC_HEAVY_IN
#define TKC_HEAVY_IN 24
#endif
#ifndef TKC_HEAVY_IN_LABELLED
#define TKC_HEAVY_IN_LABELLED 96
#endif
constexpr uint32_t kHeavyIn = TKC_HEAVY_IN;
constexpr uint32_t kHeavyInLabelled = TKC_HEAVY_IN_LABELLED;

// Device-resident state of one persistent BFSCut run (one graph).
struct Ctl {
  // grid barrier, alone in its cache line
  unsigned int bar_count;
  unsigned int bar_gen;
  unsigned int bar_pad[30];
  int err;
  int err_where;
  // loop state
  int step;          // 0 = level, 1 = clear + seed, 2 = compact the frontier list to the active slots
  int done;
  int dir;           // 0 = top-down, 1 = bottom-up
  int cur;           // which frontier buffer / list is current
  unsigned int level_id;  // global level stamp
  unsigned int cursor;    // next position in the source order
  unsigned int fl_count;  // current frontier list size
  unsigned int vl_count;  // visited-list size (vertices with a non-zero seen row)
  unsigned int pad0;
  unsigned long long fl_arcs;    // arcs out of the current frontier list
  unsigned long long nl_packed;  // next list: count << 38 | arcs
  unsigned long long active[kMaxWords];
  // counters
  unsigned long long edges_visited;
  unsigned long long edges_scanned;
  unsigned long long bfs_started;
  unsigned long long bfs_cut;
  unsigned long long bfs_finished;
  unsigned long long levels;
  unsigned long long batches;
  // cost-model bytes of the levels and this level's bottom-up scan statistics
  unsigned long long alg_bytes;
  unsigned long long lvl_scan_v;
  unsigned long long lvl_scan_a;
  unsigned long long lvl_scan_r;  // this level's frontier rows loaded by the bottom-up walks
  unsigned long long trace_n;  // records written to the optional trace
  unsigned int bdepth;         // depth reached by the current batch (0 after seeding)
  unsigned int pad1;
  // per-level totals of the run (tkc_last_run_stats)
  unsigned long long st_td_levels, st_td_frontier, st_td_arcs, st_td_new;
  unsigned long long st_bu_levels, st_bu_scan_v, st_bu_scan_a, st_bu_new, st_bu_frontier, st_bu_rows;
  unsigned long long st_seeded, st_cleared;
  unsigned long long st_compactions, st_compact_dropped;
  int lcur;          // which list buffer holds the current frontier list (compaction swaps it alone)
  int pad2;
};

// State shared by all teams of one run.
struct Shared {
  unsigned int cursor;   // next position in the source order (teams take chunks)
  int lock;              // guards the k-lists while a team merges
  int err;               // first error of any team
  unsigned int first_done;  // team 0 has finished its first batch (other teams may start)
};

struct Slot {
  unsigned long long S;   // sum of distances of the discovered levels
  unsigned long long nd;  // size of the discovered ball
  unsigned long long g;   // upper bound on the next level's size
  unsigned long long arcs;  // arcs out of the newest level (expanded next)
  unsigned int v;         // source vertex
  unsigned int d;         // deepest discovered level
  unsigned int alpha, omega;
  int state;              // 0 free, 1 active, 2 done (waiting for the clear step)
  unsigned int graph;     // graph of the source (several graphs in one run)
  unsigned int nocut;     // 1: searched to the end (threshold seeding)
  unsigned int pad;
  double H;               // harmonic runs: sum over discovered levels of |level| / level
};

struct RunParams {
  // graph
  uint32_t n;
  int directed;
  uint64_t arcs;
  const uint32_t *off, *col, *ioff, *icol;
  // labels of the search's rows (nullptr: a vertex's label is its id).
  // off/col/ioff/icol, bu_list and every per-vertex row, bit and list of the
  // search are indexed by label; the source order, alpha, omega, lb_key, gid,
  // res_S/res_r, lvl and every id in a slot or list entry by id.
  const uint32_t *lab;    // id -> label
  const uint32_t *unlab;  // label -> id
  const uint32_t *alpha, *omega;
  // bottom-up levels sweep bu_list[0, n_bu): the vertices with an in-arc, the
  // n_bu_heavy with more than heavy_in in-arcs first (longest first), then the
  // others by label (nullptr: every vertex, by label)
  const uint32_t *bu_list;
  uint32_t n_bu, n_bu_heavy;
  uint32_t heavy_in;  // in-rows longer than this are walked by the whole warp
  uint32_t large_blocks;  // tkc_options.large_blocks: 0 = by size, 1 = larger blocks, 2 = 512 threads
  const uint32_t *order;
  uint32_t norder;  // sources in `order` to examine (all have out-degree >= 1)
  // search configuration
  // teams: independent groups of `gridDim.x / teams` blocks, each running its
  // own batches; per-team buffers sit at team * stride from the base pointers
  uint32_t teams;
  uint32_t team;         // this block's team (set by the kernel)
  uint64_t row_stride;   // 64-bit words between the teams' seen/F0/F1/N rows
  uint64_t vtx_stride;   // 32-bit words between the teams' lists and stamps
  uint64_t fb_stride;    // 32-bit words between the teams' frontier bitmaps
  Shared *sh;
  // published k-th entry of each graph's list (seqlock: odd = being written)
  unsigned int *x_seq;
  unsigned long long *x_S;
  uint32_t *x_r, *x_id;
  // several graphs in one run, as their disjoint union (ng = 1: one graph)
  uint32_t ng;
  const uint32_t *gid;        // graph of each vertex (nullptr: every vertex in graph 0)
  // sources graph by graph after every graph's opening batch: one past each
  // graph's last order position (nullable), and the first position after the
  // openings (a stop there may skip the rest of its graph at once)
  const uint32_t *g_end;
  uint32_t g_rest;
  const uint8_t *g_directed;  // per graph (nullptr: `directed` for all)
  unsigned int *g_ntop;       // entries in each graph's top list
  unsigned long long *g_ctr;  // per graph: edges_visited, bfs_started, bfs_cut, bfs_finished (nullable)
  uint32_t kk;        // min(k, n); 0 never reaches the kernel
  uint32_t B;         // active slots per batch (1..64*W)
  int nocut;          // 1: never cut (exact S, r for every source)
  int harmonic;       // 1: rank by harmonic centrality (list keys are the FP64 bits of h, largest first)
  uint32_t nocut_prefix;  // sources at order positions below this are never cut
  // NBCut (nullptr: off): per-vertex floor(2^46 * bound on S/(r-1)^2), the
  // order sorted by it; seeding stops at the first source whose key exceeds
  // its graph's k-th farness strictly.  Harmonic runs: ~(FP64 bits of the
  // upper bound on h), stop when the bound is below the k-th h.
  const unsigned long long *lb_key;
  unsigned int *g_stop;  // several graphs: graph g's search has stopped (its later sources are skipped)
  // updateBoundsLB (nullptr: off; every search complete, one batch per team):
  // the level at which each vertex is found by each slot of each team,
  // lvl[v * lvl_stride + team * B + slot] (0xffff: not found), each slot's
  // level sizes hist[(team * B + slot) * hist_cap + level], and its source
  // lvl_src[team * B + slot]
  uint16_t *lvl;
  uint32_t *hist;
  uint32_t *lvl_src;
  uint32_t hist_cap;
  uint32_t lvl_stride;
  uint32_t bu_num, bu_den;
  uint64_t timeout;
  // workspace
  unsigned long long *seen, *F0, *F1, *N;
  uint32_t *FB0, *FB1;      // one bit per vertex: row of F0 / F1 is non-zero
  uint32_t *L0, *L1;        // frontier lists
  uint32_t *Loff0, *Loff1;  // exclusive arc prefix of each list entry
  uint32_t *VL;             // visited list
  uint32_t *stamp;
  Slot *slots;
  unsigned int *cnt;             // per-slot level counts
  unsigned long long *wsum;      // per-slot sums of out-degree over the new level
  unsigned long long *top_S;     // graph g's list at [g * kk, (g + 1) * kk)
  uint32_t *top_r, *top_id;
  unsigned long long *res_S;     // per-vertex S of finished searches
  uint32_t *res_r;               // per-vertex r of finished searches (0 = not finished)
  Ctl *ctl;
  // optional per-step trace (16 words per record), nullptr when off
  unsigned long long *trace;
  uint32_t trace_cap;
};

struct Workspace {
  uint32_t n_cap = 0;
  int words_cap = 0;
  unsigned long long *seen = nullptr, *F0 = nullptr, *F1 = nullptr, *N = nullptr;
  uint32_t *FB0 = nullptr, *FB1 = nullptr;
  uint32_t *L0 = nullptr, *L1 = nullptr, *Loff0 = nullptr, *Loff1 = nullptr, *VL = nullptr, *stamp = nullptr;
  unsigned long long *res_S = nullptr;
  uint32_t *res_r = nullptr;
  Slot *slots = nullptr;
  unsigned int *cnt = nullptr;
  unsigned long long *wsum = nullptr;
  unsigned long long *top_S = nullptr;
  uint32_t *top_r = nullptr, *top_id = nullptr;
  Ctl *ctl = nullptr;
  unsigned long long *out_S = nullptr;
  uint32_t *out_r = nullptr, *out_id = nullptr;
  double *out_f = nullptr, *out_c = nullptr;
  unsigned int *tied = nullptr;     // per graph
  unsigned int *g_ntop = nullptr;   // per graph
  unsigned int *g_stop = nullptr;   // per graph: NBCut stop reached
  unsigned long long *g_ctr = nullptr;  // 4 per graph
  Shared *sh = nullptr;
  unsigned int *x_seq = nullptr;
  unsigned long long *x_S = nullptr;
  uint32_t *x_r = nullptr, *x_id = nullptr;
  uint32_t top_cap = 0;   // entries of top_* / out_* (graphs x k)
  uint32_t ng_cap = 0;    // graphs of tied / g_ntop / g_ctr / x_*
  uint32_t teams_cap = 0; // teams the per-team buffers are sized for
  unsigned int level_base = 0;  // stamp epoch carried across runs
};

}  // namespace tkc

// Source-order model: 5 -> 64 -> 64 -> 1 MLP, fp32 master weights with a
// bf16 copy for the forward passes, Adam moments.
struct MlpState {
  float *w = nullptr;             // TKC_MLP_PARAMS fp32 master weights
  unsigned short *wb = nullptr;   // bf16 copy used by the forward passes
  float *m = nullptr, *v = nullptr;  // Adam moments
  float *grad = nullptr;          // gradient scratch
  float *loss = nullptr;          // loss accumulator
  uint64_t step = 0;
  uint64_t version = 0;           // bumped whenever the weights change
  bool ready = false;
};

// Autotuner choice for one graph class.
struct TuneEntry {
  uint32_t batch_bits, teams, bu_num, bu_den;
  double ms;
  uint32_t large_blocks;  // tkc_options.large_blocks of the fastest run (1 or 2)
};

struct tkc_ctx {
  int device = 0;
  tkc_run_stats last_stats{};  // per-level totals of the latest search-kernel run
  const tkc_graph *last_shard = nullptr;  // graph of the latest run, when it was a shard run
  MlpState mlp;
  std::map<std::string, TuneEntry> tune;  // graph class -> fastest parameters
  cudaStream_t stream = nullptr;
  tkc_options opt{};
  int num_sms = 0;
  tkc::Workspace ws;
  cudaEvent_t ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  cudaStream_t aux = nullptr;    // helper stream: the labelled copy, built while `stream` preprocesses
  cudaEvent_t aux_in = nullptr;  // orders the helper stream after `stream`'s work so far
  int graphs_alive = 0;
};

struct tkc_graph {
  tkc_ctx *ctx = nullptr;
  uint32_t n = 0;
  uint64_t arcs = 0;
  int directed = 0;
  uint32_t *off = nullptr, *col = nullptr;    // out-arcs
  mutable uint32_t *ioff = nullptr, *icol = nullptr;  // in-arcs (aliases of out-arcs when undirected; directed: built
                                                      // on first use, ensure_in_csr)
  uint32_t *deg_order = nullptr;              // computeBoundsDeg order (all n vertices)
  uint32_t n_src_deg = 0;                     // vertices with out-degree >= 1 (prefix of deg_order)
  mutable uint32_t *zero_ids = nullptr;       // vertices of out-degree 0, id order (ensure_zero_list)
  mutable uint32_t n_zero = 0;
  mutable bool have_zero = false;
  uint32_t *given_order = nullptr;            // filtered caller order
  uint32_t n_src_given = 0;
  uint32_t *alpha = nullptr, *omega = nullptr;
  uint32_t *scc_size = nullptr;               // size of the SCC (component, if undirected) of each vertex
  uint32_t *comp = nullptr;                   // SCC (component, if undirected) id of each vertex
  bool have_order = false, have_reach = false;
  float *features = nullptr;                  // standardized vertex features, n x TKC_MLP_FEATURES
  uint32_t *learned_order = nullptr;          // filtered order by predicted farness
  uint32_t n_src_learned = 0;
  uint64_t learned_version = 0;               // model version the learned order was computed with
  uint32_t *seeded_order = nullptr;           // predicted-closest prefix, then the degree or NB order
  uint64_t seeded_version = 0;
  uint32_t seeded_prefix = 0;
  int seeded_base = -1;                       // 0: degree order after the prefix, 1: NB order
  uint32_t seeded_nb_cap = 0;                 // nb_cap of the NB order it was built from
  uint32_t *nb_order = nullptr;               // NBCut order: out-degree >= 1, by (nb_key, id)
  uint32_t n_src_nb = 0;
  uint32_t nb_cap = 0;                        // level cap the bounds were computed with (0 = none yet)
  uint32_t nb_levels = 0;                     // sweeps run
  unsigned long long *nb_S = nullptr;         // neighbourhood bound: S~ at the minimising reach
  uint32_t *nb_r = nullptr;                   //   that reach (1: out-degree 0)
  unsigned long long *nb_key = nullptr;       //   floor(S~ * 2^46 / (r-1)^2)
  unsigned long long *nb_hkey = nullptr;      // harmonic: ~(FP64 bits of the upper bound on h)
  uint32_t *nb_horder = nullptr;              // harmonic NBCut order: by (nb_hkey, id)
  // the graph as the search kernel walks it (ensure_search_csr): s_mode 0 =
  // the graph itself, 1 = a copy whose vertex i is vertex s_unlab[i] (s_lab is
  // the inverse), vertices by in-degree, largest first; -1 = not built yet
  mutable int s_mode = -1;
  mutable uint32_t *s_off = nullptr, *s_col = nullptr, *s_ioff = nullptr, *s_icol = nullptr;
  mutable uint32_t *s_lab = nullptr, *s_unlab = nullptr;
  mutable uint32_t *s_cnt = nullptr;          // device: the bottom-up list's counts (n_bu, n_bu_heavy)
  mutable cudaEvent_t s_ready = nullptr;      // the copy is being built on the context's helper stream
  mutable uint32_t *bu_list = nullptr;        // bottom-up sweep order of that CSR: vertices with an in-arc, hubs first
  mutable uint32_t n_bu = 0, n_bu_heavy = 0;
  mutable uint32_t heavy_in = 0;              // the list's long-row threshold (kHeavyIn or kHeavyInLabelled)
};

namespace tkc {
// tkc_prep.cu
int validate_graph(tkc_graph *g);
int enqueue_validate(const tkc_graph *g, uint32_t *flag);   // no host wait
int enqueue_symmetric(const tkc_graph *g, uint32_t *flag);  // after enqueue_validate passed
int build_in_csr(const tkc_graph *g);
int ensure_in_csr(const tkc_graph *g);
int ensure_degree_order(tkc_graph *g);
int ensure_zero_list(const tkc_graph *g);
// gid/ng (several graphs as one union, graphs in contiguous vertex ranges):
// one pivot per graph in the first forward-backward round
int ensure_reach_bounds(tkc_graph *g, const uint32_t *gid = nullptr, uint32_t ng = 0);
// the search kernel's CSR and bottom-up list (relabel: the in-degree labelling)
int ensure_search_csr(const tkc_graph *g, bool relabel);
int start_search_csr(const tkc_graph *g);  // the labelled copy, on the helper stream
void free_search_csr(const tkc_graph *g);
int filter_order(tkc_graph *g, const uint32_t *d_order_all, uint32_t *d_out, uint32_t *count);
// tkc_nb.cu
// gid/g_directed (several graphs as one union): per-vertex directedness
int ensure_nb_bounds(tkc_graph *g, uint32_t max_levels, const uint32_t *gid = nullptr,
                     const uint8_t *g_directed = nullptr);
int nb_sort_sources(tkc_graph *g, const unsigned long long *key, uint32_t *order, uint32_t *count);
// tkc_lb.cu
int lb_init(tkc_graph *g, const unsigned long long *S0, const uint32_t *r0, const unsigned long long *key0,
            unsigned long long *bS, uint32_t *bR, unsigned long long *key, uint8_t *done);
int lb_sorted_candidates(tkc_graph *g, const uint32_t *order0, uint32_t n0, const uint8_t *done,
                         const unsigned long long *key, uint32_t *cand, uint32_t *count, uint32_t *scratch_pos,
                         uint32_t *scratch_tmp, uint32_t *scratch_lo, unsigned long long *scratch_max);
int lb_gather_keys(tkc_graph *g, uint32_t cnt, const uint32_t *cand, const unsigned long long *key,
                   unsigned long long *out);
int lb_update(tkc_graph *g, uint32_t B, uint32_t nsrc, const uint32_t *srcs, uint16_t *lvl, uint32_t *hist,
              uint32_t cap, uint32_t *depth, unsigned long long *Ltab, const uint32_t *res_r, unsigned long long *bS,
              uint32_t *bR, unsigned long long *key, uint8_t *done);
// tkc_mlp.cu
int ensure_features(tkc_graph *g);
int ensure_learned_order(tkc_graph *g);
// prefix predicted-closest sources, then the degree order (nb = false) or the
// NB order (nb = true; ensure_nb_bounds must have run) without them
int ensure_seeded_order(tkc_graph *g, uint32_t prefix, bool nb);
void free_mlp(tkc_ctx *ctx);
// tkc_bfscut.cu
int ensure_workspace(tkc_ctx *ctx, uint32_t n, int words, uint32_t top_entries, uint32_t ng, uint32_t teams);
int run_bfscut(tkc_ctx *ctx, const RunParams &p, int words, int blocks);  // blocks: a multiple of p.teams
int max_coresident_blocks(tkc_ctx *ctx, int words);
}  // namespace tkc
