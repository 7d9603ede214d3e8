// Reach bounds alpha(v) <= r(v) <= omega(v) for directed graphs on the GPU
// (Section 8.4, Algorithm 6).
//
//  1. Strongly connected components:
//     trim   vertices with no active in-arc or no active out-arc are their own
//            SCC (repeated until nothing changes);
//     FW-BW  the SCC of a pivot (largest in-degree x out-degree among the rest)
//            is the intersection of its forward and backward reach;
//     colour the rest: every vertex takes the largest id that reaches it
//            (max propagation along arcs); a vertex whose colour is its own id
//            is a root, and its SCC is the set of same-colour vertices that
//            reach it (backward propagation); repeat on what is left.
//     Each SCC is named by one of its vertices.
//  2. The biggest SCC (ties: the one holding the smallest vertex id) gets its
//     exact reach from one BFS; a backward BFS marks the SCCs that reach it.
//  3. Condensation arcs (SCC pairs) are sorted and deduplicated, so the DAG's
//     arc set has no repeats, and Algorithm 6's recurrences are evaluated
//     sinks-first by peeling: an SCC is ready once all its successors are.
//       alpha(X) = w(X) + max alpha(Y), omega(X) = w(X) + sum omega(Y), or
//       omega(X) = w(X) + omega(C~) + sum of omega(Y) over successors Y not
//       reachable from C~ when X reaches C~;  omega clamped to n.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "tkc_internal.cuh"

namespace tkc {

typedef uint32_t u32;
typedef unsigned long long u64;
static constexpr unsigned FULL = 0xffffffffu;
static constexpr u32 INF = 0xffffffffu;

// scan / sort helpers of tkc_prep.cu
int scan_exclusive_u32(const u32 *in, u32 *out, u64 len, u32 *tmp, cudaStream_t st);
int radix_sort_u32_pairs(u32 *key, u32 *val, u32 n, int bits, cudaStream_t st);

namespace {

unsigned grid_of(u64 work, unsigned tpb = 256, unsigned cap = 152 * 16) {
  u64 b = (work + tpb - 1) / tpb;
  return (unsigned)std::max<u64>(1, std::min<u64>(b, cap));
}

// ---------------------------------------------------------------- trimming

__global__ void k_trim_init(const u32 *off, const u32 *ioff, u32 n, u32 *outd, u32 *ind, uint8_t *active) {
  for (u32 v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    outd[v] = off[v + 1] - off[v];
    ind[v] = ioff[v + 1] - ioff[v];
    active[v] = 1;
  }
}

// Removes vertices without an active in-arc or out-arc (each is its own SCC)
// and lowers the counters of their neighbours.  One warp per removed vertex
// walks its arcs.
__global__ void k_trim_round(const u32 *off, const u32 *col, const u32 *ioff, const u32 *icol, u32 n, u32 *outd,
                             u32 *ind, uint8_t *active, u32 *comp, u32 *changed) {
  const int lane = threadIdx.x & 31;
  for (u32 base = (blockIdx.x * blockDim.x + threadIdx.x) & ~31u; base < n; base += gridDim.x * blockDim.x) {
    u32 v = base + lane;
    bool rm = v < n && active[v] && (outd[v] == 0 || ind[v] == 0);
    if (rm) {
      active[v] = 0;
      comp[v] = v;
    }
    u32 mask = __ballot_sync(FULL, rm);
    if (mask && lane == 0) *changed = 1;
    while (mask) {
      int src = __ffs(mask) - 1;
      mask &= mask - 1;
      u32 x = base + src;
      for (u32 i = off[x] + lane; i < off[x + 1]; i += 32) atomicSub(&ind[col[i]], 1u);
      for (u32 i = ioff[x] + lane; i < ioff[x + 1]; i += 32) atomicSub(&outd[icol[i]], 1u);
    }
  }
}

// ---------------------------------------------------------------- level BFS by sweeps

// One level of a BFS restricted to `active` (nullable): vertices at `level`
// label their unlabelled neighbours with level + 1.  Warps collect the
// frontier vertices of 32 consecutive ids and expand each with all lanes.
// Frontier vertices of out-degree above this are expanded by the whole grid.
constexpr u32 kBfsHeavy = 2048;

// One BFS level: the vertices at `level` relax their arcs (a warp per vertex);
// those of degree above kBfsHeavy are listed for k_bfs_heavy instead, so that
// a hub does not keep one warp busy while the rest of the grid waits.
__global__ void k_bfs_sweep(const u32 *off, const u32 *col, u32 n, const uint8_t *active, u32 *dist, u32 level,
                            u32 *changed, u32 *heavy, u32 *nheavy) {
  const int lane = threadIdx.x & 31;
  for (u32 base = (blockIdx.x * blockDim.x + threadIdx.x) & ~31u; base < n; base += gridDim.x * blockDim.x) {
    u32 v = base + lane;
    u32 mask = __ballot_sync(FULL, v < n && dist[v] == level);
    u32 ch = 0;
    while (mask) {
      int src = __ffs(mask) - 1;
      mask &= mask - 1;
      u32 x = base + src;
      const u32 b = off[x], e = off[x + 1];
      if (e - b > kBfsHeavy) {
        if (lane == 0) heavy[atomicAdd(nheavy, 1u)] = x;
        continue;
      }
      for (u32 i = b + lane; i < e; i += 32) {
        u32 w = col[i];
        if ((!active || active[w]) && dist[w] == INF) {
          dist[w] = level + 1;
          ch = 1;
        }
      }
    }
    if (__any_sync(FULL, ch) && lane == 0) *changed = 1;
  }
}

// The listed heavy vertices of the level: one block per vertex, and the whole
// grid for the few above kBfsHuge out-arcs.
constexpr u32 kBfsHuge = 1u << 16;

__global__ void k_bfs_heavy(const u32 *off, const u32 *col, const uint8_t *active, u32 *dist, u32 level,
                            u32 *changed, const u32 *heavy, const u32 *nheavy) {
  const u32 nh = *nheavy;
  u32 ch = 0;
  for (u32 h = 0; h < nh; ++h) {
    const u32 x = heavy[h];
    const u32 b = off[x], e = off[x + 1];
    u32 first, step;
    if (e - b > kBfsHuge) {
      first = b + blockIdx.x * blockDim.x + threadIdx.x;
      step = gridDim.x * blockDim.x;
    } else if (h % gridDim.x == blockIdx.x) {
      first = b + threadIdx.x;
      step = blockDim.x;
    } else {
      continue;
    }
    for (u32 i = first; i < e; i += step) {
      u32 w = col[i];
      if ((!active || active[w]) && dist[w] == INF) {
        dist[w] = level + 1;
        ch = 1;
      }
    }
  }
  if (__any_sync(FULL, ch) && (threadIdx.x & 31) == 0) *changed = 1;
}

// BFS levels from src over the arcs (off, col), restricted to active vertices
// (nullptr: all); flag must hold 2 words.
int bfs_levels(const u32 *off, const u32 *col, u32 n, u64 arcs, const uint8_t *active, u32 *dist, u32 src,
               u32 *flag, cudaStream_t st) {
  u32 *heavy = nullptr;
  TKC_TRY(cudaMallocAsync(&heavy, (size_t)(arcs / kBfsHeavy + 1) * sizeof(u32), st));
  TKC_TRY(cudaMemsetAsync(dist, 0xff, (size_t)n * sizeof(u32), st));
  TKC_TRY(cudaMemsetAsync(dist + src, 0, sizeof(u32), st));
  for (u32 level = 0;; ++level) {
    if (level > n) return TKC_ETIMEOUT;
    TKC_TRY(cudaMemsetAsync(flag, 0, 2 * sizeof(u32), st));
    TKC_LAUNCH(k_bfs_sweep<<<grid_of(n), 256, 0, st>>>(off, col, n, active, dist, level, flag, heavy, flag + 1));
    TKC_LAUNCH(k_bfs_heavy<<<grid_of(arcs / 8 + 1), 256, 0, st>>>(off, col, active, dist, level, flag, heavy, flag + 1));
    u32 h = 0;
    TKC_TRY(cudaMemcpyAsync(&h, flag, sizeof(u32), cudaMemcpyDeviceToHost, st));
    TKC_TRY(cudaStreamSynchronize(st));
    if (!h) break;
  }
  TKC_TRY(cudaFreeAsync(heavy, st));
  return TKC_OK;
}

// ---------------------------------------------------------------- pivot and FW-BW

__global__ void k_pivot(const u32 *outd, const u32 *ind, const uint8_t *active, u32 n, u64 *best) {
  u64 b = 0;
  for (u32 v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    if (active[v]) {
      u64 score = (u64)outd[v] * (u64)ind[v];
      score = score > 0xffffffffull ? 0xffffffffull : score;
      u64 key = (score << 32) | (u64)(0xffffffffu - v);  // larger score, then smaller id
      b = key > b ? key : b;
    }
  for (int o = 16; o; o >>= 1) {
    u64 t = __shfl_down_sync(FULL, b, o);
    b = t > b ? t : b;
  }
  if ((threadIdx.x & 31) == 0 && b) atomicMax(best, b);
}

__global__ void k_fwbw_mark(const u32 *fw, const u32 *bw, u32 n, uint8_t *active, u32 *comp, u32 pivot) {
  for (u32 v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    if (active[v] && fw[v] != INF && bw[v] != INF) {
      comp[v] = pivot;
      active[v] = 0;
    }
}

// ---------------------------------------------------------------- colouring

__global__ void k_color_init(const uint8_t *active, u32 n, u32 *color, u32 *found, u32 *cnt) {
  u32 c = 0;
  for (u32 v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    color[v] = active[v] ? v : INF;
    found[v] = 0;
    c += active[v];
  }
  c = __reduce_add_sync(FULL, c);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(cnt, c);
}

// colour[w] = max(colour[w], colour[v]) over active arcs v -> w
__global__ void k_color_prop(const u32 *off, const u32 *col, u32 n, const uint8_t *active, u32 *color,
                             u32 *changed) {
  const int lane = threadIdx.x & 31;
  for (u32 base = (blockIdx.x * blockDim.x + threadIdx.x) & ~31u; base < n; base += gridDim.x * blockDim.x) {
    u32 v = base + lane;
    u32 mask = __ballot_sync(FULL, v < n && active[v]);
    u32 ch = 0;
    while (mask) {
      int src = __ffs(mask) - 1;
      mask &= mask - 1;
      u32 x = base + src;
      u32 cx = color[x];
      for (u32 i = off[x] + lane; i < off[x + 1]; i += 32) {
        u32 w = col[i];
        if (active[w] && color[w] < cx) {
          atomicMax(&color[w], cx);
          ch = 1;
        }
      }
    }
    if (__any_sync(FULL, ch) && lane == 0) *changed = 1;
  }
}

__global__ void k_roots(const uint8_t *active, const u32 *color, u32 n, u32 *found) {
  for (u32 v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    if (active[v] && color[v] == v) found[v] = 1;
}

// found spreads backwards (along in-arcs) among vertices of the same colour
__global__ void k_back_prop(const u32 *ioff, const u32 *icol, u32 n, const uint8_t *active, const u32 *color,
                            u32 *found, u32 *changed) {
  const int lane = threadIdx.x & 31;
  for (u32 base = (blockIdx.x * blockDim.x + threadIdx.x) & ~31u; base < n; base += gridDim.x * blockDim.x) {
    u32 v = base + lane;
    u32 mask = __ballot_sync(FULL, v < n && active[v] && found[v]);
    u32 ch = 0;
    while (mask) {
      int src = __ffs(mask) - 1;
      mask &= mask - 1;
      u32 x = base + src;
      u32 cx = color[x];
      for (u32 i = ioff[x] + lane; i < ioff[x + 1]; i += 32) {
        u32 u = icol[i];
        if (active[u] && color[u] == cx && !found[u]) {
          found[u] = 1;
          ch = 1;
        }
      }
    }
    if (__any_sync(FULL, ch) && lane == 0) *changed = 1;
  }
}

__global__ void k_color_assign(u32 n, uint8_t *active, const u32 *color, const u32 *found, u32 *comp) {
  for (u32 v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    if (active[v] && found[v]) {
      comp[v] = color[v];
      active[v] = 0;
    }
}

// ---------------------------------------------------------------- component statistics

__global__ void k_comp_stats(const u32 *comp, u32 n, u32 *wgt, u32 *minid) {
  for (u32 v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    atomicAdd(&wgt[comp[v]], 1u);
    atomicMin(&minid[comp[v]], v);
  }
}

__global__ void k_biggest(const u32 *wgt, const u32 *minid, u32 n, u64 *best) {
  u64 b = 0;
  for (u32 c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x)
    if (wgt[c]) {
      u64 key = ((u64)wgt[c] << 32) | (u64)(0xffffffffu - minid[c]);
      b = key > b ? key : b;
    }
  for (int o = 16; o; o >>= 1) {
    u64 t = __shfl_down_sync(FULL, b, o);
    b = t > b ? t : b;
  }
  if ((threadIdx.x & 31) == 0 && b) atomicMax(best, b);
}

__global__ void k_count_reached(const u32 *dist, u32 n, u32 *cnt) {
  u32 c = 0;
  for (u32 v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) c += dist[v] != INF;
  c = __reduce_add_sync(FULL, c);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(cnt, c);
}

// ---------------------------------------------------------------- condensation

__global__ void k_cross_count(const u32 *off, const u32 *col, const u32 *comp, u32 n, u32 *cnt) {
  const int lane = threadIdx.x & 31;
  u32 c = 0;
  for (u32 v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += (gridDim.x * blockDim.x) >> 5)
    for (u32 i = off[v] + lane; i < off[v + 1]; i += 32) c += comp[col[i]] != comp[v];
  c = __reduce_add_sync(FULL, c);
  if (lane == 0 && c) atomicAdd(cnt, c);
}

__global__ void k_cross_emit(const u32 *off, const u32 *col, const u32 *comp, u32 n, u32 *cursor, u32 *cu,
                             u32 *cv) {
  const int lane = threadIdx.x & 31;
  for (u32 v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += (gridDim.x * blockDim.x) >> 5) {
    u32 a = comp[v];
    for (u32 i0 = off[v]; i0 < off[v + 1]; i0 += 32) {
      u32 i = i0 + lane;
      u32 b = i < off[v + 1] ? comp[col[i]] : a;
      bool cross = b != a;
      u32 m = __ballot_sync(FULL, cross);
      u32 pos = 0;
      if (lane == 0 && m) pos = atomicAdd(cursor, (u32)__popc(m));
      pos = __shfl_sync(FULL, pos, 0);
      if (cross) {
        u32 k = pos + __popc(m & ((1u << lane) - 1u));
        cu[k] = a;
        cv[k] = b;
      }
    }
  }
}

// flag[i] = 1 for the first of each run of equal (cu, cv) pairs (sorted input)
__global__ void k_unique_flags(const u32 *cu, const u32 *cv, u32 m, u32 *flag) {
  for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
    flag[i] = (i == 0 || cu[i] != cu[i - 1] || cv[i] != cv[i - 1]) ? 1u : 0u;
  if (blockIdx.x == 0 && threadIdx.x == 0) flag[m] = 0;
}

__global__ void k_unique_compact(const u32 *cu, const u32 *cv, const u32 *pos, u32 m, u32 *ou, u32 *ov,
                                 u32 *succ_cnt, u32 *pred_cnt) {
  for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
    if (pos[i + 1] != pos[i]) {
      ou[pos[i]] = cu[i];
      ov[pos[i]] = cv[i];
      atomicAdd(&succ_cnt[cu[i]], 1u);
      atomicAdd(&pred_cnt[cv[i]], 1u);
    }
}

__global__ void k_pred_scatter(const u32 *ou, const u32 *ov, u32 m, const u32 *poff, u32 *pcur, u32 *pred) {
  for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    u32 c = ov[i];
    pred[poff[c] + atomicAdd(&pcur[c], 1u)] = ou[i];
  }
}

// ---------------------------------------------------------------- Algorithm 6, sinks first

__global__ void k_sinks(const u32 *wgt, const u32 *soff, u32 n, u32 *rem, u32 *list, u32 *count) {
  for (u32 c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
    if (!wgt[c]) continue;
    u32 d = soff[c + 1] - soff[c];
    rem[c] = d;
    if (d == 0) list[atomicAdd(count, 1u)] = c;
  }
}

// Evaluates alpha/omega of the ready SCCs (all successors done), one warp
// per SCC reducing over its successors.
__global__ void k_dp_eval(const u32 *list, u32 cnt, const u32 *soff, const u32 *succ, const u32 *wgt,
                          const u32 *dist_from_big, const u32 *dist_to_big, u32 big, u64 reach_big, u32 n, u64 *A,
                          u64 *O, u32 *npred, const u32 *poff) {
  const int lane = threadIdx.x & 31;
  for (u32 i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < cnt; i += (gridDim.x * blockDim.x) >> 5) {
    u32 c = list[i];
    u64 amax = 0, osum = 0, onot = 0;
    if (c != big) {
      for (u32 e = soff[c] + lane; e < soff[c + 1]; e += 32) {
        u32 y = succ[e];
        amax = A[y] > amax ? A[y] : amax;
        osum += O[y];
        if (dist_from_big[y] == INF) onot += O[y];
      }
      for (int o = 16; o; o >>= 1) {
        u64 t = __shfl_down_sync(FULL, amax, o);
        amax = t > amax ? t : amax;
        osum += __shfl_down_sync(FULL, osum, o);
        onot += __shfl_down_sync(FULL, onot, o);
      }
    }
    if (lane == 0) {
      u64 a, o;
      if (c == big) {
        a = o = reach_big;
      } else {
        if (dist_to_big[c] != INF) osum = onot + O[big];
        a = amax + wgt[c];
        o = osum + wgt[c];
        if (o > n) o = n;
      }
      A[c] = a;
      O[c] = o;
      npred[i] = poff[c + 1] - poff[c];
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) npred[cnt] = 0;
}

// Releases the predecessors of the SCCs just evaluated, one thread per
// predecessor arc (pos: exclusive prefix of the predecessor counts); an SCC
// whose last successor this was joins the next ready list.
__global__ void k_dp_release(const u32 *list, u32 cnt, const u32 *pos, const u32 *poff, const u32 *pred, u32 *rem,
                             u32 *next, u32 *next_cnt) {
  const u32 total = pos[cnt];
  for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    u32 lo = 0, hi = cnt;  // last j with pos[j] <= i
    while (hi - lo > 1) {
      u32 mid = (lo + hi) >> 1;
      if (pos[mid] <= i) lo = mid;
      else hi = mid;
    }
    u32 c = list[lo];
    u32 p = pred[poff[c] + (i - pos[lo])];
    if (atomicSub(&rem[p], 1u) == 1u) next[atomicAdd(next_cnt, 1u)] = p;
  }
}

__global__ void k_write_bounds(const u32 *comp, u32 n, const u64 *A, const u64 *O, const u32 *wgt, u32 *alpha,
                               u32 *omega, u32 *scc_size) {
  for (u32 v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    u32 c = comp[v];
    alpha[v] = (u32)A[c];
    omega[v] = (u32)(O[c] < n ? O[c] : n);
    scc_size[v] = wgt[c];
  }
}

struct DevBufs {
  std::vector<void *> ptrs;
  cudaStream_t st;
  ~DevBufs() {
    for (void *p : ptrs) cudaFreeAsync(p, st);
  }
  template <typename T>
  cudaError_t get(T **p, size_t count) {
    cudaError_t e = cudaMallocAsync((void **)p, std::max<size_t>(count, 1) * sizeof(T), st);
    if (e == cudaSuccess) ptrs.push_back(*p);
    return e;
  }
};

u32 read_u32(const u32 *d, cudaStream_t st, int *rc) {
  u32 h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, d, sizeof(u32), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    tkc_set_last_cuda_error(e, "readback", __FILE__, __LINE__);
    *rc = TKC_ECUDA;
  }
  return h;
}

}  // namespace

int reach_directed_gpu(tkc_graph *g) {
  cudaStream_t st = g->ctx->stream;
  const u32 n = g->n;
  DevBufs b;
  b.st = st;
  u32 *outd, *ind, *comp, *fw, *bw, *color, *found, *flag, *wgt, *minid;
  uint8_t *active;
  u64 *best;
  TKC_TRY(b.get(&outd, n));
  TKC_TRY(b.get(&ind, n));
  TKC_TRY(b.get(&comp, n));
  TKC_TRY(b.get(&fw, n));
  TKC_TRY(b.get(&bw, n));
  TKC_TRY(b.get(&color, n));
  TKC_TRY(b.get(&found, n));
  TKC_TRY(b.get(&flag, 4));
  TKC_TRY(b.get(&active, n));
  TKC_TRY(b.get(&best, 1));
  int rc = TKC_OK;
  u32 pivot0 = INF;  // the first pivot, whose full forward and backward reach fw/bw keep
  TKC_LAUNCH(k_trim_init<<<grid_of(n), 256, 0, st>>>(g->off, g->ioff, n, outd, ind, active));
  for (int round = 0;; ++round) {
    // trim until stable
    for (int it = 0;; ++it) {
      if (it > (int)n + 1) return TKC_ETIMEOUT;
      TKC_TRY(cudaMemsetAsync(flag, 0, sizeof(u32), st));
      TKC_LAUNCH(k_trim_round<<<grid_of(n), 256, 0, st>>>(g->off, g->col, g->ioff, g->icol, n, outd, ind, active,
                                                          comp, flag));
      if (!read_u32(flag, st, &rc)) break;
      TKC_RC(rc);
    }
    TKC_RC(rc);
    // pivot of the largest remaining SCC candidate
    TKC_TRY(cudaMemsetAsync(best, 0, sizeof(u64), st));
    TKC_LAUNCH(k_pivot<<<grid_of(n), 256, 0, st>>>(outd, ind, active, n, best));
    u64 hb = 0;
    TKC_TRY(cudaMemcpyAsync(&hb, best, sizeof(u64), cudaMemcpyDeviceToHost, st));
    TKC_TRY(cudaStreamSynchronize(st));
    if (hb == 0) break;  // nothing left
    if (round == 0) {
      // The BFS run over the whole graph, not only the untrimmed vertices: a
      // trimmed vertex is its own SCC, so the intersection is the same, and
      // the full reach sets serve again below when this SCC is the biggest.
      u32 pivot = 0xffffffffu - (u32)(hb & 0xffffffffu);
      TKC_RC(bfs_levels(g->off, g->col, n, g->arcs, nullptr, fw, pivot, flag, st));
      TKC_RC(bfs_levels(g->ioff, g->icol, n, g->arcs, nullptr, bw, pivot, flag, st));
      TKC_LAUNCH(k_fwbw_mark<<<grid_of(n), 256, 0, st>>>(fw, bw, n, active, comp, pivot));
      pivot0 = pivot;
      continue;  // trim again, then colour
    }
    // colouring round over the remaining vertices
    TKC_TRY(cudaMemsetAsync(flag + 1, 0, sizeof(u32), st));
    TKC_LAUNCH(k_color_init<<<grid_of(n), 256, 0, st>>>(active, n, color, found, flag + 1));
    for (int it = 0;; ++it) {
      if (it > (int)n + 1) return TKC_ETIMEOUT;
      TKC_TRY(cudaMemsetAsync(flag, 0, sizeof(u32), st));
      TKC_LAUNCH(k_color_prop<<<grid_of(n), 256, 0, st>>>(g->off, g->col, n, active, color, flag));
      if (!read_u32(flag, st, &rc)) break;
      TKC_RC(rc);
    }
    TKC_RC(rc);
    TKC_LAUNCH(k_roots<<<grid_of(n), 256, 0, st>>>(active, color, n, found));
    for (int it = 0;; ++it) {
      if (it > (int)n + 1) return TKC_ETIMEOUT;
      TKC_TRY(cudaMemsetAsync(flag, 0, sizeof(u32), st));
      TKC_LAUNCH(k_back_prop<<<grid_of(n), 256, 0, st>>>(g->ioff, g->icol, n, active, color, found, flag));
      if (!read_u32(flag, st, &rc)) break;
      TKC_RC(rc);
    }
    TKC_RC(rc);
    TKC_LAUNCH(k_color_assign<<<grid_of(n), 256, 0, st>>>(n, active, color, found, comp));
  }
  TKC_TRY(cudaMemcpyAsync(g->comp, comp, (size_t)n * sizeof(u32), cudaMemcpyDeviceToDevice, st));
  // component sizes and the biggest SCC
  TKC_TRY(b.get(&wgt, n));
  TKC_TRY(b.get(&minid, n));
  TKC_TRY(cudaMemsetAsync(wgt, 0, (size_t)n * sizeof(u32), st));
  TKC_TRY(cudaMemsetAsync(minid, 0xff, (size_t)n * sizeof(u32), st));
  TKC_LAUNCH(k_comp_stats<<<grid_of(n), 256, 0, st>>>(comp, n, wgt, minid));
  TKC_TRY(cudaMemsetAsync(best, 0, sizeof(u64), st));
  TKC_LAUNCH(k_biggest<<<grid_of(n), 256, 0, st>>>(wgt, minid, n, best));
  u64 hb = 0;
  TKC_TRY(cudaMemcpyAsync(&hb, best, sizeof(u64), cudaMemcpyDeviceToHost, st));
  TKC_TRY(cudaStreamSynchronize(st));
  const u32 big_min = 0xffffffffu - (u32)(hb & 0xffffffffu);
  u32 big = 0;
  TKC_TRY(cudaMemcpyAsync(&big, comp + big_min, sizeof(u32), cudaMemcpyDeviceToHost, st));
  TKC_TRY(cudaStreamSynchronize(st));
  // exact reach of the biggest SCC (forward), and the SCCs that reach it
  // (backward); only reachability is used, the same from every vertex of the
  // SCC, so the first pivot's sweeps serve when it lies in the biggest SCC
  if (big != pivot0) {
    TKC_RC(bfs_levels(g->off, g->col, n, g->arcs, nullptr, fw, big, flag, st));
    TKC_RC(bfs_levels(g->ioff, g->icol, n, g->arcs, nullptr, bw, big, flag, st));
  }
  TKC_TRY(cudaMemsetAsync(flag, 0, sizeof(u32), st));
  TKC_LAUNCH(k_count_reached<<<grid_of(n), 256, 0, st>>>(fw, n, flag));
  const u64 reach_big = read_u32(flag, st, &rc);
  TKC_RC(rc);
  // condensation arcs, sorted by (cu, cv) and deduplicated
  TKC_TRY(cudaMemsetAsync(flag, 0, sizeof(u32), st));
  TKC_LAUNCH(k_cross_count<<<grid_of((u64)n * 32), 256, 0, st>>>(g->off, g->col, comp, n, flag));
  const u32 m = read_u32(flag, st, &rc);
  TKC_RC(rc);
  u32 *cu, *cv, *pos, *tmp, *su, *sv, *soff, *poff, *pcur, *pred, *rem, *listA, *listB;
  u64 *A, *O;
  TKC_TRY(b.get(&cu, m));
  TKC_TRY(b.get(&cv, m));
  TKC_TRY(b.get(&pos, (size_t)m + 1));
  TKC_TRY(b.get(&su, m));
  TKC_TRY(b.get(&sv, m));
  TKC_TRY(b.get(&soff, (size_t)n + 1));
  TKC_TRY(b.get(&poff, (size_t)n + 1));
  TKC_TRY(b.get(&pcur, n));
  TKC_TRY(b.get(&tmp, (std::max<size_t>(m, n) + 1) / 4096 + 2));
  TKC_TRY(cudaMemsetAsync(flag, 0, sizeof(u32), st));
  TKC_LAUNCH(k_cross_emit<<<grid_of((u64)n * 32), 256, 0, st>>>(g->off, g->col, comp, n, flag, cu, cv));
  int bits = 0;
  while (bits < 32 && ((n - 1) >> bits) != 0) ++bits;
  TKC_RC(radix_sort_u32_pairs(cv, cu, m, bits, st));  // by target
  TKC_RC(radix_sort_u32_pairs(cu, cv, m, bits, st));  // then by source, stable
  TKC_LAUNCH(k_unique_flags<<<grid_of(m), 256, 0, st>>>(cu, cv, m, pos));
  TKC_RC(scan_exclusive_u32(pos, pos, (u64)m + 1, tmp, st));
  TKC_TRY(cudaMemsetAsync(soff, 0, ((size_t)n + 1) * sizeof(u32), st));
  TKC_TRY(cudaMemsetAsync(poff, 0, ((size_t)n + 1) * sizeof(u32), st));
  TKC_LAUNCH(k_unique_compact<<<grid_of(m), 256, 0, st>>>(cu, cv, pos, m, su, sv, soff, poff));
  const u32 mu = read_u32(pos + m, st, &rc);
  TKC_RC(rc);
  TKC_RC(scan_exclusive_u32(soff, soff, (u64)n + 1, tmp, st));
  TKC_RC(scan_exclusive_u32(poff, poff, (u64)n + 1, tmp, st));
  TKC_TRY(b.get(&pred, mu));
  TKC_TRY(cudaMemsetAsync(pcur, 0, (size_t)n * sizeof(u32), st));
  TKC_LAUNCH(k_pred_scatter<<<grid_of(mu), 256, 0, st>>>(su, sv, mu, poff, pcur, pred));
  // su is sorted by source with unique pairs, so sv is the successor list
  // indexed by soff; Algorithm 6 sinks first
  TKC_TRY(b.get(&rem, n));
  TKC_TRY(b.get(&listA, n));
  TKC_TRY(b.get(&listB, n));
  TKC_TRY(b.get(&A, n));
  TKC_TRY(b.get(&O, n));
  TKC_TRY(cudaMemsetAsync(flag, 0, 2 * sizeof(u32), st));
  TKC_LAUNCH(k_sinks<<<grid_of(n), 256, 0, st>>>(wgt, soff, n, rem, listA, flag));
  u32 cnt = read_u32(flag, st, &rc);
  TKC_RC(rc);
  u32 *cur_list = listA, *nxt_list = listB, *ppos = nullptr, *ptmp = nullptr;
  TKC_TRY(b.get(&ppos, (size_t)n + 1));
  TKC_TRY(b.get(&ptmp, ((size_t)n + 1) / 4096 + 2));
  for (u32 round = 0; cnt > 0; ++round) {
    if (round > n) return TKC_ETIMEOUT;
    TKC_TRY(cudaMemsetAsync(flag + 1, 0, sizeof(u32), st));
    TKC_LAUNCH(k_dp_eval<<<grid_of((u64)cnt * 32), 256, 0, st>>>(cur_list, cnt, soff, sv, wgt, fw, bw, big,
                                                                    reach_big, n, A, O, ppos, poff));
    TKC_RC(scan_exclusive_u32(ppos, ppos, (u64)cnt + 1, ptmp, st));
    TKC_LAUNCH(k_dp_release<<<grid_of((u64)cnt * 8), 256, 0, st>>>(cur_list, cnt, ppos, poff, pred, rem, nxt_list,
                                                                     flag + 1));
    TKC_TRY(cudaGetLastError());
    cnt = read_u32(flag + 1, st, &rc);
    TKC_RC(rc);
    std::swap(cur_list, nxt_list);
  }
  TKC_LAUNCH(k_write_bounds<<<grid_of(n), 256, 0, st>>>(comp, n, A, O, wgt, g->alpha, g->omega, g->scc_size));
  TKC_TRY(cudaGetLastError());
  TKC_TRY(cudaStreamSynchronize(st));
  return TKC_OK;
}

}  // namespace tkc
