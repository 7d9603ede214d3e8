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

#include "tkc_arcs.cuh"
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

// ---------------------------------------------------------------- reach BFS, one cooperative launch

// Control block of the reach BFS: grid barrier alone in its cache line, then
// the frontier queues' packed counters (count << 38 | out-arcs).
struct BfsCtl {
  unsigned bar_count, bar_gen, bar_pad[30];
  int err;
  unsigned level;
  unsigned long long q[2];
};

constexpr int kBfsThreads = 512;
constexpr int kQShift = 38;
constexpr u64 kQArcs = (1ull << kQShift) - 1;

__device__ __forceinline__ unsigned ld_acq(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_rel(unsigned *p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid barrier of the cooperative launch; the last block to arrive runs
// `epi` (thread 0) first.  Every wait is bounded: on expiry the kernel
// records TKC_ETIMEOUT and returns false, as do all blocks once it is set.
template <typename Epi>
__device__ bool bfs_sync(BfsCtl *c, u64 timeout, Epi epi) {
  __shared__ int s_last;
  __shared__ unsigned s_gen;
  __syncthreads();
  if (threadIdx.x == 0) {
    s_gen = ld_acq(&c->bar_gen);
    __threadfence();
    s_last = atomicAdd(&c->bar_count, 1u) + 1u == gridDim.x;
  }
  __syncthreads();
  if (s_last) {
    if (threadIdx.x == 0) {
      __threadfence();
      epi();
      c->bar_count = 0;
      __threadfence();
      st_rel(&c->bar_gen, s_gen + 1u);
    }
  } else if (threadIdx.x == 0) {
    const long long t0 = clock64();
    unsigned ns = 32;
    while (ld_acq(&c->bar_gen) == s_gen) {
      if (*(volatile int *)&c->err) break;
      if ((u64)(clock64() - t0) > timeout) {
        atomicCAS(&c->err, 0, TKC_ETIMEOUT);
        break;
      }
      __nanosleep(ns);
      if (ns < 256) ns <<= 1;
    }
    __threadfence();
  }
  __syncthreads();
  return *(volatile int *)&c->err == 0;
}

// Appends the lanes with `pred` to a queue whose counter packs count << 38 |
// out-arcs (one atomic per warp); qo[pos] = the arcs of the entries before.
__device__ __forceinline__ void q_append(bool pred, u32 v, u32 od, unsigned long long *packed, u32 *q, u64 *qo,
                                         int lane) {
  const unsigned m = __ballot_sync(FULL, pred);
  if (!m) return;
  u32 a = pred ? od : 0u;
  u32 incl = a;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const u32 t = __shfl_up_sync(FULL, incl, o);
    if (lane >= o) incl += t;
  }
  const u32 tot = __shfl_sync(FULL, incl, 31);
  const int leader = __ffs(m) - 1;
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(packed, ((unsigned long long)__popc(m) << kQShift) | tot);
  base = __shfl_sync(FULL, base, leader);
  if (pred) {
    const u32 pos = (u32)(base >> kQShift) + __popc(m & ((1u << lane) - 1u));
    q[pos] = v;
    qo[pos] = (base & kQArcs) + (incl - a);
  }
}

// Reachability from src along the arcs (off, col); (roff, rcol) are the same
// arcs reversed.  mark[v] = the step at which v was reached, INF if never
// (src: 0).  A step expands the frontier queue top-down (its arcs split evenly
// over the warps, so a hub's row is shared by many; a vertex is claimed by
// compare-and-swap) or, when the frontier's arcs exceed 1/8 of all arcs,
// bottom-up: every unreached vertex looks for any reached in-neighbour and
// stops at the first (only reachability is asked for).
__global__ void __launch_bounds__(kBfsThreads) k_bfs_reach(const u32 *off, const u32 *col, const u32 *roff,
                                                          const u32 *rcol, u32 n, u64 arcs, u32 *mark, u32 *q0,
                                                          u32 *q1, u64 *qo0, u64 *qo1, BfsCtl *c, u64 timeout) {
  const int lane = threadIdx.x & 31;
  const u32 gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int cur = 0;; cur ^= 1) {
    const unsigned long long qp = ((volatile BfsCtl *)c)->q[cur];
    const u32 qn = (u32)(qp >> kQShift);
    const u64 qa = qp & kQArcs;
    if (qn == 0) break;
    const u32 step = ((volatile BfsCtl *)c)->level + 1;
    const u32 *Q = cur ? q1 : q0;
    const u64 *QO = cur ? qo1 : qo0;
    u32 *NQ = cur ? q0 : q1;
    u64 *NQO = cur ? qo0 : qo1;
    unsigned long long *npk = &c->q[cur ^ 1];
    if (qa * 8 <= arcs) {
      // about two arc ranges per warp, whole warp steps of 32 arcs
      u64 ch = (qa + 2ull * nwarps - 1) / (2ull * nwarps);
      ch = (ch + 31) / 32 * 32;
      for (u64 a0 = (u64)gwarp * ch; a0 < qa; a0 += (u64)nwarps * ch) {
        const u64 a1 = a0 + ch < qa ? a0 + ch : qa;
        u32 lo = 0, hi = qn;  // last entry with QO <= a0
        while (hi - lo > 1) {
          const u32 mid = (lo + hi) >> 1;
          if (QO[mid] <= a0) lo = mid;
          else hi = mid;
        }
        u32 ent = lo;
        for (u64 s0 = a0; s0 < a1; s0 += 32) {
          const u64 a = s0 + lane;
          u32 w = 0;
          bool got = false;
          u32 e = ent;
          if (a < a1) {
            while (e + 1 < qn && QO[e + 1] <= a) ++e;
            w = col[off[Q[e]] + (u32)(a - QO[e])];
            got = mark[w] == INF && atomicCAS(&mark[w], INF, step) == INF;
          }
          q_append(got, w, got ? off[w + 1] - off[w] : 0u, npk, NQ, NQO, lane);
          ent = __reduce_max_sync(FULL, e);
        }
      }
    } else {
      for (u32 base = gwarp * 32; base < n; base += nwarps * 32) {
        const u32 v = base + lane;
        bool got = false;
        u32 b = 0, e = 0;
        if (v < n && mark[v] == INF) {
          b = roff[v];
          e = roff[v + 1];
        }
        const bool light = e - b <= 32;
        // short in-rows: the lane alone, four in-neighbours per step
        if (light)
          for (u32 k = b; k < e && !got; k += 4) {
            u32 mu[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) mu[j] = k + j < e ? mark[rcol[k + j]] : INF;
#pragma unroll
            for (int j = 0; j < 4; ++j) got |= mu[j] < step;
          }
        // long in-rows: the whole warp, 32 in-neighbours per step, until one is reached
        for (unsigned hv = __ballot_sync(FULL, !light); hv; hv &= hv - 1) {
          const int src = __ffs(hv) - 1;
          const u32 hb = __shfl_sync(FULL, b, src), he = __shfl_sync(FULL, e, src);
          bool hit = false;
          for (u32 k0 = hb; k0 < he && !hit; k0 += 32) {
            const u32 k = k0 + lane;
            hit = __any_sync(FULL, k < he && mark[rcol[k]] < step);
          }
          if (lane == src) got = hit;
        }
        if (got) mark[v] = step;
        q_append(got, v, got ? off[v + 1] - off[v] : 0u, npk, NQ, NQO, lane);
      }
    }
    const bool ok = bfs_sync(c, timeout, [&] {
      c->q[cur] = 0;
      c->level = step;
    });
    if (!ok) return;
  }
}

__global__ void k_bfs_start(const u32 *off, u32 *mark, u32 *q0, u64 *qo0, BfsCtl *c, u32 src) {
  mark[src] = 0;
  q0[0] = src;
  qo0[0] = 0;
  c->q[0] = (1ull << kQShift) | (unsigned long long)(off[src + 1] - off[src]);
}

// Several sources at once (nsrc distinct vertices, device array): all at step 0.
__global__ void k_bfs_start_many(const u32 *off, const u32 *src, u32 nsrc, u32 *mark, u32 *q0, u64 *qo0,
                                 BfsCtl *c) {
  u64 arcs = 0;
  for (u32 i = 0; i < nsrc; ++i) {
    const u32 v = src[i];
    mark[v] = 0;
    q0[i] = v;
    qo0[i] = arcs;
    arcs += off[v + 1] - off[v];
  }
  c->q[0] = ((unsigned long long)nsrc << kQShift) | arcs;
}

// Reachability from src (or, with srcs, from the nsrc vertices of the device
// array srcs) along (off, col) into mark (see k_bfs_reach); one cooperative
// launch.
int bfs_reach(tkc_ctx *ctx, const u32 *off, const u32 *col, const u32 *roff, const u32 *rcol, u32 n, u64 arcs,
              u32 *mark, u32 src, cudaStream_t st, const u32 *srcs = nullptr, u32 nsrc = 0) {
  static int per_sm = 0;
  if (!per_sm) {
    TKC_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bfs_reach, kBfsThreads, 0));
    if (per_sm <= 0) return TKC_ECUDA;
  }
  u32 *q = nullptr;
  u64 *qo = nullptr;
  BfsCtl *c = nullptr;
  TKC_TRY(cudaMallocAsync(&q, (size_t)2 * n * sizeof(u32), st));
  TKC_TRY(cudaMallocAsync(&qo, (size_t)2 * n * sizeof(u64), st));
  TKC_TRY(cudaMallocAsync(&c, sizeof(BfsCtl), st));
  TKC_TRY(cudaMemsetAsync(c, 0, sizeof(BfsCtl), st));
  TKC_TRY(cudaMemsetAsync(mark, 0xff, (size_t)n * sizeof(u32), st));
  u32 *q0 = q, *q1 = q + n;
  u64 *qo0 = qo, *qo1 = qo + n;
  if (srcs) {
    TKC_LAUNCH(k_bfs_start_many<<<1, 1, 0, st>>>(off, srcs, nsrc, mark, q0, qo0, c));
  } else {
    TKC_LAUNCH(k_bfs_start<<<1, 1, 0, st>>>(off, mark, q0, qo0, c, src));
  }
  u64 timeout = ctx->opt.timeout_cycles ? ctx->opt.timeout_cycles : (1ull << 34);
  void *args[] = {(void *)&off,  (void *)&col, (void *)&roff, (void *)&rcol, (void *)&n,
                  (void *)&arcs, (void *)&mark, (void *)&q0,  (void *)&q1,   (void *)&qo0,
                  (void *)&qo1,  (void *)&c,    (void *)&timeout};
  const int blocks = std::max(1, std::min(per_sm * ctx->num_sms, (int)((n + kBfsThreads - 1) / kBfsThreads)));
  note_launches(1);
  TKC_TRY(cudaLaunchCooperativeKernel((const void *)k_bfs_reach, dim3(blocks), dim3(kBfsThreads), args, 0, st));
  int err = 0;
  TKC_TRY(cudaMemcpyAsync(&err, &c->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  TKC_TRY(cudaStreamSynchronize(st));
  TKC_TRY(cudaFreeAsync(q, st));
  TKC_TRY(cudaFreeAsync(qo, st));
  TKC_TRY(cudaFreeAsync(c, st));
  return err ? err : TKC_OK;
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

// Several graphs as one union (gid: graph of each vertex, graphs in
// contiguous vertex ranges): the pivot of every graph, best[g] packed like
// k_pivot's.  Lanes of one graph first take their warp's maximum, so each
// graph sees about one atomic per warp.
__global__ void k_pivot_many(const u32 *outd, const u32 *ind, const uint8_t *active, const u32 *gid, u32 n,
                             u64 *best) {
  for (u32 base = (blockIdx.x * blockDim.x + threadIdx.x) & ~31u; base < n; base += gridDim.x * blockDim.x) {
    const u32 v = base + (threadIdx.x & 31);
    u32 score = 0, g = 0xffffffffu;
    if (v < n) {
      g = gid[v];
      if (active[v]) {
        const u64 s = (u64)outd[v] * (u64)ind[v];
        score = s > 0xffffffffull ? 0xffffffffu : (u32)s;
      }
    }
    const unsigned peers = __match_any_sync(FULL, g);
    const u32 hi = __reduce_max_sync(peers, score);
    const u32 lo = __reduce_max_sync(peers, score == hi && v < n ? 0xffffffffu - v : 0u);
    if (v < n && hi > 0 && (int)(threadIdx.x & 31) == __ffs(peers) - 1)
      atomicMax(&best[g], ((u64)hi << 32) | (u64)lo);
  }
}

// The graphs' pivots as a list (graphs without one are skipped); count in *cnt.
__global__ void k_pivot_list(const u64 *best, u32 ng, u32 *piv, u32 *list, u32 *cnt) {
  for (u32 g = blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += gridDim.x * blockDim.x) {
    const u64 b = best[g];
    piv[g] = b ? 0xffffffffu - (u32)(b & 0xffffffffu) : INF;
    if (b) list[atomicAdd(cnt, 1u)] = piv[g];
  }
}

// fw, bw: reach from / to all pivots at once.  The graphs are disjoint, so a
// vertex reached either way is reached by its own graph's pivot only, and it
// lies in that pivot's SCC when reached both ways.
__global__ void k_fwbw_mark_many(const u32 *fw, const u32 *bw, const u32 *gid, const u32 *piv, u32 n,
                                 uint8_t *active, u32 *comp) {
  for (u32 v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    if (active[v] && fw[v] != INF && bw[v] != INF) {
      comp[v] = piv[gid[v]];
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

// Size and smallest vertex of every SCC.  Lanes holding the same SCC add up
// in the warp first: one big SCC would otherwise take one atomic per vertex on
// a single address.
__global__ void k_comp_stats(const u32 *comp, u32 n, u32 *wgt, u32 *minid) {
  const int lane = threadIdx.x & 31;
  for (u32 base = (blockIdx.x * blockDim.x + threadIdx.x) & ~31u; base < n; base += gridDim.x * blockDim.x) {
    const u32 v = base + lane;
    const bool valid = v < n;
    const u32 c = valid ? comp[v] : INF;
    const unsigned grp = __match_any_sync(FULL, c);
    if (valid && lane == __ffs(grp) - 1) {
      atomicAdd(&wgt[c], (u32)__popc(grp));
      atomicMin(&minid[c], v);  // the group's first lane holds its smallest id
    }
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

// Arcs between different SCCs.  Arcs are dealt to warps in fixed chunks with
// their sources found by search (tkc_arcs.cuh), so a hub's out-row is spread
// over many warps.  The count pass writes each block's count; after an
// exclusive scan of those, the emit pass (same grid, so the same arcs per
// block) writes each block's arcs from its offset on, placed by a
// shared-memory cursor: no global atomics.  (The pairs are sorted afterwards,
// so their order within a block does not matter.)
template <bool emit>
__global__ void k_cross(const u32 *off, const u32 *col, const u32 *comp, u32 n, u64 arcs, u32 *blk, u32 *cu,
                        u32 *cv) {
  __shared__ u32 s_cnt;
  const int lane = threadIdx.x & 31;
  if (threadIdx.x == 0) s_cnt = 0;
  __syncthreads();
  const u32 base = emit ? blk[blockIdx.x] : 0u;
  u32 c = 0;
  grid_walk_arcs(off, n, arcs, [&](u32 u, u64 i, bool valid, u32) {
    const u32 a = valid ? comp[u] : 0u;
    const u32 t = valid ? comp[col[i]] : 0u;
    const bool cross = valid && t != a;
    if (!emit) {
      c += cross;
      return;
    }
    const unsigned m = __ballot_sync(FULL, cross);
    if (!m) return;
    u32 pos = 0;
    if (lane == 0) pos = atomicAdd(&s_cnt, (u32)__popc(m));
    pos = __shfl_sync(FULL, pos, 0);
    if (cross) {
      const u32 k = base + pos + __popc(m & ((1u << lane) - 1u));
      cu[k] = a;
      cv[k] = t;
    }
  });
  if (!emit) {
    c = __reduce_add_sync(FULL, c);
    if (lane == 0 && c) atomicAdd(&s_cnt, c);
    __syncthreads();
    if (threadIdx.x == 0) blk[blockIdx.x] = s_cnt;
  }
}

// flag[i] = 1 for the first of each run of equal (cu, cv) pairs (sorted input)
__global__ void k_unique_flags(const u32 *cu, const u32 *cv, u32 m, u32 *flag) {
  for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
    flag[i] = (i == 0 || cu[i] != cu[i - 1] || cv[i] != cv[i - 1]) ? 1u : 0u;
  if (blockIdx.x == 0 && threadIdx.x == 0) flag[m] = 0;
}

// Keeps the first of each run of equal pairs and counts successors and
// predecessors per SCC; lanes holding the same SCC add up in the warp first
// (one SCC may be the target of a large share of all pairs).
__global__ void k_unique_compact(const u32 *cu, const u32 *cv, const u32 *pos, u32 m, u32 *ou, u32 *ov,
                                 u32 *succ_cnt, u32 *pred_cnt) {
  const int lane = threadIdx.x & 31;
  for (u32 base = (blockIdx.x * blockDim.x + threadIdx.x) & ~31u; base < m; base += gridDim.x * blockDim.x) {
    const u32 i = base + lane;
    const bool keep = i < m && pos[i + 1] != pos[i];
    const u32 a = keep ? cu[i] : INF, t = keep ? cv[i] : INF;
    if (keep) {
      ou[pos[i]] = a;
      ov[pos[i]] = t;
    }
    const unsigned ga = __match_any_sync(FULL, a), gt = __match_any_sync(FULL, t);
    if (keep && lane == __ffs(ga) - 1) atomicAdd(&succ_cnt[a], (u32)__popc(ga));
    if (keep && lane == __ffs(gt) - 1) atomicAdd(&pred_cnt[t], (u32)__popc(gt));
  }
}

// Predecessor lists: each pair's source into its target's list (positions
// claimed once per warp and target SCC).
__global__ void k_pred_scatter(const u32 *ou, const u32 *ov, u32 m, const u32 *poff, u32 *pcur, u32 *pred) {
  const int lane = threadIdx.x & 31;
  for (u32 base = (blockIdx.x * blockDim.x + threadIdx.x) & ~31u; base < m; base += gridDim.x * blockDim.x) {
    const u32 i = base + lane;
    const u32 c = i < m ? ov[i] : INF;
    const unsigned grp = __match_any_sync(FULL, c);
    const int leader = __ffs(grp) - 1;
    u32 at = 0;
    if (c != INF && lane == leader) at = atomicAdd(&pcur[c], (u32)__popc(grp));
    at = __shfl_sync(FULL, at, leader);
    if (c != INF) pred[poff[c] + at + __popc(grp & ((1u << lane) - 1u))] = ou[i];
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

// Evaluates alpha/omega of the ready SCCs (all successors done).  A lane
// reduces over the successors of its own SCC when there are at most 32; the
// whole warp over longer successor lists.
__global__ void k_dp_eval(const u32 *list, u32 cnt, const u32 *soff, const u32 *succ, const u32 *wgt,
                          const u32 *dist_from_big, const u32 *dist_to_big, u32 big, u64 reach_big, u32 n, u64 *A,
                          u64 *O) {
  const int lane = threadIdx.x & 31;
  for (u32 base = (blockIdx.x * blockDim.x + threadIdx.x) & ~31u; base < cnt; base += gridDim.x * blockDim.x) {
    const u32 i = base + lane;
    const u32 c = i < cnt ? list[i] : INF;
    u32 b = 0, e = 0;
    if (c != INF && c != big) {
      b = soff[c];
      e = soff[c + 1];
    }
    const bool light = e - b <= 32;
    u64 amax = 0, osum = 0, onot = 0;
    if (light)
      for (u32 k = b; k < e; ++k) {
        const u32 y = succ[k];
        amax = A[y] > amax ? A[y] : amax;
        osum += O[y];
        if (dist_from_big[y] == INF) onot += O[y];
      }
    for (unsigned hv = __ballot_sync(FULL, !light); hv; hv &= hv - 1) {
      const int src = __ffs(hv) - 1;
      const u32 hb = __shfl_sync(FULL, b, src), he = __shfl_sync(FULL, e, src);
      u64 wa = 0, wo = 0, wn = 0;
      for (u32 k = hb + lane; k < he; k += 32) {
        const u32 y = succ[k];
        wa = A[y] > wa ? A[y] : wa;
        wo += O[y];
        if (dist_from_big[y] == INF) wn += O[y];
      }
      for (int o = 16; o; o >>= 1) {
        const u64 t = __shfl_xor_sync(FULL, wa, o);
        wa = t > wa ? t : wa;
        wo += __shfl_xor_sync(FULL, wo, o);
        wn += __shfl_xor_sync(FULL, wn, o);
      }
      if (lane == src) {
        amax = wa;
        osum = wo;
        onot = wn;
      }
    }
    if (c == INF) continue;
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
  }
}

// Predecessor lists longer than this are released by the whole grid.
constexpr u32 kDpHuge = 4096;

// Appends the lanes with `rel` to the ready list (one atomic per warp).
__device__ __forceinline__ void ready_append(bool rel, u32 p, u32 *next, u32 *next_cnt, int lane) {
  const unsigned m = __ballot_sync(FULL, rel);
  if (!m) return;
  u32 pos = 0;
  if (lane == 0) pos = atomicAdd(next_cnt, (u32)__popc(m));
  pos = __shfl_sync(FULL, pos, 0);
  if (rel) next[pos + __popc(m & ((1u << lane) - 1u))] = p;
}

// Releases the predecessors of the SCCs just evaluated: an SCC whose last
// unevaluated successor this was joins the next ready list.  A lane walks
// lists of at most 32, the warp longer ones; lists above kDpHuge are left to
// k_dp_release_huge (listed in huge[]).
__global__ void k_dp_release(const u32 *list, u32 cnt, const u32 *poff, const u32 *pred, u32 *rem, u32 *next,
                             u32 *next_cnt, u32 *huge, u32 *nhuge) {
  const int lane = threadIdx.x & 31;
  for (u32 base = (blockIdx.x * blockDim.x + threadIdx.x) & ~31u; base < cnt; base += gridDim.x * blockDim.x) {
    const u32 i = base + lane;
    u32 b = 0, e = 0;
    if (i < cnt) {
      const u32 c = list[i];
      b = poff[c];
      e = poff[c + 1];
      if (e - b > kDpHuge) {
        huge[atomicAdd(nhuge, 1u)] = c;
        e = b;
      }
    }
    const bool light = e - b <= 32;
    const u32 np = light ? e - b : 0;
    const u32 maxn = __reduce_max_sync(FULL, np);
    for (u32 j = 0; j < maxn; ++j) {
      u32 p = 0;
      bool rel = false;
      if (j < np) {
        p = pred[b + j];
        rel = atomicSub(&rem[p], 1u) == 1u;
      }
      ready_append(rel, p, next, next_cnt, lane);
    }
    for (unsigned hv = __ballot_sync(FULL, !light); hv; hv &= hv - 1) {
      const int src = __ffs(hv) - 1;
      const u32 hb = __shfl_sync(FULL, b, src), he = __shfl_sync(FULL, e, src);
      for (u32 k0 = hb; k0 < he; k0 += 32) {
        const u32 k = k0 + lane;
        u32 p = 0;
        bool rel = false;
        if (k < he) {
          p = pred[k];
          rel = atomicSub(&rem[p], 1u) == 1u;
        }
        ready_append(rel, p, next, next_cnt, lane);
      }
    }
  }
}

// The listed SCCs with more than kDpHuge predecessors, each by the whole grid.
__global__ void k_dp_release_huge(const u32 *huge, const u32 *nhuge, const u32 *poff, const u32 *pred, u32 *rem,
                                  u32 *next, u32 *next_cnt) {
  const int lane = threadIdx.x & 31;
  const u32 nh = *nhuge;
  for (u32 h = 0; h < nh; ++h) {
    const u32 c = huge[h];
    const u32 b = poff[c], e = poff[c + 1];
    for (u32 k0 = b + ((blockIdx.x * blockDim.x + threadIdx.x) & ~31u); k0 < e; k0 += gridDim.x * blockDim.x) {
      const u32 k = k0 + lane;
      u32 p = 0;
      bool rel = false;
      if (k < e) {
        p = pred[k];
        rel = atomicSub(&rem[p], 1u) == 1u;
      }
      ready_append(rel, p, next, next_cnt, lane);
    }
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

int reach_directed_gpu(tkc_graph *g, const u32 *gid, u32 ng) {
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
    if (round == 0 && gid && ng > 1) {
      // Several graphs: one pivot per graph and one forward and one backward
      // search from all of them, so that every graph's largest SCC is found in
      // this round (with a single pivot, only one graph's would be, and the
      // colouring rounds would take the rest).
      u64 *gbest;
      u32 *piv, *plist, *pcnt;
      TKC_TRY(b.get(&gbest, ng));
      TKC_TRY(b.get(&piv, ng));
      TKC_TRY(b.get(&plist, ng));
      TKC_TRY(b.get(&pcnt, 1));
      TKC_TRY(cudaMemsetAsync(gbest, 0, (size_t)ng * sizeof(u64), st));
      TKC_TRY(cudaMemsetAsync(pcnt, 0, sizeof(u32), st));
      TKC_LAUNCH(k_pivot_many<<<grid_of(n), 256, 0, st>>>(outd, ind, active, gid, n, gbest));
      TKC_LAUNCH(k_pivot_list<<<grid_of(ng), 256, 0, st>>>(gbest, ng, piv, plist, pcnt));
      const u32 np = read_u32(pcnt, st, &rc);
      TKC_RC(rc);
      TKC_RC(bfs_reach(g->ctx, g->off, g->col, g->ioff, g->icol, n, g->arcs, fw, 0, st, plist, np));
      TKC_RC(bfs_reach(g->ctx, g->ioff, g->icol, g->off, g->col, n, g->arcs, bw, 0, st, plist, np));
      TKC_LAUNCH(k_fwbw_mark_many<<<grid_of(n), 256, 0, st>>>(fw, bw, gid, piv, n, active, comp));
      continue;  // trim again, then colour; pivot0 stays INF (fw/bw hold no single vertex's reach)
    }
    if (round == 0) {
      // The BFS run over the whole graph, not only the untrimmed vertices: a
      // trimmed vertex is its own SCC, so the intersection is the same, and
      // the full reach sets serve again below when this SCC is the biggest.
      u32 pivot = 0xffffffffu - (u32)(hb & 0xffffffffu);
      TKC_RC(bfs_reach(g->ctx, g->off, g->col, g->ioff, g->icol, n, g->arcs, fw, pivot, st));
      TKC_RC(bfs_reach(g->ctx, g->ioff, g->icol, g->off, g->col, n, g->arcs, bw, pivot, st));
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
    TKC_RC(bfs_reach(g->ctx, g->off, g->col, g->ioff, g->icol, n, g->arcs, fw, big, st));
    TKC_RC(bfs_reach(g->ctx, g->ioff, g->icol, g->off, g->col, n, g->arcs, bw, big, st));
  }
  TKC_TRY(cudaMemsetAsync(flag, 0, sizeof(u32), st));
  TKC_LAUNCH(k_count_reached<<<grid_of(n), 256, 0, st>>>(fw, n, flag));
  const u64 reach_big = read_u32(flag, st, &rc);
  TKC_RC(rc);
  // condensation arcs, sorted by (cu, cv) and deduplicated
  const unsigned cross_grid = grid_of((g->arcs + kArcChunk - 1) / kArcChunk * 32);
  u32 *blk = nullptr, *blk_tmp = nullptr;
  TKC_TRY(b.get(&blk, (size_t)cross_grid + 1));
  TKC_TRY(b.get(&blk_tmp, ((size_t)cross_grid + 1) / 4096 + 2));
  TKC_TRY(cudaMemsetAsync(blk + cross_grid, 0, sizeof(u32), st));
  TKC_LAUNCH(k_cross<false><<<cross_grid, 256, 0, st>>>(g->off, g->col, comp, n, g->arcs, blk, nullptr, nullptr));
  TKC_RC(scan_exclusive_u32(blk, blk, (u64)cross_grid + 1, blk_tmp, st));
  const u32 m = read_u32(blk + cross_grid, st, &rc);
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
  TKC_LAUNCH(k_cross<true><<<cross_grid, 256, 0, st>>>(g->off, g->col, comp, n, g->arcs, blk, cu, cv));
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
  u32 *cur_list = listA, *nxt_list = listB, *huge = nullptr;
  TKC_TRY(b.get(&huge, (size_t)mu / kDpHuge + 1));
  for (u32 round = 0; cnt > 0; ++round) {
    if (round > n) return TKC_ETIMEOUT;
    TKC_TRY(cudaMemsetAsync(flag + 1, 0, 2 * sizeof(u32), st));
    TKC_LAUNCH(k_dp_eval<<<grid_of(cnt), 256, 0, st>>>(cur_list, cnt, soff, sv, wgt, fw, bw, big, reach_big, n, A,
                                                         O));
    TKC_LAUNCH(k_dp_release<<<grid_of(cnt), 256, 0, st>>>(cur_list, cnt, poff, pred, rem, nxt_list, flag + 1, huge,
                                                            flag + 2));
    TKC_LAUNCH(k_dp_release_huge<<<grid_of((u64)mu / 4 + 1), 256, 0, st>>>(huge, flag + 2, poff, pred, rem,
                                                                             nxt_list, flag + 1));
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
