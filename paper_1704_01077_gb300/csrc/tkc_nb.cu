// computeBoundsNB (Section 5, Algorithm 3; Eq. 3 for directed graphs; Eq. 6
// for reach known only within [alpha, omega]): a lower bound on the farness of
// every vertex from upper bounds on its level sizes, and the source order of
// NBCut (increasing bound, ties by id).
//
// All vertices advance one level per sweep.  Level k needs, for every vertex
// s, the sum of N~_{k-1} over its out-neighbours (Eq. 2 subtracts the
// backtracking walks on undirected graphs, Eq. 3 does not).  A sweep is one
// gather over the CSR plus one per-vertex pass that turns the sum into N~_k,
// evaluates the reach candidates of Eq. 6 that fall on level k's linear piece
// and counts the vertices still unfinished.  The host loop stops when none is
// left or after max_levels sweeps.
//
// Counts are exact below 2^32 and stored as 2^32 from there on (any count >= n
// bounds a level; a count computed from a capped one is capped).  Per-vertex
// state is 40 bytes plus three count arrays; the gather reads every column
// once per sweep and the previous counts (8 bytes per vertex, L2-resident up
// to ~16M vertices) once per arc.
//
// Gather layout, balanced for skewed degrees: one warp per 32 consecutive
// vertices; a vertex of degree <= 8 is summed by its own lane, one of degree
// <= kHeavy by the whole warp (coalesced column reads), and a heavier one by
// one warp per kSeg-arc segment from a segment list built once per call, with
// an atomic add of each segment's capped partial sum.
#include <cuda_runtime.h>
#include <stdint.h>

#include <string.h>

#include <algorithm>
#include <vector>

#include "tkc_internal.cuh"

namespace tkc {

typedef uint32_t u32;
typedef unsigned long long u64;
typedef unsigned __int128 u128;
static constexpr unsigned FULL = 0xffffffffu;

constexpr u64 kCap = 1ull << 32;      // counts at or above this are stored as this
constexpr int kKeyFrac = 46;          // order key = floor(S * 2^46 / (r-1)^2)
constexpr u32 kHeavy = 1024;          // degrees above this go to the segment list
constexpr u32 kSeg = 1024;            // arcs per segment
constexpr u32 kLight = 8;             // degrees up to this are summed by one lane

int radix_sort_u32_pairs(u32 *key, u32 *val, u32 n, int bits, cudaStream_t st);
int scan_exclusive_u32(const u32 *in, u32 *out, u64 len, u32 *tmp, cudaStream_t st);

namespace {

unsigned grid_of(u64 work, unsigned tpb = 256, unsigned cap = 152 * 16) {
  u64 b = (work + tpb - 1) / tpb;
  return (unsigned)std::max<u64>(1, std::min<u64>(b, cap));
}

enum : uint8_t { kFinished = 1, kHave = 2 };

// ---------------------------------------------------------------- gather

__device__ __forceinline__ u64 warp_sum(u64 x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
  return x;
}

// sum[v] = sum of prev[w] over out-neighbours w, capped at kCap; heavy rows
// get 0 here and their segments are added by k_nb_gather_heavy.
__global__ void k_nb_gather(u32 n, const u32 *__restrict__ off, const u32 *__restrict__ col,
                            const u64 *__restrict__ prev, u64 *__restrict__ sum) {
  const int lane = threadIdx.x & 31;
  const u64 nwarps = (u64)gridDim.x * (blockDim.x >> 5);
  for (u64 w = (u64)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w * 32 < n; w += nwarps) {
    const u32 v = (u32)(w * 32) + lane;
    u32 b = 0, e = 0;
    if (v < n) {
      b = off[v];
      e = off[v + 1];
    }
    const u32 deg = e - b;
    u64 s = 0;
    if (deg <= kLight) {
      for (u32 a = b; a < e; ++a) s += prev[col[a]];
    }
    // medium rows: the whole warp, one row at a time
    unsigned mid = __ballot_sync(FULL, deg > kLight && deg <= kHeavy);
    while (mid) {
      const int src = __ffs(mid) - 1;
      mid &= mid - 1;
      const u32 rb = __shfl_sync(FULL, b, src), re = __shfl_sync(FULL, e, src);
      u64 part = 0;
      u32 a = rb + lane;
      for (; a + 96 < re; a += 128) {
        const u32 c0 = col[a], c1 = col[a + 32], c2 = col[a + 64], c3 = col[a + 96];
        part += prev[c0] + prev[c1] + prev[c2] + prev[c3];
      }
      for (; a < re; a += 32) part += prev[col[a]];
      part = warp_sum(part);
      if (lane == src) s = part;
    }
    if (v < n) sum[v] = deg > kHeavy ? 0 : (s < kCap ? s : kCap);
  }
}

__global__ void k_nb_gather_heavy(u32 nseg, const u32 *__restrict__ seg_row, const u32 *__restrict__ seg_begin,
                                  const u32 *__restrict__ off, const u32 *__restrict__ col,
                                  const u64 *__restrict__ prev, u64 *__restrict__ sum) {
  const int lane = threadIdx.x & 31;
  const u64 nwarps = (u64)gridDim.x * (blockDim.x >> 5);
  for (u64 w = (u64)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < nseg; w += nwarps) {
    const u32 row = seg_row[w], rb = seg_begin[w];
    const u32 re = min(rb + kSeg, off[row + 1]);
    u64 part = 0;
    u32 a = rb + lane;
    for (; a + 96 < re; a += 128) {
      const u32 c0 = col[a], c1 = col[a + 32], c2 = col[a + 64], c3 = col[a + 96];
      part += prev[c0] + prev[c1] + prev[c2] + prev[c3];
    }
    for (; a < re; a += 32) part += prev[col[a]];
    part = warp_sum(part);
    if (lane == 0) atomicAdd(&sum[row], part < kCap ? part : kCap);
  }
}

// segment list of the heavy rows
__global__ void k_seg_count(u32 n, const u32 *off, u32 *cnt) {
  for (u32 v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const u32 d = off[v + 1] - off[v];
    cnt[v] = d > kHeavy ? (d + kSeg - 1) / kSeg : 0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) cnt[n] = 0;
}

__global__ void k_seg_emit(u32 n, const u32 *off, const u32 *pos, u32 *seg_row, u32 *seg_begin) {
  for (u32 v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const u32 p0 = pos[v], p1 = pos[v + 1];
    for (u32 j = p0; j < p1; ++j) {
      seg_row[j] = v;
      seg_begin[j] = off[v] + (j - p0) * kSeg;
    }
  }
}

// ---------------------------------------------------------------- level pass

struct NbState {
  u64 *c;       // nVisited: c_{k-1} = sum of N~_i for i < k
  u64 *P;       // sum of i N~_i for i < k
  u64 *bS;      // best candidate's sum bound
  u32 *bR;      // best candidate's reach
  uint8_t *flag;
  double *hU;   // harmonic centrality: running upper bound on h
};

__device__ __forceinline__ void candidate(u64 S, u64 r, bool &have, u64 &bS, u64 &br) {
  if (!have) {
    have = true;
    bS = S;
    br = r;
    return;
  }
  const u128 lhs = (u128)S * (u128)((br - 1) * (br - 1));
  const u128 rhs = (u128)bS * (u128)((r - 1) * (r - 1));
  if (lhs < rhs) {
    bS = S;
    br = r;
  }
}

// Level k: cur holds the gathered sums (k >= 2) and receives N~_k; prev2 holds
// N~_{k-2}.  Unfinished vertices are counted into *left; an impossible
// subtraction or an empty candidate set raises *err.
__global__ void k_nb_level(u32 n, u32 k, u32 K, int directed, const u32 *__restrict__ gid,
                           const uint8_t *__restrict__ gdir, const u32 *__restrict__ off,
                           const u32 *__restrict__ alpha, const u32 *__restrict__ omega,
                           const u64 *__restrict__ prev2, u64 *__restrict__ cur, NbState st, u32 *left,
                           int *err) {
  u32 mine = 0;
  for (u32 v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const u64 deg = off[v + 1] - off[v];
    u64 x;
    if (k == 1) {
      x = deg;
    } else {
      const u64 sum = cur[v] < kCap ? cur[v] : kCap;
      if (gdir ? gdir[gid[v]] : directed) {
        x = sum;
      } else {
        const u64 p2 = prev2[v];
        if (sum >= kCap || p2 >= kCap) {
          x = kCap;
        } else {
          const u64 sub = p2 * (k == 2 ? deg : deg - 1);  // both factors < 2^32
          if (sub > sum) {
            atomicOr(err, 1);
            x = 0;
          } else {
            x = sum - sub;
          }
        }
      }
    }
    cur[v] = x;
    uint8_t f = st.flag[v];
    if (f & kFinished) continue;
    bool have = f & kHave;
    u64 bS = have ? st.bS[v] : 0, br = have ? st.bR[v] : 0;
    const u64 a = alpha[v], o = omega[v], c0 = st.c[v], P0 = st.P[v];
    double hU = st.hU[v];
    bool fin = false;
    if (x == 0) {
      // no walk continues: r(v) <= c0, nothing above c0 is a candidate
      fin = true;
      if (!have) {
        if (c0 != 1) atomicOr(err, 2);
        have = true;
        bS = 0;
        br = 1;  // out-degree 0: closeness 0
      }
    } else {
      const u64 c1 = c0 + x;
      if (a > c0 && a <= c1) candidate(P0 + (u64)k * (a - c0), a, have, bS, br);
      if (c1 > a && c1 < o) candidate(P0 + (u64)k * x, c1, have, bS, br);
      if (o <= c1) {
        candidate(P0 + (u64)k * (o - c0), o, have, bS, br);
        hU = __dadd_rn(hU, __ddiv_rn((double)(o - c0), (double)k));
        fin = true;
      } else {
        const u64 P1 = P0 + (u64)k * x;
        st.c[v] = c1;
        st.P[v] = P1;
        hU = __dadd_rn(hU, __ddiv_rn((double)x, (double)k));
        if (k == K) {
          // level K+1 unbounded: slope K+1 from c_K up to omega
          if (a > c1) candidate(P1 + (u64)(k + 1) * (a - c1), a, have, bS, br);
          candidate(P1 + (u64)(k + 1) * (o - c1), o, have, bS, br);
          hU = __dadd_rn(hU, __ddiv_rn((double)(o - c1), (double)(k + 1)));
          fin = true;
        }
      }
      st.hU[v] = hU;
    }
    if (have) {
      st.bS[v] = bS;
      st.bR[v] = (u32)br;
    }
    st.flag[v] = (uint8_t)((fin ? kFinished : 0) | (have ? kHave : 0));
    mine += fin ? 0 : 1;
  }
  mine = __reduce_add_sync(FULL, mine);
  if ((threadIdx.x & 31) == 0 && mine) atomicAdd(left, mine);
}

__global__ void k_nb_init(u32 n, NbState st, u64 *prev1, u64 *prev2) {
  for (u32 v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    st.c[v] = 1;
    st.P[v] = 0;
    st.flag[v] = 0;
    st.hU[v] = 0.0;
    prev1[v] = 1;  // N~_0
    prev2[v] = 0;
  }
}

// order keys of every vertex, and its bounds in the graph's arrays; the
// harmonic key is the complement of the bound's FP64 bits (h >= 0), so that an
// ascending sort puts the largest bound first
__global__ void k_nb_keys(u32 n, NbState st, u64 *S_out, u32 *r_out, u64 *key, u64 *hkey, int *err) {
  for (u32 v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    if (!(st.flag[v] & kHave)) {
      atomicOr(err, 4);  // every vertex finishes with a candidate
      continue;
    }
    hkey[v] = ~(u64)__double_as_longlong(st.hU[v]);
    const u64 S = st.bS[v];
    const u64 r = st.bR[v];
    S_out[v] = S;
    r_out[v] = (u32)r;
    key[v] = r <= 1 ? ~0ull : (u64)(((u128)S << kKeyFrac) / (u128)((r - 1) * (r - 1)));
  }
}

__global__ void k_iota(u32 n, u32 *a) {
  for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) a[i] = i;
}

// split keys of the listed sources, and the largest key
__global__ void k_key_parts(u32 ns, const u32 *src, const u64 *key, u32 *lo, u64 *maxkey) {
  u64 m = 0;
  for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < ns; i += gridDim.x * blockDim.x) {
    const u64 kv = key[src[i]];
    lo[i] = (u32)kv;
    m = max(m, kv);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, (u64)__shfl_xor_sync(FULL, m, o));
  if ((threadIdx.x & 31) == 0 && m) atomicMax(maxkey, m);
}

__global__ void k_key_hi(u32 ns, const u32 *val, const u64 *key, u32 *hi) {
  for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < ns; i += gridDim.x * blockDim.x)
    hi[i] = (u32)(key[val[i]] >> 32);
}

}  // namespace

// The vertices of g with out-degree >= 1, sorted by (key, id): stable LSD radix
// passes over the low and then the high 32 key bits, ids starting ascending.
// Writes *count of them to order (device); synchronises the stream.
int nb_sort_sources(tkc_graph *g, const u64 *key, u32 *order, u32 *count) {
  cudaStream_t st = g->ctx->stream;
  const u32 n = g->n;
  *count = 0;
  if (n == 0) return TKC_OK;
  u32 *ids = nullptr, *lo = nullptr;
  u64 *maxkey = nullptr;
  TKC_TRY(cudaMallocAsync(&ids, (size_t)n * sizeof(u32), st));
  TKC_TRY(cudaMallocAsync(&lo, (size_t)n * sizeof(u32), st));
  TKC_TRY(cudaMallocAsync(&maxkey, sizeof(u64), st));
  TKC_TRY(cudaMemsetAsync(maxkey, 0, sizeof(u64), st));
  TKC_LAUNCH(k_iota<<<grid_of(n), 256, 0, st>>>(n, ids));
  TKC_RC(filter_order(g, ids, order, count));  // synchronises
  const u32 ns = *count;
  if (ns) {
    TKC_LAUNCH(k_key_parts<<<grid_of(ns), 256, 0, st>>>(ns, order, key, lo, maxkey));
    u64 mk = 0;
    TKC_TRY(cudaMemcpyAsync(&mk, maxkey, sizeof(u64), cudaMemcpyDeviceToHost, st));
    TKC_TRY(cudaStreamSynchronize(st));
    int bits = 0;
    while (bits < 64 && (mk >> bits) != 0) ++bits;
    if (bits <= 32) {
      TKC_RC(radix_sort_u32_pairs(lo, order, ns, bits, st));
    } else {
      TKC_RC(radix_sort_u32_pairs(lo, order, ns, 32, st));
      TKC_LAUNCH(k_key_hi<<<grid_of(ns), 256, 0, st>>>(ns, order, key, lo));
      TKC_RC(radix_sort_u32_pairs(lo, order, ns, bits - 32, st));
    }
  }
  TKC_TRY(cudaFreeAsync(ids, st));
  TKC_TRY(cudaFreeAsync(lo, st));
  TKC_TRY(cudaFreeAsync(maxkey, st));
  TKC_TRY(cudaStreamSynchronize(st));
  return TKC_OK;
}

// Computes the bound, the order keys and the NBCut order of g (cached until the
// level cap changes).
int ensure_nb_bounds(tkc_graph *g, u32 K, const u32 *gid, const uint8_t *gdir) {
  if (K == 0 || K > 65535) return TKC_EINVAL;
  if (g->nb_order && g->nb_cap == K) return TKC_OK;
  TKC_RC(ensure_reach_bounds(g));
  tkc_ctx *ctx = g->ctx;
  cudaStream_t st = ctx->stream;
  const u32 n = g->n;
  const size_t n1 = std::max<size_t>(n, 1);
  if (!g->nb_order) {
    TKC_TRY(cudaMallocAsync(&g->nb_order, n1 * sizeof(u32), st));
    TKC_TRY(cudaMallocAsync(&g->nb_S, n1 * sizeof(u64), st));
    TKC_TRY(cudaMallocAsync(&g->nb_r, n1 * sizeof(u32), st));
    TKC_TRY(cudaMallocAsync(&g->nb_key, n1 * sizeof(u64), st));
    TKC_TRY(cudaMallocAsync(&g->nb_hkey, n1 * sizeof(u64), st));
    TKC_TRY(cudaMallocAsync(&g->nb_horder, n1 * sizeof(u32), st));
  }
  if (n == 0) {
    g->n_src_nb = 0;
    g->nb_levels = 0;
    g->nb_cap = K;
    return TKC_OK;
  }
  // scratch: three count arrays, state, heavy segments, counters
  u64 *N[3] = {nullptr, nullptr, nullptr};
  NbState s{};
  u32 *segpos = nullptr, *seg_row = nullptr, *seg_begin = nullptr, *tmp = nullptr;
  u32 *left = nullptr;
  int *err = nullptr;
  for (int i = 0; i < 3; ++i) TKC_TRY(cudaMallocAsync(&N[i], n1 * sizeof(u64), st));
  TKC_TRY(cudaMallocAsync(&s.c, n1 * sizeof(u64), st));
  TKC_TRY(cudaMallocAsync(&s.P, n1 * sizeof(u64), st));
  TKC_TRY(cudaMallocAsync(&s.bS, n1 * sizeof(u64), st));
  TKC_TRY(cudaMallocAsync(&s.bR, n1 * sizeof(u32), st));
  TKC_TRY(cudaMallocAsync(&s.flag, n1, st));
  TKC_TRY(cudaMallocAsync(&s.hU, n1 * sizeof(double), st));
  TKC_TRY(cudaMallocAsync(&segpos, (n1 + 1) * sizeof(u32), st));
  TKC_TRY(cudaMallocAsync(&tmp, ((n1 + 1) / 4096 + 16) * sizeof(u32), st));
  TKC_TRY(cudaMallocAsync(&left, 2 * sizeof(u32), st));
  TKC_TRY(cudaMallocAsync(&err, sizeof(int), st));
  TKC_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));
  // heavy-row segments
  TKC_LAUNCH(k_seg_count<<<grid_of(n), 256, 0, st>>>(n, g->off, segpos));
  TKC_RC(scan_exclusive_u32(segpos, segpos, (u64)n + 1, tmp, st));
  u32 nseg = 0;
  TKC_TRY(cudaMemcpyAsync(&nseg, segpos + n, sizeof(u32), cudaMemcpyDeviceToHost, st));
  TKC_TRY(cudaStreamSynchronize(st));
  if (nseg) {
    TKC_TRY(cudaMallocAsync(&seg_row, (size_t)nseg * sizeof(u32), st));
    TKC_TRY(cudaMallocAsync(&seg_begin, (size_t)nseg * sizeof(u32), st));
    TKC_LAUNCH(k_seg_emit<<<grid_of(n), 256, 0, st>>>(n, g->off, segpos, seg_row, seg_begin));
  }
  // sweeps: N[i % 3] holds N~_i
  TKC_LAUNCH(k_nb_init<<<grid_of(n), 256, 0, st>>>(n, s, N[0], N[2]));
  u32 levels = 0;
  const unsigned gwarps = grid_of((u64)((n + 31) / 32) * 32, 256);
  for (u32 k = 1; k <= K; ++k) {
    u64 *cur = N[k % 3], *prev1 = N[(k + 2) % 3], *prev2 = N[(k + 1) % 3];
    if (k >= 2) {
      TKC_LAUNCH(k_nb_gather<<<gwarps, 256, 0, st>>>(n, g->off, g->col, prev1, cur));
      if (nseg) TKC_LAUNCH(k_nb_gather_heavy<<<grid_of((u64)nseg * 32, 256), 256, 0, st>>>(
                    nseg, seg_row, seg_begin, g->off, g->col, prev1, cur));
    }
    TKC_TRY(cudaMemsetAsync(left, 0, sizeof(u32), st));
    TKC_LAUNCH(k_nb_level<<<grid_of(n), 256, 0, st>>>(n, k, K, g->directed, gid, gdir, g->off, g->alpha, g->omega,
                                                      prev2, cur, s, left, err));
    TKC_TRY(cudaGetLastError());
    u32 h_left = 0;
    TKC_TRY(cudaMemcpyAsync(&h_left, left, sizeof(u32), cudaMemcpyDeviceToHost, st));
    TKC_TRY(cudaStreamSynchronize(st));
    levels = k;
    if (h_left == 0) break;
  }
  TKC_LAUNCH(k_nb_keys<<<grid_of(n), 256, 0, st>>>(n, s, g->nb_S, g->nb_r, g->nb_key, g->nb_hkey, err));
  int h_err = 0;
  TKC_TRY(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  TKC_RC(nb_sort_sources(g, g->nb_key, g->nb_order, &g->n_src_nb));
  u32 nh = 0;
  TKC_RC(nb_sort_sources(g, g->nb_hkey, g->nb_horder, &nh));
  TKC_TRY(cudaStreamSynchronize(st));
  for (int i = 0; i < 3; ++i) TKC_TRY(cudaFreeAsync(N[i], st));
  void *frees[] = {s.c, s.P, s.bS, s.bR, s.flag, s.hU, segpos, seg_row, seg_begin, tmp, left, err};
  for (void *p : frees)
    if (p) TKC_TRY(cudaFreeAsync(p, st));
  if (h_err) return TKC_EGRAPH;
  g->nb_levels = levels;
  g->nb_cap = K;
  return TKC_OK;
}

}  // namespace tkc

using namespace tkc;

extern "C" {

int tkc_nb_bounds(tkc_graph *g, uint32_t max_levels, uint64_t *S_lb, uint32_t *r_lb, uint64_t *key,
                  uint32_t *order, uint32_t *n_order, uint32_t *levels) {
  if (!g || max_levels > 65535) return TKC_EINVAL;
  TKC_TRY(cudaSetDevice(g->ctx->device));
  TKC_RC(ensure_nb_bounds(g, max_levels ? max_levels : 256u));
  cudaStream_t st = g->ctx->stream;
  const size_t n = g->n;
  if (n) {
    if (S_lb) TKC_TRY(cudaMemcpyAsync(S_lb, g->nb_S, n * sizeof(u64), cudaMemcpyDeviceToHost, st));
    if (r_lb) TKC_TRY(cudaMemcpyAsync(r_lb, g->nb_r, n * sizeof(u32), cudaMemcpyDeviceToHost, st));
    if (key) TKC_TRY(cudaMemcpyAsync(key, g->nb_key, n * sizeof(u64), cudaMemcpyDeviceToHost, st));
    if (order && g->n_src_nb)
      TKC_TRY(cudaMemcpyAsync(order, g->nb_order, (size_t)g->n_src_nb * sizeof(u32), cudaMemcpyDeviceToHost, st));
  }
  TKC_TRY(cudaStreamSynchronize(st));
  if (n_order) *n_order = g->n_src_nb;
  if (levels) *levels = g->nb_levels;
  return TKC_OK;
}

int tkc_nb_harmonic_bounds(tkc_graph *g, uint32_t max_levels, double *h_ub, uint32_t *order, uint32_t *n_order) {
  if (!g || max_levels > 65535) return TKC_EINVAL;
  TKC_TRY(cudaSetDevice(g->ctx->device));
  TKC_RC(ensure_nb_bounds(g, max_levels ? max_levels : 256u));
  cudaStream_t st = g->ctx->stream;
  const size_t n = g->n;
  if (n && h_ub) {
    std::vector<u64> keys(n);
    TKC_TRY(cudaMemcpyAsync(keys.data(), g->nb_hkey, n * sizeof(u64), cudaMemcpyDeviceToHost, st));
    TKC_TRY(cudaStreamSynchronize(st));
    for (size_t i = 0; i < n; ++i) {
      const u64 b = ~keys[i];
      memcpy(&h_ub[i], &b, sizeof(double));
    }
  }
  if (n && order && g->n_src_nb)
    TKC_TRY(cudaMemcpyAsync(order, g->nb_horder, (size_t)g->n_src_nb * sizeof(u32), cudaMemcpyDeviceToHost, st));
  TKC_TRY(cudaStreamSynchronize(st));
  if (n_order) *n_order = g->n_src_nb;
  return TKC_OK;
}

}  // extern "C"
