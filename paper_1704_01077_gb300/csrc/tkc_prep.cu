// Preprocessing for Algorithm 1: CSR validation and in-arc CSR, the
// computeBoundsDeg source order (Section 4), and the reach bounds alpha/omega
// (exact component sizes for undirected graphs here; Algorithm 6 of Section
// 8.4 for directed graphs in tkc_scc.cu).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "tkc_arcs.cuh"
#include "tkc_internal.cuh"

namespace tkc {

typedef uint32_t u32;
typedef unsigned long long u64;
static constexpr unsigned FULL = 0xffffffffu;

// ------------------------------------------------------------------ device-wide exclusive scan

static constexpr int kScanTPB = 1024;
static constexpr int kScanItems = 4;
static constexpr int kScanTile = kScanTPB * kScanItems;

__device__ __forceinline__ u32 block_exscan_1024(u32 x, u32 *s_warp, u32 *total) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  u32 incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    u32 t = __shfl_up_sync(FULL, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) s_warp[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    u32 v = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : 0;
    u32 vi = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      u32 t = __shfl_up_sync(FULL, vi, o);
      if (lane >= o) vi += t;
    }
    s_warp[lane] = vi - v;
    if (lane == 31) s_warp[32] = vi;
  }
  __syncthreads();
  u32 res = s_warp[wid] + incl - x;
  *total = s_warp[32];
  __syncthreads();
  return res;
}

__global__ void k_scan_bsum(const u32 *in, u64 len, u32 *bsum) {
  __shared__ u32 s_warp[33];
  u64 base = (u64)blockIdx.x * kScanTile + (u64)threadIdx.x * kScanItems;
  u32 s = 0;
  for (int i = 0; i < kScanItems; ++i)
    if (base + i < len) s += in[base + i];
  u32 total;
  block_exscan_1024(s, s_warp, &total);
  if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

__global__ void k_scan_small(u32 *a, u32 len) {
  __shared__ u32 s_warp[33];
  u32 per = (len + kScanTPB - 1) / kScanTPB;
  u32 lo = threadIdx.x * per, hi = min(len, lo + per);
  u32 s = 0;
  for (u32 i = lo; i < hi; ++i) s += a[i];
  u32 total;
  u32 pre = block_exscan_1024(s, s_warp, &total);
  for (u32 i = lo; i < hi; ++i) {
    u32 t = a[i];
    a[i] = pre;
    pre += t;
  }
}

__global__ void k_scan_apply(const u32 *in, u32 *out, u64 len, const u32 *bsum) {
  __shared__ u32 s_warp[33];
  u64 base = (u64)blockIdx.x * kScanTile + (u64)threadIdx.x * kScanItems;
  u32 v[kScanItems];
  u32 s = 0;
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = base + i < len ? in[base + i] : 0;
    s += v[i];
  }
  u32 total;
  u32 pre = block_exscan_1024(s, s_warp, &total) + bsum[blockIdx.x];
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < len) out[base + i] = pre;
    pre += v[i];
  }
}

// out[i] = sum of in[0..i); in and out may alias.  tmp holds ceil(len/4096) words.
static int scan_exclusive(const u32 *in, u32 *out, u64 len, u32 *tmp, cudaStream_t st) {
  if (len == 0) return TKC_OK;
  u64 nb = (len + kScanTile - 1) / kScanTile;
  if (nb > (u64)kScanTPB * 4096) return TKC_EOVERFLOW;
  TKC_LAUNCH(k_scan_bsum<<<(unsigned)nb, kScanTPB, 0, st>>>(in, len, tmp));
  TKC_LAUNCH(k_scan_small<<<1, kScanTPB, 0, st>>>(tmp, (u32)nb));
  TKC_LAUNCH(k_scan_apply<<<(unsigned)nb, kScanTPB, 0, st>>>(in, out, len, tmp));
  TKC_TRY(cudaGetLastError());
  return TKC_OK;
}

// ------------------------------------------------------------------ CSR validation and transpose

enum : u32 { kBadOffsets = 1, kBadRange = 2, kSelfLoop = 4, kUnsorted = 8, kAsymmetric = 16 };

// Offsets from 0 to arcs, monotone and within arcs (a thread per vertex); ids
// in range, no self-loop, each row strictly increasing (sorted, no
// duplicates), checked arc by arc.
__global__ void k_validate(const u32 *off, const u32 *col, u32 n, u64 arcs, u32 *flags) {
  const int lane = threadIdx.x & 31;
  u32 f = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0 && (off[0] != 0 || off[n] != arcs)) f |= kBadOffsets;
  for (u64 v = (u64)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (u64)gridDim.x * blockDim.x) {
    const u32 b = off[v], e = off[v + 1];
    if (e < b || e > arcs) f |= kBadOffsets;
  }
  // the arcs in chunks with their sources (tkc_arcs.cuh: a hub's row is
  // spread over many warps; reads stay in bounds even when the offsets are
  // bad, which the loop above reports)
  grid_walk_arcs<true>(off, n, arcs, [&](u32 u, u64 i, bool valid, u32 rs) {
    if (!valid) return;
    const u32 c = col[i];
    if (c >= n) f |= kBadRange;
    if (c == u) f |= kSelfLoop;
    if (i > rs && col[i - 1] >= c) f |= kUnsorted;
  });
  f = __reduce_or_sync(FULL, f);
  if (lane == 0 && f) atomicOr(flags, f);
}

// Undirected input: every arc u->v needs the arc v->u (binary search in v's
// row; the graph already passed k_validate, so rows are sorted).  Arcs in
// chunks with their sources (tkc_arcs.cuh), so a hub's row is spread over
// many warps.
__global__ void k_symmetric(const u32 *off, const u32 *col, u32 n, u64 arcs, u32 *flags) {
  const int lane = threadIdx.x & 31;
  u32 f = 0;
  grid_walk_arcs(off, n, arcs, [&](u32 u, u64 i, bool valid, u32) {
    if (!valid) return;
    const u32 v = col[i];
    u32 lo = off[v], hi = off[v + 1];
    const u32 end = hi;
    while (lo < hi) {
      const u32 mid = (lo + hi) >> 1;
      if (col[mid] < u) lo = mid + 1;
      else hi = mid;
    }
    if (lo >= end || col[lo] != u) f |= kAsymmetric;
  });
  f = __reduce_or_sync(FULL, f);
  if (lane == 0 && f) atomicOr(flags, f);
}

// In-degrees: cnt[v] += 1 per arc u -> v, 32 consecutive arcs per warp step
// (coalesced column reads).  Lanes adding to the same vertex (the hubs of
// skewed in-degree distributions) add their count in one atomic.
__global__ void k_in_count(const u32 *__restrict__ col, u64 arcs, u32 *__restrict__ cnt) {
  const int lane = threadIdx.x & 31;
  for (u64 base = ((u64)blockIdx.x * blockDim.x + threadIdx.x) & ~31ull; base < arcs;
       base += (u64)gridDim.x * blockDim.x) {
    const u64 i = base + lane;
    const bool valid = i < arcs;
    const u32 v = valid ? col[i] : 0xffffffffu;
    const unsigned peers = __match_any_sync(FULL, v);
    if (valid && __ffs(peers) - 1 == lane) atomicAdd(&cnt[v], (u32)__popc(peers));
  }
}

// The in-arc columns: arc u -> v takes slot cursor[v]++ of v's in-row (cursor
// starts at ioff).  Arcs are dealt to warps in fixed chunks with their
// sources found by search (tkc_arcs.cuh), so a hub's out-row is spread over
// many warps.  Lanes writing the same in-row take consecutive slots from one
// atomic.  In-rows come out roughly in ascending source order (chunks are
// taken in arc order).
__global__ void k_in_fill(const u32 *__restrict__ off, const u32 *__restrict__ col, u32 n, u64 arcs,
                          u32 *__restrict__ cursor, u32 *__restrict__ icol) {
  const int lane = threadIdx.x & 31;
  grid_walk_arcs(off, n, arcs, [&](u32 u, u64 i, bool valid, u32) {
    const u32 v = valid ? col[i] : 0xffffffffu;
    const unsigned peers = __match_any_sync(FULL, v);
    const int leader = __ffs(peers) - 1;
    u32 pos = 0;
    if (valid && leader == lane) pos = atomicAdd(&cursor[v], (u32)__popc(peers));
    pos = __shfl_sync(FULL, pos, leader) + (u32)__popc(peers & ((1u << lane) - 1u));
    if (valid) icol[pos] = u;
  });
}

static unsigned grid_for(u64 work, unsigned tpb, unsigned cap = 152 * 16) {
  u64 b = (work + tpb - 1) / tpb;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (unsigned)b;
}

// Enqueues the structural checks of g's CSR (offsets, ids, self-loops, row
// order); violations are ORed into the device word *flag.  No host wait.
int enqueue_validate(const tkc_graph *g, u32 *flag) {
  if (g->n == 0) return TKC_OK;
  cudaStream_t st = g->ctx->stream;
  TKC_LAUNCH(k_validate<<<grid_for(std::max<u64>(g->n, (g->arcs + kArcChunk - 1) / kArcChunk * 32), 256), 256, 0,
                          st>>>(g->off, g->col, g->n, g->arcs, flag));
  TKC_TRY(cudaGetLastError());
  return TKC_OK;
}

// Enqueues the symmetry check of an undirected graph into *flag; only for a
// CSR that passed enqueue_validate (it searches rows for ids).
int enqueue_symmetric(const tkc_graph *g, u32 *flag) {
  if (g->n == 0 || g->directed) return TKC_OK;
  cudaStream_t st = g->ctx->stream;
  TKC_LAUNCH(k_symmetric<<<grid_for((g->arcs + kArcChunk - 1) / kArcChunk * 32, 256), 256, 0, st>>>(
      g->off, g->col, g->n, g->arcs, flag));
  TKC_TRY(cudaGetLastError());
  return TKC_OK;
}

int validate_graph(tkc_graph *g) {
  cudaStream_t st = g->ctx->stream;
  if (g->n == 0) return TKC_OK;
  u32 *flags = nullptr;
  TKC_TRY(cudaMallocAsync(&flags, sizeof(u32), st));
  TKC_TRY(cudaMemsetAsync(flags, 0, sizeof(u32), st));
  TKC_RC(enqueue_validate(g, flags));
  u32 hf = 0;
  TKC_TRY(cudaMemcpyAsync(&hf, flags, sizeof(u32), cudaMemcpyDeviceToHost, st));
  TKC_TRY(cudaStreamSynchronize(st));
  if (hf == 0 && !g->directed) {
    TKC_RC(enqueue_symmetric(g, flags));
    TKC_TRY(cudaMemcpyAsync(&hf, flags, sizeof(u32), cudaMemcpyDeviceToHost, st));
    TKC_TRY(cudaStreamSynchronize(st));
  }
  TKC_TRY(cudaFreeAsync(flags, st));
  if (hf) return TKC_EGRAPH;
  if (!g->directed) {
    g->ioff = g->off;
    g->icol = g->col;
  }
  return TKC_OK;  // a directed graph's in-arc CSR is built on first use (ensure_in_csr)
}

// Fills the in-arc columns of the CSR (off, col) with n vertices into icol,
// given its in-row offsets ioff (rows not sorted: an in-row holds its arcs in
// the order the fill reached them, roughly ascending source id).
static int fill_in_arcs(const u32 *off, const u32 *col, u32 n, u64 arcs, const u32 *ioff, u32 *icol,
                        cudaStream_t st) {
  if (!arcs) return TKC_OK;
  u32 *cursor = nullptr;
  TKC_TRY(cudaMallocAsync(&cursor, (size_t)n * sizeof(u32), st));
  TKC_TRY(cudaMemcpyAsync(cursor, ioff, (size_t)n * sizeof(u32), cudaMemcpyDeviceToDevice, st));
  TKC_LAUNCH(k_in_fill<<<grid_for((arcs + kArcChunk - 1) / kArcChunk * 32, 256), 256, 0, st>>>(
      off, col, n, arcs, cursor, icol));
  TKC_TRY(cudaGetLastError());
  TKC_TRY(cudaFreeAsync(cursor, st));
  return TKC_OK;
}

// Transpose of the CSR (off, col) with n vertices: the in-arc CSR.  *ioff and
// *icol are allocated here.
static int transpose_csr(const u32 *off, const u32 *col, u32 n, u64 arcs, u32 **ioff, u32 **icol,
                         cudaStream_t st) {
  u32 *tmp = nullptr;
  TKC_TRY(cudaMallocAsync(ioff, ((size_t)n + 1) * sizeof(u32), st));
  TKC_TRY(cudaMallocAsync(icol, std::max<size_t>(arcs, 1) * sizeof(u32), st));
  TKC_TRY(cudaMallocAsync(&tmp, (((size_t)n + 1) / kScanTile + 2) * sizeof(u32), st));
  TKC_TRY(cudaMemsetAsync(*ioff, 0, ((size_t)n + 1) * sizeof(u32), st));
  if (arcs) {
    TKC_LAUNCH(k_in_count<<<grid_for(arcs, 256), 256, 0, st>>>(col, arcs, *ioff));
    TKC_TRY(cudaGetLastError());
  }
  TKC_RC(scan_exclusive(*ioff, *ioff, (u64)n + 1, tmp, st));
  TKC_RC(fill_in_arcs(off, col, n, arcs, *ioff, *icol, st));
  TKC_TRY(cudaFreeAsync(tmp, st));
  return TKC_OK;
}

// In-arc CSR of g.
int build_in_csr(const tkc_graph *g) {
  if (g->n == 0) return TKC_OK;
  return transpose_csr(g->off, g->col, g->n, g->arcs, &g->ioff, &g->icol, g->ctx->stream);
}

// The in-arc CSR, built the first time a step needs it (a graph loaded only
// to join a multi-graph launch never does: the union builds its own).
int ensure_in_csr(const tkc_graph *g) {
  if (g->ioff || g->n == 0) return TKC_OK;
  return build_in_csr(g);
}

// ------------------------------------------------------------------ stable LSD radix sort (4-bit digits)

static constexpr int kRsTPB = 256;
static constexpr int kRsRounds = 4;
static constexpr int kRsTile = kRsTPB * kRsRounds;

__global__ void k_rs_count(const u32 *key, u32 n, int shift, u32 *hist, u32 ntiles) {
  __shared__ u32 cnt[16];
  if (threadIdx.x < 16) cnt[threadIdx.x] = 0;
  __syncthreads();
  for (int r = 0; r < kRsRounds; ++r) {
    u64 i = (u64)blockIdx.x * kRsTile + r * kRsTPB + threadIdx.x;
    if (i < n) atomicAdd(&cnt[(key[i] >> shift) & 15u], 1u);
  }
  __syncthreads();
  if (threadIdx.x < 16) hist[threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

// Stable scatter: element order inside a tile is kept by ranking each round's
// 256 elements by (warp, lane) and carrying per-digit running counts.
__global__ void k_rs_scatter(const u32 *key, const u32 *val, u32 *key_out, u32 *val_out, u32 n, int shift,
                             const u32 *hist, u32 ntiles) {
  __shared__ u32 running[16];
  __shared__ u32 wcnt[kRsTPB / 32][16];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (threadIdx.x < 16) running[threadIdx.x] = 0;
  for (int r = 0; r < kRsRounds; ++r) {
    for (int i = threadIdx.x; i < (kRsTPB / 32) * 16; i += kRsTPB) (&wcnt[0][0])[i] = 0;
    __syncthreads();
    u64 idx = (u64)blockIdx.x * kRsTile + r * kRsTPB + threadIdx.x;
    bool valid = idx < n;
    u32 k = valid ? key[idx] : 0u;
    u32 d = valid ? ((k >> shift) & 15u) : 16u;
    u32 peers = __match_any_sync(FULL, d);
    u32 rank = __popc(peers & ((1u << lane) - 1u));
    if (valid && rank == 0) wcnt[wid][d] = __popc(peers);
    __syncthreads();
    if (valid) {
      u32 pos = hist[d * ntiles + blockIdx.x] + running[d] + rank;
      for (int w = 0; w < wid; ++w) pos += wcnt[w][d];
      key_out[pos] = k;
      val_out[pos] = val[idx];
    }
    __syncthreads();
    if (threadIdx.x < 16) {
      u32 s = 0;
      for (int w = 0; w < kRsTPB / 32; ++w) s += wcnt[w][threadIdx.x];
      running[threadIdx.x] += s;
    }
    __syncthreads();
  }
}

// Sorts (key, val) by key ascending, keeping the input order of equal keys.
// Only the low `bits` bits of the keys are looked at.  Result lands in key/val.
static int radix_sort_pairs(u32 *key, u32 *val, u32 n, int bits, cudaStream_t st) {
  if (n <= 1 || bits <= 0) return TKC_OK;
  u32 ntiles = (n + kRsTile - 1) / kRsTile;
  u32 *k2 = nullptr, *v2 = nullptr, *hist = nullptr, *tmp = nullptr;
  size_t hlen = (size_t)16 * ntiles;
  TKC_TRY(cudaMallocAsync(&k2, (size_t)n * sizeof(u32), st));
  TKC_TRY(cudaMallocAsync(&v2, (size_t)n * sizeof(u32), st));
  TKC_TRY(cudaMallocAsync(&hist, hlen * sizeof(u32), st));
  TKC_TRY(cudaMallocAsync(&tmp, (hlen / kScanTile + 2) * sizeof(u32), st));
  u32 *ka = key, *va = val, *kb = k2, *vb = v2;
  int passes = (bits + 3) / 4;
  for (int ps = 0; ps < passes; ++ps) {
    TKC_LAUNCH(k_rs_count<<<ntiles, kRsTPB, 0, st>>>(ka, n, 4 * ps, hist, ntiles));
    TKC_RC(scan_exclusive(hist, hist, hlen, tmp, st));
    TKC_LAUNCH(k_rs_scatter<<<ntiles, kRsTPB, 0, st>>>(ka, va, kb, vb, n, 4 * ps, hist, ntiles));
    TKC_TRY(cudaGetLastError());
    std::swap(ka, kb);
    std::swap(va, vb);
  }
  if (ka != key) {
    TKC_TRY(cudaMemcpyAsync(key, ka, (size_t)n * sizeof(u32), cudaMemcpyDeviceToDevice, st));
    TKC_TRY(cudaMemcpyAsync(val, va, (size_t)n * sizeof(u32), cudaMemcpyDeviceToDevice, st));
  }
  TKC_TRY(cudaFreeAsync(k2, st));
  TKC_TRY(cudaFreeAsync(v2, st));
  TKC_TRY(cudaFreeAsync(hist, st));
  TKC_TRY(cudaFreeAsync(tmp, st));
  return TKC_OK;
}

int scan_exclusive_u32(const u32 *in, u32 *out, u64 len, u32 *tmp, cudaStream_t st) {
  return scan_exclusive(in, out, len, tmp, st);
}

int radix_sort_u32_pairs(u32 *key, u32 *val, u32 n, int bits, cudaStream_t st) {
  return radix_sort_pairs(key, val, n, bits, st);
}

// ------------------------------------------------------------------ computeBoundsDeg

__global__ void k_maxdeg(const u32 *off, u32 n, u32 *maxd, u32 *nzero) {
  u32 m = 0, z = 0;
  for (u32 v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    u32 d = off[v + 1] - off[v];
    m = max(m, d);
    z += d == 0;
  }
  m = __reduce_max_sync(FULL, m);
  z = __reduce_add_sync(FULL, z);
  if ((threadIdx.x & 31) == 0) {
    atomicMax(maxd, m);
    atomicAdd(nzero, z);
  }
}

__global__ void k_deg_keys(const u32 *off, u32 n, u32 maxd, u32 *key, u32 *val) {
  for (u32 v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    key[v] = maxd - (off[v + 1] - off[v]);  // larger degree -> smaller key
    val[v] = v;                              // ids ascending: the sort is stable
  }
}

int ensure_degree_order(tkc_graph *g) {
  if (g->have_order) return TKC_OK;
  cudaStream_t st = g->ctx->stream;
  const u32 n = g->n;
  if (n == 0) {
    g->have_order = true;
    return TKC_OK;
  }
  u32 *keys = nullptr, *stats = nullptr;
  if (!g->deg_order) TKC_TRY(cudaMallocAsync(&g->deg_order, (size_t)n * sizeof(u32), st));
  TKC_TRY(cudaMallocAsync(&keys, (size_t)n * sizeof(u32), st));
  TKC_TRY(cudaMallocAsync(&stats, 2 * sizeof(u32), st));
  TKC_TRY(cudaMemsetAsync(stats, 0, 2 * sizeof(u32), st));
  TKC_LAUNCH(k_maxdeg<<<grid_for(n, 256), 256, 0, st>>>(g->off, n, stats, stats + 1));
  TKC_TRY(cudaGetLastError());
  u32 hs[2];
  TKC_TRY(cudaMemcpyAsync(hs, stats, sizeof(hs), cudaMemcpyDeviceToHost, st));
  TKC_TRY(cudaStreamSynchronize(st));
  TKC_LAUNCH(k_deg_keys<<<grid_for(n, 256), 256, 0, st>>>(g->off, n, hs[0], keys, g->deg_order));
  TKC_TRY(cudaGetLastError());
  int bits = 0;
  while (bits < 32 && (hs[0] >> bits) != 0) ++bits;
  TKC_RC(radix_sort_pairs(keys, g->deg_order, n, bits, st));
  TKC_TRY(cudaFreeAsync(keys, st));
  TKC_TRY(cudaFreeAsync(stats, st));
  g->n_src_deg = n - hs[1];
  g->have_order = true;
  return TKC_OK;
}

// ------------------------------------------------------------------ vertices of out-degree 0

__global__ void k_zero_flag(const u32 *off, u32 n, u32 *flag) {
  for (u32 v = blockIdx.x * blockDim.x + threadIdx.x; v <= n; v += gridDim.x * blockDim.x)
    flag[v] = v < n && off[v + 1] == off[v];
}

__global__ void k_zero_out(const u32 *off, const u32 *pos, u32 n, u32 *out) {
  for (u32 v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    if (off[v + 1] == off[v]) out[pos[v]] = v;
}

// The vertices of out-degree 0 in id order (closeness 0: they end a list
// that fewer than k vertices with reach above 1 fill), by one compaction;
// the degree order's tail holds the same, but needs a sort.
int ensure_zero_list(const tkc_graph *g) {
  if (g->have_zero) return TKC_OK;
  cudaStream_t st = g->ctx->stream;
  const u32 n = g->n;
  if (n == 0) {
    g->have_zero = true;
    return TKC_OK;
  }
  u32 *flag = nullptr, *tmp = nullptr;
  TKC_TRY(cudaMallocAsync(&flag, ((size_t)n + 1) * sizeof(u32), st));
  TKC_TRY(cudaMallocAsync(&tmp, (((size_t)n + 1) / kScanTile + 2) * sizeof(u32), st));
  if (!g->zero_ids) TKC_TRY(cudaMallocAsync(&g->zero_ids, (size_t)n * sizeof(u32), st));
  TKC_LAUNCH(k_zero_flag<<<grid_for((u64)n + 1, 256), 256, 0, st>>>(g->off, n, flag));
  TKC_RC(scan_exclusive(flag, flag, (u64)n + 1, tmp, st));
  TKC_LAUNCH(k_zero_out<<<grid_for(n, 256), 256, 0, st>>>(g->off, flag, n, g->zero_ids));
  TKC_TRY(cudaGetLastError());
  u32 cnt = 0;
  TKC_TRY(cudaMemcpyAsync(&cnt, flag + n, sizeof(u32), cudaMemcpyDeviceToHost, st));
  TKC_TRY(cudaFreeAsync(flag, st));
  TKC_TRY(cudaFreeAsync(tmp, st));
  TKC_TRY(cudaStreamSynchronize(st));
  g->n_zero = cnt;
  g->have_zero = true;
  return TKC_OK;
}

// ------------------------------------------------------------------ bottom-up work order

__global__ void k_bu_keys(const u32 *ioff, u32 n, u32 heavy_in, u32 *key, u32 *val, u32 *count) {
  u32 any = 0, heavy = 0;
  for (u32 v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const u32 indeg = ioff[v + 1] - ioff[v];
    // rows walked by a whole warp: by bit length of the in-degree, longest
    // first; then the other vertices with an in-arc; none last
    key[v] = indeg > heavy_in ? (u32)__clz(indeg) : indeg ? 32u : 33u;
    val[v] = v;  // ids ascending: the sort is stable
    any += indeg != 0;
    heavy += indeg > heavy_in;
  }
  for (int o = 16; o > 0; o >>= 1) {
    any += __shfl_down_sync(0xffffffffu, any, o);
    heavy += __shfl_down_sync(0xffffffffu, heavy, o);
  }
  if ((threadIdx.x & 31) == 0 && any) atomicAdd(&count[0], any);
  if ((threadIdx.x & 31) == 0 && heavy) atomicAdd(&count[1], heavy);
}

// The vertices that bottom-up levels sweep, for the in-arc CSR `ioff`: those
// with an in-arc (no other vertex can be discovered bottom-up; a source is
// seeded directly).  First the n_heavy vertices of more than heavy_in in-arcs,
// whose rows a whole warp walks, longest rows first (bit length of the
// in-degree, then id); then the others by id, so that a warp's 32 entries
// share a few frontier-bitmap words.  Only the order of work depends on it,
// not any result.  *list is allocated here; cnt (device, 2 words) receives
// the number of vertices with an in-arc and of long rows.
static int build_bu_list(const u32 *ioff, u32 n, u32 heavy_in, cudaStream_t st, u32 **list, u32 *cnt) {
  u32 *keys = nullptr, *ids = nullptr;
  TKC_TRY(cudaMallocAsync(&ids, (size_t)n * sizeof(u32), st));
  TKC_TRY(cudaMallocAsync(&keys, (size_t)n * sizeof(u32), st));
  TKC_TRY(cudaMemsetAsync(cnt, 0, 2 * sizeof(u32), st));
  TKC_LAUNCH(k_bu_keys<<<grid_for(n, 256), 256, 0, st>>>(ioff, n, heavy_in, keys, ids, cnt));
  TKC_TRY(cudaGetLastError());
  TKC_RC(radix_sort_pairs(keys, ids, n, 6, st));
  TKC_TRY(cudaFreeAsync(keys, st));
  *list = ids;
  return TKC_OK;
}

// ------------------------------------------------------------------ the search kernel's copy of the graph

// Relabelling key: in-degree, larger first (top is at least every in-degree;
// the stable sort keeps ids ascending among equal in-degrees).
__global__ void k_relabel_keys(const u32 *ioff, u32 n, u32 top, u32 *key, u32 *val) {
  for (u32 v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    key[v] = top - (ioff[v + 1] - ioff[v]);
    val[v] = v;
  }
}

// lab = the inverse of unlab; out_len[i] and in_len[i] = out- and in-degree
// of vertex unlab[i] (in_len may be null).
__global__ void k_relabel_rows(const u32 *unlab, const u32 *off, const u32 *ioff, u32 n, u32 *lab, u32 *out_len,
                               u32 *in_len) {
  for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const u32 v = unlab[i];
    lab[v] = i;
    out_len[i] = off[v + 1] - off[v];
    if (in_len) in_len[i] = ioff[v + 1] - ioff[v];
  }
}

// Row i of the relabelled out-CSR: the out-row of vertex unlab[i], each target
// replaced by its label.  Arcs are dealt to warps in fixed ranges.
__global__ void k_relabel_cols(const u32 *__restrict__ s_off, const u32 *__restrict__ unlab,
                               const u32 *__restrict__ off, const u32 *__restrict__ col,
                               const u32 *__restrict__ lab, u32 n, u64 arcs, u32 *__restrict__ s_col) {
  grid_walk_arcs<true>(s_off, n, arcs, [&](u32 i, u64 a, bool valid, u32 rs) {
    if (valid) s_col[a] = lab[col[off[unlab[i]] + (u32)(a - rs)]];
  });
}

void free_search_csr(const tkc_graph *g) {
  cudaStream_t st = g->ctx->stream;  // stream-ordered: after the work that used them
  if (g->s_ready) {  // a copy still being built on the helper stream
    cudaStreamWaitEvent(st, g->s_ready, 0);
    cudaEventDestroy(g->s_ready);
    g->s_ready = nullptr;
  }
  if (g->s_ioff && g->s_ioff != g->s_off) cudaFreeAsync(g->s_ioff, st);
  if (g->s_icol && g->s_icol != g->s_col) cudaFreeAsync(g->s_icol, st);
  void *ptrs[] = {g->s_off, g->s_col, g->s_lab, g->s_unlab, g->bu_list, g->s_cnt};
  for (void *q : ptrs)
    if (q) cudaFreeAsync(q, st);
  g->s_off = g->s_col = g->s_ioff = g->s_icol = g->s_lab = g->s_unlab = g->s_cnt = nullptr;
  g->bu_list = nullptr;
  g->n_bu = g->n_bu_heavy = 0;
  g->s_mode = -1;
}

// The graph as the search kernel walks it (ensure_search_csr below).  Plain: the graph itself.
// Relabelled: vertex i of the copy is vertex unlab[i] of the graph, the
// vertices taken by in-degree, largest first.  Bottom-up levels gather the
// frontier rows of in-neighbours, and in-neighbours are mostly vertices of
// large degree; with those first, the rows and frontier bits that levels
// touch most sit together in a few megabytes that stay in L2 (R-MAT 22,
// NBCut: search kernel 51 -> 35 ms).  The copy's in-rows come out in
// ascending label order, largest in-degree first, so that a walk meets the
// likely frontier vertices early.  An undirected graph's copy serves both
// directions (its transpose is itself).  Every result is the same: sources,
// slots, ties and outputs keep the graph's own ids; only the search's rows
// are indexed by labels.
// The labelled copy and its bottom-up list, enqueued on `st` without a host
// wait (the list's counts land in g->s_cnt).  The graph's in-arc CSR exists.
static int build_labelled_copy(const tkc_graph *g, cudaStream_t st) {
  const u32 n = g->n;
  u32 *keys = nullptr, *gcol = nullptr, *tmp = nullptr;
  TKC_TRY(cudaMallocAsync(&g->s_cnt, 2 * sizeof(u32), st));
  TKC_TRY(cudaMallocAsync(&g->s_unlab, (size_t)n * sizeof(u32), st));
  TKC_TRY(cudaMallocAsync(&g->s_lab, (size_t)n * sizeof(u32), st));
  TKC_TRY(cudaMallocAsync(&g->s_off, ((size_t)n + 1) * sizeof(u32), st));
  TKC_TRY(cudaMallocAsync(&g->s_ioff, ((size_t)n + 1) * sizeof(u32), st));
  TKC_TRY(cudaMallocAsync(&g->s_icol, std::max<size_t>(g->arcs, 1) * sizeof(u32), st));
  TKC_TRY(cudaMallocAsync(&gcol, std::max<size_t>(g->arcs, 1) * sizeof(u32), st));
  TKC_TRY(cudaMallocAsync(&keys, (size_t)n * sizeof(u32), st));
  TKC_TRY(cudaMallocAsync(&tmp, (((size_t)n + 1) / kScanTile + 2) * sizeof(u32), st));
  // key n - indegree (in [1, n]: no vertex has n in-arcs), ascending
  TKC_LAUNCH(k_relabel_keys<<<grid_for(n, 256), 256, 0, st>>>(g->ioff, n, n, keys, g->s_unlab));
  TKC_TRY(cudaGetLastError());
  int bits = 0;
  while (bits < 32 && (n >> bits) != 0) ++bits;
  TKC_RC(radix_sort_pairs(keys, g->s_unlab, n, bits, st));
  // the copy's row lengths are the graph's degrees in label order: its
  // in-rows need no counting pass
  TKC_TRY(cudaMemsetAsync(g->s_off + n, 0, sizeof(u32), st));
  TKC_TRY(cudaMemsetAsync(g->s_ioff + n, 0, sizeof(u32), st));
  TKC_LAUNCH(k_relabel_rows<<<grid_for(n, 256), 256, 0, st>>>(g->s_unlab, g->off, g->ioff, n, g->s_lab, g->s_off,
                                                              g->s_ioff));
  TKC_TRY(cudaGetLastError());
  TKC_RC(scan_exclusive(g->s_off, g->s_off, (u64)n + 1, tmp, st));
  TKC_RC(scan_exclusive(g->s_ioff, g->s_ioff, (u64)n + 1, tmp, st));
  if (g->arcs) {
    TKC_LAUNCH(k_relabel_cols<<<grid_for((g->arcs + kArcChunk - 1) / kArcChunk * 32, 256), 256, 0, st>>>(
        g->s_off, g->s_unlab, g->off, g->col, g->s_lab, n, g->arcs, gcol));
    TKC_TRY(cudaGetLastError());
  }
  // in-rows by transposition, so that each runs in ascending label order
  TKC_RC(fill_in_arcs(g->s_off, gcol, n, g->arcs, g->s_ioff, g->s_icol, st));
  if (g->directed) {
    g->s_col = gcol;
  } else {
    TKC_TRY(cudaFreeAsync(g->s_off, st));
    TKC_TRY(cudaFreeAsync(gcol, st));
    g->s_off = g->s_ioff;
    g->s_col = g->s_icol;
  }
  TKC_TRY(cudaFreeAsync(keys, st));
  TKC_TRY(cudaFreeAsync(tmp, st));
  g->heavy_in = kHeavyInLabelled;
  return build_bu_list(g->s_ioff, n, g->heavy_in, st, &g->bu_list, g->s_cnt);
}

// Reads the bottom-up list's counts once the work that writes them is done.
static int read_bu_counts(const tkc_graph *g) {
  cudaStream_t st = g->ctx->stream;
  u32 c[2] = {0, 0};
  TKC_TRY(cudaMemcpyAsync(c, g->s_cnt, sizeof(c), cudaMemcpyDeviceToHost, st));
  TKC_TRY(cudaStreamSynchronize(st));
  g->n_bu = c[0];
  g->n_bu_heavy = c[1];
  return TKC_OK;
}

// A copy started on the helper stream: the context's stream waits for it.
static int finish_started_copy(const tkc_graph *g) {
  if (!g->s_ready) return TKC_OK;
  TKC_TRY(cudaStreamWaitEvent(g->ctx->stream, g->s_ready, 0));
  TKC_TRY(cudaEventDestroy(g->s_ready));
  g->s_ready = nullptr;
  return read_bu_counts(g);
}

int ensure_search_csr(const tkc_graph *g, bool relabel) {
  TKC_RC(finish_started_copy(g));
  const int want = relabel ? 1 : 0;
  if (g->s_mode == want || g->n == 0) return TKC_OK;
  TKC_RC(ensure_in_csr(g));
  free_search_csr(g);  // the other labelling's copy, or what a failed build left
  cudaStream_t st = g->ctx->stream;
  if (!relabel) {
    g->heavy_in = kHeavyIn;
    TKC_TRY(cudaMallocAsync(&g->s_cnt, 2 * sizeof(u32), st));
    TKC_RC(build_bu_list(g->ioff, g->n, g->heavy_in, st, &g->bu_list, g->s_cnt));
  } else {
    TKC_RC(build_labelled_copy(g, st));
  }
  TKC_RC(read_bu_counts(g));
  g->s_mode = want;
  return TKC_OK;
}

// Starts the labelled copy on the context's helper stream, so that it is
// built while the context's stream runs the preprocessing (degree order,
// reach bounds, NB bounds) with its host waits: it needs only the CSR and
// the in-arc CSR.  ensure_search_csr completes it.
int start_search_csr(const tkc_graph *g) {
  if (g->s_mode == 1 || g->s_ready || g->n == 0) return TKC_OK;
  TKC_RC(ensure_in_csr(g));
  free_search_csr(g);
  tkc_ctx *ctx = g->ctx;
  if (!ctx->aux) {
    TKC_TRY(cudaStreamCreateWithFlags(&ctx->aux, cudaStreamNonBlocking));
    TKC_TRY(cudaEventCreateWithFlags(&ctx->aux_in, cudaEventDisableTiming));
  }
  TKC_TRY(cudaEventRecord(ctx->aux_in, ctx->stream));
  TKC_TRY(cudaStreamWaitEvent(ctx->aux, ctx->aux_in, 0));
  TKC_RC(build_labelled_copy(g, ctx->aux));
  cudaEvent_t ready = nullptr;
  TKC_TRY(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
  TKC_TRY(cudaEventRecord(ready, ctx->aux));
  g->s_ready = ready;
  g->s_mode = 1;
  return TKC_OK;
}

// Keeps the vertices of out-degree >= 1 of a full order, in order.
__global__ void k_flag_src(const u32 *order, const u32 *off, u32 n, u32 *flag) {
  for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    u32 v = order[i];
    flag[i] = off[v + 1] > off[v];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) flag[n] = 0;
}

__global__ void k_compact(const u32 *order, const u32 *pos, u32 n, u32 *out) {
  for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    if (pos[i + 1] != pos[i]) out[pos[i]] = order[i];
}

int filter_order(tkc_graph *g, const u32 *d_order_all, u32 *d_out, u32 *count) {
  cudaStream_t st = g->ctx->stream;
  const u32 n = g->n;
  u32 *pos = nullptr, *tmp = nullptr;
  TKC_TRY(cudaMallocAsync(&pos, ((size_t)n + 1) * sizeof(u32), st));
  TKC_TRY(cudaMallocAsync(&tmp, (((size_t)n + 1) / kScanTile + 2) * sizeof(u32), st));
  TKC_LAUNCH(k_flag_src<<<grid_for(n, 256), 256, 0, st>>>(d_order_all, g->off, n, pos));
  TKC_RC(scan_exclusive(pos, pos, (u64)n + 1, tmp, st));
  TKC_LAUNCH(k_compact<<<grid_for(n, 256), 256, 0, st>>>(d_order_all, pos, n, d_out));
  TKC_TRY(cudaGetLastError());
  TKC_TRY(cudaMemcpyAsync(count, pos + n, sizeof(u32), cudaMemcpyDeviceToHost, st));
  TKC_TRY(cudaStreamSynchronize(st));
  TKC_TRY(cudaFreeAsync(pos, st));
  TKC_TRY(cudaFreeAsync(tmp, st));
  return TKC_OK;
}

// ------------------------------------------------------------------ reach: undirected components

__device__ __forceinline__ u32 cc_root(const u32 *parent, u32 x) {
  u32 p = parent[x];
  while (p != x) {
    x = p;
    p = parent[x];
  }
  return x;
}

__global__ void k_cc_init(u32 *parent, u32 n) {
  for (u32 v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) parent[v] = v;
}

// Hooks the larger root of every edge's endpoints under the smaller one.
// parent[x] <= x always holds, so pointers only decrease and no cycle forms.
__global__ void k_cc_hook(const u32 *off, const u32 *col, u32 n, u32 *parent, u32 *changed) {
  int lane = threadIdx.x & 31;
  u32 warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  u32 nw = (gridDim.x * blockDim.x) >> 5;
  u32 ch = 0;
  for (u32 u = warp; u < n; u += nw) {
    for (u32 i = off[u] + lane; i < off[u + 1]; i += 32) {
      u32 v = col[i];
      if (v < u) continue;
      u32 ru = cc_root(parent, u), rv = cc_root(parent, v);
      if (ru != rv) {
        u32 hi = max(ru, rv), lo = min(ru, rv);
        atomicMin(&parent[hi], lo);
        ch = 1;
      }
    }
  }
  ch = __reduce_or_sync(FULL, ch);
  if (lane == 0 && ch) *changed = 1;
}

__global__ void k_cc_compress(u32 *parent, u32 n) {
  for (u32 v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    parent[v] = cc_root(parent, v);
}

__global__ void k_cc_size(const u32 *parent, u32 n, u32 *size) {
  for (u32 v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    atomicAdd(&size[parent[v]], 1u);
}

__global__ void k_cc_out(const u32 *parent, const u32 *size, u32 n, u32 *alpha, u32 *omega, u32 *scc_size) {
  for (u32 v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    u32 s = size[parent[v]];
    alpha[v] = s;
    omega[v] = s;
    scc_size[v] = s;
  }
}

static int reach_undirected(tkc_graph *g) {
  cudaStream_t st = g->ctx->stream;
  const u32 n = g->n;
  u32 *parent = nullptr, *size = nullptr, *changed = nullptr;
  TKC_TRY(cudaMallocAsync(&parent, (size_t)n * sizeof(u32), st));
  TKC_TRY(cudaMallocAsync(&size, (size_t)n * sizeof(u32), st));
  TKC_TRY(cudaMallocAsync(&changed, sizeof(u32), st));
  TKC_LAUNCH(k_cc_init<<<grid_for(n, 256), 256, 0, st>>>(parent, n));
  for (int it = 0;; ++it) {
    if (it > 4096) return TKC_ETIMEOUT;
    TKC_TRY(cudaMemsetAsync(changed, 0, sizeof(u32), st));
    TKC_LAUNCH(k_cc_hook<<<grid_for((u64)n * 32, 256), 256, 0, st>>>(g->off, g->col, n, parent, changed));
    TKC_LAUNCH(k_cc_compress<<<grid_for(n, 256), 256, 0, st>>>(parent, n));
    TKC_TRY(cudaGetLastError());
    u32 hc = 0;
    TKC_TRY(cudaMemcpyAsync(&hc, changed, sizeof(u32), cudaMemcpyDeviceToHost, st));
    TKC_TRY(cudaStreamSynchronize(st));
    if (!hc) break;
  }
  TKC_TRY(cudaMemsetAsync(size, 0, (size_t)n * sizeof(u32), st));
  TKC_LAUNCH(k_cc_size<<<grid_for(n, 256), 256, 0, st>>>(parent, n, size));
  TKC_LAUNCH(k_cc_out<<<grid_for(n, 256), 256, 0, st>>>(parent, size, n, g->alpha, g->omega, g->scc_size));
  TKC_TRY(cudaGetLastError());
  TKC_TRY(cudaMemcpyAsync(g->comp, parent, (size_t)n * sizeof(u32), cudaMemcpyDeviceToDevice, st));
  TKC_TRY(cudaFreeAsync(parent, st));
  TKC_TRY(cudaFreeAsync(size, st));
  TKC_TRY(cudaFreeAsync(changed, st));
  return TKC_OK;
}

// ------------------------------------------------------------------ reach: directed

// SCCs and Algorithm 6 run on the device (tkc_scc.cu).
int reach_directed_gpu(tkc_graph *g, const u32 *gid, u32 ng);

int ensure_reach_bounds(tkc_graph *g, const u32 *gid, u32 ng) {
  if (g->have_reach) return TKC_OK;
  cudaStream_t st = g->ctx->stream;
  if (g->n == 0) {
    g->have_reach = true;
    return TKC_OK;
  }
  if (!g->alpha) TKC_TRY(cudaMallocAsync(&g->alpha, (size_t)g->n * sizeof(u32), st));
  if (!g->omega) TKC_TRY(cudaMallocAsync(&g->omega, (size_t)g->n * sizeof(u32), st));
  if (!g->scc_size) TKC_TRY(cudaMallocAsync(&g->scc_size, (size_t)g->n * sizeof(u32), st));
  if (!g->comp) TKC_TRY(cudaMallocAsync(&g->comp, (size_t)g->n * sizeof(u32), st));
  TKC_RC(ensure_in_csr(g));
  TKC_RC(g->directed ? reach_directed_gpu(g, gid, ng) : reach_undirected(g));
  g->have_reach = true;
  return TKC_OK;
}

}  // namespace tkc
