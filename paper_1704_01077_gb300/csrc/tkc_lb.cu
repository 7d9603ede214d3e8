// updateBoundsLB (Section 7, Algorithm 5; Eq. 4 for undirected graphs, Eq. 5
// for directed ones): after a complete BFS from s, every vertex w whose reach
// equals s's (its component; its SCC if directed) has
//   S(w) >= L(l(w)) - outdeg(w),
//   L(i) = 2 sum_{|j-i| <= 1} g_j + sum_{|j-i| > 1} g_j |j-i| - 2     (undirected)
//   L(i) = 2 sum_{j-i <= 1} g_j  + sum_{j-i > 1} g_j (j-i) - 2        (directed)
// with g_j the size of level j of the BFS from s (g_0 = 1: s itself).
//
// Algorithm 1 runs in rounds: the B unsearched vertices of smallest bound key
// (ties by their position in the initial order) are searched completely by the
// persistent kernel, which records for every vertex the level at which each
// slot found it and each slot's level sizes; then one thread per source turns
// its level sizes into L(i) (O(depth), prefix sums), and one thread per vertex
// raises the vertex's bound with every slot that found it.  The host loop ends
// when the head of the order has a key above the k-th farness.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "tkc_internal.cuh"

namespace tkc {

typedef uint32_t u32;
typedef unsigned long long u64;
typedef unsigned __int128 u128;
static constexpr unsigned FULL = 0xffffffffu;
constexpr int kKeyFrac = 46;  // key = floor(S * 2^46 / (r-1)^2), as the NB order keys

int radix_sort_u32_pairs(u32 *key, u32 *val, u32 n, int bits, cudaStream_t st);
int scan_exclusive_u32(const u32 *in, u32 *out, u64 len, u32 *tmp, cudaStream_t st);

namespace {

unsigned grid_of(u64 work, unsigned tpb = 256, unsigned cap = 152 * 16) {
  u64 b = (work + tpb - 1) / tpb;
  return (unsigned)std::max<u64>(1, std::min<u64>(b, cap));
}

// flag[i] = order0[i] is still a candidate (not searched, out-degree >= 1)
__global__ void k_lb_flags(const u32 *order0, u32 n0, const u32 *off, const uint8_t *done, u32 *flag) {
  for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < n0; i += gridDim.x * blockDim.x) {
    const u32 v = order0[i];
    flag[i] = !done[v] && off[v + 1] > off[v];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) flag[n0] = 0;
}

__global__ void k_lb_compact(const u32 *order0, const u32 *pos, u32 n0, u32 *out) {
  for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < n0; i += gridDim.x * blockDim.x)
    if (pos[i + 1] != pos[i]) out[pos[i]] = order0[i];
}

__global__ void k_lb_key_lo(u32 m, const u32 *cand, const u64 *key, u32 *lo, u64 *maxkey) {
  u64 mx = 0;
  for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    const u64 kv = key[cand[i]];
    lo[i] = (u32)kv;
    mx = max(mx, kv);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, (u64)__shfl_xor_sync(FULL, mx, o));
  if ((threadIdx.x & 31) == 0 && mx) atomicMax(maxkey, mx);
}

__global__ void k_lb_key_hi(u32 m, const u32 *cand, const u64 *key, u32 *hi) {
  for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) hi[i] = (u32)(key[cand[i]] >> 32);
}

// One thread per source: L(i) for every level i of its BFS, from the level
// sizes with running prefix sums G(j) = sum_{t<=j} g_t, M(j) = sum_{t<=j} t g_t:
//   sum_{j <= i-2} g_j (i-j)  = i G(i-2) - M(i-2)
//   sum_{j >= i+2} g_j (j-i)  = (M_all - M(i+1)) - i (G_all - G(i+1))
__global__ void k_lb_table(u32 nsrc, u32 *hist, u32 cap, const u32 *depth, int directed, u64 *Ltab) {
  const u32 s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nsrc) return;
  u32 *g = hist + (size_t)s * cap;
  u64 *L = Ltab + (size_t)s * cap;
  const u32 D = depth[s];
  g[0] = 1;  // the source
  u64 Gall = 0, Mall = 0;
  for (u32 j = 0; j <= D; ++j) {
    Gall += g[j];
    Mall += (u64)j * g[j];
  }
  // G(i-2), M(i-2) and G(i+1), M(i+1) advance with i
  u64 Glo = 0, Mlo = 0;         // up to i-2
  u64 Ghi = g[0], Mhi = 0;      // up to i+1, start at i = 0: levels 0 and 1
  if (D >= 1) {
    Ghi += g[1];
    Mhi += g[1];
  }
  for (u32 i = 0; i <= D; ++i) {
    if (i >= 2) {
      Glo += g[i - 2];
      Mlo += (u64)(i - 2) * g[i - 2];
    }
    const u64 above = (Mall - Mhi) - (u64)i * (Gall - Ghi);
    u64 v;
    if (directed) {
      v = 2 * Ghi + above - 2;
    } else {
      const u64 near = (i >= 1 ? g[i - 1] : 0) + g[i] + (i + 1 <= D ? g[i + 1] : 0);
      const u64 below = (u64)i * Glo - Mlo;
      v = 2 * near + below + above - 2;
    }
    L[i] = v;
    if (i + 2 <= D) {
      Ghi += g[i + 2];
      Mhi += (u64)(i + 2) * g[i + 2];
    }
  }
}

// Depth of each slot's BFS: its deepest non-empty level.
__global__ void k_lb_depth(u32 nsrc, const u32 *hist, u32 cap, u32 *depth) {
  const u32 s = blockIdx.x;
  if (s >= nsrc) return;
  u32 best = 0;
  for (u32 j = 1 + threadIdx.x; j < cap; j += blockDim.x)
    if (hist[(size_t)s * cap + j]) best = max(best, j);
  best = __reduce_max_sync(FULL, best);
  __shared__ u32 wbest[32];
  if ((threadIdx.x & 31) == 0) wbest[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x == 0) {
    u32 b = 0;
    for (u32 i = 0; i < blockDim.x / 32; ++i) b = max(b, wbest[i]);
    depth[s] = b;
  }
}

// One thread per vertex: raise its bound with every slot that found it, then
// reset its level row for the next round.
__global__ void k_lb_update(u32 n, u32 B, u32 nsrc, uint16_t *lvl, const u32 *srcs, const u32 *comp, const u32 *off,
                            const u64 *Ltab, u32 cap, const u32 *res_r, u64 *bS, u32 *bR, u64 *key) {
  for (u32 w = blockIdx.x * blockDim.x + threadIdx.x; w < n; w += gridDim.x * blockDim.x) {
    uint16_t *row = lvl + (size_t)w * B;
    const u64 od = off[w + 1] - off[w];
    const u32 cw = comp[w];
    u64 S = bS[w], r = bR[w];
    bool changed = false;
    for (u32 s = 0; s < nsrc; ++s) {
      const uint16_t l = row[s];
      if (l == 0xffffu) continue;
      row[s] = 0xffffu;
      const u32 src = srcs[s];
      if (src == 0xffffffffu || src == w || comp[src] != cw || od == 0) continue;
      const u64 cS = Ltab[(size_t)s * cap + l] - od;
      const u64 cr = res_r[src];
      // keep the larger of cS/(cr-1)^2 and S/(r-1)^2 (r <= 1: no bound yet)
      if (cr <= 1) continue;
      if (r <= 1 || (u128)cS * (u128)((r - 1) * (r - 1)) > (u128)S * (u128)((cr - 1) * (cr - 1))) {
        S = cS;
        r = cr;
        changed = true;
      }
    }
    if (changed) {
      bS[w] = S;
      bR[w] = (u32)r;
      key[w] = (u64)(((u128)S << kKeyFrac) / (u128)((r - 1) * (r - 1)));
    }
  }
}

__global__ void k_lb_gather(u32 cnt, const u32 *cand, const u64 *key, u64 *out) {
  const u32 i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < cnt) out[i] = key[cand[i]];
}

__global__ void k_lb_done(u32 nsrc, const u32 *srcs, uint8_t *done) {
  const u32 i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nsrc && srcs[i] != 0xffffffffu) done[srcs[i]] = 1;
}

__global__ void k_lb_init(u32 n, const u64 *S0, const u32 *r0, const u64 *key0, u64 *bS, u32 *bR, u64 *key,
                          uint8_t *done) {
  for (u32 v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    bS[v] = S0 ? S0[v] : 0;
    bR[v] = S0 ? r0[v] : 2;  // bound 0
    key[v] = S0 ? key0[v] : 0;
    done[v] = 0;
  }
}

}  // namespace

int lb_init(tkc_graph *g, const u64 *S0, const u32 *r0, const u64 *key0, u64 *bS, u32 *bR, u64 *key,
            uint8_t *done) {
  cudaStream_t st = g->ctx->stream;
  TKC_LAUNCH(k_lb_init<<<grid_of(g->n), 256, 0, st>>>(g->n, S0, r0, key0, bS, bR, key, done));
  TKC_TRY(cudaGetLastError());
  return TKC_OK;
}

// The candidates (initial order, not searched, out-degree >= 1) sorted by
// (key, position in the initial order): a stable compaction, then stable
// radix passes over the low and the high 32 key bits.  Writes *count of them
// to cand (device); synchronises the stream.
int lb_sorted_candidates(tkc_graph *g, const u32 *order0, u32 n0, const uint8_t *done, const u64 *key, u32 *cand,
                         u32 *count, u32 *scratch_pos, u32 *scratch_tmp, u32 *scratch_lo, u64 *scratch_max) {
  cudaStream_t st = g->ctx->stream;
  *count = 0;
  if (n0 == 0) return TKC_OK;
  TKC_LAUNCH(k_lb_flags<<<grid_of(n0), 256, 0, st>>>(order0, n0, g->off, done, scratch_pos));
  TKC_RC(scan_exclusive_u32(scratch_pos, scratch_pos, (u64)n0 + 1, scratch_tmp, st));
  TKC_LAUNCH(k_lb_compact<<<grid_of(n0), 256, 0, st>>>(order0, scratch_pos, n0, cand));
  u32 m = 0;
  TKC_TRY(cudaMemcpyAsync(&m, scratch_pos + n0, sizeof(u32), cudaMemcpyDeviceToHost, st));
  TKC_TRY(cudaMemsetAsync(scratch_max, 0, sizeof(u64), st));
  TKC_TRY(cudaStreamSynchronize(st));
  if (m) {
    TKC_LAUNCH(k_lb_key_lo<<<grid_of(m), 256, 0, st>>>(m, cand, key, scratch_lo, scratch_max));
    u64 mk = 0;
    TKC_TRY(cudaMemcpyAsync(&mk, scratch_max, sizeof(u64), cudaMemcpyDeviceToHost, st));
    TKC_TRY(cudaStreamSynchronize(st));
    int bits = 0;
    while (bits < 64 && (mk >> bits) != 0) ++bits;
    if (bits <= 32) {
      TKC_RC(radix_sort_u32_pairs(scratch_lo, cand, m, bits, st));
    } else {
      TKC_RC(radix_sort_u32_pairs(scratch_lo, cand, m, 32, st));
      TKC_LAUNCH(k_lb_key_hi<<<grid_of(m), 256, 0, st>>>(m, cand, key, scratch_lo));
      TKC_RC(radix_sort_u32_pairs(scratch_lo, cand, m, bits - 32, st));
    }
  }
  TKC_TRY(cudaStreamSynchronize(st));
  *count = m;
  return TKC_OK;
}

int lb_gather_keys(tkc_graph *g, u32 cnt, const u32 *cand, const u64 *key, u64 *out) {
  TKC_LAUNCH(k_lb_gather<<<(cnt + 255) / 256, 256, 0, g->ctx->stream>>>(cnt, cand, key, out));
  TKC_TRY(cudaGetLastError());
  return TKC_OK;
}

// After a round of complete searches from srcs[0..nsrc) (0xffffffff: slot
// unused): level bounds per source, then every vertex's bound.  lvl rows (B =
// row length) are reset to 0xffff.
int lb_update(tkc_graph *g, u32 B, u32 nsrc, const u32 *srcs, uint16_t *lvl, u32 *hist, u32 cap, u32 *depth,
              u64 *Ltab, const u32 *res_r, u64 *bS, u32 *bR, u64 *key, uint8_t *done) {
  cudaStream_t st = g->ctx->stream;
  TKC_LAUNCH(k_lb_depth<<<nsrc, 256, 0, st>>>(nsrc, hist, cap, depth));
  TKC_LAUNCH(k_lb_table<<<(nsrc + 63) / 64, 64, 0, st>>>(nsrc, hist, cap, depth, g->directed, Ltab));
  TKC_LAUNCH(k_lb_update<<<grid_of(g->n), 256, 0, st>>>(g->n, B, nsrc, lvl, srcs, g->comp, g->off, Ltab, cap, res_r,
                                                         bS, bR, key));
  TKC_LAUNCH(k_lb_done<<<(nsrc + 255) / 256, 256, 0, st>>>(nsrc, srcs, done));
  TKC_TRY(cudaGetLastError());
  return TKC_OK;
}

}  // namespace tkc
