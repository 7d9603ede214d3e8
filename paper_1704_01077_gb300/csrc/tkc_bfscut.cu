// Batched BFSCut: Algorithm 1 with updateBoundsBFSCut (Algorithm 4) for up to
// 512 sources at once, as one persistent cooperative kernel per call.
//
// Sources of one batch occupy bit "slots" of a per-vertex row of W 64-bit
// words: seen (visited by slot b), F (frontier of slot b) and N (next level of
// slot b, top-down only).  One loop iteration advances every active slot by one
// BFS level:
//   phase A  expand: top-down over the frontier list (atomic OR into N) or
//            bottom-up over all vertices (OR of in-neighbours' F rows, stopping
//            once every missing bit is found), direction chosen per level;
//   phase B  finalize: new = N, seen |= new, F' = new, per-slot level sizes and
//            out-degree sums by warp bit-transpose + popcount; old F rows cleared;
//   epilogue (last block to reach the grid barrier): per-slot S, n_d, gamma,
//            merge of finished searches into the top-k, x = k-th farness, the
//            BFSCut test of the Section 6 lemma at r in [alpha', omega] (Section 8.2), and
//            the next step's direction.
// When every slot of a batch is done, a clear step zeroes the rows the batch
// touched and the epilogue seeds the next batch from the source order,
// abandoning sources already at level 0 when their bound exceeds x.
//
// Every grid-wide wait is bounded by a clock64 budget; on expiry the kernel
// records TKC_ETIMEOUT and every block returns.
#include <cuda_runtime.h>
#include <stdint.h>

#include "tkc_internal.cuh"

namespace tkc {

typedef unsigned long long u64;
typedef uint32_t u32;
typedef unsigned __int128 u128;

static constexpr unsigned FULL = 0xffffffffu;
static constexpr int kPackShift = 38;
static constexpr u64 kArcMask = (1ull << kPackShift) - 1;
static constexpr int kTopMax = TKC_MAX_K;

// ------------------------------------------------------------------ memory ordering

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(unsigned *p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_volatile_i32(const int *p) { return *(volatile const int *)p; }

// Barrier over the `nblocks` blocks of one team (all co-resident: the launch
// is cooperative).  The last block to arrive runs `epi` (whole block) before
// releasing the others.  Returns false when the run must stop: an error
// recorded by this team or any other, including a timed-out wait.
template <typename Epi>
__device__ __forceinline__ bool team_sync(Ctl *ctl, Shared *sh, unsigned nblocks, uint64_t timeout, Epi epi) {
  __shared__ int s_last;
  __shared__ unsigned s_gen;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned gen = ld_acquire_u32(&ctl->bar_gen);
    s_gen = gen;
    __threadfence();
    unsigned arrived = atomicAdd(&ctl->bar_count, 1u) + 1u;
    s_last = (arrived == nblocks);
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    epi();
    __syncthreads();
    if (threadIdx.x == 0) {
      ctl->bar_count = 0;
      __threadfence();
      st_release_u32(&ctl->bar_gen, s_gen + 1u);
    }
  } else if (threadIdx.x == 0) {
    long long t0 = clock64();
    unsigned ns = 32;
    while (ld_acquire_u32(&ctl->bar_gen) == s_gen) {
      if (ld_volatile_i32(&ctl->err) != 0 || ld_volatile_i32(&sh->err) != 0) break;
      if ((uint64_t)(clock64() - t0) > timeout) {
        atomicCAS(&ctl->err, 0, TKC_ETIMEOUT);
        atomicCAS(&sh->err, 0, TKC_ETIMEOUT);
        atomicCAS(&ctl->err_where, 0, 1);
        break;
      }
      __nanosleep(ns);
      if (ns < 256) ns <<= 1;
    }
    __threadfence();
  }
  __syncthreads();
  return ld_volatile_i32(&ctl->err) == 0 && ld_volatile_i32(&sh->err) == 0;
}

// ------------------------------------------------------------------ exact arithmetic

// The Section 6 lemma at radius d, evaluated at reach r >= nd:
//   L = S_d + (d+1)(r - n_d) + max(0, r - n_d - g)
__device__ __forceinline__ u64 cut_sum(u64 Sd, u64 d, u64 nd, u64 g, u64 r) {
  u64 rem = r - nd;
  return Sd + (d + 1) * rem + (rem > g ? rem - g : 0);
}

// a/(ra-1)^2 < b/(rb-1)^2 for ra, rb >= 2
__device__ __forceinline__ bool ratio_less(u64 a, u64 ra, u64 b, u64 rb) {
  return (u128)a * (u128)((rb - 1) * (rb - 1)) < (u128)b * (u128)((ra - 1) * (ra - 1));
}

// True when the farness lower bound exceeds x = (Sx, rx) strictly for every
// r in [max(lo, nd), hi].  The bound divided by (r-1)^2 is linear-over-square
// on [lo', kink] and on [kink, hi] (kink = nd + g), so by the Section 8 lemma
// on such bounds its minimum over the interval is at lo', hi or the kink.
__device__ bool cut_exceeds(u64 Sd, u64 d, u64 nd, u64 g, u64 lo, u64 hi, u64 Sx, u64 rx) {
  if (lo < nd) lo = nd;
  if (hi < lo) hi = lo;
  u64 kink = nd + g;
  u64 cand[3] = {lo, hi, kink};
  int nc = (kink > lo && kink < hi) ? 3 : 2;
  for (int i = 0; i < nc; ++i) {
    u64 r = cand[i];
    if (r <= 1) continue;  // r = 1 is farness +inf, above any finite x
    u64 L = cut_sum(Sd, d, nd, g, r);
    // not (L/(r-1)^2 > Sx/(rx-1)^2)  ->  keep searching
    if (!ratio_less(Sx, rx, L, r)) return false;
  }
  return true;
}

// NBCut's stop (Algorithm 1 with computeBoundsNB): the source's order key
// floor(2^46 L') with L' <= S/(r-1)^2 exceeds x = Sx/(rx-1)^2 strictly.  The
// order is sorted by key, so every later source of the graph exceeds x too.
__device__ __forceinline__ bool nb_exceeds(u64 key, u64 Sx, u64 rx) {
  return (u128)key * (u128)((rx - 1) * (rx - 1)) > ((u128)Sx << 46);
}

// List order.  Closeness: (S, r, id) by farness ascending, then id ascending
// (r >= 2 here).  Harmonic: the key is the FP64 bit pattern of h >= 0, which
// orders like the value; larger h first, then smaller id.
__device__ __forceinline__ bool entry_less(bool harmonic, u64 Sa, u32 ra, u32 ia, u64 Sb, u32 rb, u32 ib) {
  if (harmonic) return Sa != Sb ? Sa > Sb : ia < ib;
  u128 lhs = (u128)Sa * (u128)((u64)(rb - 1) * (u64)(rb - 1));
  u128 rhs = (u128)Sb * (u128)((u64)(ra - 1) * (u64)(ra - 1));
  if (lhs != rhs) return lhs < rhs;
  return ia < ib;
}

// Harmonic centrality (the paper's closing generalisation to sums of f(d) with
// f = 1/d): after level d, the vertices not yet found lie at distance >= d+1,
// at most g of them at d+1, and there are at most omega - n_d of them, so
//   h <= U = H_d + min(g, w)/(d+1) + max(0, w - g)/(d+2),  w = omega - n_d.
// The search is abandoned when fl(U * (1 + 2^-20)) < x: the margin covers the
// rounding of H_d and U and of the FP64 h it is compared with (depths < 2^32).
constexpr double kHMargin = 1.0 + 1.0 / 1048576.0;


// Bottom-up walks, batches of at most 256 bits: in-arcs a lane takes per step
// when it walks a short in-row alone (U), and per lane per step when the warp
// walks a long one (HU).  Measured on R-MAT 22, NBCut: 4 and 4 beat 2 and 8
// either way (2 to 5% slower).
#ifndef TKC_BU_U
#define TKC_BU_U 4
#endif
#ifndef TKC_BU_HU
#define TKC_BU_HU 4
#endif

// Threads per block of the search kernel (one block per SM).  The level loops
// wait on dependent row gathers, so more resident warps hide more latency:
// the 64- and 128-bit kernels run 32 warps per SM, at the price of a few
// spilled registers (measured on R-MAT 22, NBCut: 1024 threads beat 768 by 5%
// for 128-bit batches; DegCut and NBCut, 64-bit: 1024 beat 512 by 30%).
#ifndef TKC_THREADS_W2
#define TKC_THREADS_W2 1024
#endif
template <int W>
constexpr int kThreads = W == 1 ? 1024 : W == 2 ? TKC_THREADS_W2 : 512;
// Small graphs and one-source searches: short levels, where the block-wide
// barriers and scans of the larger blocks cost more than they hide.
constexpr int kMinThreads = 512;
constexpr int kMaxThreads = 1024;

__device__ __forceinline__ bool harmonic_below(double Hd, u64 d, u64 nd, u64 g, u64 omega, u64 xbits) {
  const u64 w = omega > nd ? omega - nd : 0;
  const u64 near_ = g < w ? g : w, far_ = w > g ? w - g : 0;
  const double t1 = __ddiv_rn((double)near_, (double)(d + 1));
  const double t2 = __ddiv_rn((double)far_, (double)(d + 2));
  const double U = __dadd_rn(__dadd_rn(Hd, t1), t2);
  return __dmul_rn(U, kHMargin) < __longlong_as_double((long long)xbits);
}

// ------------------------------------------------------------------ warp helpers

// 32x32 bit-matrix transpose across a warp: afterwards bit l of lane i equals
// bit i of lane l's input.
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t x, int lane) {
  uint32_t m = 0x0000FFFFu;
#pragma unroll
  for (int j = 16; j > 0; j >>= 1) {
    uint32_t y = __shfl_xor_sync(FULL, x, j);
    x = (lane & j) ? ((x & ~m) | ((y >> j) & m)) : ((x & m) | ((y & m) << j));
    m ^= m << (j >> 1);
  }
  return x;
}

// OR of a 64-bit word over the warp: one warp reduction per 32-bit half
// (measured 5% off the search kernel against five rounds of shuffles).
__device__ __forceinline__ u64 warp_or(u64 x) {
  const uint32_t lo = __reduce_or_sync(FULL, (uint32_t)x), hi = __reduce_or_sync(FULL, (uint32_t)(x >> 32));
  return ((u64)hi << 32) | lo;
}

// Adds, for every slot bit of the 32 lanes' rows, the number of lanes with
// the bit set and the sum of those lanes' `od` into the block counters.
template <int W>
__device__ __forceinline__ void warp_count_slots(const u64 (&nw)[W], uint32_t od, unsigned *s_cnt,
                                                 u64 *s_wsum, int lane) {
  uint32_t anyw = 0;
#pragma unroll
  for (int j = 0; j < W; ++j) anyw |= (nw[j] != 0);
  if (__ballot_sync(FULL, anyw) == 0) return;
  uint32_t odm = anyw ? od : 0u;
  uint32_t maxod = __reduce_max_sync(FULL, odm);
  int planes = 32 - __clz(maxod);
  // all 2W halves transposed first, so that the out-degree bit planes (one
  // ballot each) serve every half
  uint32_t colv[2 * W], cv[2 * W];
  uint32_t cmax = 0;
#pragma unroll
  for (int jh = 0; jh < 2 * W; ++jh) {
    const uint32_t x = (uint32_t)(nw[jh >> 1] >> (32 * (jh & 1)));
    colv[jh] = __ballot_sync(FULL, x != 0) ? warp_transpose32(x, lane) : 0u;
    cv[jh] = __popc(colv[jh]);
    cmax = cv[jh] > cmax ? cv[jh] : cmax;
  }
  const uint32_t maxc = __reduce_max_sync(FULL, cmax);
  u64 ws[2 * W];
#pragma unroll
  for (int jh = 0; jh < 2 * W; ++jh) ws[jh] = 0;
  // about 6 instructions per half for a walk step or a plane, 1 more per plane
  if ((int)maxc * 12 * W <= planes * (1 + 12 * W)) {
    // walk the set bits: fetch each contributing lane's out-degree
    for (uint32_t it = 0; it < maxc; ++it) {
#pragma unroll
      for (int jh = 0; jh < 2 * W; ++jh) {
        const int src = colv[jh] ? (__ffs(colv[jh]) - 1) : 0;
        const uint32_t v = __shfl_sync(FULL, odm, src);
        if (colv[jh]) {
          ws[jh] += v;
          colv[jh] &= colv[jh] - 1;
        }
      }
    }
  } else {
    // bit planes of the out-degrees: sum = sum_p 2^p popc(col & plane_p)
    for (int p = 0; p < planes; ++p) {
      const uint32_t plane = __ballot_sync(FULL, (odm >> p) & 1u);
#pragma unroll
      for (int jh = 0; jh < 2 * W; ++jh) ws[jh] += (u64)__popc(colv[jh] & plane) << p;
    }
  }
#pragma unroll
  for (int jh = 0; jh < 2 * W; ++jh) {
    if (cv[jh]) {
      const int slot = 32 * jh + lane;
      atomicAdd(&s_cnt[slot], cv[jh]);
      atomicAdd(&s_wsum[slot], ws[jh]);
    }
  }
}

// Warp-aggregated append of the lanes with `pred` to a list whose counter
// packs count << 38 | arcs.  Writes list[pos] = v and loff[pos] = arc prefix.
__device__ __forceinline__ void warp_append(bool pred, uint32_t v, uint32_t od, u64 *packed, uint32_t *list,
                                            uint32_t *loff, int lane) {
  uint32_t mask = __ballot_sync(FULL, pred);
  if (mask == 0) return;
  uint32_t a = pred ? od : 0u;
  // inclusive scan of arcs over lanes
  uint32_t incl = a;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t t = __shfl_up_sync(FULL, incl, o);
    if (lane >= o) incl += t;
  }
  uint32_t total = __shfl_sync(FULL, incl, 31);
  int leader = __ffs(mask) - 1;
  u64 base = 0;
  if (lane == leader) base = atomicAdd(packed, ((u64)__popc(mask) << kPackShift) | (u64)total);
  base = __shfl_sync(FULL, base, leader);
  if (pred) {
    uint32_t pos = (uint32_t)(base >> kPackShift) + __popc(mask & ((1u << lane) - 1u));
    list[pos] = v;
    loff[pos] = (uint32_t)((base & kArcMask) + (incl - a));
  }
}

__device__ __forceinline__ void warp_append_plain(bool pred, uint32_t v, unsigned *counter, uint32_t *list,
                                                  int lane) {
  uint32_t mask = __ballot_sync(FULL, pred);
  if (mask == 0) return;
  int leader = __ffs(mask) - 1;
  uint32_t base = 0;
  if (lane == leader) base = atomicAdd(counter, (unsigned)__popc(mask));
  base = __shfl_sync(FULL, base, leader);
  if (pred) list[base + __popc(mask & ((1u << lane) - 1u))] = v;
}

template <int W>
__device__ __forceinline__ void load_row(const u64 *base, uint32_t v, u64 (&r)[W]) {
  const u64 *p = base + (size_t)v * W;
  if constexpr (W == 1) {
    r[0] = p[0];
  } else {
#pragma unroll
    for (int j = 0; j < W; j += 2) {
      ulonglong2 t = *reinterpret_cast<const ulonglong2 *>(p + j);
      r[j] = t.x;
      r[j + 1] = t.y;
    }
  }
}

template <int W>
__device__ __forceinline__ void store_row(u64 *base, uint32_t v, const u64 (&r)[W]) {
  u64 *p = base + (size_t)v * W;
  if constexpr (W == 1) {
    p[0] = r[0];
  } else {
#pragma unroll
    for (int j = 0; j < W; j += 2) *reinterpret_cast<ulonglong2 *>(p + j) = make_ulonglong2(r[j], r[j + 1]);
  }
}

template <int W>
__device__ __forceinline__ bool row_nonzero(const u64 (&r)[W]) {
  u64 a = 0;
#pragma unroll
  for (int j = 0; j < W; ++j) a |= r[j];
  return a != 0;
}

// Zeroes the frontier rows of the listed vertices and their frontier bits.
// A long list clears the whole bitmap instead of one bit per vertex.
template <int W>
__device__ __forceinline__ void clear_frontier(u64 *F, uint32_t *FB, const uint32_t *list, uint32_t count, uint32_t n,
                                               uint64_t gthread, uint64_t nthreads) {
  for (uint64_t i = gthread; i < (uint64_t)count * W; i += nthreads) {
    uint32_t v = list[i / W];
    F[(size_t)v * W + (i % W)] = 0;
  }
  if (count > n / 32) {
    for (uint64_t i = gthread; i < n / 32 + 1; i += nthreads) FB[i] = 0;
  } else {
    for (uint64_t i = gthread; i < count; i += nthreads) {
      uint32_t v = list[i];
      atomicAnd(&FB[v >> 5], ~(1u << (v & 31)));
    }
  }
}

// updateBoundsLB: the slots whose bits are new in this vertex's row found it at
// this depth.
template <int W>
__device__ __forceinline__ void record_levels(const RunParams &p, uint32_t w, const u64 (&nw)[W], uint32_t depth) {
  const uint32_t v = p.unlab ? p.unlab[w] : w;  // the vertex whose search label is w
  uint16_t *row = p.lvl + (size_t)v * p.lvl_stride + (size_t)p.team * p.B;
#pragma unroll
  for (int q = 0; q < W; ++q) {
    u64 b = nw[q];
    while (b) {
      const int j = __ffsll((long long)b) - 1;
      b &= b - 1;
      row[64 * q + j] = (uint16_t)depth;
    }
  }
}

// ------------------------------------------------------------------ shared state

template <int W>
struct Smem {
  unsigned cnt[64 * W];
  u64 wsum[64 * W];
  u64 active[W];
  // epilogue scratch
  u64 tS[kTopMax];
  uint32_t tr[kTopMax], tid[kTopMax];
  u64 cS[64 * W];
  uint32_t cr[64 * W], cid[64 * W], cg[64 * W];
  unsigned ncand;
  unsigned nactive;
  unsigned scan[kMaxThreads / 32 + 1];
  u64 scan64[kMaxThreads / 32 + 1];
  u64 acc[4];
  unsigned bu_next;  // bottom-up level: next of this block's vertex chunks
};

// Block-wide exclusive scan of one uint32 per thread; returns the prefix and
// writes the total to *total.
template <int W>
__device__ uint32_t block_exscan(Smem<W> &sm, uint32_t x, uint32_t *total) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t t = __shfl_up_sync(FULL, incl, o);
    if (lane >= o) incl += t;
  }
  __syncthreads();
  if (lane == 31) sm.scan[wid] = incl;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      uint32_t t = sm.scan[i];
      sm.scan[i] = run;
      run += t;
    }
    sm.scan[blockDim.x >> 5] = run;
  }
  __syncthreads();
  uint32_t res = sm.scan[wid] + incl - x;
  *total = sm.scan[blockDim.x >> 5];
  __syncthreads();
  return res;
}

template <int W>
__device__ u64 block_exscan64(Smem<W> &sm, u64 x, u64 *total) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  u64 incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    u64 t = __shfl_up_sync(FULL, incl, o);
    if (lane >= o) incl += t;
  }
  __syncthreads();
  if (lane == 31) sm.scan64[wid] = incl;
  __syncthreads();
  if (threadIdx.x == 0) {
    u64 run = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      u64 t = sm.scan64[i];
      sm.scan64[i] = run;
      run += t;
    }
    sm.scan64[blockDim.x >> 5] = run;
  }
  __syncthreads();
  u64 res = sm.scan64[wid] + incl - x;
  *total = sm.scan64[blockDim.x >> 5];
  __syncthreads();
  return res;
}

// ------------------------------------------------------------------ epilogues

// The k-th entry of graph g's list as last published (seqlock: the writer
// makes the sequence odd, writes, makes it even).  A read that keeps seeing
// a write in progress reports no threshold, which only means no cut.
struct Thresh {
  bool have;
  u64 S;
  uint32_t r, id;
};

__device__ __forceinline__ Thresh thresh_of(const RunParams &p, uint32_t g) {
  Thresh t;
  t.have = false;
  t.S = 0;
  t.r = t.id = 0;
  for (int tries = 0; tries < 64; ++tries) {
    unsigned s1 = ld_acquire_u32(&p.x_seq[g]);
    if (s1 & 1u) continue;
    u64 S = *(volatile const u64 *)&p.x_S[g];
    uint32_t r = *(volatile const uint32_t *)&p.x_r[g];
    uint32_t id = *(volatile const uint32_t *)&p.x_id[g];
    __threadfence();
    unsigned s2 = *(volatile const unsigned *)&p.x_seq[g];
    if (s1 == s2) {
      t.have = r != 0;
      t.S = S;
      t.r = r;
      t.id = id;
      return t;
    }
  }
  return t;
}

// Publishes graph g's current k-th entry (caller holds the merge lock).
__device__ __forceinline__ void publish_thresh(const RunParams &p, uint32_t g) {
  if (p.g_ntop[g] != p.kk) return;
  size_t i = (size_t)g * p.kk + p.kk - 1;
  unsigned s = p.x_seq[g];
  *(volatile unsigned *)&p.x_seq[g] = s + 1u;
  __threadfence();
  *(volatile u64 *)&p.x_S[g] = p.top_S[i];
  *(volatile uint32_t *)&p.x_id[g] = p.top_id[i];
  *(volatile uint32_t *)&p.x_r[g] = p.top_r[i];
  __threadfence();
  st_release_u32(&p.x_seq[g], s + 2u);
}

// Merge lock shared by the teams; a wait beyond the budget is an error.
__device__ __forceinline__ bool lock_lists(const RunParams &p) {
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    long long t0 = clock64();
    unsigned ns = 32;
    int ok = 1;
    while (atomicCAS(&p.sh->lock, 0, 1) != 0) {
      if (ld_volatile_i32(&p.sh->err) != 0 || (uint64_t)(clock64() - t0) > p.timeout) {
        atomicCAS(&p.sh->err, 0, TKC_ETIMEOUT);
        atomicCAS(&p.ctl->err, 0, TKC_ETIMEOUT);
        ok = 0;
        break;
      }
      __nanosleep(ns);
      if (ns < 256) ns <<= 1;
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

__device__ __forceinline__ void unlock_lists(const RunParams &p) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicExch(&p.sh->lock, 0);
  }
}

// Merges the block's candidate list (sm.cS/cr/cid, sm.ncand entries) into the
// global top list.  Every entry's new position is its rank among the old list
// and the candidates (keys are unique: farness then id), so each position below
// k gets exactly one writer and the old list is read from a shared copy.
template <int W>
__device__ void merge_topk_one(const RunParams &p, Smem<W> &sm) {
  const uint32_t kk = p.kk;
  uint32_t ntop = p.g_ntop[0];
  uint32_t nc = sm.ncand;
  if (nc == 0) return;
  for (uint32_t i = threadIdx.x; i < ntop; i += blockDim.x) {
    sm.tS[i] = p.top_S[i];
    sm.tr[i] = p.top_r[i];
    sm.tid[i] = p.top_id[i];
  }
  __syncthreads();
  // rank of each candidate among existing entries and other candidates
  for (uint32_t i = threadIdx.x; i < nc; i += blockDim.x) {
    u64 S = sm.cS[i];
    uint32_t r = sm.cr[i], id = sm.cid[i];
    uint32_t lo = 0, hi = ntop;  // first existing entry not less than the candidate
    while (lo < hi) {
      uint32_t mid = (lo + hi) >> 1;
      if (entry_less(p.harmonic, sm.tS[mid], sm.tr[mid], sm.tid[mid], S, r, id)) lo = mid + 1;
      else hi = mid;
    }
    uint32_t rank = lo;
    for (uint32_t j = 0; j < nc; ++j)
      if (j != i && entry_less(p.harmonic, sm.cS[j], sm.cr[j], sm.cid[j], S, r, id)) ++rank;
    if (rank < kk) {
      p.top_S[rank] = S;
      p.top_r[rank] = r;
      p.top_id[rank] = id;
    }
  }
  for (uint32_t i = threadIdx.x; i < ntop; i += blockDim.x) {
    uint32_t rank = i;
    for (uint32_t j = 0; j < nc; ++j)
      if (entry_less(p.harmonic, sm.cS[j], sm.cr[j], sm.cid[j], sm.tS[i], sm.tr[i], sm.tid[i])) ++rank;
    if (rank < kk) {
      p.top_S[rank] = sm.tS[i];
      p.top_r[rank] = sm.tr[i];
      p.top_id[rank] = sm.tid[i];
    }
  }
  __syncthreads();
  uint32_t nnew = ntop + nc < kk ? ntop + nc : kk;
  if (threadIdx.x == 0) p.g_ntop[0] = nnew;
  __syncthreads();
}

// Several graphs: the thread holding a graph's first candidate inserts that
// graph's candidates into its list one by one (each list has one writer).
template <int W>
__device__ void merge_topk_many(const RunParams &p, Smem<W> &sm) {
  const uint32_t kk = p.kk;
  const uint32_t nc = sm.ncand;
  for (uint32_t i = threadIdx.x; i < nc; i += blockDim.x) {
    const uint32_t g = sm.cg[i];
    bool first = true;
    for (uint32_t j = 0; j < i && first; ++j) first = sm.cg[j] != g;
    if (!first) continue;
    u64 *tS = p.top_S + (size_t)g * kk;
    uint32_t *tr = p.top_r + (size_t)g * kk, *ti = p.top_id + (size_t)g * kk;
    uint32_t cnt = p.g_ntop[g];
    for (uint32_t j = i; j < nc; ++j) {
      if (sm.cg[j] != g) continue;
      u64 S = sm.cS[j];
      uint32_t r = sm.cr[j], id = sm.cid[j];
      if (cnt == kk && !entry_less(p.harmonic, S, r, id, tS[kk - 1], tr[kk - 1], ti[kk - 1])) continue;
      uint32_t pos = cnt < kk ? cnt++ : kk - 1;
      while (pos > 0 && entry_less(p.harmonic, S, r, id, tS[pos - 1], tr[pos - 1], ti[pos - 1])) {
        tS[pos] = tS[pos - 1];
        tr[pos] = tr[pos - 1];
        ti[pos] = ti[pos - 1];
        --pos;
      }
      tS[pos] = S;
      tr[pos] = r;
      ti[pos] = id;
    }
    p.g_ntop[g] = cnt;
    publish_thresh(p, g);
  }
  __syncthreads();
}

template <int W>
__device__ __forceinline__ void merge_topk(const RunParams &p, Smem<W> &sm) {
  if (sm.ncand == 0) return;
  if (!lock_lists(p)) return;
  __threadfence();
  if (p.ng == 1) {
    merge_topk_one(p, sm);
    if (threadIdx.x == 0) publish_thresh(p, 0);
  } else {
    merge_topk_many(p, sm);
  }
  unlock_lists(p);
}

__device__ __forceinline__ void graph_count(const RunParams &p, uint32_t g, int which, u64 v) {
  if (p.g_ctr && v) atomicAdd(&p.g_ctr[(size_t)g * 4 + which], v);
}

// Adds a finished search to the candidate list if it can enter the top list.
template <int W>
__device__ __forceinline__ void offer_candidate(const RunParams &p, Smem<W> &sm, u64 S, uint32_t r, uint32_t v,
                                                uint32_t g) {
  Thresh x = thresh_of(p, g);
  if (x.have && !entry_less(p.harmonic, S, r, v, x.S, x.r, x.id)) return;
  unsigned pos = atomicAdd(&sm.ncand, 1u);
  sm.cS[pos] = S;
  sm.cr[pos] = r;
  sm.cid[pos] = v;
  sm.cg[pos] = g;
}

// Epilogue after a level: update every active slot, merge finished searches,
// apply the cut test, choose the next step.
__device__ __forceinline__ void trace_stamp(const RunParams &p, int slot) {
  if (p.trace && threadIdx.x == 0) {
    u64 idx = ((volatile Ctl *)p.ctl)->trace_n;
    if (idx < p.trace_cap) {
      u64 t;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
      p.trace[idx * 16 + slot] = t;
    }
  }
}

// Direction of the next level: bottom-up when the frontier's arcs are a large
// share of all arcs.
__device__ __forceinline__ int choose_dir(const RunParams &p, u64 fl_arcs) {
  return ((u128)fl_arcs * p.bu_num > (u128)p.arcs * p.bu_den) ? 1 : 0;
}

// Frontier lists at most this long are never compacted (the pass and its
// barrier would cost more than the dead entries).
constexpr uint32_t kCompactMin = 4096;

template <int W>
__device__ void epilogue_level(const RunParams &p, Smem<W> &sm) {
  Ctl *c = p.ctl;
  const uint32_t B = p.B;
  trace_stamp(p, 13);
  if (threadIdx.x == 0) {
    sm.ncand = 0;
    sm.nactive = 0;
  }
  if (threadIdx.x < W) sm.active[threadIdx.x] = 0;
  for (int i = threadIdx.x; i < 4; i += blockDim.x) sm.acc[i] = 0;
  __syncthreads();
  // 1. per-slot level update
  int cont[(64 * W + kMinThreads - 1) / kMinThreads];
  uint32_t finished = 0;
#pragma unroll
  for (int t = 0; t < (64 * W + kMinThreads - 1) / kMinThreads; ++t) {
    uint32_t s = threadIdx.x + t * blockDim.x;
    cont[t] = 0;
    if (s >= B) continue;
    Slot sl = p.slots[s];
    if (sl.state != 1) continue;
    unsigned cn = p.cnt[s];
    u64 ws = p.wsum[s];
    p.cnt[s] = 0;
    p.wsum[s] = 0;
    if (cn == 0) {
      // the BFS from sl.v is complete: S and r = n_d are exact
      sl.state = 2;
      const u64 key = p.harmonic ? (u64)__double_as_longlong(sl.H) : sl.S;
      p.res_S[sl.v] = key;
      p.res_r[sl.v] = (uint32_t)sl.nd;
      ++finished;
      graph_count(p, sl.graph, 3, 1);
      offer_candidate(p, sm, key, (uint32_t)sl.nd, sl.v, sl.graph);
    } else {
      const int directed = p.g_directed ? p.g_directed[sl.graph] : p.directed;
      sl.d += 1;
      if (p.hist) {
        if (sl.d < p.hist_cap)
          p.hist[((size_t)p.team * p.B + s) * p.hist_cap + sl.d] = cn;
        else
          atomicCAS(&c->err, 0, TKC_EOVERFLOW);
      }
      sl.S += (u64)sl.d * cn;
      sl.H = __dadd_rn(sl.H, __ddiv_rn((double)cn, (double)sl.d));
      sl.nd += cn;
      sl.g = ws - (directed ? 0ull : (u64)cn);
      sl.arcs = ws;
      cont[t] = 1;
    }
    p.slots[s] = sl;
  }
  if (finished) atomicAdd(&sm.acc[0], (u64)finished);
  __syncthreads();
  // 2. top-k merge and the new threshold
  merge_topk(p, sm);
  // 3. BFSCut test for the slots that continue
  uint32_t cuts = 0;
  u64 visited = 0;
#pragma unroll
  for (int t = 0; t < (64 * W + kMinThreads - 1) / kMinThreads; ++t) {
    uint32_t s = threadIdx.x + t * blockDim.x;
    if (!cont[t]) continue;
    Slot sl = p.slots[s];
    Thresh x = thresh_of(p, sl.graph);
    const bool below = x.have && (p.harmonic ? harmonic_below(sl.H, sl.d, sl.nd, sl.g, sl.omega, x.S)
                                             : cut_exceeds(sl.S, sl.d, sl.nd, sl.g, sl.alpha, sl.omega, x.S, x.r));
    if (!p.nocut && !sl.nocut && below) {
      sl.state = 2;
      ++cuts;
      graph_count(p, sl.graph, 2, 1);
      p.slots[s] = sl;
    } else {
      visited += sl.arcs;
      graph_count(p, sl.graph, 0, sl.arcs);
      atomicOr(&sm.active[s >> 6], 1ull << (s & 63));
      atomicAdd(&sm.nactive, 1u);
    }
  }
  if (cuts) atomicAdd(&sm.acc[1], (u64)cuts);
  if (visited) atomicAdd(&sm.acc[2], visited);
  __syncthreads();
  if (threadIdx.x == 0) {
    c->bfs_finished += sm.acc[0];
    c->bfs_cut += sm.acc[1];
    c->edges_visited += sm.acc[2];
    c->levels += 1;
    u64 packed = c->nl_packed;
    {
      // cost model of the level just run (bytes that must move):
      //  top-down : per frontier vertex list+offsets (16) + F row read and clear;
      //             per frontier arc column (4) + seen row read + N row update;
      //             per new vertex list (8) + N read/clear, seen read/write, F write
      //  bottom-up: per swept list entry (vertices with an in-arc) the entry (4)
      //             and its seen row; per scanned vertex in-offsets (8); per
      //             scanned in-arc its column (4) and frontier-bitmap word (4);
      //             per frontier in-neighbour found its F row; per new vertex
      //             seen/F writes + list (8); per old frontier vertex list (4) +
      //             F row clear
      const u64 rb = 8ull * W;
      const u64 fl = c->fl_count, fa = c->fl_arcs, nl = packed >> kPackShift;
      u64 bytes;
      if (c->dir == 0) {
        bytes = fl * (16 + 2 * rb) + fa * (4 + 2 * rb) + nl * (8 + 5 * rb);
        c->st_td_levels += 1;
        c->st_td_frontier += fl;
        c->st_td_arcs += fa;
        c->st_td_new += nl;
      } else {
        const u64 swept = p.bu_list ? p.n_bu : p.n;
        bytes = swept * (4 + rb) + c->lvl_scan_v * 8 + c->lvl_scan_a * 8 + c->lvl_scan_r * rb + nl * (8 + 2 * rb) +
                fl * (4 + rb);
        c->st_bu_levels += 1;
        c->st_bu_rows += c->lvl_scan_r;
        c->st_bu_scan_v += c->lvl_scan_v;
        c->st_bu_scan_a += c->lvl_scan_a;
        c->st_bu_new += nl;
        c->st_bu_frontier += fl;
      }
      c->alg_bytes += bytes;
      if (p.trace) {
        u64 idx = c->trace_n++;
        if (idx < p.trace_cap) {
          u64 t;
          asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
          u64 *rec = p.trace + idx * 16;
          rec[0] = t;
          rec[1] = (u64)c->dir;
          rec[2] = fl;
          rec[3] = fa;
          rec[4] = nl;
          rec[5] = c->lvl_scan_v;
          rec[6] = c->lvl_scan_a;
          rec[7] = sm.nactive;
        }
      }
      c->lvl_scan_v = 0;
      c->lvl_scan_a = 0;
      c->lvl_scan_r = 0;
    }
    c->nl_packed = 0;
    c->cur ^= 1;
    c->lcur ^= 1;
    c->bdepth += 1;
    c->fl_count = (uint32_t)(packed >> kPackShift);
    c->fl_arcs = packed & kArcMask;
    c->level_id += 1;
    for (int j = 0; j < W; ++j) c->active[j] = sm.active[j];
    if (sm.nactive == 0) {
      c->step = 1;  // clear the batch's rows, then seed the next batch
    } else if (c->fl_count > kCompactMin && sm.acc[2] * 2 < c->fl_arcs) {
      // the new frontier list was built before this level's cuts: when the
      // surviving searches' own frontier arcs (sm.acc[2], an upper bound on
      // the arcs of the list entries they still use) are less than half of
      // the list's, compact it first, so that the level neither expands nor
      // (bottom-up) matches against rows of abandoned searches
      c->step = 2;
    } else {
      c->step = 0;
      c->dir = choose_dir(p, c->fl_arcs);
    }
  }
  __syncthreads();
}

// Epilogue after a compaction step: the compacted list (built in the next-list
// buffer) becomes the frontier list, and the level's direction is chosen from
// its arcs.
template <int W>
__device__ void epilogue_compact(const RunParams &p, Smem<W> &sm) {
  Ctl *c = p.ctl;
  if (threadIdx.x == 0) {
    const u64 packed = c->nl_packed;
    const u64 before = c->fl_count, after = packed >> kPackShift;
    c->nl_packed = 0;
    c->lcur ^= 1;
    c->fl_count = (uint32_t)after;
    c->fl_arcs = packed & kArcMask;
    c->st_compactions += 1;
    c->st_compact_dropped += before - after;
    // list entry and row read per old entry, row cleared per dropped one, list written per kept one
    c->alg_bytes += before * (4 + 8ull * W) + (before - after) * 8ull * W + after * 8;
    c->step = 0;
    c->dir = choose_dir(p, c->fl_arcs);
  }
  __syncthreads();
}

// Epilogue after a clear step: seed the next batch of up to B sources.
template <int W>
__device__ void epilogue_seed(const RunParams &p, Smem<W> &sm) {
  Ctl *c = p.ctl;
  trace_stamp(p, 13);
  const uint32_t B = p.B;
  u64 *Fcur = c->cur ? p.F1 : p.F0;
  uint32_t *FBcur = c->cur ? p.FB1 : p.FB0;
  uint32_t *FL = c->lcur ? p.L1 : p.L0;
  uint32_t *FLoff = c->lcur ? p.Loff1 : p.Loff0;
  uint32_t assigned = 0, last_base = 0;
  u64 arcs_total = 0, started = 0, cut0 = 0;
  __shared__ uint32_t s_base;
  __shared__ int s_gate;
  if (threadIdx.x < W) sm.active[threadIdx.x] = 0;
  // One graph and several teams, no threshold yet: the other teams start only
  // after team 0's first batch.  Until then every source they took would be
  // searched to the end; afterwards most are abandoned at once.
  if (threadIdx.x == 0) {
    volatile Shared *vsh = p.sh;
    if (p.team == 0 && c->batches >= 1) vsh->first_done = 1u;
    s_gate = p.teams > 1 && p.team != 0 && p.ng == 1 && !p.nocut && vsh->first_done == 0u &&
             vsh->cursor < p.norder && vsh->err == 0 && !thresh_of(p, 0).have;
  }
  __syncthreads();
  if (s_gate) {
    if (threadIdx.x == 0) {
      __nanosleep(2000);
      c->fl_count = 0;
      c->fl_arcs = 0;
      c->vl_count = 0;
      c->nl_packed = 0;
      c->level_id += 1;
      for (int j = 0; j < W; ++j) c->active[j] = 0;
      c->step = 1;  // another empty clear step, then this check again
    }
    for (uint32_t s = threadIdx.x; s < B; s += blockDim.x) p.slots[s].state = 0;
    __syncthreads();
    return;
  }
  // take sources from the shared cursor, `room` positions at a time, so that
  // every position taken is either abandoned at level 0 or gets a slot
  // (updateBoundsLB runs: one batch per team, its levels are read afterwards)
  const bool lb_done = p.lvl && c->batches >= 1;
  while (!lb_done && assigned < B) {
    const uint32_t room = B - assigned;
    if (threadIdx.x == 0) s_base = atomicAdd(&p.sh->cursor, room);
    __syncthreads();
    const uint32_t base = s_base;
    __syncthreads();
    if (base >= p.norder) break;
    last_base = base;
    const uint32_t cnt = room < p.norder - base ? room : p.norder - base;
    const uint32_t idx = base + threadIdx.x;
    const bool valid = threadIdx.x < cnt;
    uint32_t v = valid ? p.order[idx] : 0;
    const uint32_t sv = valid && p.lab ? p.lab[v] : v;  // its row's label
    uint32_t od = valid ? p.off[sv + 1] - p.off[sv] : 0;
    uint32_t a = valid ? p.alpha[v] : 0, o = valid ? p.omega[v] : 0;
    uint32_t gv = (valid && p.gid) ? p.gid[v] : 0;
    // level 0: S_0 = 0, n_0 = 1, gamma_1 = out-degree
    bool cut = false, stop = false;
    // several graphs: a graph whose search stopped skips its later sources
    const bool stopped = valid && p.lb_key && p.gid && *(volatile unsigned *)&p.g_stop[gv];
    if (valid && !stopped && !p.nocut && idx >= p.nocut_prefix) {
      Thresh x = thresh_of(p, gv);
      if (p.harmonic) {
        stop = x.have && p.lb_key &&
               __dmul_rn(__longlong_as_double((long long)~p.lb_key[v]), kHMargin) <
                   __longlong_as_double((long long)x.S);
        cut = !stop && x.have && harmonic_below(0.0, 0, 1, od, o, x.S);
      } else {
        stop = x.have && p.lb_key && nb_exceeds(p.lb_key[v], x.S, x.r);
        cut = !stop && x.have && cut_exceeds(0, 0, 1, od, a, o, x.S, x.r);
      }
    }
    // nothing after a stopped position of its graph is searched, by any team
    if (stop) {
      if (!p.gid) {
        atomicMax(&p.sh->cursor, p.norder);
      } else {
        *(volatile unsigned *)&p.g_stop[gv] = 1u;
        // sources graph by graph: the rest of this graph's run is skipped at
        // once (only after the openings, where the run is contiguous)
        if (p.g_end && idx >= p.g_rest) atomicMax(&p.sh->cursor, p.g_end[gv]);
      }
    }
    if (stopped && p.g_end && idx >= p.g_rest) atomicMax(&p.sh->cursor, p.g_end[gv]);
    const bool take = valid && !cut && !stop && !stopped;
    uint32_t total;
    uint32_t pre = block_exscan(sm, take ? 1u : 0u, &total);
    if (cut) {
      graph_count(p, gv, 1, 1);
      graph_count(p, gv, 2, 1);
    }
    uint32_t s = assigned + pre;
    u64 myarcs = take ? od : 0;
    u64 arcs_pre_total;
    u64 arcs_pre = block_exscan64(sm, myarcs, &arcs_pre_total);
    if (take) {
      Slot sl;
      sl.S = 0;
      sl.nd = 1;
      sl.g = od;
      sl.arcs = od;
      sl.v = v;
      sl.d = 0;
      sl.alpha = a;
      sl.omega = o;
      sl.state = 1;
      sl.graph = gv;
      sl.nocut = idx < p.nocut_prefix;
      sl.pad = 0;
      sl.H = 0.0;
      if (p.lvl_src) p.lvl_src[p.team * B + s] = v;
      p.slots[s] = sl;
      graph_count(p, gv, 1, 1);
      graph_count(p, gv, 0, od);
      u64 bit = 1ull << (s & 63);
      p.seen[(size_t)sv * W + (s >> 6)] = bit;
      Fcur[(size_t)sv * W + (s >> 6)] = bit;
      atomicOr(&FBcur[sv >> 5], 1u << (sv & 31));
      FL[s] = sv;
      FLoff[s] = (uint32_t)(arcs_total + arcs_pre);
      p.VL[s] = sv;
      atomicOr(&sm.active[s >> 6], bit);
    }
    uint32_t ncut;
    block_exscan(sm, cut ? 1u : 0u, &ncut);
    assigned += total;
    arcs_total += arcs_pre_total;
    started += total + ncut;
    cut0 += ncut;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // the clear step just zeroed these rows
    c->alg_bytes += (u64)(c->vl_count + c->fl_count) * (4 + 8ull * W);
    c->st_cleared += (u64)c->vl_count + c->fl_count;
    c->st_seeded += assigned;
    c->cursor = last_base;
    c->bfs_started += started;
    c->bfs_cut += cut0;
    c->edges_visited += arcs_total;
    c->fl_count = assigned;
    c->fl_arcs = arcs_total;
    c->vl_count = assigned;
    c->bdepth = 0;
    c->nl_packed = 0;
    c->level_id += 1;
    if (p.trace) {
      u64 idx = c->trace_n++;
      if (idx < p.trace_cap) {
        u64 t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        u64 *rec = p.trace + idx * 16;
        rec[0] = t;
        rec[1] = 2;  // seed step
        rec[2] = assigned;
        rec[3] = arcs_total;
        rec[4] = last_base;
        rec[5] = cut0;
        rec[6] = c->vl_count;
        rec[7] = p.g_ntop[0];
      }
    }
    c->batches += 1;
    for (int j = 0; j < W; ++j) c->active[j] = sm.active[j];
    if (assigned == 0) {
      c->done = 1;
      if (p.team == 0) ((volatile Shared *)p.sh)->first_done = 1u;
    } else {
      c->step = 0;
      c->dir = choose_dir(p, arcs_total);
    }
  }
  // slots beyond `assigned` are free
  for (uint32_t s = assigned + threadIdx.x; s < B; s += blockDim.x) p.slots[s].state = 0;
  __syncthreads();
}

// ------------------------------------------------------------------ the kernel

template <int W, int TPB>
__global__ void __launch_bounds__(TPB, 1) bfscut_kernel(RunParams p0) {
  __shared__ Smem<W> sm;
  // this block's team: its own control block, slots, rows, lists and stamps
  __shared__ RunParams p;
  const uint32_t bpt = gridDim.x / p0.teams;  // blocks per team
  const uint32_t team = blockIdx.x / bpt;
  const uint32_t tb = blockIdx.x % bpt;
  if (threadIdx.x == 0) {
    p = p0;
    p.team = team;
    p.ctl = p0.ctl + team;
    p.slots = p0.slots + (size_t)team * 64 * kMaxWords;
    p.cnt = p0.cnt + (size_t)team * 64 * kMaxWords;
    p.wsum = p0.wsum + (size_t)team * 64 * kMaxWords;
    p.seen = p0.seen + team * p0.row_stride;
    p.F0 = p0.F0 + team * p0.row_stride;
    p.F1 = p0.F1 + team * p0.row_stride;
    p.N = p0.N + team * p0.row_stride;
    p.FB0 = p0.FB0 + team * p0.fb_stride;
    p.FB1 = p0.FB1 + team * p0.fb_stride;
    p.L0 = p0.L0 + team * p0.vtx_stride;
    p.L1 = p0.L1 + team * p0.vtx_stride;
    p.Loff0 = p0.Loff0 + team * p0.vtx_stride;
    p.Loff1 = p0.Loff1 + team * p0.vtx_stride;
    p.VL = p0.VL + team * p0.vtx_stride;
    p.stamp = p0.stamp + team * p0.vtx_stride;
    if (p0.trace) {
      p.trace_cap = p0.trace_cap / p0.teams;
      p.trace = p0.trace + (size_t)team * p.trace_cap * 16;
    }
  }
  __syncthreads();
  Ctl *c = p.ctl;
  const int lane = threadIdx.x & 31;
  const uint32_t gwarp = (tb * TPB + threadIdx.x) >> 5;
  const uint32_t nwarps = (bpt * TPB) >> 5;
  const uint32_t gthread = tb * TPB + threadIdx.x;
  const uint32_t nthreads = bpt * TPB;

  while (true) {
    const int step = ld_volatile_i32(&c->step);
    if (ld_volatile_i32(&c->done)) break;
    volatile Ctl *vc = c;
    const int cur = vc->cur;
    u64 *Fcur = cur ? p.F1 : p.F0;
    u64 *Fnext = cur ? p.F0 : p.F1;
    uint32_t *FBcur = cur ? p.FB1 : p.FB0;
    uint32_t *FBnext = cur ? p.FB0 : p.FB1;
    const int lcur = vc->lcur;
    uint32_t *FL = lcur ? p.L1 : p.L0;
    uint32_t *FLoff = lcur ? p.Loff1 : p.Loff0;
    uint32_t *NL = lcur ? p.L0 : p.L1;
    uint32_t *NLoff = lcur ? p.Loff0 : p.Loff1;
    const uint32_t fl_count = vc->fl_count;
    if (step == 1) {
      if (tb == 0) trace_stamp(p, 8);
      // ---- clear step: zero the rows touched by the finished batch
      const uint32_t vl = vc->vl_count;
      for (uint64_t i = gthread; i < (uint64_t)vl * W; i += nthreads) {
        uint32_t v = p.VL[i / W];
        p.seen[(size_t)v * W + (i % W)] = 0;
      }
      clear_frontier<W>(Fcur, FBcur, FL, fl_count, p.n, gthread, nthreads);
      if (tb == 0) trace_stamp(p, 12);
      if (!team_sync(c, p.sh, bpt, p.timeout, [&] { epilogue_seed<W>(p, sm); })) break;
      continue;
    }
    if (step == 2) {
      // ---- compaction: keep the frontier entries with a bit of a search
      // still active (rows masked to those bits); zero the rows and frontier
      // bits of the others, which only abandoned or finished searches used
      u64 act[W];
#pragma unroll
      for (int q = 0; q < W; ++q) act[q] = vc->active[q];
      for (uint32_t base = gwarp * 32; base < fl_count; base += nwarps * 32) {
        const uint32_t i = base + lane;
        const bool valid = i < fl_count;
        uint32_t u = 0, od = 0;
        bool keep = false;
        if (valid) {
          u = FL[i];
          u64 row[W], f[W];
          load_row<W>(Fcur, u, row);
          bool same = true;
#pragma unroll
          for (int q = 0; q < W; ++q) {
            f[q] = row[q] & act[q];
            same &= f[q] == row[q];
          }
          keep = row_nonzero<W>(f);
          if (!keep) atomicAnd(&FBcur[u >> 5], ~(1u << (u & 31)));
          if (!same) store_row<W>(Fcur, u, f);
          if (keep) od = p.off[u + 1] - p.off[u];
        }
        warp_append(keep, u, od, &c->nl_packed, NL, NLoff, lane);
      }
      if (!team_sync(c, p.sh, bpt, p.timeout, [&] { epilogue_compact<W>(p, sm); })) break;
      continue;
    }
    if (tb == 0) trace_stamp(p, 8);
    const int dir = vc->dir;
    const uint32_t level_id = vc->level_id;
    const uint32_t depth = vc->bdepth + 1;  // depth of the level being discovered
    const u64 fl_arcs = vc->fl_arcs;
    if (threadIdx.x < W) sm.active[threadIdx.x] = vc->active[threadIdx.x];
    for (int i = threadIdx.x; i < 64 * W; i += TPB) {
      sm.cnt[i] = 0;
      sm.wsum[i] = 0;
    }
    if (threadIdx.x == 0) {
      sm.acc[2] = 0;
      sm.acc[3] = 0;
      sm.bu_next = 0;
    }
    __syncthreads();
    u64 scanned = 0, scanned_v = 0;
    uint32_t rows_read = 0;
    if (dir == 0) {
      // ---- phase A, top-down: OR each frontier row into its out-neighbours' N rows
      constexpr uint32_t APS = 32 / W;  // arcs per warp step
      // arcs per warp task: about two tasks per warp, at least one step, so a
      // small level still spreads over every warp (each step is a chain of
      // dependent loads)
      constexpr int TU = W <= 2 ? 4 : 2;  // warp steps unrolled per iteration
      u64 CH = (fl_arcs + 2ull * nwarps - 1) / (2ull * nwarps);
      CH = (CH + TU * APS - 1) / (TU * APS) * (TU * APS);
      if (CH < TU * APS) CH = TU * APS;
      const int grp = lane / W, j = lane % W;
      const u64 actj = sm.active[j];
      for (u64 base = (u64)gwarp * CH; base < fl_arcs; base += (u64)nwarps * CH) {
        u64 end = base + CH < fl_arcs ? base + CH : fl_arcs;
        // entry holding arc `base`: last i with FLoff[i] <= base
        uint32_t lo = 0, hi = fl_count;
        while (hi - lo > 1) {
          uint32_t mid = (lo + hi) >> 1;
          if (FLoff[mid] <= base) lo = mid;
          else hi = mid;
        }
        uint32_t ent = lo;
        // TU warp steps per iteration: every arc's loads are issued before
        // any arc's atomic
        for (u64 e0 = base; e0 < end; e0 += TU * APS) {
          u64 ew[TU];
          uint32_t iw[TU], uw[TU], ww[TU];
          u64 fw[TU], bw[TU], cw[TU];
          uint32_t ii = ent;
#pragma unroll
          for (int t = 0; t < TU; ++t) {
            ew[t] = e0 + (u64)t * APS + grp;
            if (ew[t] < end)
              while (ii + 1 < fl_count && FLoff[ii + 1] <= ew[t]) ++ii;
            iw[t] = ii;
          }
#pragma unroll
          for (int t = 0; t < TU; ++t) uw[t] = ew[t] < end ? FL[iw[t]] : 0;
#pragma unroll
          for (int t = 0; t < TU; ++t) fw[t] = ew[t] < end ? Fcur[(size_t)uw[t] * W + j] & actj : 0;
#pragma unroll
          for (int t = 0; t < TU; ++t) ww[t] = fw[t] ? p.col[p.off[uw[t]] + (uint32_t)(ew[t] - FLoff[iw[t]])] : 0;
#pragma unroll
          for (int t = 0; t < TU; ++t) bw[t] = fw[t] ? fw[t] & ~p.seen[(size_t)ww[t] * W + j] : 0;
#pragma unroll
          for (int t = 0; t < TU; ++t) cw[t] = bw[t] ? *(volatile u64 *)(p.N + (size_t)ww[t] * W + j) : 0;
#pragma unroll
          for (int t = 0; t < TU; ++t) {
            bool app = false;
            if (bw[t] & ~cw[t]) {
              u64 old = atomicOr(p.N + (size_t)ww[t] * W + j, bw[t]);
              if (old == 0) app = atomicExch(&p.stamp[ww[t]], level_id) != level_id;
            }
            uint32_t od = app ? p.off[ww[t] + 1] - p.off[ww[t]] : 0;
            warp_append(app, ww[t], od, &c->nl_packed, NL, NLoff, lane);
          }
          ent = __reduce_max_sync(FULL, ii);
        }
      }
      scanned = 0;
      if (gthread == 0) atomicAdd(&c->edges_scanned, fl_arcs);
      if (tb == 0) trace_stamp(p, 9);
      if (!team_sync(c, p.sh, bpt, p.timeout, [] {})) break;
      if (tb == 0) trace_stamp(p, 10);
      // ---- phase B: finalize the next level, clear the old frontier rows
      const uint32_t nl_count = (uint32_t)(((volatile Ctl *)c)->nl_packed >> kPackShift);
      for (uint32_t base = gwarp * 32; base < nl_count; base += nwarps * 32) {
        uint32_t i = base + lane;
        bool valid = i < nl_count;
        u64 nw[W], sr[W];
        uint32_t w = 0, od = 0;
        bool was_empty = false;
#pragma unroll
        for (int q = 0; q < W; ++q) nw[q] = 0;
        if (valid) {
          w = NL[i];
          od = p.off[w + 1] - p.off[w];
          load_row<W>(p.N, w, nw);
          load_row<W>(p.seen, w, sr);
          was_empty = !row_nonzero<W>(sr);
          u64 z[W];
#pragma unroll
          for (int q = 0; q < W; ++q) {
            sr[q] |= nw[q];
            z[q] = 0;
          }
          store_row<W>(p.seen, w, sr);
          store_row<W>(Fnext, w, nw);
          store_row<W>(p.N, w, z);
          atomicOr(&FBnext[w >> 5], 1u << (w & 31));
          if (p.lvl) record_levels<W>(p, w, nw, depth);
        }
        warp_count_slots<W>(nw, od, sm.cnt, sm.wsum, lane);
        warp_append_plain(valid && was_empty, w, &c->vl_count, p.VL, lane);
      }
      clear_frontier<W>(Fcur, FBcur, FL, fl_count, p.n, gthread, nthreads);
    } else {
      // ---- phase A, bottom-up: each vertex ORs its in-neighbours' frontier rows
      u64 act[W];
#pragma unroll
      for (int q = 0; q < W; ++q) act[q] = sm.active[q];
      // Work items of the sweep list (vertices with an in-arc), dealt
      // round-robin to the team's blocks, whose warps take them from a shared
      // counter as they finish: first groups of 32 long in-rows, group j
      // holding list entries j, j + hg, j + 2 hg, ... so that the longest rows
      // land in different warps; then chunks of kBuChunkVerts consecutive
      // entries of the shorter rows (labels ascending).
      const uint32_t nheavy = p.bu_list ? p.n_bu_heavy : 0u;
      const uint32_t nlight = p.bu_list ? p.n_bu - nheavy : p.n;
      const uint32_t hg = (nheavy + 31) / 32;
      const uint32_t nitems = hg + (nlight + kBuChunkVerts - 1) / kBuChunkVerts;
      for (;;) {
        uint32_t j = 0;
        if (lane == 0) j = atomicAdd(&sm.bu_next, 1u);
        j = __shfl_sync(FULL, j, 0);
        const u64 gi64 = (u64)tb + (u64)bpt * j;
        if (gi64 >= nitems) break;
        const uint32_t gi = (uint32_t)gi64;
        const bool hitem = gi < hg;
        const uint32_t g0 = hitem ? 0u : (gi - hg) * kBuChunkVerts;
        const uint32_t g1 = hitem ? 32u : (g0 + kBuChunkVerts < nlight ? g0 + kBuChunkVerts : nlight);
        for (uint32_t base = g0; base < g1; base += 32) {
          bool valid;
          uint32_t w;
          if (hitem) {
            const uint32_t e = gi + hg * (uint32_t)lane;
            valid = e < nheavy;
            w = valid ? p.bu_list[e] : 0;
          } else {
            valid = base + lane < g1;
            w = valid ? (p.bu_list ? p.bu_list[nheavy + base + lane] : base + lane) : 0;
          }
          u64 nw[W], sr[W], miss[W];
          uint32_t od = 0, e0 = 0, ee = 0;
          bool was_empty = false, any = false, heavy = false;
#pragma unroll
          for (int q = 0; q < W; ++q) {
            nw[q] = 0;
            miss[q] = 0;
          }
          if (valid) {
            load_row<W>(p.seen, w, sr);
            was_empty = !row_nonzero<W>(sr);
#pragma unroll
            for (int q = 0; q < W; ++q) {
              miss[q] = act[q] & ~sr[q];
              any |= miss[q] != 0;
            }
            e0 = p.ioff[w];
            ee = p.ioff[w + 1];
            heavy = any && ee - e0 > p.heavy_in;
            if (any && !heavy) {
              // U in-arcs per step, software-pipelined: step i's rows (of the
              // in-neighbours on a frontier) are loaded together with step
              // i+1's frontier bits and step i+2's columns, so a step waits on
              // one round trip instead of three (1.5% off the kernel on R-MAT
              // 22); the early exit is tested once per step (extra rows only
              // repeat found bits)
              constexpr int U = W >= 8 ? 2 : TKC_BU_U;
              uint32_t e = e0;
              uint32_t c0[U], c1[U], f0[U];
#pragma unroll
              for (int j = 0; j < U; ++j) {
                c0[j] = e + j < ee ? p.icol[e + j] : 0xffffffffu;
                c1[j] = e + U + j < ee ? p.icol[e + U + j] : 0xffffffffu;
              }
#pragma unroll
              for (int j = 0; j < U; ++j)
                f0[j] = c0[j] != 0xffffffffu ? (FBcur[c0[j] >> 5] >> (c0[j] & 31)) & 1u : 0u;
              for (; e < ee; e += U) {
                uint32_t c2[U], f1[U];
#pragma unroll
                for (int j = 0; j < U; ++j) c2[j] = e + 2 * U + j < ee ? p.icol[e + 2 * U + j] : 0xffffffffu;
#pragma unroll
                for (int j = 0; j < U; ++j)
                  f1[j] = c1[j] != 0xffffffffu ? (FBcur[c1[j] >> 5] >> (c1[j] & 31)) & 1u : 0u;
#pragma unroll
                for (int j = 0; j < U; ++j) {
                  if (f0[j]) {
                    u64 fr[W];
                    load_row<W>(Fcur, c0[j], fr);
                    ++rows_read;
#pragma unroll
                    for (int q = 0; q < W; ++q) nw[q] |= fr[q] & miss[q];
                  }
                }
                bool full = true;
#pragma unroll
                for (int q = 0; q < W; ++q) full &= nw[q] == miss[q];
                if (full) {
                  e += U;
                  break;
                }
#pragma unroll
                for (int j = 0; j < U; ++j) {
                  c0[j] = c1[j];
                  c1[j] = c2[j];
                  f0[j] = f1[j];
                }
              }
              scanned += (e < ee ? e : ee) - e0;
              scanned_v += 1;
            }
          }
          // vertices of high in-degree: the whole warp walks their in-arcs
          // (coalesced column reads, HU per lane per step) so that one lane does
          // not hold the level up; same result as the lane loop (the OR of the
          // frontier rows of in-neighbours, or every missing bit found)
          for (unsigned hv = __ballot_sync(FULL, heavy); hv; hv &= hv - 1) {
            const int src = __ffs(hv) - 1;
            const uint32_t hb = __shfl_sync(FULL, e0, src), he = __shfl_sync(FULL, ee, src);
            u64 hm[W], acc[W];
#pragma unroll
            for (int q = 0; q < W; ++q) {
              hm[q] = __shfl_sync(FULL, miss[q], src);
              acc[q] = 0;
            }
            constexpr int HU = W >= 8 ? 1 : W >= 4 ? 2 : TKC_BU_HU;
            uint32_t e = hb;
            // the next step's columns are loaded before this step's frontier
            // bits and rows are waited on, so their latency overlaps
            uint32_t nx[HU];
#pragma unroll
            for (int j = 0; j < HU; ++j) {
              const uint32_t i = hb + 32 * j + lane;
              nx[j] = i < he ? p.icol[i] : 0xffffffffu;
            }
            for (; e < he; e += 32 * HU) {
              uint32_t uu[HU], fb[HU];
#pragma unroll
              for (int j = 0; j < HU; ++j) {
                uu[j] = nx[j];
                const uint32_t i = e + 32 * HU + 32 * j + lane;
                nx[j] = i < he ? p.icol[i] : 0xffffffffu;
              }
#pragma unroll
              for (int j = 0; j < HU; ++j)
                fb[j] = uu[j] != 0xffffffffu ? (FBcur[uu[j] >> 5] >> (uu[j] & 31)) & 1u : 0u;
#pragma unroll
              for (int j = 0; j < HU; ++j) {
                if (fb[j]) {
                  u64 fr[W];
                  load_row<W>(Fcur, uu[j], fr);
                  ++rows_read;
#pragma unroll
                  for (int q = 0; q < W; ++q) acc[q] |= fr[q] & hm[q];
                }
              }
              // early exit once every missing bit is found
              bool full = true;
#pragma unroll
              for (int q = 0; q < W; ++q) full &= warp_or(acc[q]) == hm[q];
              if (full) {
                e += 32 * HU;
                break;
              }
            }
#pragma unroll
            for (int q = 0; q < W; ++q) acc[q] = warp_or(acc[q]);
            if (lane == src) {
#pragma unroll
              for (int q = 0; q < W; ++q) nw[q] = acc[q];
              scanned += (e < he ? e : he) - hb;
              scanned_v += 1;
            }
          }
          bool isnew = valid && row_nonzero<W>(nw);
          if (isnew) {
            od = p.off[w + 1] - p.off[w];
#pragma unroll
            for (int q = 0; q < W; ++q) sr[q] |= nw[q];
            store_row<W>(p.seen, w, sr);
            store_row<W>(Fnext, w, nw);
            if (p.lvl) record_levels<W>(p, w, nw, depth);
          }
          // the next frontier's bitmap starts all zero (each level clears the
          // bits of its own frontier), so setting the new vertices' bits
          // suffices: one atomic per bitmap word the group's new vertices share
          // (shorter rows: labels ascending, a few words), one per vertex for the
          // long rows (labels scattered)
          if (hitem) {
            if (isnew) atomicOr(&FBnext[w >> 5], 1u << (w & 31));
          } else {
            for (unsigned pend = __ballot_sync(FULL, isnew); pend;) {
              const int l = __ffs(pend) - 1;
              const uint32_t word = __shfl_sync(FULL, w >> 5, l);
              const bool mine = isnew && (w >> 5) == word;
              const unsigned bits = __reduce_or_sync(FULL, mine ? 1u << (w & 31) : 0u);
              if (lane == l) atomicOr(&FBnext[word], bits);
              pend &= ~__ballot_sync(FULL, mine);
            }
          }
          warp_count_slots<W>(nw, od, sm.cnt, sm.wsum, lane);
          warp_append(isnew, w, od, &c->nl_packed, NL, NLoff, lane);
          warp_append_plain(isnew && was_empty, w, &c->vl_count, p.VL, lane);
        }
      }
      if (tb == 0) trace_stamp(p, 9);
      if (!team_sync(c, p.sh, bpt, p.timeout, [] {})) break;
      if (tb == 0) trace_stamp(p, 10);
      // ---- phase B: only the old frontier rows need clearing
      clear_frontier<W>(Fcur, FBcur, FL, fl_count, p.n, gthread, nthreads);
    }
    if (tb == 0) trace_stamp(p, 11);
    // flush the block's per-slot counters
    u64 rows64 = rows_read;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      scanned += __shfl_down_sync(FULL, scanned, o);
      scanned_v += __shfl_down_sync(FULL, scanned_v, o);
      rows64 += __shfl_down_sync(FULL, rows64, o);
    }
    if (lane == 0 && scanned) atomicAdd(&sm.acc[3], scanned);
    if (lane == 0 && scanned_v) atomicAdd(&sm.acc[2], scanned_v);
    if (lane == 0 && rows64) atomicAdd(&c->lvl_scan_r, rows64);
    __syncthreads();
    for (int i = threadIdx.x; i < 64 * W; i += TPB) {
      if (sm.cnt[i]) {
        atomicAdd(&p.cnt[i], sm.cnt[i]);
        atomicAdd(&p.wsum[i], sm.wsum[i]);
      }
    }
    if (threadIdx.x == 0 && sm.acc[3]) {
      atomicAdd(&c->edges_scanned, sm.acc[3]);
      atomicAdd(&c->lvl_scan_a, sm.acc[3]);
    }
    if (threadIdx.x == 0 && sm.acc[2]) atomicAdd(&c->lvl_scan_v, sm.acc[2]);
    if (tb == 0) trace_stamp(p, 12);
    if (!team_sync(c, p.sh, bpt, p.timeout, [&] { epilogue_level<W>(p, sm); })) break;
  }
}

// ------------------------------------------------------------------ host side

// The larger blocks pay off on batched searches of large graphs (R-MAT 20 and
// 22); one-source searches and graphs below 2^20 vertices (BA 10^6: 1.75 ms of
// kernel time at 512 threads, 1.98 ms at 768) run 512 threads per block.
static bool wide_blocks(const RunParams &p) {
  if (p.large_blocks) return p.large_blocks == 1;
  return p.B > 1 && p.n >= (1u << 20);
}

template <int W, int TPB>
static int occupancy_of(int *blocks_per_sm) {
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, bfscut_kernel<W, TPB>, TPB, 0);
  return e == cudaSuccess ? TKC_OK : TKC_ECUDA;
}

// Co-resident blocks of the W-word kernel, the smaller of its two block sizes'
// (either may be launched with this count).
template <int W>
static int occupancy_both(int *blocks_per_sm) {
  int a = 0, b = 0;
  int rc = occupancy_of<W, kThreads<W>>(&a);
  if (rc == TKC_OK) rc = occupancy_of<W, kMinThreads>(&b);
  if (rc != TKC_OK) return rc;
  *blocks_per_sm = a < b ? a : b;
  return TKC_OK;
}

int max_coresident_blocks(tkc_ctx *ctx, int words) {
  int per_sm = 0;
  int rc = TKC_OK;
  switch (words) {
    case 1: rc = occupancy_both<1>(&per_sm); break;
    case 2: rc = occupancy_both<2>(&per_sm); break;
    case 4: rc = occupancy_both<4>(&per_sm); break;
    case 8: rc = occupancy_both<8>(&per_sm); break;
    default: return 0;
  }
  if (rc != TKC_OK) return 0;
  return per_sm * ctx->num_sms;
}

template <int W, int TPB>
static cudaError_t launch_tpb(const RunParams &p, int blocks, cudaStream_t st) {
  void *args[] = {(void *)&p};
  note_launches(1);
  return cudaLaunchCooperativeKernel((const void *)bfscut_kernel<W, TPB>, dim3(blocks), dim3(TPB), args, 0, st);
}

template <int W>
static cudaError_t launch(const RunParams &p, int blocks, cudaStream_t st) {
  if (kThreads<W> != kMinThreads && wide_blocks(p)) return launch_tpb<W, kThreads<W>>(p, blocks, st);
  return launch_tpb<W, kMinThreads>(p, blocks, st);
}

int run_bfscut(tkc_ctx *ctx, const RunParams &p, int words, int blocks) {
  cudaError_t e;
  switch (words) {
    case 1: e = launch<1>(p, blocks, ctx->stream); break;
    case 2: e = launch<2>(p, blocks, ctx->stream); break;
    case 4: e = launch<4>(p, blocks, ctx->stream); break;
    case 8: e = launch<8>(p, blocks, ctx->stream); break;
    default: return TKC_EINVAL;
  }
  TKC_TRY(e);
  return TKC_OK;
}

}  // namespace tkc
