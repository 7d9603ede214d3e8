// Warp-cooperative walks over the arcs of a CSR graph, balanced by arcs.
//
// Kernels that visit every arc u -> v with its source u (in-arc CSR build,
// SCC condensation) give each warp a fixed range of arc indices instead of a
// set of vertices: a vertex with a long out-row (an R-MAT hub holds about
// 10^5 arcs) is then spread over many warps rather than walked by one, and
// short rows are taken 32 at a time.  The source of each arc comes from a
// 32-way search of the offsets and a window of 32 consecutive row ends held
// one per lane.
#pragma once

#include <cstdint>

namespace tkc {

// Largest u in [0, n) with off[u] <= a, for a < off[n] (so that u's row holds
// arc a).  32-way search: each round every lane probes one of 32 evenly
// spaced offsets and the range shrinks to one gap.  Called by all 32 lanes
// with the same arguments; every lane returns the same u.
__device__ __forceinline__ uint32_t warp_arc_source(const uint32_t *off, uint32_t n, uint64_t a, int lane) {
  uint32_t lo = 0, hi = n;  // off[lo] <= a; the answer lies in [lo, hi)
  while (hi - lo > 1) {
    const uint32_t step = (hi - lo + 31) / 32;
    const uint32_t p = lo + step * (uint32_t)lane;
    const bool ok = p < hi && off[p] <= a;  // true on a prefix of the lanes, lane 0 included
    const unsigned m = __ballot_sync(0xffffffffu, ok);
    const uint32_t l = 31u - (uint32_t)__clz(m);
    lo += step * l;
    hi = lo + step < hi ? lo + step : hi;
  }
  return lo;
}

// Calls f(u, i, valid, rs) for the arcs i of [a0, a1), 32 at a time (lane j
// takes arc t0 + j of each group; `valid` is false past a1, and then u and i
// are not arcs of the graph), u the source of arc i and rs the first arc of
// u's row (only with kRowStart; 0 otherwise).  a0 < a1 <= off[n].  All 32
// lanes run the same number of groups, so f may use warp collectives.  With
// offsets that are not nondecreasing the sources are meaningless, but every
// offset read stays within off[0 .. n] and the walk ends.
template <bool kRowStart = false, typename F>
__device__ __forceinline__ void warp_walk_arcs(const uint32_t *off, uint32_t n, uint64_t a0, uint64_t a1, int lane,
                                               F &&f) {
  uint32_t u = warp_arc_source(off, n, a0, lane);
  uint32_t wstart = kRowStart ? off[u] : 0u;  // first arc of the window's first row
  while (a0 < a1) {
    // row ends of the window u .. u + 31 (past the last vertex: no end)
    const uint64_t w = (uint64_t)u + 1 + (uint32_t)lane;
    const uint32_t vend = w <= n ? off[w] : 0xffffffffu;
    const uint32_t wlast = __shfl_sync(0xffffffffu, vend, 31);
    const uint64_t stop = a1 < (uint64_t)wlast ? a1 : (uint64_t)wlast;
    for (uint64_t t0 = a0; t0 < stop; t0 += 32) {
      const uint64_t i = t0 + (uint32_t)lane;
      // rows of the window ending at or before i (vend is nondecreasing)
      uint32_t cnt = 0;
#pragma unroll
      for (uint32_t s = 16; s > 0; s >>= 1) {
        const uint32_t x = __shfl_sync(0xffffffffu, vend, (int)(cnt + s - 1));
        if ((uint64_t)x <= i) cnt += s;
      }
      uint32_t rs = 0;
      if (kRowStart) {
        const uint32_t prev = __shfl_sync(0xffffffffu, vend, (int)((cnt + 31) & 31));
        rs = cnt ? prev : wstart;
      }
      f(u + cnt, i, i < stop, rs);
    }
    if (stop > a0) a0 = stop;
    wstart = wlast;
    u += 32;
  }
}

// Arcs per warp task of the walks above: a few window and search rounds per
// task against 64 groups of 32 arcs.
constexpr uint32_t kArcChunk = 2048;

// Calls f(u, i, valid, rs) for every arc of the graph, the arcs dealt to the
// grid's warps in tasks of kArcChunk consecutive indices (task c to warp
// c mod warps: a kernel launched twice with the same grid gives each block
// the same arcs).
template <bool kRowStart = false, typename F>
__device__ __forceinline__ void grid_walk_arcs(const uint32_t *off, uint32_t n, uint64_t arcs, F &&f) {
  const int lane = threadIdx.x & 31;
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t a0 = warp * kArcChunk; a0 < arcs; a0 += nwarps * kArcChunk) {
    const uint64_t a1 = a0 + kArcChunk < arcs ? a0 + kArcChunk : arcs;
    warp_walk_arcs<kRowStart>(off, n, a0, a1, lane, f);
  }
}

}  // namespace tkc
