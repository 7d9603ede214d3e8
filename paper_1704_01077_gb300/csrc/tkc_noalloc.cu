// Allocation-free exact distance sums for small graphs.
//
// Some callers cannot allocate device memory at the point where they need a
// result: runtimes that hand out a fixed device-memory budget up front (an
// allocation later would exceed it or fail), and latency-bound services that
// cannot afford the device-wide synchronisation an allocation may imply.  For
// them this file offers one entry point that allocates nothing: every scratch
// buffer of the batched BFS (bit rows, frontier lists, per-slot state, control
// block) lives in one file-scope device array of fixed size, and the caller
// passes device pointers for the graph, the sources and the outputs.
//
// Limits: at most TKC_NOALLOC_MAX_N vertices; sources are searched 64 at a
// time.  The array is shared by every call on a device and keeps the previous
// call's contents; each call clears what must start at zero.  Calls whose GPU
// work overlaps (different streams, or different host threads on one device)
// race on the array and must be serialised by the caller.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "tkc_internal.cuh"

namespace tkc {
namespace {

typedef uint32_t u32;
typedef unsigned long long u64;

constexpr u32 kNaMaxN = TKC_NOALLOC_MAX_N;
constexpr int kWords = 1;       // 64-bit rows: 64 sources per batch
constexpr u32 kSlots = 64 * kWords;

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Byte offsets of every buffer inside the static array.
struct Layout {
  static constexpr size_t rows = align256(sizeof(u64) * kNaMaxN * kWords);
  static constexpr size_t u32n = align256(sizeof(u32) * kNaMaxN);
  static constexpr size_t bits = align256(sizeof(u32) * (kNaMaxN / 32 + 1));
  static constexpr size_t seen = 0;
  static constexpr size_t F0 = seen + rows;
  static constexpr size_t F1 = F0 + rows;
  static constexpr size_t N = F1 + rows;
  static constexpr size_t FB0 = N + rows;
  static constexpr size_t FB1 = FB0 + bits;
  static constexpr size_t dup = FB1 + bits;
  static constexpr size_t L0 = dup + bits;
  static constexpr size_t L1 = L0 + u32n;
  static constexpr size_t Loff0 = L1 + u32n;
  static constexpr size_t Loff1 = Loff0 + u32n;
  static constexpr size_t VL = Loff1 + u32n;
  static constexpr size_t stamp = VL + u32n;
  static constexpr size_t alpha = stamp + u32n;
  static constexpr size_t omega = alpha + u32n;
  static constexpr size_t res_r = omega + u32n;
  static constexpr size_t res_S = res_r + u32n;
  static constexpr size_t slots = res_S + align256(sizeof(u64) * kNaMaxN);
  static constexpr size_t cnt = slots + align256(sizeof(Slot) * kSlots);
  static constexpr size_t wsum = cnt + align256(sizeof(unsigned) * kSlots);
  static constexpr size_t top_S = wsum + align256(sizeof(u64) * kSlots);
  static constexpr size_t top_r = top_S + 256;
  static constexpr size_t top_id = top_r + 256;
  static constexpr size_t g_ntop = top_id + 256;
  static constexpr size_t shared = g_ntop + 256;
  static constexpr size_t x_seq = shared + 256;
  static constexpr size_t x_S = x_seq + 256;
  static constexpr size_t x_r = x_S + 256;
  static constexpr size_t x_id = x_r + 256;
  static constexpr size_t flag = x_id + 256;
  static constexpr size_t ctl = flag + 256;
  static constexpr size_t total = ctl + align256(sizeof(Ctl));
};

// The scratch of every call on this device (about 5.5 MB).
static __device__ __align__(256) unsigned char g_scratch[Layout::total];

// Range checks that keep every later access in bounds, and distinct sources
// (two slots of one batch must not share a source row).
__global__ void k_check(const u32 *off, const u32 *col, u32 n, u64 arcs, const u32 *srcs, u32 nsrc, u32 *dup,
                        int *flag) {
  u32 tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
  if (tid == 0 && (off[0] != 0 || off[n] != arcs)) atomicCAS(flag, 0, TKC_EGRAPH);
  for (u32 v = tid; v < n; v += nth) {
    u32 b = off[v], e = off[v + 1];
    if (e < b || e > arcs) {
      atomicCAS(flag, 0, TKC_EGRAPH);
      continue;
    }
    for (u32 i = b; i < e; ++i)
      if (col[i] >= n) atomicCAS(flag, 0, TKC_EGRAPH);
  }
  for (u32 i = tid; i < nsrc; i += nth) {
    u32 v = srcs[i];
    if (v >= n) {
      atomicCAS(flag, 0, TKC_EINVAL);
      continue;
    }
    u32 bit = 1u << (v & 31);
    if (atomicOr(&dup[v >> 5], bit) & bit) atomicCAS(flag, 0, TKC_EINVAL);
  }
}

// Control block of the persistent kernel: an empty clear step first, whose
// epilogue seeds the first batch; a failed check ends the run before it starts.
__global__ void k_init_ctl(Ctl *ctl, const int *flag) {
  ctl->step = 1;
  ctl->level_id = 0;
  ctl->cur = 0;
  if (*flag) {
    ctl->err = *flag;
    ctl->done = 1;
  }
}

__global__ void k_gather(const u32 *srcs, u32 nsrc, const u64 *res_S, const u32 *res_r, const Ctl *ctl, u64 *S,
                         u32 *r) {
  if (ctl->err) return;
  for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < nsrc; i += gridDim.x * blockDim.x) {
    u32 v = srcs[i];
    S[i] = res_S[v];
    r[i] = res_r[v];
  }
}

// Device address of g_scratch on the current device.  The symbol's host-side
// name is not a device address, so it is looked up on every call: the lookup
// allocates nothing, and an address cached across calls would go stale after a
// device reset reloads the module.
int scratch_for_device(unsigned char **out) {
  void *p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
  if (e != cudaSuccess) {
    tkc_set_last_cuda_error(e, "cudaGetSymbolAddress(g_scratch)", __FILE__, __LINE__);
    return TKC_ECUDA;
  }
  *out = (unsigned char *)p;
  return TKC_OK;
}

}  // namespace
}  // namespace tkc

using namespace tkc;

extern "C" int tkc_distance_sums_noalloc(const uint32_t *offsets, const uint32_t *cols, uint32_t n, uint64_t arcs,
                                         uint32_t nsrc, const uint32_t *srcs, uint64_t *S, uint32_t *r,
                                         void *stream) {
  if (n > kNaMaxN) return TKC_EINVAL;
  if (arcs >= (1ull << 32)) return TKC_EOVERFLOW;
  if (nsrc == 0) return TKC_OK;
  if (n == 0 || !offsets || (arcs && !cols) || !srcs || !S || !r) return TKC_EINVAL;
  int dev = 0;
  TKC_TRY(cudaGetDevice(&dev));
  unsigned char *base = nullptr;
  TKC_RC(scratch_for_device(&base));
  cudaStream_t st = (cudaStream_t)stream;
  typedef Layout L;
  // what must start at zero: bit rows, frontier bitmaps, duplicate map,
  // per-vertex results, per-slot counters, the flag and the control block;
  // stamps start at all-ones so that level 0 never matches a stale stamp
  TKC_TRY(cudaMemsetAsync(base + L::seen, 0, L::FB0 - L::seen, st));
  TKC_TRY(cudaMemsetAsync(base + L::FB0, 0, L::L0 - L::FB0, st));
  TKC_TRY(cudaMemsetAsync(base + L::stamp, 0xff, L::alpha - L::stamp, st));
  TKC_TRY(cudaMemsetAsync(base + L::alpha, 0, L::slots - L::alpha, st));
  TKC_TRY(cudaMemsetAsync(base + L::cnt, 0, L::total - L::cnt, st));
  int *flag = (int *)(base + L::flag);
  Ctl *ctl = (Ctl *)(base + L::ctl);
  TKC_LAUNCH(k_check<<<64, 256, 0, st>>>(offsets, cols, n, arcs, srcs, nsrc, (u32 *)(base + L::dup), flag));
  TKC_LAUNCH(k_init_ctl<<<1, 1, 0, st>>>(ctl, flag));
  TKC_TRY(cudaGetLastError());

  RunParams p;
  memset(&p, 0, sizeof(p));
  p.n = n;
  p.directed = 1;  // only out-arcs are read; gamma bounds are unused without cutting
  p.arcs = arcs;
  p.off = offsets;
  p.col = cols;
  p.ioff = offsets;  // never read: every level runs top-down (bu_num = 0)
  p.icol = cols;
  p.alpha = (const u32 *)(base + L::alpha);
  p.omega = (const u32 *)(base + L::omega);
  p.order = srcs;
  p.norder = nsrc;
  p.teams = 1;
  p.row_stride = 0;
  p.vtx_stride = 0;
  p.fb_stride = 0;
  p.sh = (Shared *)(base + L::shared);
  p.x_seq = (unsigned *)(base + L::x_seq);
  p.x_S = (u64 *)(base + L::x_S);
  p.x_r = (u32 *)(base + L::x_r);
  p.x_id = (u32 *)(base + L::x_id);
  p.ng = 1;
  p.gid = nullptr;
  p.g_directed = nullptr;
  p.g_ntop = (unsigned *)(base + L::g_ntop);
  p.g_ctr = nullptr;
  p.kk = 1;
  p.B = kSlots;
  p.nocut = 1;
  p.bu_num = 0;
  p.bu_den = 1;
  p.timeout = 1ull << 34;
  p.seen = (u64 *)(base + L::seen);
  p.F0 = (u64 *)(base + L::F0);
  p.F1 = (u64 *)(base + L::F1);
  p.N = (u64 *)(base + L::N);
  p.FB0 = (u32 *)(base + L::FB0);
  p.FB1 = (u32 *)(base + L::FB1);
  p.L0 = (u32 *)(base + L::L0);
  p.L1 = (u32 *)(base + L::L1);
  p.Loff0 = (u32 *)(base + L::Loff0);
  p.Loff1 = (u32 *)(base + L::Loff1);
  p.VL = (u32 *)(base + L::VL);
  p.stamp = (u32 *)(base + L::stamp);
  p.slots = (Slot *)(base + L::slots);
  p.cnt = (unsigned *)(base + L::cnt);
  p.wsum = (u64 *)(base + L::wsum);
  p.top_S = (u64 *)(base + L::top_S);
  p.top_r = (u32 *)(base + L::top_r);
  p.top_id = (u32 *)(base + L::top_id);
  p.res_S = (u64 *)(base + L::res_S);
  p.res_r = (u32 *)(base + L::res_r);
  p.ctl = ctl;
  p.trace = nullptr;
  p.trace_cap = 0;

  tkc_ctx lc;  // launch configuration only: no workspace, no events
  lc.device = dev;
  lc.stream = st;
  TKC_TRY(cudaDeviceGetAttribute(&lc.num_sms, cudaDevAttrMultiProcessorCount, dev));
  int maxb = max_coresident_blocks(&lc, kWords);
  if (maxb <= 0) return TKC_ECUDA;
  int blocks = (int)((n + 511) / 512);
  blocks = blocks < 8 ? 8 : blocks;
  blocks = blocks > maxb ? maxb : blocks;
  TKC_RC(run_bfscut(&lc, p, kWords, blocks));
  TKC_LAUNCH(k_gather<<<(nsrc + 255) / 256 < 1024 ? (nsrc + 255) / 256 : 1024, 256, 0, st>>>(
      srcs, nsrc, p.res_S, p.res_r, ctl, (u64 *)S, r));
  TKC_TRY(cudaGetLastError());
  int err = 0;
  TKC_TRY(cudaMemcpyAsync(&err, &ctl->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  TKC_TRY(cudaStreamSynchronize(st));
  return err;
}
