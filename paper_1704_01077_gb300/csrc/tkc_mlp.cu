// Learned source order: per-vertex features, a 5 -> 64 -> 64 -> 1 MLP
// (bf16 weights, fp32 accumulation) with hand-written forward, backward and
// Adam kernels, and the order of sources by predicted farness.
//
// The paper orders sources by a degree bound (computeBoundsDeg, Section 4);
// any order gives the same exact top-k (Algorithm 1 only prunes), so a model
// that predicts farness can only change how soon the k-th threshold x becomes
// tight.  Without a model the degree order is used.
//
// Parameter layout (TKC_MLP_PARAMS floats):
//   W1[64][5] at 0, b1[64] at 320, W2[64][64] at 384, b2[64] at 4480,
//   w3[64] at 4544, b3 at 4608.
// y = w3 . relu(W2 relu(W1 x + b1) + b2) + b3.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "tkc_internal.cuh"

namespace tkc {

typedef uint32_t u32;
typedef unsigned long long u64;
static constexpr unsigned FULL = 0xffffffffu;

constexpr int F = TKC_MLP_FEATURES;
constexpr int H = TKC_MLP_HIDDEN;
constexpr int P = TKC_MLP_PARAMS;
constexpr int oW1 = 0, oB1 = H * F, oW2 = oB1 + H, oB2 = oW2 + H * H, oW3 = oB2 + H, oB3 = oW3 + H;
static_assert(oB3 + 1 == P, "parameter layout");

int radix_sort_u32_pairs(u32 *key, u32 *val, u32 n, int bits, cudaStream_t st);

namespace {

unsigned grid_of(u64 work, unsigned tpb = 256, unsigned cap = 152 * 16) {
  u64 b = (work + tpb - 1) / tpb;
  return (unsigned)std::max<u64>(1, std::min<u64>(b, cap));
}

// ---------------------------------------------------------------- features

// 2-walk count: sum of out-degrees of the out-neighbours (the gamma bound of
// the Section 6 lemma at d = 1, an upper bound on the 2-hop ball), one warp per vertex.
__global__ void k_two_walks(const u32 *off, const u32 *col, u32 n, float *w2) {
  const int lane = threadIdx.x & 31;
  for (u32 v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += (gridDim.x * blockDim.x) >> 5) {
    u64 s = 0;
    for (u32 i = off[v] + lane; i < off[v + 1]; i += 32) {
      u32 u = col[i];
      s += off[u + 1] - off[u];
    }
    for (int o = 16; o; o >>= 1) s += __shfl_down_sync(FULL, s, o);
    if (lane == 0) w2[v] = (float)s;
  }
}

__global__ void k_core_init(const u32 *off, const u32 *ioff, u32 n, int directed, u32 *c) {
  for (u32 v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    c[v] = (off[v + 1] - off[v]) + (directed ? ioff[v + 1] - ioff[v] : 0u);
}

// One h-index step of the core-number iteration (Lu, Zhou, Zhang, Stanley,
// Nat. Commun. 2016): c'(v) = the largest h such that at least h neighbours
// have c >= h, neighbours taken over out-arcs (and in-arcs when directed,
// so a vertex linked both ways counts twice: the graph with arc directions
// dropped).  Started from the degree it never rises, and once no value
// changes it is the core number.  Only vertices with a neighbour whose value
// changed in the previous step (dirty_in) are recomputed; a vertex whose value
// changes marks its neighbours in dirty_out and sets *changed.
constexpr int kCoreTPB = 256;      // threads per block of k_core_step
constexpr u32 kCoreBuckets = 256;  // histogram buckets per warp

__global__ void __launch_bounds__(kCoreTPB) k_core_step(const u32 *off, const u32 *col, const u32 *ioff,
                                                        const u32 *icol, u32 n, int directed, const u32 *c, u32 *c2,
                                                        const uint8_t *dirty_in, uint8_t *dirty_out, u32 *changed) {
  __shared__ u32 hist_all[kCoreTPB / 32][kCoreBuckets];
  const int lane = threadIdx.x & 31;
  u32 *hist = hist_all[threadIdx.x >> 5];
  for (u32 base = (blockIdx.x * blockDim.x + threadIdx.x) & ~31u; base < n; base += gridDim.x * blockDim.x) {
    // lane per vertex: copy the clean ones; the warp then takes the dirty ones
    const u32 mine = base + lane;
    bool dirty = false;
    if (mine < n) {
      dirty = dirty_in[mine] != 0;
      if (!dirty) c2[mine] = c[mine];
    }
    for (unsigned dm = __ballot_sync(FULL, dirty); dm; dm &= dm - 1) {
      const u32 v = base + (__ffs(dm) - 1);
      const u32 cv = c[v];
      // neighbours' values (out-arcs, and in-arcs when directed), visited by the warp
      auto for_each_value = [&](auto &&f) {
        for (u32 i = off[v] + lane; i < off[v + 1]; i += 32) f(c[col[i]]);
        if (directed)
          for (u32 i = ioff[v] + lane; i < ioff[v + 1]; i += 32) f(c[icol[i]]);
      };
      // the value never rises: one pass checks whether it stays (the common
      // case once most values have settled)
      u32 cnt = 0;
      for_each_value([&](u32 x) { cnt += x >= cv; });
      u32 above = __reduce_add_sync(FULL, cnt);  // neighbours with a value above the range searched
      u32 lo = 0, hi = cv;                       // the new value h lies in [lo, hi]
      if (above >= cv) {
        lo = cv;
      } else {
        // h < cv: h = the largest h with (neighbours whose value is >= h) >= h.
        // Each pass spreads [lo, hi] over 256 buckets, counts the neighbours'
        // values per bucket, and keeps the highest bucket whose start still
        // satisfies the condition (the count only falls as h rises, and h = lo
        // always satisfies it): one pass when cv <= 256, at most three below
        // 2^24 -- instead of one pass per halving of [0, cv].
        hi = cv - 1;
        while (lo < hi) {
          const u32 width = (hi - lo) / kCoreBuckets + 1;
          for (u32 j = lane; j < kCoreBuckets; j += 32) hist[j] = 0;
          __syncwarp();
          for_each_value([&](u32 x) {
            if (x >= lo && x <= hi) atomicAdd(&hist[(x - lo) / width], 1u);
          });
          __syncwarp();
          // lane j holds buckets 8j .. 8j+7; suffix sums over the warp from the top
          u32 loc[kCoreBuckets / 32];
          u32 part = 0;
#pragma unroll
          for (int q = kCoreBuckets / 32 - 1; q >= 0; --q) {
            part += hist[lane * (kCoreBuckets / 32) + q];
            loc[q] = part;  // buckets q.. of this lane's group
          }
          u32 incl = part;  // this lane's group total, then the sum of groups j..31
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const u32 t = __shfl_down_sync(FULL, incl, o);
            if (lane + o < 32) incl += t;
          }
          const u32 later = incl - part;  // groups above this lane's
          // highest bucket b with above + (count in buckets >= b) >= lo + b * width
          int best = -1;
#pragma unroll
          for (int q = kCoreBuckets / 32 - 1; q >= 0; --q) {
            const u32 b = lane * (kCoreBuckets / 32) + q;
            const u64 start = (u64)lo + (u64)b * width;
            if (best < 0 && start <= hi && (u64)above + later + loc[q] >= start) best = (int)b;
          }
          const unsigned has = __ballot_sync(FULL, best >= 0);
          const int src = 31 - __clz(has);  // the highest group with such a bucket (group 0 always has one)
          const u32 b = (u32)__shfl_sync(FULL, best, src);
          // neighbours in buckets above b
          const u32 b_above = __shfl_sync(FULL, later + loc[b % (kCoreBuckets / 32)] -
                                                     hist[lane * (kCoreBuckets / 32) + b % (kCoreBuckets / 32)],
                                          src);
          __syncwarp();
          const u32 nlo = lo + b * width;
          const u32 nhi = (u64)nlo + width - 1 < hi ? nlo + width - 1 : hi;
          above += b_above;
          lo = nlo;
          hi = nhi;
        }
      }
      if (lane == 0) c2[v] = lo;
      if (lo != cv) {
        if (lane == 0) *changed = 1;
        for (u32 i = off[v] + lane; i < off[v + 1]; i += 32) dirty_out[col[i]] = 1;
        if (directed)
          for (u32 i = ioff[v] + lane; i < ioff[v + 1]; i += 32) dirty_out[icol[i]] = 1;
      }
    }
  }
}

__global__ void k_features_raw(const u32 *off, const u32 *ioff, const float *w2, const u32 *core, const u32 *scc,
                               u32 n, float *x, double *sums) {
  double s[F] = {0}, q[F] = {0};
  for (u32 v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    float f[F];
    f[0] = log1pf((float)(off[v + 1] - off[v]));
    f[1] = log1pf((float)(ioff[v + 1] - ioff[v]));
    f[2] = log1pf(w2[v]);
    f[3] = log1pf((float)core[v]);
    f[4] = log1pf((float)scc[v]);
#pragma unroll
    for (int j = 0; j < F; ++j) {
      x[(size_t)v * F + j] = f[j];
      s[j] += f[j];
      q[j] += (double)f[j] * f[j];
    }
  }
#pragma unroll
  for (int j = 0; j < F; ++j) {
    for (int o = 16; o; o >>= 1) {
      s[j] += __shfl_down_sync(FULL, s[j], o);
      q[j] += __shfl_down_sync(FULL, q[j], o);
    }
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(&sums[j], s[j]);
      atomicAdd(&sums[F + j], q[j]);
    }
  }
}

__global__ void k_features_standardize(float *x, u32 n, const double *sums) {
  __shared__ float mean[F], inv[F];
  if (threadIdx.x < F) {
    double m = sums[threadIdx.x] / n;
    double var = sums[F + threadIdx.x] / n - m * m;
    mean[threadIdx.x] = (float)m;
    inv[threadIdx.x] = (float)(1.0 / sqrt(var > 1e-12 ? var : 1e-12));
  }
  __syncthreads();
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < (u64)n * F; i += (u64)gridDim.x * blockDim.x) {
    int j = (int)(i % F);
    x[i] = (x[i] - mean[j]) * inv[j];
  }
}

// ---------------------------------------------------------------- MLP kernels

__device__ __forceinline__ void load_weights(const unsigned short *wb, float *ws) {
  for (int i = threadIdx.x; i < P; i += blockDim.x) ws[i] = __bfloat162float(__ushort_as_bfloat16(wb[i]));
  __syncthreads();
}

constexpr int FT = 64;  // samples per forward block

// y[i] for m samples, one thread per sample; the first hidden layer of the
// block's samples is kept in shared memory, unit-major so that the threads
// of a warp read consecutive words.
__global__ void __launch_bounds__(FT) k_mlp_forward(const float *x, u32 m, const unsigned short *wb, float *y) {
  __shared__ float ws[P];
  __shared__ float h1[H][FT];
  load_weights(wb, ws);
  const int t = threadIdx.x;
  for (u32 i0 = blockIdx.x * FT; i0 < m; i0 += gridDim.x * FT) {
    const u32 i = i0 + t;
    const bool valid = i < m;
    float xi[F];
#pragma unroll
    for (int f = 0; f < F; ++f) xi[f] = valid ? x[(size_t)i * F + f] : 0.f;
    for (int o = 0; o < H; ++o) {
      float a = ws[oB1 + o];
#pragma unroll
      for (int f = 0; f < F; ++f) a = fmaf(ws[oW1 + o * F + f], xi[f], a);
      h1[o][t] = a > 0.f ? a : 0.f;
    }
    float out = ws[oB3];
    for (int o = 0; o < H; ++o) {
      float a = ws[oB2 + o];
#pragma unroll 16
      for (int j = 0; j < H; ++j) a = fmaf(ws[oW2 + o * H + j], h1[j][t], a);
      out = fmaf(ws[oW3 + o], a > 0.f ? a : 0.f, out);
    }
    if (valid) y[i] = out;
  }
}

constexpr int TS = 64;  // samples per gradient tile

// Gradient of the mean squared error L = (1/m) sum (y_i - t_i)^2 with
// respect to the parameters, the forward pass using the bf16 weights.  One
// block per tile of 64 samples; dense tile products in shared memory; block
// sums added to grad with atomics.
__global__ void k_mlp_grad(const float *x, const float *t, u32 m, const unsigned short *wb, float *grad,
                           float *loss) {
  extern __shared__ float sm[];
  float *ws = sm;                 // P
  float *X = ws + P + 3;          // TS x F   (+3 keeps the tiles 16-byte apart)
  float *H1 = X + TS * F;         // TS x H   post-activation
  float *H2 = H1 + TS * H;        // TS x H   post-activation
  float *D2 = H2 + TS * H;        // TS x H   dL/d(pre-activation 2)
  float *D1 = D2 + TS * H;        // TS x H   dL/d(pre-activation 1)
  float *dy = D1 + TS * H;        // TS
  load_weights(wb, ws);
  const u32 base = blockIdx.x * TS;
  for (int i = threadIdx.x; i < TS * F; i += blockDim.x) {
    u32 s = base + i / F;
    X[i] = s < m ? x[(size_t)s * F + i % F] : 0.f;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < TS * H; i += blockDim.x) {
    int s = i / H, o = i % H;
    float a = ws[oB1 + o];
    for (int f = 0; f < F; ++f) a = fmaf(ws[oW1 + o * F + f], X[s * F + f], a);
    H1[i] = a > 0.f ? a : 0.f;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < TS * H; i += blockDim.x) {
    int s = i / H, o = i % H;
    float a = ws[oB2 + o];
    for (int j = 0; j < H; ++j) a = fmaf(ws[oW2 + o * H + j], H1[s * H + j], a);
    H2[i] = a > 0.f ? a : 0.f;
  }
  __syncthreads();
  if (threadIdx.x < TS) {
    int s = threadIdx.x;
    float yv = ws[oB3];
    for (int o = 0; o < H; ++o) yv = fmaf(ws[oW3 + o], H2[s * H + o], yv);
    bool valid = base + s < m;
    float e = valid ? yv - t[base + s] : 0.f;
    dy[s] = 2.f * e / (float)m;
    float l = e * e / (float)m;
    for (int o = 16; o; o >>= 1) l += __shfl_down_sync(FULL, l, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, l);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < TS * H; i += blockDim.x) {
    int s = i / H, o = i % H;
    D2[i] = H2[i] > 0.f ? dy[s] * ws[oW3 + o] : 0.f;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < TS * H; i += blockDim.x) {
    int s = i / H, j = i % H;
    float a = 0.f;
    for (int o = 0; o < H; ++o) a = fmaf(D2[s * H + o], ws[oW2 + o * H + j], a);
    D1[i] = H1[i] > 0.f ? a : 0.f;
  }
  __syncthreads();
  // parameter gradients: sums over the tile's samples
  for (int p = threadIdx.x; p < P; p += blockDim.x) {
    float g = 0.f;
    if (p < oB1) {
      int o = p / F, f = p % F;
      for (int s = 0; s < TS; ++s) g = fmaf(D1[s * H + o], X[s * F + f], g);
    } else if (p < oW2) {
      int o = p - oB1;
      for (int s = 0; s < TS; ++s) g += D1[s * H + o];
    } else if (p < oB2) {
      int o = (p - oW2) / H, j = (p - oW2) % H;
      for (int s = 0; s < TS; ++s) g = fmaf(D2[s * H + o], H1[s * H + j], g);
    } else if (p < oW3) {
      int o = p - oB2;
      for (int s = 0; s < TS; ++s) g += D2[s * H + o];
    } else if (p < oB3) {
      int o = p - oW3;
      for (int s = 0; s < TS; ++s) g = fmaf(dy[s], H2[s * H + o], g);
    } else {
      for (int s = 0; s < TS; ++s) g += dy[s];
    }
    if (g != 0.f) atomicAdd(&grad[p], g);
  }
}

// Adam (Kingma & Ba 2015) on the fp32 master weights; refreshes the bf16 copy.
__global__ void k_adam(float *w, unsigned short *wb, float *mo, float *ve, const float *g, float lr, float b1,
                       float b2, float c1, float c2, float eps) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P; i += gridDim.x * blockDim.x) {
    float gi = g[i];
    float m = b1 * mo[i] + (1.f - b1) * gi;
    float v = b2 * ve[i] + (1.f - b2) * gi * gi;
    mo[i] = m;
    ve[i] = v;
    float wi = w[i] - lr * (m / c1) / (sqrtf(v / c2) + eps);
    w[i] = wi;
    wb[i] = __bfloat16_as_ushort(__float2bfloat16_rn(wi));
  }
}

__global__ void k_to_bf16(const float *w, unsigned short *wb) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P; i += gridDim.x * blockDim.x)
    wb[i] = __bfloat16_as_ushort(__float2bfloat16_rn(w[i]));
}

// He-uniform weights from splitmix64(seed ^ index); biases zero.
__global__ void k_mlp_init(float *w, u64 seed) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P; i += gridDim.x * blockDim.x) {
    u64 z = (seed ^ (u64)i) + 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    z ^= z >> 31;
    float u = (float)(z >> 40) * (1.0f / 16777216.0f) * 2.f - 1.f;  // [-1, 1)
    float fan_in = i < oB1 ? (float)F : (i >= oW2 && i < oB2) || (i >= oW3 && i < oB3) ? (float)H : 0.f;
    w[i] = fan_in > 0.f ? u * sqrtf(6.f / fan_in) : 0.f;
  }
}

// Order keys for predicted farness: smaller prediction first (float bits
// mapped to an order-preserving unsigned integer).
__global__ void k_score_keys(const float *y, u32 n, u32 *key, u32 *val) {
  for (u32 v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    u32 b = __float_as_uint(y[v]);
    key[v] = (b & 0x80000000u) ? ~b : (b | 0x80000000u);
    val[v] = v;
  }
}

}  // namespace

int filter_order(tkc_graph *g, const u32 *d_order_all, u32 *d_out, u32 *count);

static int ensure_mlp(tkc_ctx *ctx) {
  MlpState &s = ctx->mlp;
  if (s.w) return TKC_OK;
  TKC_TRY(cudaMalloc(&s.w, P * sizeof(float)));
  TKC_TRY(cudaMalloc(&s.wb, P * sizeof(unsigned short)));
  TKC_TRY(cudaMalloc(&s.m, P * sizeof(float)));
  TKC_TRY(cudaMalloc(&s.v, P * sizeof(float)));
  TKC_TRY(cudaMalloc(&s.grad, P * sizeof(float)));
  TKC_TRY(cudaMalloc(&s.loss, sizeof(float)));
  return TKC_OK;
}

void free_mlp(tkc_ctx *ctx) {
  MlpState &s = ctx->mlp;
  void *ptrs[] = {s.w, s.wb, s.m, s.v, s.grad, s.loss};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  s = MlpState();
}

static int reset_adam(tkc_ctx *ctx) {
  MlpState &s = ctx->mlp;
  TKC_TRY(cudaMemsetAsync(s.m, 0, P * sizeof(float), ctx->stream));
  TKC_TRY(cudaMemsetAsync(s.v, 0, P * sizeof(float), ctx->stream));
  s.step = 0;
  s.version++;
  s.ready = true;
  return TKC_OK;
}

int ensure_features(tkc_graph *g) {
  if (g->features) return TKC_OK;
  TKC_RC(ensure_reach_bounds(g));  // provides the SCC sizes
  TKC_RC(ensure_in_csr(g));
  cudaStream_t st = g->ctx->stream;
  const u32 n = g->n;
  if (n == 0) return TKC_OK;
  float *w2 = nullptr;
  u32 *c0 = nullptr, *c1 = nullptr;
  double *sums = nullptr;
  TKC_TRY(cudaMallocAsync(&g->features, (size_t)n * F * sizeof(float), st));
  TKC_TRY(cudaMallocAsync(&w2, (size_t)n * sizeof(float), st));
  TKC_TRY(cudaMallocAsync(&c0, (size_t)n * sizeof(u32), st));
  TKC_TRY(cudaMallocAsync(&c1, (size_t)n * sizeof(u32), st));
  TKC_TRY(cudaMallocAsync(&sums, 2 * F * sizeof(double), st));
  TKC_LAUNCH(k_two_walks<<<grid_of((u64)n * 32), 256, 0, st>>>(g->off, g->col, n, w2));
  TKC_LAUNCH(k_core_init<<<grid_of(n), 256, 0, st>>>(g->off, g->ioff, n, g->directed, c0));
  u32 *flag = nullptr;
  uint8_t *d0 = nullptr, *d1 = nullptr;
  TKC_TRY(cudaMallocAsync(&flag, sizeof(u32), st));
  TKC_TRY(cudaMallocAsync(&d0, n, st));
  TKC_TRY(cudaMallocAsync(&d1, n, st));
  TKC_TRY(cudaMemsetAsync(d0, 1, n, st));  // every vertex is computed in the first step
  for (u64 it = 0;; ++it) {
    // a step that changes something lowers at least one value, and the values
    // start at the degrees: 2 arcs + 1 steps suffice
    if (it > 2 * g->arcs + 1) return TKC_ETIMEOUT;
    TKC_TRY(cudaMemsetAsync(flag, 0, sizeof(u32), st));
    TKC_TRY(cudaMemsetAsync(d1, 0, n, st));
    TKC_LAUNCH(k_core_step<<<grid_of(n, kCoreTPB), kCoreTPB, 0, st>>>(g->off, g->col, g->ioff, g->icol, n, g->directed, c0, c1, d0,
                                                       d1, flag));
    std::swap(c0, c1);
    std::swap(d0, d1);
    u32 h = 0;
    TKC_TRY(cudaMemcpyAsync(&h, flag, sizeof(u32), cudaMemcpyDeviceToHost, st));
    TKC_TRY(cudaStreamSynchronize(st));
    if (!h) break;
  }
  TKC_TRY(cudaFreeAsync(flag, st));
  TKC_TRY(cudaFreeAsync(d0, st));
  TKC_TRY(cudaFreeAsync(d1, st));
  TKC_TRY(cudaMemsetAsync(sums, 0, 2 * F * sizeof(double), st));
  TKC_LAUNCH(k_features_raw<<<grid_of(n), 256, 0, st>>>(g->off, g->ioff, w2, c0, g->scc_size, n, g->features, sums));
  TKC_LAUNCH(k_features_standardize<<<grid_of((u64)n * F), 256, 0, st>>>(g->features, n, sums));
  TKC_TRY(cudaGetLastError());
  TKC_TRY(cudaFreeAsync(w2, st));
  TKC_TRY(cudaFreeAsync(c0, st));
  TKC_TRY(cudaFreeAsync(c1, st));
  TKC_TRY(cudaFreeAsync(sums, st));
  return TKC_OK;
}

static int forward(tkc_ctx *ctx, const float *x, u32 m, float *y) {
  if (m == 0) return TKC_OK;
  TKC_LAUNCH(k_mlp_forward<<<grid_of(m, FT), FT, 0, ctx->stream>>>(x, m, ctx->mlp.wb, y));
  TKC_TRY(cudaGetLastError());
  return TKC_OK;
}

int ensure_learned_order(tkc_graph *g) {
  tkc_ctx *ctx = g->ctx;
  if (!ctx->mlp.ready) return TKC_EINVAL;
  if (g->learned_order && g->learned_version == ctx->mlp.version) return TKC_OK;
  TKC_RC(ensure_features(g));
  cudaStream_t st = ctx->stream;
  const u32 n = g->n;
  if (!g->learned_order) TKC_TRY(cudaMallocAsync(&g->learned_order, std::max<size_t>(n, 1) * sizeof(u32), st));
  if (n == 0) {
    g->n_src_learned = 0;
    g->learned_version = ctx->mlp.version;
    return TKC_OK;
  }
  float *y = nullptr;
  u32 *key = nullptr, *val = nullptr;
  TKC_TRY(cudaMallocAsync(&y, (size_t)n * sizeof(float), st));
  TKC_TRY(cudaMallocAsync(&key, (size_t)n * sizeof(u32), st));
  TKC_TRY(cudaMallocAsync(&val, (size_t)n * sizeof(u32), st));
  TKC_RC(forward(ctx, g->features, n, y));
  TKC_LAUNCH(k_score_keys<<<grid_of(n), 256, 0, st>>>(y, n, key, val));
  TKC_RC(radix_sort_u32_pairs(key, val, n, 32, st));  // stable: equal predictions keep id order
  TKC_RC(filter_order(g, val, g->learned_order, &g->n_src_learned));
  TKC_TRY(cudaFreeAsync(y, st));
  TKC_TRY(cudaFreeAsync(key, st));
  TKC_TRY(cudaFreeAsync(val, st));
  g->learned_version = ctx->mlp.version;
  return TKC_OK;
}

namespace {
__global__ void k_mark_prefix(const u32 *order, u32 count, uint8_t *mark) {
  for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) mark[order[i]] = 1;
}

__global__ void k_unmarked_flags(const u32 *order, u32 n, const uint8_t *mark, u32 *flag) {
  for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) flag[i] = !mark[order[i]];
  if (blockIdx.x == 0 && threadIdx.x == 0) flag[n] = 0;
}

__global__ void k_compact_into(const u32 *order, const u32 *pos, u32 n, u32 *out) {
  for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    if (pos[i + 1] != pos[i]) out[pos[i]] = order[i];
}
}  // namespace

int scan_exclusive_u32(const u32 *in, u32 *out, u64 len, u32 *tmp, cudaStream_t st);

// Seeded order: the `prefix` sources the model predicts closest first (they
// are searched without cutting and set x from exact farness), then every
// other source in the degree order.
int ensure_seeded_order(tkc_graph *g, u32 prefix, bool nb) {
  tkc_ctx *ctx = g->ctx;
  TKC_RC(ensure_learned_order(g));
  TKC_RC(ensure_degree_order(g));
  if (nb && !g->nb_order) return TKC_EINVAL;
  prefix = std::min(prefix, g->n_src_learned);
  const int base_kind = nb ? 1 : 0;
  if (g->seeded_order && g->seeded_version == ctx->mlp.version && g->seeded_prefix == prefix &&
      g->seeded_base == base_kind && (!nb || g->seeded_nb_cap == g->nb_cap))
    return TKC_OK;
  cudaStream_t st = ctx->stream;
  const u32 *base = nb ? g->nb_order : g->deg_order;
  const u32 ns = nb ? g->n_src_nb : g->n_src_deg;
  if (!g->seeded_order) TKC_TRY(cudaMallocAsync(&g->seeded_order, std::max<size_t>(g->n, 1) * sizeof(u32), st));
  uint8_t *mark = nullptr;
  u32 *pos = nullptr, *tmp = nullptr;
  TKC_TRY(cudaMallocAsync(&mark, std::max<size_t>(g->n, 1), st));
  TKC_TRY(cudaMallocAsync(&pos, ((size_t)ns + 1) * sizeof(u32), st));
  TKC_TRY(cudaMallocAsync(&tmp, ((size_t)ns + 1) / 4096 * sizeof(u32) + 16, st));
  TKC_TRY(cudaMemsetAsync(mark, 0, std::max<size_t>(g->n, 1), st));
  if (prefix) {
    TKC_LAUNCH(k_mark_prefix<<<grid_of(prefix), 256, 0, st>>>(g->learned_order, prefix, mark));
    TKC_TRY(cudaMemcpyAsync(g->seeded_order, g->learned_order, prefix * sizeof(u32), cudaMemcpyDeviceToDevice, st));
  }
  TKC_LAUNCH(k_unmarked_flags<<<grid_of(ns + 1), 256, 0, st>>>(base, ns, mark, pos));
  TKC_RC(scan_exclusive_u32(pos, pos, (u64)ns + 1, tmp, st));
  TKC_LAUNCH(k_compact_into<<<grid_of(ns), 256, 0, st>>>(base, pos, ns, g->seeded_order + prefix));
  TKC_TRY(cudaGetLastError());
  TKC_TRY(cudaFreeAsync(mark, st));
  TKC_TRY(cudaFreeAsync(pos, st));
  TKC_TRY(cudaFreeAsync(tmp, st));
  TKC_TRY(cudaStreamSynchronize(st));
  g->seeded_version = ctx->mlp.version;
  g->seeded_prefix = prefix;
  g->seeded_base = base_kind;
  g->seeded_nb_cap = nb ? g->nb_cap : 0;
  return TKC_OK;
}

}  // namespace tkc

using namespace tkc;

extern "C" {

int tkc_mlp_init(tkc_ctx *ctx, uint64_t seed) {
  if (!ctx) return TKC_EINVAL;
  TKC_TRY(cudaSetDevice(ctx->device));
  TKC_RC(ensure_mlp(ctx));
  TKC_LAUNCH(k_mlp_init<<<grid_of(P), 256, 0, ctx->stream>>>(ctx->mlp.w, seed));
  TKC_LAUNCH(k_to_bf16<<<grid_of(P), 256, 0, ctx->stream>>>(ctx->mlp.w, ctx->mlp.wb));
  TKC_RC(reset_adam(ctx));
  TKC_TRY(cudaStreamSynchronize(ctx->stream));
  return TKC_OK;
}

int tkc_set_source_model(tkc_ctx *ctx, const float *params, uint32_t nparams) {
  if (!ctx || !params || nparams != (uint32_t)P) return TKC_EINVAL;
  TKC_TRY(cudaSetDevice(ctx->device));
  TKC_RC(ensure_mlp(ctx));
  TKC_TRY(cudaMemcpyAsync(ctx->mlp.w, params, P * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
  TKC_LAUNCH(k_to_bf16<<<grid_of(P), 256, 0, ctx->stream>>>(ctx->mlp.w, ctx->mlp.wb));
  TKC_RC(reset_adam(ctx));
  TKC_TRY(cudaStreamSynchronize(ctx->stream));
  return TKC_OK;
}

int tkc_get_source_model(tkc_ctx *ctx, float *params, uint32_t nparams) {
  if (!ctx || !params || nparams != (uint32_t)P || !ctx->mlp.ready) return TKC_EINVAL;
  TKC_TRY(cudaSetDevice(ctx->device));
  TKC_TRY(cudaMemcpyAsync(params, ctx->mlp.w, P * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
  TKC_TRY(cudaStreamSynchronize(ctx->stream));
  return TKC_OK;
}

int tkc_vertex_features(tkc_graph *g, float *x) {
  if (!g || (!x && g->n)) return TKC_EINVAL;
  TKC_TRY(cudaSetDevice(g->ctx->device));
  TKC_RC(ensure_features(g));
  if (g->n)
    TKC_TRY(cudaMemcpyAsync(x, g->features, (size_t)g->n * F * sizeof(float), cudaMemcpyDeviceToDevice,
                            g->ctx->stream));
  TKC_TRY(cudaStreamSynchronize(g->ctx->stream));
  return TKC_OK;
}

int tkc_mlp_forward(tkc_ctx *ctx, const float *x, uint32_t m, float *y) {
  if (!ctx || (m && (!x || !y)) || !ctx->mlp.ready) return TKC_EINVAL;
  TKC_TRY(cudaSetDevice(ctx->device));
  TKC_RC(forward(ctx, x, m, y));
  TKC_TRY(cudaStreamSynchronize(ctx->stream));
  return TKC_OK;
}

static int gradient(tkc_ctx *ctx, const float *x, const float *t, u32 m, float *loss) {
  cudaStream_t st = ctx->stream;
  MlpState &s = ctx->mlp;
  TKC_TRY(cudaMemsetAsync(s.grad, 0, P * sizeof(float), st));
  TKC_TRY(cudaMemsetAsync(s.loss, 0, sizeof(float), st));
  size_t smem = (P + 3 + TS * F + 4 * TS * H + TS) * sizeof(float);
  TKC_TRY(cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  TKC_LAUNCH(k_mlp_grad<<<(m + TS - 1) / TS, 256, smem, st>>>(x, t, m, s.wb, s.grad, s.loss));
  TKC_TRY(cudaGetLastError());
  if (loss) TKC_TRY(cudaMemcpyAsync(loss, s.loss, sizeof(float), cudaMemcpyDeviceToHost, st));
  return TKC_OK;
}

int tkc_mlp_gradient(tkc_ctx *ctx, const float *x, const float *t, uint32_t m, float *grad, float *loss) {
  if (!ctx || !x || !t || !grad || m == 0 || !ctx->mlp.ready) return TKC_EINVAL;
  TKC_TRY(cudaSetDevice(ctx->device));
  TKC_RC(gradient(ctx, x, t, m, loss));
  TKC_TRY(cudaMemcpyAsync(grad, ctx->mlp.grad, P * sizeof(float), cudaMemcpyDeviceToDevice, ctx->stream));
  TKC_TRY(cudaStreamSynchronize(ctx->stream));
  return TKC_OK;
}

int tkc_mlp_train_step(tkc_ctx *ctx, const float *x, const float *t, uint32_t m, float lr, float *loss) {
  if (!ctx || !x || !t || m == 0 || !ctx->mlp.ready || !(lr > 0.f)) return TKC_EINVAL;
  TKC_TRY(cudaSetDevice(ctx->device));
  MlpState &s = ctx->mlp;
  TKC_RC(gradient(ctx, x, t, m, loss));
  s.step++;
  const double b1 = 0.9, b2 = 0.999;
  float c1 = (float)(1.0 - pow(b1, (double)s.step)), c2 = (float)(1.0 - pow(b2, (double)s.step));
  TKC_LAUNCH(k_adam<<<grid_of(P), 256, 0, ctx->stream>>>(s.w, s.wb, s.m, s.v, s.grad, lr, (float)b1, (float)b2, c1,
                                                         c2, 1e-8f));
  TKC_TRY(cudaGetLastError());
  s.version++;
  TKC_TRY(cudaStreamSynchronize(ctx->stream));
  return TKC_OK;
}

}  // extern "C"
