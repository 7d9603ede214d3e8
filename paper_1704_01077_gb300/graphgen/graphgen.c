/*
 * Seeded synthetic graph generators shared by the tests, the benchmark and the
 * CPU oracle's test inputs.  This file holds input generation only: no BFS, no
 * distance sums, no bounds.  Every generator is deterministic in its seed and
 * independent of the number of threads.
 *
 * Random numbers: splitmix64 (Steele, Lea, Flood, "Fast splittable pseudorandom
 * number generators", OOPSLA 2014), one stream per fixed-size chunk of work so
 * that chunks can be generated in parallel with identical output.
 *
 * Output format: CSR with uint32 row offsets (n+1) and uint32 column ids, every
 * row sorted ascending, no self-loops, no duplicate arcs.  Undirected graphs are
 * returned with both arc directions present.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define GG_OK 0
#define GG_ENOMEM -3
#define GG_EINVAL -1

static inline uint64_t sm64_next(uint64_t *state) {
  uint64_t z = (*state += 0x9e3779b97f4a7c15ULL);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

/* One splitmix64 output of a given input, used to derive sub-seeds. */
uint64_t gg_splitmix64(uint64_t x) {
  uint64_t s = x;
  return sm64_next(&s);
}

/* uniform integer in [0, bound) by the multiply-high method */
static inline uint32_t uniform_below(uint64_t *st, uint32_t bound) {
  unsigned __int128 p = (unsigned __int128)sm64_next(st) * (unsigned __int128)bound;
  return (uint32_t)(p >> 64);
}

static inline double uniform01(uint64_t *st) {
  return (double)(sm64_next(st) >> 11) * (1.0 / 9007199254740992.0);
}

void gg_free(void *p) { free(p); }

/* ---------------------------------------------------------------------- */
/* Edge list -> sorted, deduplicated CSR                                  */
/* ---------------------------------------------------------------------- */

static int cmp_u32(const void *a, const void *b) {
  uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
  return (x > y) - (x < y);
}

static void sort_small(uint32_t *a, uint64_t len) {
  if (len < 32) {
    for (uint64_t i = 1; i < len; ++i) {
      uint32_t v = a[i];
      uint64_t j = i;
      while (j > 0 && a[j - 1] > v) { a[j] = a[j - 1]; --j; }
      a[j] = v;
    }
  } else {
    qsort(a, (size_t)len, sizeof(uint32_t), cmp_u32);
  }
}

/*
 * Builds a CSR from arcs (src[i] -> dst[i]).  If symmetric != 0 every arc is
 * inserted in both directions.  Self-loops and duplicates are dropped.
 * Returns malloc'ed offsets / columns.
 */
static int build_csr(uint32_t n, uint64_t narcs, const uint32_t *src, const uint32_t *dst,
                     int symmetric, uint32_t **off_out, uint32_t **col_out, uint64_t *m_out) {
  uint64_t *cnt = (uint64_t *)calloc((size_t)n + 1, sizeof(uint64_t));
  if (!cnt) return GG_ENOMEM;
  for (uint64_t i = 0; i < narcs; ++i) {
    if (src[i] == dst[i]) continue;
    cnt[src[i] + 1]++;
    if (symmetric) cnt[dst[i] + 1]++;
  }
  for (uint32_t v = 0; v < n; ++v) cnt[v + 1] += cnt[v];
  uint64_t total = cnt[n];
  uint32_t *tmp = (uint32_t *)malloc((size_t)(total ? total : 1) * sizeof(uint32_t));
  uint64_t *pos = (uint64_t *)malloc(((size_t)n + 1) * sizeof(uint64_t));
  if (!tmp || !pos) { free(cnt); free(tmp); free(pos); return GG_ENOMEM; }
  memcpy(pos, cnt, ((size_t)n + 1) * sizeof(uint64_t));
  for (uint64_t i = 0; i < narcs; ++i) {
    if (src[i] == dst[i]) continue;
    tmp[pos[src[i]]++] = dst[i];
    if (symmetric) tmp[pos[dst[i]]++] = src[i];
  }
  free(pos);
  /* sort and deduplicate each row in place, then compact */
  uint32_t *off = (uint32_t *)malloc(((size_t)n + 1) * sizeof(uint32_t));
  if (!off) { free(cnt); free(tmp); return GG_ENOMEM; }
  uint64_t w = 0;
  for (uint32_t v = 0; v < n; ++v) {
    uint64_t b = cnt[v], e = cnt[v + 1];
    sort_small(tmp + b, e - b);
    off[v] = (uint32_t)w;
    for (uint64_t i = b; i < e; ++i) {
      if (i > b && tmp[i] == tmp[i - 1]) continue;
      tmp[w++] = tmp[i];
    }
  }
  off[n] = (uint32_t)w;
  free(cnt);
  uint32_t *col = (uint32_t *)realloc(tmp, (size_t)(w ? w : 1) * sizeof(uint32_t));
  if (!col) col = tmp;
  *off_out = off;
  *col_out = col;
  *m_out = w;
  return GG_OK;
}

/* CSR from an explicit arc list (used for small hand-made graphs). */
int gg_from_arcs(uint32_t n, uint64_t narcs, const uint32_t *src, const uint32_t *dst, int symmetric,
                 uint32_t **off, uint32_t **col, uint64_t *m) {
  for (uint64_t i = 0; i < narcs; ++i)
    if (src[i] >= n || dst[i] >= n) return GG_EINVAL;
  return build_csr(n, narcs, src, dst, symmetric, off, col, m);
}

/* ---------------------------------------------------------------------- */
/* Barabasi-Albert preferential attachment                                 */
/* ---------------------------------------------------------------------- */
/*
 * Starts from the complete graph on m0 = medges+1 vertices.  Every later vertex
 * v attaches to medges distinct earlier vertices, each drawn with probability
 * proportional to its current degree by sampling a uniform position in the list
 * of all edge endpoints (rejecting repeats).  The result is connected and
 * undirected with C(m0,2) + medges*(n-m0) edges.
 */
int gg_barabasi_albert(uint32_t n, uint32_t medges, uint64_t seed,
                       uint32_t **off, uint32_t **col, uint64_t *m) {
  if (medges == 0 || n < medges + 1) return GG_EINVAL;
  uint32_t m0 = medges + 1;
  uint64_t nedges = (uint64_t)m0 * (m0 - 1) / 2 + (uint64_t)medges * (n - m0);
  uint32_t *src = (uint32_t *)malloc((size_t)nedges * sizeof(uint32_t));
  uint32_t *dst = (uint32_t *)malloc((size_t)nedges * sizeof(uint32_t));
  uint32_t *ends = (uint32_t *)malloc((size_t)nedges * 2 * sizeof(uint32_t));
  uint32_t *pick = (uint32_t *)malloc((size_t)medges * sizeof(uint32_t));
  if (!src || !dst || !ends || !pick) { free(src); free(dst); free(ends); free(pick); return GG_ENOMEM; }
  uint64_t e = 0, ne = 0;
  for (uint32_t a = 0; a < m0; ++a)
    for (uint32_t b = a + 1; b < m0; ++b) {
      src[e] = a; dst[e] = b; ++e;
      ends[ne++] = a; ends[ne++] = b;
    }
  uint64_t st = seed;
  for (uint32_t v = m0; v < n; ++v) {
    uint32_t got = 0;
    while (got < medges) {
      uint64_t idx;
      {
        unsigned __int128 p = (unsigned __int128)sm64_next(&st) * (unsigned __int128)ne;
        idx = (uint64_t)(p >> 64);
      }
      uint32_t t = ends[idx];
      int dup = 0;
      for (uint32_t j = 0; j < got; ++j) if (pick[j] == t) { dup = 1; break; }
      if (!dup) pick[got++] = t;
    }
    for (uint32_t j = 0; j < medges; ++j) {
      src[e] = v; dst[e] = pick[j]; ++e;
      ends[ne++] = v; ends[ne++] = pick[j];
    }
  }
  free(ends); free(pick);
  int rc = build_csr(n, e, src, dst, 1, off, col, m);
  free(src); free(dst);
  return rc;
}

/* ---------------------------------------------------------------------- */
/* R-MAT (Chakrabarti, Zhan, Faloutsos 2004), directed                     */
/* ---------------------------------------------------------------------- */
#define GG_CHUNK (1u << 20)

/*
 * ef * 2^scale arcs; each arc descends `scale` levels of the adjacency matrix
 * choosing quadrant a/b/c/d (no noise).  Self-loops and duplicate arcs are
 * removed.  If permute != 0 vertex ids are relabelled by a seeded Fisher-Yates
 * shuffle so that ids carry no degree information.
 */
int gg_rmat(uint32_t scale, uint32_t edge_factor, double a, double b, double c, uint64_t seed,
            int permute, int symmetric, uint32_t **off, uint32_t **col, uint64_t *m) {
  if (scale == 0 || scale > 30) return GG_EINVAL;
  uint32_t n = 1u << scale;
  uint64_t narcs = (uint64_t)edge_factor << scale;
  uint32_t *src = (uint32_t *)malloc((size_t)(narcs ? narcs : 1) * sizeof(uint32_t));
  uint32_t *dst = (uint32_t *)malloc((size_t)(narcs ? narcs : 1) * sizeof(uint32_t));
  uint32_t *perm = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
  if (!src || !dst || !perm) { free(src); free(dst); free(perm); return GG_ENOMEM; }
  /* cumulative thresholds on 16-bit uniforms */
  uint32_t ta = (uint32_t)(a * 65536.0), tb = (uint32_t)((a + b) * 65536.0),
           tc = (uint32_t)((a + b + c) * 65536.0);
  int64_t nchunks = (int64_t)((narcs + GG_CHUNK - 1) / GG_CHUNK);
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t ch = 0; ch < nchunks; ++ch) {
    uint64_t st = gg_splitmix64(seed ^ (0xA5A5A5A5ULL * (uint64_t)(ch + 1)));
    uint64_t lo = (uint64_t)ch * GG_CHUNK, hi = lo + GG_CHUNK;
    if (hi > narcs) hi = narcs;
    for (uint64_t i = lo; i < hi; ++i) {
      uint32_t u = 0, v = 0;
      uint64_t r = 0;
      for (uint32_t lvl = 0; lvl < scale; ++lvl) {
        if ((lvl & 3) == 0) r = sm64_next(&st);
        uint32_t x = (uint32_t)(r & 0xFFFF);
        r >>= 16;
        uint32_t bit = scale - 1 - lvl;
        if (x < ta) {
        } else if (x < tb) {
          v |= 1u << bit;
        } else if (x < tc) {
          u |= 1u << bit;
        } else {
          u |= 1u << bit;
          v |= 1u << bit;
        }
      }
      src[i] = u;
      dst[i] = v;
    }
  }
  for (uint32_t i = 0; i < n; ++i) perm[i] = i;
  if (permute) {
    uint64_t st = gg_splitmix64(seed ^ 0x5EED5EEDULL);
    for (uint32_t i = n - 1; i > 0; --i) {
      uint32_t j = uniform_below(&st, i + 1);
      uint32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)narcs; ++i) {
      src[i] = perm[src[i]];
      dst[i] = perm[dst[i]];
    }
  }
  free(perm);
  int rc = build_csr(n, narcs, src, dst, symmetric, off, col, m);
  free(src); free(dst);
  return rc;
}

/* ---------------------------------------------------------------------- */
/* Erdos-Renyi with a fixed number of uniform arcs                         */
/* ---------------------------------------------------------------------- */
int gg_erdos_renyi(uint32_t n, uint64_t narcs, uint64_t seed, int symmetric,
                   uint32_t **off, uint32_t **col, uint64_t *m) {
  if (n == 0) return GG_EINVAL;
  uint32_t *src = (uint32_t *)malloc((size_t)(narcs ? narcs : 1) * sizeof(uint32_t));
  uint32_t *dst = (uint32_t *)malloc((size_t)(narcs ? narcs : 1) * sizeof(uint32_t));
  if (!src || !dst) { free(src); free(dst); return GG_ENOMEM; }
  uint64_t st = seed;
  for (uint64_t i = 0; i < narcs; ++i) {
    src[i] = uniform_below(&st, n);
    dst[i] = uniform_below(&st, n);
  }
  int rc = build_csr(n, narcs, src, dst, symmetric, off, col, m);
  free(src); free(dst);
  return rc;
}

/* Uniform double in [0,1) from a seed and an index, for Python-side recipes. */
double gg_uniform(uint64_t seed, uint64_t index) {
  uint64_t st = gg_splitmix64(seed ^ (index * 0x9E3779B97F4A7C15ULL));
  return uniform01(&st);
}
