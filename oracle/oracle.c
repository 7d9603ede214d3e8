/*
 * CPU oracle for exact top-k closeness centrality (Bergamini, Borassi,
 * Crescenzi, Marino, Meyerhenke, "Computing top-k Closeness Centrality Faster
 * in Unweighted Graphs", arXiv 1704.01077).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA path is checked against.  It shares no code, header, table or helper
 * with the CUDA library and must never be linked into, or called by, the
 * product path.  Only the tests, the package's smoke check and the benchmark's
 * CPU-baseline leg use it.
 *
 * Graph input everywhere: CSR, uint32 row offsets off[0..n], uint32 column ids
 * col[0..off[n]), out-arcs of each vertex (undirected graphs hold both arc
 * directions).
 *
 * Definitions followed (Section 2, notation table):
 *   R(v) = vertices reachable from v (v included), r(v) = |R(v)|,
 *   S(v) = sum over w in R(v) of d(v,w),
 *   f(v) = (n-1) S(v) / (r(v)-1)^2,  c(v) = 1/f(v), and c(v) = 0 when r(v) = 1.
 *
 * Parity status of each function is stated beside it.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef unsigned __int128 u128;

#define ORC_OK 0
#define ORC_EINVAL -1
#define ORC_ENOMEM -3

/* ---------------------------------------------------------------------- */
/* Textbook BFS (Section 1: "the textbook algorithm", one BFS per vertex)  */
/* ---------------------------------------------------------------------- */

/* BFS from one source with a FIFO queue; returns S(v), r(v), arcs scanned.
 * dist must hold n entries set to UINT32_MAX and is restored on return. */
static void bfs_one(uint32_t n, const uint32_t *off, const uint32_t *col, uint32_t s,
                    uint32_t *dist, uint32_t *queue, uint64_t *S_out, uint32_t *r_out) {
  (void)n;
  uint32_t head = 0, tail = 0;
  uint64_t S = 0;
  dist[s] = 0;
  queue[tail++] = s;
  while (head < tail) {
    uint32_t u = queue[head++];
    for (uint32_t e = off[u]; e < off[u + 1]; ++e) {
      uint32_t w = col[e];
      if (dist[w] == UINT32_MAX) {
        dist[w] = dist[u] + 1;
        S += dist[w];
        queue[tail++] = w;
      }
    }
  }
  for (uint32_t i = 0; i < tail; ++i) dist[queue[i]] = UINT32_MAX;
  *S_out = S;
  *r_out = tail;
}

/* S(v) and r(v) for the listed sources (all vertices if srcs == NULL).
 * Pinned by: Floyd-Warshall on small graphs, closed forms, networkx. */
int orc_bfs_sums(uint32_t n, const uint32_t *off, const uint32_t *col, uint32_t nsrc,
                 const uint32_t *srcs, uint64_t *S, uint32_t *r, int nthreads) {
  if (n == 0) return ORC_OK;
  int rc = ORC_OK;
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel num_threads(nthreads)
#endif
  {
    uint32_t *dist = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
    uint32_t *queue = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
    if (!dist || !queue) {
      rc = ORC_ENOMEM;
    } else {
      for (uint32_t i = 0; i < n; ++i) dist[i] = UINT32_MAX;
      int64_t cnt = srcs ? (int64_t)nsrc : (int64_t)n;
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 16)
#endif
      for (int64_t i = 0; i < cnt; ++i) {
        uint32_t s = srcs ? srcs[i] : (uint32_t)i;
        bfs_one(n, off, col, s, dist, queue, &S[i], &r[i]);
      }
    }
    free(dist);
    free(queue);
  }
  (void)nthreads;
  return rc;
}

/* All-pairs distances by Floyd-Warshall on a dense matrix (n <= 64); an
 * independent route to S(v) and r(v) used to pin the BFS above. */
int orc_floyd_warshall(uint32_t n, const uint32_t *off, const uint32_t *col, uint64_t *S, uint32_t *r) {
  if (n > 64) return ORC_EINVAL;
  const uint32_t INF = 1u << 20;
  uint32_t D[64][64];
  for (uint32_t i = 0; i < n; ++i)
    for (uint32_t j = 0; j < n; ++j) D[i][j] = (i == j) ? 0 : INF;
  for (uint32_t u = 0; u < n; ++u)
    for (uint32_t e = off[u]; e < off[u + 1]; ++e) D[u][col[e]] = 1;
  for (uint32_t m = 0; m < n; ++m)
    for (uint32_t i = 0; i < n; ++i)
      for (uint32_t j = 0; j < n; ++j)
        if (D[i][m] + D[m][j] < D[i][j]) D[i][j] = D[i][m] + D[m][j];
  for (uint32_t i = 0; i < n; ++i) {
    uint64_t s = 0;
    uint32_t c = 0;
    for (uint32_t j = 0; j < n; ++j)
      if (D[i][j] < INF) { s += D[i][j]; ++c; }
    S[i] = s;
    r[i] = c;
  }
  return ORC_OK;
}

/* ---------------------------------------------------------------------- */
/* Exact ordering by farness                                               */
/* ---------------------------------------------------------------------- */

/* Compares f(a) with f(b) exactly: f = (n-1) S / (r-1)^2, (n-1) cancels, so
 * compare S_a (r_b-1)^2 with S_b (r_a-1)^2 in 128-bit integers.  r = 1 means
 * closeness 0, i.e. farness +infinity (Section 2).  Returns -1, 0, 1. */
static int cmp_farness(uint64_t Sa, uint32_t ra, uint64_t Sb, uint32_t rb) {
  int inf_a = ra <= 1, inf_b = rb <= 1;
  if (inf_a || inf_b) return inf_a - inf_b;
  u128 lhs = (u128)Sa * (u128)((uint64_t)(rb - 1) * (uint64_t)(rb - 1));
  u128 rhs = (u128)Sb * (u128)((uint64_t)(ra - 1) * (uint64_t)(ra - 1));
  return (lhs > rhs) - (lhs < rhs);
}

int orc_cmp_farness(uint64_t Sa, uint32_t ra, uint64_t Sb, uint32_t rb) {
  return cmp_farness(Sa, ra, Sb, rb);
}

typedef struct {
  uint64_t S;
  uint32_t r;
  uint32_t id;
} entry_t;

static int cmp_entry(const void *pa, const void *pb) {
  const entry_t *a = (const entry_t *)pa, *b = (const entry_t *)pb;
  int c = cmp_farness(a->S, a->r, b->S, b->r);
  if (c) return c;
  return (a->id > b->id) - (a->id < b->id);
}

/* Top-k by closeness (Section 4: the k vertices of smallest farness), ties
 * broken by id; n_tied = number of vertices whose farness equals that of the
 * k-th returned vertex (the paper returns all of them).  Returns the number of
 * ids written, min(k, n). */
int orc_topk(uint32_t n, const uint64_t *S, const uint32_t *r, uint32_t k, uint32_t *ids,
             uint32_t *n_tied) {
  if (n == 0 || k == 0) { if (n_tied) *n_tied = 0; return 0; }
  entry_t *e = (entry_t *)malloc((size_t)n * sizeof(entry_t));
  if (!e) return ORC_ENOMEM;
  for (uint32_t v = 0; v < n; ++v) { e[v].S = S[v]; e[v].r = r[v]; e[v].id = v; }
  qsort(e, n, sizeof(entry_t), cmp_entry);
  uint32_t kk = k < n ? k : n;
  for (uint32_t i = 0; i < kk; ++i) ids[i] = e[i].id;
  if (n_tied) {
    uint32_t t = 0;
    for (uint32_t v = 0; v < n; ++v)
      if (cmp_farness(S[v], r[v], e[kk - 1].S, e[kk - 1].r) == 0) ++t;
    *n_tied = t;
  }
  free(e);
  return (int)kk;
}

/* f(v) and c(v) in IEEE double from the exact integers: one rounded product
 * and one rounded quotient each (Section 2's definitions). */
void orc_farness(uint32_t n, uint64_t S, uint32_t r, double *farness, double *closeness) {
  if (r <= 1) {
    *farness = INFINITY;
    *closeness = 0.0;
    return;
  }
  double num = (double)(n - 1) * (double)S;
  double den = (double)((uint64_t)(r - 1) * (uint64_t)(r - 1));
  *farness = num / den;
  *closeness = den / num;
}

/* ---------------------------------------------------------------------- */
/* computeBoundsDeg (Section 4): vertices by decreasing degree             */
/* ---------------------------------------------------------------------- */

/* Counting sort by out-degree, largest first; equal degrees keep increasing
 * id order (the sort is stable).  Pinned by numpy lexsort in the tests. */
int orc_degree_order(uint32_t n, const uint32_t *off, uint32_t *order) {
  if (n == 0) return ORC_OK;
  uint32_t maxd = 0;
  for (uint32_t v = 0; v < n; ++v) {
    uint32_t d = off[v + 1] - off[v];
    if (d > maxd) maxd = d;
  }
  uint32_t *start = (uint32_t *)calloc((size_t)maxd + 2, sizeof(uint32_t));
  if (!start) return ORC_ENOMEM;
  /* bucket b holds degree maxd - b, so bucket 0 is the largest degree */
  for (uint32_t v = 0; v < n; ++v) start[maxd - (off[v + 1] - off[v]) + 1]++;
  for (uint32_t b = 0; b <= maxd; ++b) start[b + 1] += start[b];
  for (uint32_t v = 0; v < n; ++v) order[start[maxd - (off[v + 1] - off[v])]++] = v;
  free(start);
  return ORC_OK;
}

/* ---------------------------------------------------------------------- */
/* Strongly connected components (Tarjan), iterative                        */
/* ---------------------------------------------------------------------- */

/* comp[v] = index of v's SCC; components are numbered in the order Tarjan's
 * algorithm completes them, which is a reverse topological order of the SCC
 * DAG (a component is completed after every component it reaches).
 * Returns the number of components.  Pinned by mutual reachability checks. */
int64_t orc_scc(uint32_t n, const uint32_t *off, const uint32_t *col, uint32_t *comp) {
  if (n == 0) return 0;
  uint32_t *index = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
  uint32_t *low = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
  uint32_t *stack = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
  uint8_t *onstack = (uint8_t *)calloc(n, 1);
  uint32_t *cs_v = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
  uint32_t *cs_e = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
  if (!index || !low || !stack || !onstack || !cs_v || !cs_e) {
    free(index); free(low); free(stack); free(onstack); free(cs_v); free(cs_e);
    return ORC_ENOMEM;
  }
  const uint32_t UNV = UINT32_MAX;
  for (uint32_t v = 0; v < n; ++v) index[v] = UNV;
  uint32_t next_index = 0, sp = 0, ncomp = 0;
  for (uint32_t root = 0; root < n; ++root) {
    if (index[root] != UNV) continue;
    uint32_t csp = 0;
    cs_v[csp] = root;
    cs_e[csp] = off[root];
    ++csp;
    index[root] = low[root] = next_index++;
    stack[sp++] = root;
    onstack[root] = 1;
    while (csp > 0) {
      uint32_t v = cs_v[csp - 1];
      if (cs_e[csp - 1] < off[v + 1]) {
        uint32_t w = col[cs_e[csp - 1]++];
        if (index[w] == UNV) {
          index[w] = low[w] = next_index++;
          stack[sp++] = w;
          onstack[w] = 1;
          cs_v[csp] = w;
          cs_e[csp] = off[w];
          ++csp;
        } else if (onstack[w] && index[w] < low[v]) {
          low[v] = index[w];
        }
      } else {
        if (low[v] == index[v]) {
          uint32_t w;
          do {
            w = stack[--sp];
            onstack[w] = 0;
            comp[w] = ncomp;
          } while (w != v);
          ++ncomp;
        }
        --csp;
        if (csp > 0) {
          uint32_t u = cs_v[csp - 1];
          if (low[v] < low[u]) low[u] = low[v];
        }
      }
    }
  }
  free(index); free(low); free(stack); free(onstack); free(cs_v); free(cs_e);
  return (int64_t)ncomp;
}

/* ---------------------------------------------------------------------- */
/* alpha / omega bounds on r(v) (Section 8.4, Algorithm 6)                  */
/* ---------------------------------------------------------------------- */

/*
 * alpha(v) <= r(v) <= omega(v).  Steps, in the paper's order:
 *  1. SCC DAG (V, E, w) with w(C) = |C| and E a set (no repeated SCC arcs).
 *  2. C~ = the biggest SCC; ties go to the SCC holding the smallest vertex id.
 *     Its reach is computed exactly by one BFS: alpha = omega = r(C~).
 *  3. In reverse topological order, for every other X:
 *       alpha(X) = w(X) + max over successors Y of alpha(Y)
 *       omega(X) = w(X) + sum over successors Y of omega(Y)
 *     and if X reaches C~, omega(X) = w(X) + omega(C~) + sum of omega(Y) over
 *     successors Y that are not reachable from C~.
 *  4. omega is clamped to n (the sums may exceed n).
 * Undirected graphs: alpha = omega = size of the connected component.
 * Pinned by alpha <= r <= omega against brute-force reach, exact values on
 * hand-built DAGs, and exactness on the biggest SCC.
 */
int orc_alpha_omega(uint32_t n, const uint32_t *off, const uint32_t *col, int directed,
                    uint32_t *alpha, uint32_t *omega) {
  if (n == 0) return ORC_OK;
  uint32_t *comp = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
  if (!comp) return ORC_ENOMEM;
  int64_t nc64 = orc_scc(n, off, col, comp);
  if (nc64 < 0) { free(comp); return (int)nc64; }
  uint32_t nc = (uint32_t)nc64;
  uint64_t *w = (uint64_t *)calloc(nc, sizeof(uint64_t));
  uint32_t *minid = (uint32_t *)malloc((size_t)nc * sizeof(uint32_t));
  if (!w || !minid) { free(comp); free(w); free(minid); return ORC_ENOMEM; }
  for (uint32_t c = 0; c < nc; ++c) minid[c] = UINT32_MAX;
  for (uint32_t v = 0; v < n; ++v) {
    w[comp[v]]++;
    if (v < minid[comp[v]]) minid[comp[v]] = v;
  }
  if (!directed) {
    /* undirected: every SCC is a connected component and r(v) is its size */
    for (uint32_t v = 0; v < n; ++v) alpha[v] = omega[v] = (uint32_t)w[comp[v]];
    free(comp); free(w); free(minid);
    return ORC_OK;
  }
  /* condensation arcs, deduplicated per source component */
  uint64_t m = off[n];
  uint32_t *cdeg = (uint32_t *)calloc((size_t)nc + 1, sizeof(uint32_t));
  uint32_t *carc = (uint32_t *)malloc((size_t)(m ? m : 1) * sizeof(uint32_t));
  uint32_t *mark = (uint32_t *)malloc((size_t)nc * sizeof(uint32_t));
  uint32_t *members_off = (uint32_t *)calloc((size_t)nc + 1, sizeof(uint32_t));
  uint32_t *members = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
  uint64_t *A = (uint64_t *)calloc(nc, sizeof(uint64_t));
  uint64_t *O = (uint64_t *)calloc(nc, sizeof(uint64_t));
  uint8_t *from_big = (uint8_t *)calloc(nc, 1);
  uint8_t *to_big = (uint8_t *)calloc(nc, 1);
  uint32_t *coff = (uint32_t *)malloc(((size_t)nc + 1) * sizeof(uint32_t));
  if (!cdeg || !carc || !mark || !members_off || !members || !A || !O || !from_big || !to_big || !coff) {
    free(comp); free(w); free(minid); free(cdeg); free(carc); free(mark); free(members_off);
    free(members); free(A); free(O); free(from_big); free(to_big); free(coff);
    return ORC_ENOMEM;
  }
  for (uint32_t v = 0; v < n; ++v) members_off[comp[v] + 1]++;
  for (uint32_t c = 0; c < nc; ++c) members_off[c + 1] += members_off[c];
  {
    uint32_t *fill = (uint32_t *)malloc((size_t)nc * sizeof(uint32_t));
    if (!fill) return ORC_ENOMEM;
    memcpy(fill, members_off, (size_t)nc * sizeof(uint32_t));
    for (uint32_t v = 0; v < n; ++v) members[fill[comp[v]]++] = v;
    free(fill);
  }
  for (uint32_t c = 0; c < nc; ++c) mark[c] = UINT32_MAX;
  uint64_t na = 0;
  for (uint32_t c = 0; c < nc; ++c) {
    coff[c] = (uint32_t)na;
    for (uint32_t i = members_off[c]; i < members_off[c + 1]; ++i) {
      uint32_t v = members[i];
      for (uint32_t e = off[v]; e < off[v + 1]; ++e) {
        uint32_t d = comp[col[e]];
        if (d != c && mark[d] != c) {
          mark[d] = c;
          carc[na++] = d;
        }
      }
    }
  }
  coff[nc] = (uint32_t)na;
  /* biggest SCC, ties to the one holding the smallest vertex id */
  uint32_t big = 0;
  for (uint32_t c = 1; c < nc; ++c)
    if (w[c] > w[big] || (w[c] == w[big] && minid[c] < minid[big])) big = c;
  /* exact reach of the biggest SCC: BFS over the condensation from it */
  uint32_t *q = mark; /* reuse as a queue */
  uint32_t qh = 0, qt = 0;
  from_big[big] = 1;
  q[qt++] = big;
  uint64_t reach_big = 0;
  while (qh < qt) {
    uint32_t c = q[qh++];
    reach_big += w[c];
    for (uint32_t i = coff[c]; i < coff[c + 1]; ++i)
      if (!from_big[carc[i]]) { from_big[carc[i]] = 1; q[qt++] = carc[i]; }
  }
  /* Tarjan numbers components in reverse topological order: successors of c
   * have smaller numbers, so increasing c is the order Algorithm 6 needs.
   * "X reaches C~" is known once every successor is processed. */
  for (uint32_t c = 0; c < nc; ++c) {
    if (c == big) {
      A[c] = O[c] = reach_big;
      to_big[c] = 1;
      continue;
    }
    uint64_t a = 0, o = 0, o2 = 0;
    int reaches = 0;
    for (uint32_t i = coff[c]; i < coff[c + 1]; ++i) {
      uint32_t y = carc[i];
      if (A[y] > a) a = A[y];
      o += O[y];
      if (!from_big[y]) o2 += O[y];
      if (to_big[y]) reaches = 1;
    }
    if (reaches) {
      to_big[c] = 1;
      o = o2 + O[big];
    }
    A[c] = a + w[c];
    O[c] = o + w[c];
    if (O[c] > n) O[c] = n;
  }
  for (uint32_t v = 0; v < n; ++v) {
    alpha[v] = (uint32_t)A[comp[v]];
    omega[v] = (uint32_t)(O[comp[v]] > n ? n : O[comp[v]]);
  }
  free(comp); free(w); free(minid); free(cdeg); free(carc); free(mark); free(members_off);
  free(members); free(A); free(O); free(from_big); free(to_big); free(coff);
  return ORC_OK;
}

/* ---------------------------------------------------------------------- */
/* Closeness on trees (Section 5, Algorithm 2)                              */
/* ---------------------------------------------------------------------- */

/* Level counts of every vertex advance together: |N_1(s)| = deg(s); at level 2
 * |N_2(s)| = sum over neighbours w of |N_1(w)| minus deg(s); at level k > 2 it
 * is the sum of |N_{k-1}(w)| over neighbours minus |N_{k-2}(s)| (deg(s) - 1)
 * (Eq. 2).  S(s) accumulates k |N_k(s)| until every count is zero.  Exact on
 * trees (Prop. 2); used to pin the BFS on trees.  Input must be a tree. */
int orc_tree_sums(uint32_t n, const uint32_t *off, const uint32_t *col, uint64_t *S) {
  if (n == 0) return ORC_OK;
  int64_t *prev2 = (int64_t *)calloc(n, sizeof(int64_t));
  int64_t *prev1 = (int64_t *)malloc((size_t)n * sizeof(int64_t));
  int64_t *cur = (int64_t *)malloc((size_t)n * sizeof(int64_t));
  if (!prev2 || !prev1 || !cur) { free(prev2); free(prev1); free(cur); return ORC_ENOMEM; }
  for (uint32_t s = 0; s < n; ++s) {
    prev1[s] = (int64_t)(off[s + 1] - off[s]);
    S[s] = (uint64_t)prev1[s];
  }
  for (uint32_t level = 2;; ++level) {
    int any = 0;
    for (uint32_t s = 0; s < n; ++s) {
      int64_t deg = (int64_t)(off[s + 1] - off[s]);
      int64_t sum = 0;
      for (uint32_t e = off[s]; e < off[s + 1]; ++e) sum += prev1[col[e]];
      if (level == 2)
        cur[s] = sum - deg;
      else
        cur[s] = sum - prev2[s] * (deg - 1);
    }
    for (uint32_t s = 0; s < n; ++s) {
      prev2[s] = prev1[s];
      prev1[s] = cur[s];
      if (cur[s] > 0) {
        S[s] += (uint64_t)level * (uint64_t)cur[s];
        any = 1;
      }
    }
    if (!any || level > n + 1) break;
  }
  free(prev2); free(prev1); free(cur);
  return ORC_OK;
}

/* ---------------------------------------------------------------------- */
/* computeBoundsNB: neighbourhood-based lower bound (Section 5, Algorithm 3; */
/* directed graphs Eq. 3; unknown reach Section 8.1, Eq. 6)                  */
/* ---------------------------------------------------------------------- */

/* Counts are exact until they reach this value; any count >= n may stand for
 * "at least n" and every count at or above it is stored as exactly this. */
#define ORC_NB_CAP ((uint64_t)1 << 32)
/* Bits below the binary point of the order key floor(L' * 2^46), L' = S~/(r-1)^2. */
#define ORC_NB_FRAC 46

/* One candidate reach r of Eq. 6 with its sum bound S~(r); keeps the smallest
 * ratio S~/(r-1)^2 (the first one on ties: candidates come in increasing r). */
static void nb_candidate(uint64_t S, uint64_t r, int *have, uint64_t *bS, uint64_t *br) {
  if (!*have) { *have = 1; *bS = S; *br = r; return; }
  u128 lhs = (u128)S * (u128)((*br - 1) * (*br - 1));
  u128 rhs = (u128)*bS * (u128)((r - 1) * (r - 1));
  if (lhs < rhs) { *bS = S; *br = r; }
}

/*
 * Upper bounds N~_k(s) on the number of vertices at distance k from s, all
 * vertices advancing one level per sweep:
 *   N~_0(s) = 1, N~_1(s) = outdeg(s);
 *   undirected (Eq. 2, Algorithm 3): N~_2(s) = sum_{w in N(s)} N~_1(w) - deg(s),
 *     N~_k(s) = sum_{w in N(s)} N~_{k-1}(w) - N~_{k-2}(s) (deg(s) - 1) for k > 2
 *     (the count of non-backtracking walks of length k, exact on trees);
 *   directed (Eq. 3): N~_k(s) = sum_{w in Gamma(s)} N~_{k-1}(w) (walks).
 * A count that would reach ORC_NB_CAP, or that is computed from a capped
 * count, is stored as ORC_NB_CAP (it still bounds the level size, < n).
 *
 * Section 5's proposition on level-size upper bounds: with
 * c_k = sum_{i<=k} N~_i, the function
 *   S~(r) = sum_{k>=1} k * min(N~_k, max(r - c_{k-1}, 0))
 * is a lower bound on S(s) at r = r(s).  It is linear with slope k on
 * (c_{k-1}, c_k], so by the Section 8 lemma on bounds of the form
 * (n-1) S~(r)/(r-1)^2 the minimum over r in [alpha(s), omega(s)] lies at alpha,
 * at omega or at some c_l strictly between them (Eq. 6); Algorithm 3's
 * nVisited is c_k and its S~ is the running sum.  For undirected graphs
 * alpha = omega = r(s) (Algorithm 3 itself).
 *
 * Readings (where the paper is silent or its listing garbled):
 *  - Every vertex's counts advance at every level, finished or not: later
 *    levels of its neighbours need them (Algorithm 3 skips finished vertices
 *    and names s as v there).
 *  - A vertex finishes when omega(s) <= c_k (Eq. 6's third case), or when
 *    N~_k(s) = 0: no walk continues, so r(s) <= c_{k-1} and no larger r is a
 *    candidate (omega can exceed the walk count: Algorithm 6 counts the
 *    biggest SCC's reach again for every path to it).  A vertex of
 *    out-degree 0 has r = 1 (closeness 0) and gets (S, r) = (0, 1).
 *  - At most max_levels sweeps run.  A vertex still unfinished after level K
 *    takes N~_{K+1} as unbounded: S~ continues with slope K+1 from c_K, which
 *    adds the candidates alpha (if above c_K) and omega.  This is the same
 *    proposition with a weaker (still valid) count.
 *
 * Writes for every vertex the minimising candidate (S_lb, r_lb): the farness
 * bound is (n-1) S_lb / (r_lb - 1)^2, and the order key
 * floor(S_lb * 2^46 / (r_lb - 1)^2) (UINT64_MAX when r_lb = 1).  counts, if
 * not NULL, receives N~_k(v) at counts[k * n + v] for k < counts_levels
 * (sweeps continue until then even if all vertices have finished).  Returns
 * the number of sweeps run, or a negative code.  alpha/omega: Algorithm 6
 * bounds (exact component size if undirected).  h_ub, if not NULL, receives
 * the harmonic-centrality counterpart (see the harmonic section below):
 * the sum over k of min(N~_k, max(omega - c_{k-1}, 0)) / k in increasing k, plus
 * (omega - c_K) / (K+1) for a vertex unfinished at the level cap.
 */
int orc_nb_bounds(uint32_t n, const uint32_t *off, const uint32_t *col, int directed,
                  const uint32_t *alpha, const uint32_t *omega, uint32_t max_levels,
                  uint64_t *S_lb, uint32_t *r_lb, uint64_t *key, uint64_t *counts, uint32_t counts_levels,
                  double *h_ub) {
  if (n == 0) return 0;
  if (max_levels == 0 || max_levels > 65535) return ORC_EINVAL;
  uint64_t *Nk2 = (uint64_t *)malloc((size_t)n * sizeof(uint64_t)); /* N~_{k-2} */
  uint64_t *Nk1 = (uint64_t *)malloc((size_t)n * sizeof(uint64_t)); /* N~_{k-1} */
  uint64_t *Nk = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));  /* N~_k */
  uint64_t *nVisited = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
  uint64_t *Ssum = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
  uint64_t *bS = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
  uint64_t *br = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
  int *have = (int *)calloc(n, sizeof(int));
  char *finished = (char *)calloc(n, 1);
  int rc = ORC_OK;
  if (!Nk2 || !Nk1 || !Nk || !nVisited || !Ssum || !bS || !br || !have || !finished) { rc = ORC_ENOMEM; goto out; }
  uint32_t nFinished = 0;
  for (uint32_t s = 0; s < n; ++s) {
    Nk2[s] = 0;
    Nk1[s] = 1; /* N~_0 */
    nVisited[s] = 1;
    Ssum[s] = 0;
    if (h_ub) h_ub[s] = 0.0;
    if (counts && counts_levels > 0) counts[s] = 1;
  }
  uint32_t k;
  for (k = 1; k <= max_levels && (nFinished < n || k < counts_levels); ++k) {
    for (uint32_t s = 0; s < n; ++s) {
      uint64_t deg = off[s + 1] - off[s];
      if (k == 1) { Nk[s] = deg; continue; }
      uint64_t sum = 0;
      int capped = 0;
      for (uint32_t e = off[s]; e < off[s + 1]; ++e) {
        sum += Nk1[col[e]]; /* each term <= 2^32, at most 2^32 terms */
        if (sum >= ORC_NB_CAP) capped = 1;
      }
      if (directed) {
        Nk[s] = capped ? ORC_NB_CAP : sum;
      } else {
        uint64_t back = (k == 2) ? deg : deg - 1; /* N~_0 = 1 at k = 2 */
        if (capped || Nk2[s] >= ORC_NB_CAP) {
          Nk[s] = ORC_NB_CAP;
        } else {
          u128 sub = (u128)Nk2[s] * back;
          if (sub > sum) { rc = ORC_EINVAL; goto out; } /* impossible for a simple graph */
          Nk[s] = sum - (uint64_t)sub;
        }
      }
    }
    if (counts && k < counts_levels) memcpy(counts + (size_t)k * n, Nk, (size_t)n * sizeof(uint64_t));
    for (uint32_t s = 0; s < n; ++s) {
      Nk2[s] = Nk1[s];
      Nk1[s] = Nk[s];
      if (finished[s]) continue;
      const uint64_t a = alpha[s], o = omega[s], Nks = Nk[s];
      const uint64_t c0 = nVisited[s], c1 = c0 + Nks, P0 = Ssum[s];
      if (Nks == 0) {
        /* no walk continues: r(s) <= c0, nothing above c0 is a candidate */
        finished[s] = 1;
        ++nFinished;
        if (!have[s]) {
          if (c0 != 1) { rc = ORC_EINVAL; goto out; } /* alpha above every possible reach */
          bS[s] = 0; br[s] = 1; have[s] = 1;         /* out-degree 0: r = 1 */
        }
        continue;
      }
      if (a > c0 && a <= c1) nb_candidate(P0 + (uint64_t)k * (a - c0), a, &have[s], &bS[s], &br[s]);
      if (c1 > a && c1 < o) nb_candidate(P0 + (uint64_t)k * Nks, c1, &have[s], &bS[s], &br[s]);
      if (o <= c1) {
        nb_candidate(P0 + (uint64_t)k * (o - c0), o, &have[s], &bS[s], &br[s]);
        if (h_ub) h_ub[s] = h_ub[s] + (double)(o - c0) / (double)k;
        finished[s] = 1;
        ++nFinished;
        continue;
      }
      nVisited[s] = c1;
      Ssum[s] = P0 + (uint64_t)k * Nks;
      if (h_ub) h_ub[s] = h_ub[s] + (double)Nks / (double)k;
      if (k == max_levels) {
        /* level K+1 unbounded: slope K+1 from c_K up to omega */
        const uint64_t P1 = Ssum[s];
        if (a > c1) nb_candidate(P1 + (uint64_t)(k + 1) * (a - c1), a, &have[s], &bS[s], &br[s]);
        nb_candidate(P1 + (uint64_t)(k + 1) * (o - c1), o, &have[s], &bS[s], &br[s]);
        if (h_ub) h_ub[s] = h_ub[s] + (double)(o - c1) / (double)(k + 1);
        finished[s] = 1;
        ++nFinished;
      }
    }
  }
  for (uint32_t s = 0; s < n; ++s) {
    S_lb[s] = bS[s];
    r_lb[s] = (uint32_t)br[s];
    if (key) {
      if (br[s] <= 1) {
        key[s] = UINT64_MAX;
      } else {
        u128 num = (u128)bS[s] << ORC_NB_FRAC;
        key[s] = (uint64_t)(num / (u128)((br[s] - 1) * (br[s] - 1)));
      }
    }
  }
  rc = (int)(k - 1);
out:
  free(Nk2); free(Nk1); free(Nk); free(nVisited); free(Ssum); free(bS); free(br); free(have); free(finished);
  return rc;
}

/* ---------------------------------------------------------------------- */
/* BFSCut lower bound (Section 6's lemma, with the Section 8.2 reading)     */
/* ---------------------------------------------------------------------- */

/*
 * After BFS from v has discovered every level up to d:
 *   S_d  = sum of d(v,w) over the ball of radius d,   n_d = size of the ball,
 *   g    = upper bound on |Gamma_{d+1}(v)|: the sum of outdeg(w) over
 *          Gamma_d(v) for directed graphs, of deg(w)-1 for undirected graphs
 *          at d >= 1, and deg(v) at d = 0.
 * Section 6's lemma gives S(v) >= S_d - |Gamma_{d+1}| + (d+2)(r - n_d) for the true
 * r = r(v), with |Gamma_{d+1}| <= g.  Because also |Gamma_{d+1}| <= r - n_d,
 *   L_d(r) = S_d + (d+1)(r - n_d) + max(0, r - n_d - g)
 * is a lower bound on S(v) at r = r(v).  r(v) lies in [max(alpha, n_d), omega];
 * L_d(r)/(r-1)^2 is minimised over that interval at an end point or at the
 * kink r = n_d + g (it is linear on each side of the kink, and a linear L makes
 * the ratio's minimum fall at an end point of the piece, Section 8's lemma).
 *
 * Returns 1 if the farness bound exceeds the threshold (Sx, rx) strictly at
 * every candidate r, i.e. the vertex can be abandoned.  have_x = 0 means fewer
 * than k vertices are known and nothing is abandoned.
 */
static uint64_t cut_L(uint64_t Sd, uint32_t d, uint64_t nd, uint64_t g, uint64_t r) {
  uint64_t rem = r - nd;
  uint64_t extra = rem > g ? rem - g : 0;
  return Sd + (uint64_t)(d + 1) * rem + extra;
}

/* The candidate r in [max(lo, nd), hi] minimising L_d(r)/(r-1)^2, compared
 * exactly; writes that r and L_d(r).  r <= 1 stands for farness +infinity and
 * is never chosen while another candidate exists. */
static void cut_min(uint64_t Sd, uint32_t d, uint64_t nd, uint64_t g, uint64_t lo, uint64_t hi,
                    uint64_t *L_best, uint64_t *r_best) {
  if (lo < nd) lo = nd;
  if (hi < lo) hi = lo;
  uint64_t cand[3];
  int nc = 0;
  cand[nc++] = lo;
  cand[nc++] = hi;
  uint64_t kink = nd + g;
  if (kink > lo && kink < hi) cand[nc++] = kink;
  uint64_t bl = cut_L(Sd, d, nd, g, cand[0]), br = cand[0];
  for (int i = 1; i < nc; ++i) {
    uint64_t r = cand[i], L = cut_L(Sd, d, nd, g, r);
    if (r <= 1) continue;
    if (br <= 1) { bl = L; br = r; continue; }
    u128 lhs = (u128)L * (u128)((br - 1) * (br - 1));
    u128 rhs = (u128)bl * (u128)((r - 1) * (r - 1));
    if (lhs < rhs) { bl = L; br = r; }
  }
  *L_best = bl;
  *r_best = br;
}

void orc_cut_min(uint64_t Sd, uint32_t d, uint64_t nd, uint64_t g, uint64_t lo, uint64_t hi,
                 uint64_t *L_best, uint64_t *r_best) {
  cut_min(Sd, d, nd, g, lo, hi, L_best, r_best);
}

static int cut_exceeds(uint64_t Sd, uint32_t d, uint64_t nd, uint64_t g, uint64_t lo, uint64_t hi,
                       int have_x, uint64_t Sx, uint32_t rx) {
  if (!have_x) return 0;
  uint64_t L, r;
  cut_min(Sd, d, nd, g, lo, hi, &L, &r);
  if (r <= 1) return 1; /* farness +infinity exceeds any finite x */
  /* L/(r-1)^2 > Sx/(rx-1)^2 ?  (rx > 1: x is a finite farness) */
  u128 lhs = (u128)L * (u128)((uint64_t)(rx - 1) * (uint64_t)(rx - 1));
  u128 rhs = (u128)Sx * (u128)((r - 1) * (r - 1));
  return lhs > rhs;
}

/* The level-granular bound sequence L_0, L_1, ... of one source at its true
 * r(v), for the invariant tests (L_d <= S(v), non-decreasing, L_last = S(v)).
 * Returns the number of levels written (at most maxlev). */
int orc_cut_bounds(uint32_t n, const uint32_t *off, const uint32_t *col, int directed, uint32_t v,
                   uint64_t *Lout, int maxlev) {
  uint32_t *dist = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
  uint32_t *queue = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
  if (!dist || !queue) { free(dist); free(queue); return ORC_ENOMEM; }
  uint64_t Sfull;
  uint32_t rfull;
  for (uint32_t i = 0; i < n; ++i) dist[i] = UINT32_MAX;
  bfs_one(n, off, col, v, dist, queue, &Sfull, &rfull);
  /* level-by-level pass */
  uint32_t head = 0, tail = 0;
  dist[v] = 0;
  queue[tail++] = v;
  uint64_t Sd = 0, nd = 1, g = off[v + 1] - off[v];
  uint32_t d = 0;
  int nl = 0;
  while (1) {
    if (nl < maxlev) Lout[nl] = cut_L(Sd, d, nd, g, rfull);
    ++nl;
    uint32_t level_end = tail;
    uint64_t cnt = 0, gs = 0;
    while (head < level_end) {
      uint32_t u = queue[head++];
      for (uint32_t e = off[u]; e < off[u + 1]; ++e) {
        uint32_t w = col[e];
        if (dist[w] == UINT32_MAX) {
          dist[w] = d + 1;
          queue[tail++] = w;
          ++cnt;
          gs += (off[w + 1] - off[w]) - (directed ? 0u : 1u);
        }
      }
    }
    if (cnt == 0) break;
    ++d;
    Sd += (uint64_t)d * cnt;
    nd += cnt;
    g = gs;
  }
  for (uint32_t i = 0; i < tail; ++i) dist[queue[i]] = UINT32_MAX;
  free(dist); free(queue);
  return nl < maxlev ? nl : maxlev;
}

/* ---------------------------------------------------------------------- */
/* Algorithm 1 with updateBoundsBFSCut (DegCut), sequential                 */
/* ---------------------------------------------------------------------- */

typedef struct {
  uint64_t edges_visited; /* arcs scanned by the expanded BFS levels */
  uint64_t bfs_started;
  uint64_t bfs_cut;
  uint64_t bfs_finished;
} orc_counters;

/* insert (S, r, id) into the sorted top list of capacity k */
static void top_insert(entry_t *top, uint32_t *cnt, uint32_t k, uint64_t S, uint32_t r, uint32_t id) {
  entry_t e = {S, r, id};
  if (*cnt == k && cmp_entry(&e, &top[k - 1]) >= 0) return;
  uint32_t i = *cnt < k ? (*cnt)++ : k - 1;
  while (i > 0 && cmp_entry(&e, &top[i - 1]) < 0) { top[i] = top[i - 1]; --i; }
  top[i] = e;
}

/*
 * Algorithm 1 with computeBoundsDeg (L = 0, Q in decreasing degree order, or
 * the caller's order) and updateBoundsBFSCut (Algorithm 4) evaluated once per
 * completed level, r(v) bounded by alpha/omega (Algorithm 6; exact for
 * undirected graphs).  Vertices of out-degree 0 have r = 1 (closeness 0) and
 * are never searched.
 *
 * Readings where the paper leaves a choice:
 *  - A vertex is abandoned only when its farness bound is strictly greater
 *    than x, the k-th smallest farness found so far, so that every vertex tied
 *    with the final k-th is fully searched (Section 4 asks for all of them).
 *  - x is refreshed after each finished BFS (one source at a time).
 *  - The bound is checked before each level is expanded, including level 0.
 *
 * Outputs: ids/S/r of the top min(k, n) (ties by id), n_tied, counters, and
 * optionally per-vertex S/r of every finished BFS (r = 0 if not finished).
 * max_sources > 0 stops after that many searches (a timing sample only: the
 * returned list is then the top of the examined prefix, not the answer).
 *
 * lb_key (NULL = none) turns this into NBCut: lb_key[v] is the order key of
 * orc_nb_bounds, floor(2^46 L'(v)) with L'(v) a lower bound on S(v)/(r(v)-1)^2,
 * and order_in must list vertices by increasing key.  Algorithm 1 then stops
 * at the first source whose key exceeds x strictly (key / 2^46 > S_x/(r_x-1)^2):
 * every later source has a bound at least as large, hence farness > x.
 */
int orc_bfscut(uint32_t n, const uint32_t *off, const uint32_t *col, int directed, uint32_t k,
               const uint32_t *order_in, uint32_t *ids, uint64_t *S_out, uint32_t *r_out,
               uint32_t *n_tied, orc_counters *ctr, uint64_t *allS, uint32_t *allr, uint32_t max_sources,
               const uint64_t *lb_key) {
  if (k == 0 || n == 0) { if (n_tied) *n_tied = 0; return 0; }
  int rc = ORC_OK;
  uint32_t *order = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
  uint32_t *alpha = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
  uint32_t *omega = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
  uint32_t *dist = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
  uint32_t *queue = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
  uint64_t *fS = (uint64_t *)calloc(n, sizeof(uint64_t));
  uint32_t *fr = (uint32_t *)calloc(n, sizeof(uint32_t));
  uint32_t kk = k < n ? k : n;
  entry_t *top = (entry_t *)malloc((size_t)kk * sizeof(entry_t));
  if (!order || !alpha || !omega || !dist || !queue || !fS || !fr || !top) { rc = ORC_ENOMEM; goto done; }
  if (order_in)
    memcpy(order, order_in, (size_t)n * sizeof(uint32_t));
  else if ((rc = orc_degree_order(n, off, order)) != ORC_OK)
    goto done;
  if ((rc = orc_alpha_omega(n, off, col, directed, alpha, omega)) != ORC_OK) goto done;
  for (uint32_t i = 0; i < n; ++i) dist[i] = UINT32_MAX;
  orc_counters c = {0, 0, 0, 0};
  uint32_t ntop = 0;
  for (uint32_t oi = 0; oi < n; ++oi) {
    uint32_t v = order[oi];
    if (off[v + 1] == off[v]) continue; /* r(v) = 1: closeness 0 */
    if (max_sources && c.bfs_started >= max_sources) break; /* timing sample: a prefix of Q */
    int have_x = ntop == kk;
    uint64_t Sx = have_x ? top[kk - 1].S : 0;
    uint32_t rx = have_x ? top[kk - 1].r : 0;
    if (lb_key && have_x) {
      u128 lhs = (u128)lb_key[v] * (u128)((uint64_t)(rx - 1) * (uint64_t)(rx - 1));
      u128 rhs = (u128)Sx << ORC_NB_FRAC;
      if (lhs > rhs) break; /* Algorithm 1: the head of Q is bounded above x */
    }
    c.bfs_started++;
    uint32_t head = 0, tail = 0;
    dist[v] = 0;
    queue[tail++] = v;
    uint64_t Sd = 0, nd = 1, g = off[v + 1] - off[v];
    uint32_t d = 0;
    int cut = 0;
    while (1) {
      if (cut_exceeds(Sd, d, nd, g, alpha[v], omega[v], have_x, Sx, rx)) { cut = 1; break; }
      uint32_t level_end = tail;
      uint64_t cnt = 0, gs = 0;
      while (head < level_end) {
        uint32_t u = queue[head++];
        c.edges_visited += off[u + 1] - off[u];
        for (uint32_t e = off[u]; e < off[u + 1]; ++e) {
          uint32_t w = col[e];
          if (dist[w] == UINT32_MAX) {
            dist[w] = d + 1;
            queue[tail++] = w;
            ++cnt;
            gs += (off[w + 1] - off[w]) - (directed ? 0u : 1u);
          }
        }
      }
      if (cnt == 0) break;
      ++d;
      Sd += (uint64_t)d * cnt;
      nd += cnt;
      g = gs;
    }
    for (uint32_t i = 0; i < tail; ++i) dist[queue[i]] = UINT32_MAX;
    if (cut) {
      c.bfs_cut++;
      continue;
    }
    c.bfs_finished++;
    fS[v] = Sd;
    fr[v] = (uint32_t)nd;
    top_insert(top, &ntop, kk, Sd, (uint32_t)nd, v);
  }
  /* fewer than kk finished: fill with r = 1 vertices in id order */
  for (uint32_t v = 0; v < n && ntop < kk; ++v)
    if (off[v + 1] == off[v]) top_insert(top, &ntop, kk, 0, 1, v);
  for (uint32_t i = 0; i < kk; ++i) {
    ids[i] = top[i].id;
    if (S_out) S_out[i] = top[i].S;
    if (r_out) r_out[i] = top[i].r;
  }
  if (n_tied) {
    uint32_t t = 0;
    const entry_t *last = &top[kk - 1];
    for (uint32_t v = 0; v < n; ++v) {
      if (off[v + 1] == off[v]) {
        if (last->r <= 1) ++t;
      } else if (fr[v] && cmp_farness(fS[v], fr[v], last->S, last->r) == 0) {
        ++t;
      }
    }
    *n_tied = t;
  }
  if (allS) memcpy(allS, fS, (size_t)n * sizeof(uint64_t));
  if (allr) memcpy(allr, fr, (size_t)n * sizeof(uint32_t));
  if (ctr) *ctr = c;
  rc = (int)kk;
done:
  free(order); free(alpha); free(omega); free(dist); free(queue); free(fS); free(fr); free(top);
  return rc;
}

/* ---------------------------------------------------------------------- */
/* Algorithm 1 with updateBoundsBFSCut, B sources per batch (the schedule   */
/* the GPU runs with options.deterministic), level-synchronous              */
/* ---------------------------------------------------------------------- */

typedef struct {
  uint64_t edges_visited; /* arcs of every expanded level (the paper's m_vis) */
  uint64_t bfs_started;
  uint64_t bfs_cut;
  uint64_t bfs_finished;
  uint64_t levels;        /* level steps: one per BFS level of a batch, all its searches together */
} orc_bcounters;

/*
 * The same method as orc_bfscut (Algorithm 1, Algorithm 4 evaluated once per
 * level, Section 8's reach bounds), but up to B searches advance together,
 * one BFS level per step, and the threshold x changes only between steps.
 * This is the schedule of the batched GPU search with one team; the oracle
 * states it as plainly as it can so that arcs visited under batching have an
 * independent count.
 *
 *  1. Seeding a batch.  Q is the order restricted to vertices of out-degree
 *     >= 1.  Sources are taken from Q in order while the batch has free slots.
 *     With x known (k searches finished), a source at position >= nocut_prefix
 *     is first checked against Algorithm 1's stop (lb_key, NBCut: key above x
 *     ends the whole search, nothing later in Q is examined) and then against
 *     the level-0 bound of Algorithm 4 (cut before any arc is read).  A source
 *     that passes occupies a slot; its level-0 arcs (its out-degree) count as
 *     visited.  Q is read in chunks of the batch's free slots; a source cut at
 *     level 0 frees its place for the next chunk, so a batch is full unless Q
 *     runs out.
 *  2. One step.  Every active search expands its newest level (arcs already
 *     counted).  Then, in slot order: a search that found nothing new is
 *     finished (exact S, r); the others add the new level to S_d, n_d and set
 *     gamma~ (sum of out-degrees of the new level, minus its size if
 *     undirected).  All searches finished in this step enter the top list
 *     together, x becomes the new k-th entry, and only then is each
 *     continuing search tested against x (Section 6 lemma, r in
 *     [max(alpha, n_d), omega]); a search that survives counts the arcs of its
 *     new level as visited.
 *  3. When no search of the batch is active, the next batch is seeded.  The
 *     run ends when a seeding finds no source.
 * Positions below nocut_prefix are never cut nor stopped (they seed x with
 * exact values).  With B = 1 this is exactly orc_bfscut.  Outputs as
 * orc_bfscut; counters include the number of steps.
 */
int orc_bfscut_batched(uint32_t n, const uint32_t *off, const uint32_t *col, int directed, uint32_t k,
                       const uint32_t *order_in, uint32_t B, const uint64_t *lb_key, uint32_t nocut_prefix,
                       uint32_t *ids, uint64_t *S_out, uint32_t *r_out, uint32_t *n_tied, orc_bcounters *ctr,
                       uint64_t *allS, uint32_t *allr) {
  if (k == 0 || n == 0) { if (n_tied) *n_tied = 0; return 0; }
  if (B == 0) return ORC_EINVAL;
  int rc = ORC_OK;
  uint32_t kk = k < n ? k : n;
  uint32_t *order = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
  uint32_t *Q = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
  uint32_t *alpha = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
  uint32_t *omega = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
  uint64_t *fS = (uint64_t *)calloc(n, sizeof(uint64_t));
  uint32_t *fr = (uint32_t *)calloc(n, sizeof(uint32_t));
  entry_t *top = (entry_t *)malloc((size_t)kk * sizeof(entry_t));
  /* per slot: its own BFS (distance array, queue, level bounds) */
  uint32_t *dist = (uint32_t *)malloc((size_t)B * n * sizeof(uint32_t));
  uint32_t *queue = (uint32_t *)malloc((size_t)B * n * sizeof(uint32_t));
  uint32_t *head = (uint32_t *)calloc(B, sizeof(uint32_t));
  uint32_t *tail = (uint32_t *)calloc(B, sizeof(uint32_t));
  uint32_t *src = (uint32_t *)calloc(B, sizeof(uint32_t));
  uint32_t *depth = (uint32_t *)calloc(B, sizeof(uint32_t));
  uint32_t *nocut = (uint32_t *)calloc(B, sizeof(uint32_t));
  int *active = (int *)calloc(B, sizeof(int));
  uint64_t *Sd = (uint64_t *)calloc(B, sizeof(uint64_t));
  uint64_t *nd = (uint64_t *)calloc(B, sizeof(uint64_t));
  uint64_t *gam = (uint64_t *)calloc(B, sizeof(uint64_t));
  uint64_t *arcs = (uint64_t *)calloc(B, sizeof(uint64_t));
  uint64_t *cnt = (uint64_t *)calloc(B, sizeof(uint64_t));
  uint64_t *gs = (uint64_t *)calloc(B, sizeof(uint64_t));
  if (!order || !Q || !alpha || !omega || !fS || !fr || !top || !dist || !queue || !head || !tail || !src ||
      !depth || !nocut || !active || !Sd || !nd || !gam || !arcs || !cnt || !gs) {
    rc = ORC_ENOMEM;
    goto done;
  }
  if (order_in)
    memcpy(order, order_in, (size_t)n * sizeof(uint32_t));
  else if ((rc = orc_degree_order(n, off, order)) != ORC_OK)
    goto done;
  if ((rc = orc_alpha_omega(n, off, col, directed, alpha, omega)) != ORC_OK) goto done;
  uint32_t nq = 0;
  for (uint32_t i = 0; i < n; ++i)
    if (off[order[i] + 1] > off[order[i]]) Q[nq++] = order[i]; /* r = 1 vertices are never searched */
  for (size_t i = 0; i < (size_t)B * n; ++i) dist[i] = UINT32_MAX;
  orc_bcounters c = {0, 0, 0, 0, 0};
  uint32_t ntop = 0, cursor = 0;
  int stopped = 0;
  while (1) {
    /* 1. seed a batch */
    uint32_t assigned = 0;
    while (assigned < B && cursor < nq && !stopped) {
      uint32_t room = B - assigned;
      uint32_t end = cursor + room < nq ? cursor + room : nq;
      int have_x = ntop == kk;
      uint64_t Sx = have_x ? top[kk - 1].S : 0;
      uint32_t rx = have_x ? top[kk - 1].r : 0;
      for (uint32_t pos = cursor; pos < end && !stopped; ++pos) {
        uint32_t v = Q[pos];
        uint64_t od = off[v + 1] - off[v];
        int protect = pos < nocut_prefix;
        if (!protect && lb_key && have_x) {
          u128 lhs = (u128)lb_key[v] * (u128)((uint64_t)(rx - 1) * (uint64_t)(rx - 1));
          if (lhs > ((u128)Sx << ORC_NB_FRAC)) { stopped = 1; break; }
        }
        c.bfs_started++;
        if (!protect && cut_exceeds(0, 0, 1, od, alpha[v], omega[v], have_x, Sx, rx)) {
          c.bfs_cut++;
          continue;
        }
        uint32_t s = assigned++;
        uint32_t *ds = dist + (size_t)s * n, *qs = queue + (size_t)s * n;
        src[s] = v;
        nocut[s] = (uint32_t)protect;
        head[s] = 0;
        tail[s] = 0;
        ds[v] = 0;
        qs[tail[s]++] = v;
        depth[s] = 0;
        Sd[s] = 0;
        nd[s] = 1;
        gam[s] = od;
        arcs[s] = od;
        active[s] = 1;
        c.edges_visited += od;
      }
      cursor = end;
    }
    if (assigned == 0) break;
    /* 2. level steps until every search of the batch has ended */
    int any = 1;
    while (any) {
      c.levels++;
      for (uint32_t s = 0; s < assigned; ++s) {
        if (!active[s]) continue;
        uint32_t *ds = dist + (size_t)s * n, *qs = queue + (size_t)s * n;
        uint32_t level_end = tail[s];
        cnt[s] = 0;
        gs[s] = 0;
        while (head[s] < level_end) {
          uint32_t u = qs[head[s]++];
          for (uint32_t e = off[u]; e < off[u + 1]; ++e) {
            uint32_t w = col[e];
            if (ds[w] == UINT32_MAX) {
              ds[w] = depth[s] + 1;
              qs[tail[s]++] = w;
              cnt[s]++;
              gs[s] += (off[w + 1] - off[w]) - (directed ? 0u : 1u);
            }
          }
        }
      }
      /* searches that found nothing new are finished; the others advance */
      for (uint32_t s = 0; s < assigned; ++s) {
        if (!active[s]) continue;
        if (cnt[s] == 0) {
          active[s] = 0;
          c.bfs_finished++;
          fS[src[s]] = Sd[s];
          fr[src[s]] = (uint32_t)nd[s];
          top_insert(top, &ntop, kk, Sd[s], (uint32_t)nd[s], src[s]);
        } else {
          depth[s] += 1;
          Sd[s] += (uint64_t)depth[s] * cnt[s];
          nd[s] += cnt[s];
          gam[s] = gs[s];
          arcs[s] = gs[s] + (directed ? 0u : cnt[s]); /* out-degree sum of the new level */
        }
      }
      /* x after this step's merges; then the cut test of the survivors */
      int have_x = ntop == kk;
      uint64_t Sx = have_x ? top[kk - 1].S : 0;
      uint32_t rx = have_x ? top[kk - 1].r : 0;
      any = 0;
      for (uint32_t s = 0; s < assigned; ++s) {
        if (!active[s]) continue;
        uint32_t v = src[s];
        if (!nocut[s] && cut_exceeds(Sd[s], depth[s], nd[s], gam[s], alpha[v], omega[v], have_x, Sx, rx)) {
          active[s] = 0;
          c.bfs_cut++;
          continue;
        }
        c.edges_visited += arcs[s];
        any = 1;
      }
    }
    /* 3. restore the batch's distance arrays */
    for (uint32_t s = 0; s < assigned; ++s) {
      uint32_t *ds = dist + (size_t)s * n, *qs = queue + (size_t)s * n;
      for (uint32_t i = 0; i < tail[s]; ++i) ds[qs[i]] = UINT32_MAX;
    }
  }
  for (uint32_t v = 0; v < n && ntop < kk; ++v)
    if (off[v + 1] == off[v]) top_insert(top, &ntop, kk, 0, 1, v);
  for (uint32_t i = 0; i < kk; ++i) {
    ids[i] = top[i].id;
    if (S_out) S_out[i] = top[i].S;
    if (r_out) r_out[i] = top[i].r;
  }
  if (n_tied) {
    uint32_t t = 0;
    const entry_t *last = &top[kk - 1];
    for (uint32_t v = 0; v < n; ++v) {
      if (off[v + 1] == off[v]) {
        if (last->r <= 1) ++t;
      } else if (fr[v] && cmp_farness(fS[v], fr[v], last->S, last->r) == 0) {
        ++t;
      }
    }
    *n_tied = t;
  }
  if (allS) memcpy(allS, fS, (size_t)n * sizeof(uint64_t));
  if (allr) memcpy(allr, fr, (size_t)n * sizeof(uint32_t));
  if (ctr) *ctr = c;
  rc = (int)kk;
done:
  free(order); free(Q); free(alpha); free(omega); free(fS); free(fr); free(top); free(dist); free(queue);
  free(head); free(tail); free(src); free(depth); free(nocut); free(active); free(Sd); free(nd); free(gam);
  free(arcs); free(cnt); free(gs);
  return rc;
}

/* ---------------------------------------------------------------------- */
/* Harmonic centrality (Section 9, "Harmonic Centrality"): the same method  */
/* for h(v) = sum over w != v of 1/d(v,w), largest first                    */
/* ---------------------------------------------------------------------- */

/*
 * Readings (the paper states only that its bounds carry over to measures
 * sum_w f(d(v,w)) with f decreasing and f(inf) = 0):
 *  - The FP64 value of h(v) is formed per BFS level: the count c_d of vertices
 *    at distance d divided by d, these quotients added in increasing d, every
 *    operation rounded to nearest with no contraction.  The oracle and the
 *    library form it the same way, so the same counts give the same bits; the
 *    top-k is ranked by that value, ties by smaller id.
 *  - BFSCut's bound after level d (the Section 6 lemma with f = 1/d): the
 *    vertices not yet found lie at distance >= d+1, at most g of them (the same
 *    gamma as for closeness) at d+1, and there are at most omega - n_d of them,
 *    so h(v) <= U_d = H_d + min(g, w)/(d+1) + max(0, w - g)/(d+2), w = omega - n_d.
 *    U_d grows with the reach, so omega alone bounds it (alpha is not needed).
 *  - Rounding: the FP64 h may exceed the exact h by (D+1) units in the last
 *    place and the computed U_d fall short of the exact bound by (d+3); a
 *    search is abandoned only when fl(U_d * (1 + 2^-20)) < x, which implies
 *    h_fp64(v) < x for every depth below 2^32.  Strict: a vertex tied with the
 *    k-th is never abandoned.
 *  - computeBoundsNB for h: with the same level-size bounds N~_k, assigning as
 *    many vertices as possible to the nearest levels maximises sum 1/d, so
 *    h(v) <= sum_k min(N~_k, max(omega - c_{k-1}, 0)) / k (quotients added in
 *    increasing k; after a level cap K the remaining omega - c_K vertices count
 *    at distance K+1).  Sources go in decreasing order of this bound, ties by
 *    id, and Algorithm 1 stops at the first one whose bound (times 1 + 2^-20)
 *    is below x.
 */
#define ORC_H_MARGIN (1.0 + 1.0 / 1048576.0)

/* BFS from s counting each level; returns h(v) as defined above, r(v) and the
 * arcs scanned. */
static double bfs_harmonic_one(const uint32_t *off, const uint32_t *col, uint32_t s, uint32_t *dist,
                               uint32_t *queue, uint32_t *r_out) {
  uint32_t head = 0, tail = 0, d = 0;
  double h = 0.0;
  dist[s] = 0;
  queue[tail++] = s;
  while (head < tail) {
    uint32_t end = tail;
    uint64_t cnt = 0;
    while (head < end) {
      uint32_t u = queue[head++];
      for (uint32_t e = off[u]; e < off[u + 1]; ++e) {
        uint32_t w = col[e];
        if (dist[w] == UINT32_MAX) {
          dist[w] = d + 1;
          queue[tail++] = w;
          ++cnt;
        }
      }
    }
    if (cnt == 0) break;
    ++d;
    h = h + (double)cnt / (double)d;
  }
  for (uint32_t i = 0; i < tail; ++i) dist[queue[i]] = UINT32_MAX;
  *r_out = tail;
  return h;
}

/* Textbook harmonic centrality: h(v) and r(v) for the listed sources (all
 * vertices if srcs == NULL).  Pinned by exact rationals from Floyd-Warshall
 * distances (within the rounding bound), closed forms and networkx. */
int orc_harmonic_sums(uint32_t n, const uint32_t *off, const uint32_t *col, uint32_t nsrc,
                      const uint32_t *srcs, double *H, uint32_t *r, int nthreads) {
  if (n == 0) return ORC_OK;
  int rc = ORC_OK;
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel num_threads(nthreads)
#endif
  {
    uint32_t *dist = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
    uint32_t *queue = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
    if (!dist || !queue) {
      rc = ORC_ENOMEM;
    } else {
      for (uint32_t i = 0; i < n; ++i) dist[i] = UINT32_MAX;
      int64_t cnt = srcs ? (int64_t)nsrc : (int64_t)n;
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 16)
#endif
      for (int64_t i = 0; i < cnt; ++i) {
        uint32_t s = srcs ? srcs[i] : (uint32_t)i;
        H[i] = bfs_harmonic_one(off, col, s, dist, queue, &r[i]);
      }
    }
    free(dist);
    free(queue);
  }
  (void)nthreads;
  return rc;
}

typedef struct {
  double h;
  uint32_t r;
  uint32_t id;
} hentry_t;

/* larger h first, then smaller id */
static int hentry_before(const hentry_t *a, const hentry_t *b) {
  if (a->h != b->h) return a->h > b->h;
  return a->id < b->id;
}

static int cmp_hentry(const void *pa, const void *pb) {
  const hentry_t *a = (const hentry_t *)pa, *b = (const hentry_t *)pb;
  if (hentry_before(a, b)) return -1;
  if (hentry_before(b, a)) return 1;
  return 0;
}

/* Top-k by harmonic centrality (largest h, ties by id) and the number of
 * vertices whose h equals the k-th's.  Returns min(k, n). */
int orc_harmonic_topk(uint32_t n, const double *H, uint32_t k, uint32_t *ids, uint32_t *n_tied) {
  uint32_t kk = k < n ? k : n;
  if (kk == 0) { if (n_tied) *n_tied = 0; return 0; }
  hentry_t *e = (hentry_t *)malloc((size_t)n * sizeof(hentry_t));
  if (!e) return ORC_ENOMEM;
  for (uint32_t v = 0; v < n; ++v) { e[v].h = H[v]; e[v].r = 0; e[v].id = v; }
  qsort(e, n, sizeof(hentry_t), cmp_hentry);
  uint32_t t = 0;
  for (uint32_t v = 0; v < n; ++v) t += H[v] == e[kk - 1].h;
  for (uint32_t i = 0; i < kk; ++i) ids[i] = e[i].id;
  if (n_tied) *n_tied = t;
  free(e);
  return (int)kk;
}

static void htop_insert(hentry_t *top, uint32_t *cnt, uint32_t k, double h, uint32_t r, uint32_t id) {
  hentry_t e = {h, r, id};
  if (*cnt == k && !hentry_before(&e, &top[k - 1])) return;
  uint32_t i = *cnt < k ? (*cnt)++ : k - 1;
  while (i > 0 && hentry_before(&e, &top[i - 1])) { top[i] = top[i - 1]; --i; }
  top[i] = e;
}

/* U_d of the reading above, in this operation order. */
static double harmonic_cut_bound(double Hd, uint32_t d, uint64_t nd, uint64_t g, uint64_t omega) {
  uint64_t w = omega > nd ? omega - nd : 0;
  uint64_t near = g < w ? g : w;
  uint64_t far = w > g ? w - g : 0;
  double t1 = (double)near / (double)(d + 1);
  double t2 = (double)far / (double)(d + 2);
  return (Hd + t1) + t2;
}

/*
 * Algorithm 1 + BFSCut for harmonic centrality, one source at a time, in the
 * degree order (or order_in).  ub (NULL = none) is computeBoundsNB's upper bound
 * per vertex, with order_in sorted by decreasing ub: the loop stops at the first
 * source with fl(ub * (1 + 2^-20)) < x.  Vertices of out-degree 0 have h = 0 and
 * are not searched.  Outputs as orc_bfscut, with H in place of S.
 */
int orc_bfscut_harmonic(uint32_t n, const uint32_t *off, const uint32_t *col, int directed, uint32_t k,
                        const uint32_t *order_in, const double *ub, uint32_t *ids, double *H_out, uint32_t *r_out,
                        uint32_t *n_tied, orc_counters *ctr, double *allH, uint32_t *allr, uint32_t max_sources) {
  if (k == 0 || n == 0) { if (n_tied) *n_tied = 0; return 0; }
  int rc = ORC_OK;
  uint32_t *order = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
  uint32_t *alpha = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
  uint32_t *omega = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
  uint32_t *dist = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
  uint32_t *queue = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
  double *fH = (double *)calloc(n, sizeof(double));
  uint32_t *fr = (uint32_t *)calloc(n, sizeof(uint32_t));
  uint32_t kk = k < n ? k : n;
  hentry_t *top = (hentry_t *)malloc((size_t)kk * sizeof(hentry_t));
  if (!order || !alpha || !omega || !dist || !queue || !fH || !fr || !top) { rc = ORC_ENOMEM; goto done; }
  if (order_in)
    memcpy(order, order_in, (size_t)n * sizeof(uint32_t));
  else if ((rc = orc_degree_order(n, off, order)) != ORC_OK)
    goto done;
  if ((rc = orc_alpha_omega(n, off, col, directed, alpha, omega)) != ORC_OK) goto done;
  for (uint32_t i = 0; i < n; ++i) dist[i] = UINT32_MAX;
  orc_counters c = {0, 0, 0, 0};
  uint32_t ntop = 0;
  for (uint32_t oi = 0; oi < n; ++oi) {
    uint32_t v = order[oi];
    if (off[v + 1] == off[v]) continue; /* h(v) = 0 */
    if (max_sources && c.bfs_started >= max_sources) break;
    int have_x = ntop == kk;
    double xH = have_x ? top[kk - 1].h : 0.0;
    if (ub && have_x && ub[v] * ORC_H_MARGIN < xH) break; /* Algorithm 1: the head of Q is bounded below x */
    c.bfs_started++;
    uint32_t head = 0, tail = 0;
    dist[v] = 0;
    queue[tail++] = v;
    uint64_t nd = 1, g = off[v + 1] - off[v];
    uint32_t d = 0;
    double Hd = 0.0;
    int cut = 0;
    while (1) {
      if (have_x && harmonic_cut_bound(Hd, d, nd, g, omega[v]) * ORC_H_MARGIN < xH) { cut = 1; break; }
      uint32_t level_end = tail;
      uint64_t cnt = 0, gs = 0;
      while (head < level_end) {
        uint32_t u = queue[head++];
        c.edges_visited += off[u + 1] - off[u];
        for (uint32_t e = off[u]; e < off[u + 1]; ++e) {
          uint32_t w = col[e];
          if (dist[w] == UINT32_MAX) {
            dist[w] = d + 1;
            queue[tail++] = w;
            ++cnt;
            gs += (off[w + 1] - off[w]) - (directed ? 0u : 1u);
          }
        }
      }
      if (cnt == 0) break;
      ++d;
      Hd = Hd + (double)cnt / (double)d;
      nd += cnt;
      g = gs;
    }
    for (uint32_t i = 0; i < tail; ++i) dist[queue[i]] = UINT32_MAX;
    if (cut) { c.bfs_cut++; continue; }
    c.bfs_finished++;
    fH[v] = Hd;
    fr[v] = (uint32_t)nd;
    htop_insert(top, &ntop, kk, Hd, (uint32_t)nd, v);
  }
  /* fewer than kk searched: out-degree-0 vertices (h = 0) in id order */
  for (uint32_t v = 0; v < n && ntop < kk; ++v)
    if (off[v + 1] == off[v]) htop_insert(top, &ntop, kk, 0.0, 1, v);
  for (uint32_t i = 0; i < kk; ++i) {
    ids[i] = top[i].id;
    if (H_out) H_out[i] = top[i].h;
    if (r_out) r_out[i] = top[i].r;
  }
  if (n_tied) {
    uint32_t t = 0;
    const double last = top[kk - 1].h;
    for (uint32_t v = 0; v < n; ++v) {
      if (off[v + 1] == off[v]) t += last == 0.0;
      else if (fr[v] && fH[v] == last) ++t;
    }
    *n_tied = t;
  }
  if (allH) memcpy(allH, fH, (size_t)n * sizeof(double));
  if (allr) memcpy(allr, fr, (size_t)n * sizeof(uint32_t));
  if (ctr) *ctr = c;
  rc = (int)kk;
done:
  free(order); free(alpha); free(omega); free(dist); free(queue); free(fH); free(fr); free(top);
  return rc;
}

/* The bound sequence U_0, U_1, ... of one source for a given omega (>= r(v)),
 * for the invariant tests: every U_d * (1 + 2^-20) >= h(v), non-increasing in
 * exact arithmetic, and the last equals h(v) when omega = r(v).  Returns the
 * number of levels written (at most maxlev). */
int orc_harmonic_cut_bounds(uint32_t n, const uint32_t *off, const uint32_t *col, int directed, uint32_t v,
                            uint32_t omega_v, double *U, int maxlev) {
  uint32_t *dist = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
  uint32_t *queue = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
  if (!dist || !queue) { free(dist); free(queue); return ORC_ENOMEM; }
  for (uint32_t i = 0; i < n; ++i) dist[i] = UINT32_MAX;
  uint32_t head = 0, tail = 0, d = 0;
  dist[v] = 0;
  queue[tail++] = v;
  uint64_t nd = 1, g = off[v + 1] - off[v];
  double Hd = 0.0;
  int nl = 0;
  while (1) {
    if (nl < maxlev) U[nl] = harmonic_cut_bound(Hd, d, nd, g, omega_v);
    ++nl;
    uint32_t level_end = tail;
    uint64_t cnt = 0, gs = 0;
    while (head < level_end) {
      uint32_t u = queue[head++];
      for (uint32_t e = off[u]; e < off[u + 1]; ++e) {
        uint32_t w = col[e];
        if (dist[w] == UINT32_MAX) {
          dist[w] = d + 1;
          queue[tail++] = w;
          ++cnt;
          gs += (off[w + 1] - off[w]) - (directed ? 0u : 1u);
        }
      }
    }
    if (cnt == 0) break;
    ++d;
    Hd = Hd + (double)cnt / (double)d;
    nd += cnt;
    g = gs;
  }
  free(dist); free(queue);
  return nl < maxlev ? nl : maxlev;
}

/* ---------------------------------------------------------------------- */
/* updateBoundsLB (Section 7, Algorithm 5; Eq. 4 undirected, Eq. 5         */
/* directed): a full BFS from s bounds the farness of every vertex whose    */
/* reach equals s's (its component; its SCC if directed)                    */
/* ---------------------------------------------------------------------- */

/*
 * Level bound of level i of a BFS from s with level sizes g[0..D] (g[0] = 1,
 * the source itself):
 *   undirected (Eq. 4): L(i) = 2 sum_{|j-i| <= 1} g_j + sum_{|j-i| > 1} g_j |j-i| - 2
 *   directed   (Eq. 5): L(i) = 2 sum_{j - i <= 1} g_j + sum_{j - i > 1} g_j (j-i) - 2
 * and S(w) >= L(l(w)) - outdeg(w) for every w at level l(w) whose reach is
 * s's.  Readings: the sums run over all of R(s) including s at level 0 (the
 * set the bound is derived from; Section 7's lemma sets g_j = 0 for j <= 0,
 * which only weakens it), and L(i) is evaluated from its definition for
 * every level (Algorithm 5's first line, L(1) = g_1 + g_2 + sum_{>2} - 2,
 * does not match the definition, so the recurrence is not used).
 */
static uint64_t lb_level(const uint64_t *g, uint32_t D, uint32_t i, int directed) {
  uint64_t s = 0;
  for (uint32_t j = 0; j <= D; ++j) {
    int64_t diff = (int64_t)j - (int64_t)i;
    int64_t ad = diff < 0 ? -diff : diff;
    if (directed) {
      if (diff <= 1) s += 2 * g[j];
      else s += g[j] * (uint64_t)diff;
    } else {
      if (ad <= 1) s += 2 * g[j];
      else s += g[j] * (uint64_t)ad;
    }
  }
  return s - 2;
}

/* BFS from s; writes level[v] (UINT32_MAX if unreachable) and the level
 * bound of each level to L[0..D] (L must hold n entries).  Returns D + 1. */
int orc_lb_level_bounds(uint32_t n, const uint32_t *off, const uint32_t *col, int directed, uint32_t s,
                        uint32_t *level, uint64_t *L) {
  uint32_t *queue = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
  uint64_t *g = (uint64_t *)calloc((size_t)n + 1, sizeof(uint64_t));
  if (!queue || !g) { free(queue); free(g); return ORC_ENOMEM; }
  for (uint32_t i = 0; i < n; ++i) level[i] = UINT32_MAX;
  uint32_t head = 0, tail = 0, D = 0;
  level[s] = 0;
  queue[tail++] = s;
  while (head < tail) {
    uint32_t u = queue[head++];
    for (uint32_t e = off[u]; e < off[u + 1]; ++e) {
      uint32_t w = col[e];
      if (level[w] == UINT32_MAX) {
        level[w] = level[u] + 1;
        if (level[w] > D) D = level[w];
        queue[tail++] = w;
      }
    }
  }
  for (uint32_t i = 0; i < tail; ++i) g[level[queue[i]]]++;
  for (uint32_t i = 0; i <= D; ++i) L[i] = lb_level(g, D, i, directed);
  free(queue); free(g);
  return (int)(D + 1);
}

static uint64_t nb_key_of(uint64_t S, uint64_t r) {
  if (r <= 1) return UINT64_MAX;
  u128 num = (u128)S << ORC_NB_FRAC;
  return (uint64_t)(num / (u128)((r - 1) * (r - 1)));
}

/*
 * Algorithm 1 with updateBoundsLB (DegBound with init_S == NULL: every bound
 * 0; NBBound with init_S/init_r = computeBoundsNB's (S~, r)), one source at a
 * time.  Q holds the unvisited vertices of out-degree >= 1 ordered by
 * (key, position in order0), key = floor(2^46 S_lb / (r_lb - 1)^2) of the
 * vertex's current bound (the reading of the NBCut order: an exact integer
 * order whose key never exceeds the bound).  The head v of Q is searched
 * completely (no cut) unless the k-list is full and key(v) / 2^46 > x
 * strictly, which ends the loop.  After each search from s, every w with
 * comp[w] == comp[s] (its component, or its SCC if directed: then r(w) =
 * r(s)) gets bound (L(l(w)) - outdeg(w), r(s)) if that ratio is larger than
 * its current one.  Outputs as orc_bfscut (counters: edges_visited counts
 * the arcs of every search, all complete; bfs_cut stays 0).
 */
int orc_bfsbound(uint32_t n, const uint32_t *off, const uint32_t *col, int directed, uint32_t k,
                 const uint32_t *order0, const uint64_t *init_S, const uint32_t *init_r, uint32_t *ids,
                 uint64_t *S_out, uint32_t *r_out, uint32_t *n_tied, orc_counters *ctr, uint32_t max_sources) {
  if (k == 0 || n == 0) { if (n_tied) *n_tied = 0; return 0; }
  int rc = ORC_OK;
  uint32_t kk = k < n ? k : n;
  uint32_t *order = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
  uint32_t *rank0 = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
  uint32_t *comp = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
  uint32_t *level = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
  uint64_t *L = (uint64_t *)malloc(((size_t)n + 1) * sizeof(uint64_t));
  uint64_t *bS = (uint64_t *)calloc(n, sizeof(uint64_t));
  uint64_t *br = (uint64_t *)calloc(n, sizeof(uint64_t));
  uint64_t *key = (uint64_t *)calloc(n, sizeof(uint64_t));
  uint64_t *fS = (uint64_t *)calloc(n, sizeof(uint64_t));
  uint32_t *fr = (uint32_t *)calloc(n, sizeof(uint32_t));
  char *done = (char *)calloc(n, 1);
  entry_t *top = (entry_t *)malloc((size_t)kk * sizeof(entry_t));
  if (!order || !rank0 || !comp || !level || !L || !bS || !br || !key || !fS || !fr || !done || !top) {
    rc = ORC_ENOMEM;
    goto out;
  }
  if (order0) memcpy(order, order0, (size_t)n * sizeof(uint32_t));
  else if ((rc = orc_degree_order(n, off, order)) != ORC_OK) goto out;
  for (uint32_t i = 0; i < n; ++i) rank0[order[i]] = i;
  if (directed) {
    int64_t nc = orc_scc(n, off, col, comp);
    if (nc < 0) { rc = (int)nc; goto out; }
  } else {
    /* components: the SCCs of the symmetric graph */
    int64_t nc = orc_scc(n, off, col, comp);
    if (nc < 0) { rc = (int)nc; goto out; }
  }
  for (uint32_t v = 0; v < n; ++v) {
    bS[v] = init_S ? init_S[v] : 0;
    br[v] = init_S ? init_r[v] : 2; /* bound 0 */
    key[v] = nb_key_of(bS[v], br[v]);
  }
  orc_counters c = {0, 0, 0, 0};
  uint32_t ntop = 0;
  while (1) {
    /* head of Q: smallest (key, rank0) among unvisited vertices of out-degree >= 1 */
    uint32_t v = UINT32_MAX;
    for (uint32_t w = 0; w < n; ++w) {
      if (done[w] || off[w + 1] == off[w]) continue;
      if (v == UINT32_MAX || key[w] < key[v] || (key[w] == key[v] && rank0[w] < rank0[v])) v = w;
    }
    if (v == UINT32_MAX) break;
    if (max_sources && c.bfs_started >= max_sources) break;
    if (ntop == kk) {
      uint64_t Sx = top[kk - 1].S, rx = top[kk - 1].r;
      u128 lhs = (u128)key[v] * (u128)((rx - 1) * (rx - 1));
      if (lhs > ((u128)Sx << ORC_NB_FRAC)) break; /* Algorithm 1: the head of Q exceeds x */
    }
    done[v] = 1;
    c.bfs_started++;
    c.bfs_finished++;
    int nl = orc_lb_level_bounds(n, off, col, directed, v, level, L);
    if (nl < 0) { rc = nl; goto out; }
    uint64_t S = 0, r = 0;
    for (uint32_t w = 0; w < n; ++w)
      if (level[w] != UINT32_MAX) {
        S += level[w];
        ++r;
        c.edges_visited += off[w + 1] - off[w];
      }
    fS[v] = S;
    fr[v] = (uint32_t)r;
    top_insert(top, &ntop, kk, S, (uint32_t)r, v);
    if (r <= 1) continue;
    /* updateBoundsLB: vertices whose reach is R(v) */
    for (uint32_t w = 0; w < n; ++w) {
      if (level[w] == UINT32_MAX || comp[w] != comp[v] || w == v) continue;
      uint64_t lbS = L[level[w]] - (uint64_t)(off[w + 1] - off[w]);
      /* keep the larger of lbS/(r-1)^2 and the current bound */
      u128 lhs = (u128)lbS * (u128)((br[w] - 1) * (br[w] - 1));
      u128 rhs = (u128)bS[w] * (u128)((r - 1) * (r - 1));
      if (br[w] <= 1 || lhs > rhs) {
        bS[w] = lbS;
        br[w] = r;
        key[w] = nb_key_of(lbS, r);
      }
    }
  }
  for (uint32_t v = 0; v < n && ntop < kk; ++v)
    if (off[v + 1] == off[v]) top_insert(top, &ntop, kk, 0, 1, v);
  for (uint32_t i = 0; i < kk; ++i) {
    ids[i] = top[i].id;
    if (S_out) S_out[i] = top[i].S;
    if (r_out) r_out[i] = top[i].r;
  }
  if (n_tied) {
    uint32_t t = 0;
    const entry_t *last = &top[kk - 1];
    for (uint32_t v = 0; v < n; ++v) {
      if (off[v + 1] == off[v]) t += last->r <= 1;
      else if (fr[v] && cmp_farness(fS[v], fr[v], last->S, last->r) == 0) ++t;
    }
    *n_tied = t;
  }
  if (ctr) *ctr = c;
  rc = (int)kk;
out:
  free(order); free(rank0); free(comp); free(level); free(L); free(bS); free(br); free(key); free(fS); free(fr);
  free(done); free(top);
  return rc;
}
