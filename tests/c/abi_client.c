/* A plain C99 client of the C ABI: compiled and linked against libtkc.so by
 * tests/test_abi.py to show that include/tkc.h is valid C and that every call
 * below resolves.  Run on a GPU it prints the exact top-3 closeness of a
 * 4 x 4 grid, then the best vertex of two copies searched in one launch; the
 * test only builds it. */
#include <stdint.h>
#include <stdio.h>

#include "tkc.h"

int main(void) {
  /* 4 x 4 undirected grid: vertex i*4+j joined to its right and lower neighbours */
  enum { R = 4, C = 4, N = R * C };
  uint32_t off[N + 1], cols[4 * N];
  uint32_t m = 0;
  for (int v = 0; v < N; ++v) {
    int i = v / C, j = v % C;
    off[v] = m;
    if (i > 0) cols[m++] = (uint32_t)(v - C);
    if (j > 0) cols[m++] = (uint32_t)(v - 1);
    if (j < C - 1) cols[m++] = (uint32_t)(v + 1);
    if (i < R - 1) cols[m++] = (uint32_t)(v + C);
  }
  off[N] = m;
  tkc_options opt = {0};
  opt.order = TKC_ORDER_NB;
  tkc_ctx *ctx = NULL;
  int rc = tkc_create(&ctx, &opt);
  if (rc != TKC_OK) {
    fprintf(stderr, "tkc_create: %s\n", tkc_strerror(rc));
    return 1;
  }
  tkc_graph *g = NULL;
  rc = tkc_load_csr(ctx, N, m, off, cols, 0, 0, &g);
  uint32_t ids[3], reach[3];
  uint64_t S[3];
  double far[3], clo[3];
  tkc_result res = {0};
  res.ids = ids;
  res.dist_sum = S;
  res.reach = reach;
  res.farness = far;
  res.closeness = clo;
  res.capacity = 3;
  if (rc == TKC_OK) rc = tkc_topk_closeness(g, 3, &res);
  if (rc == TKC_OK)
    for (uint32_t i = 0; i < res.n_returned; ++i)
      printf("%u S=%llu r=%u farness=%.6f\n", ids[i], (unsigned long long)S[i], reach[i], far[i]);
  else
    fprintf(stderr, "tkc: %s\n", tkc_strerror(rc));
  tkc_free_graph(g);
  /* the same grid twice, loaded together, then both in one launch */
  if (rc == TKC_OK) {
    const uint32_t ns[2] = {N, N};
    const uint64_t ms[2] = {m, m};
    const uint32_t *offs[2] = {off, off}, *colss[2] = {cols, cols};
    const int dirs[2] = {0, 0};
    tkc_graph *gs[2] = {NULL, NULL};
    uint32_t bad = 2;
    rc = tkc_load_csr_many(ctx, 2, ns, ms, offs, colss, dirs, 0, gs, &bad);
    uint32_t ids2[2][3];
    tkc_result outs[2] = {{0}, {0}};
    for (int i = 0; i < 2; ++i) {
      outs[i].ids = ids2[i];  /* the other arrays may stay NULL */
      outs[i].capacity = 3;
    }
    if (rc == TKC_OK) rc = tkc_topk_closeness_multi(ctx, gs, 2, 3, outs);
    if (rc == TKC_OK)
      printf("two grids in one launch: best %u and %u\n", ids2[0][0], ids2[1][0]);
    else
      fprintf(stderr, "tkc (graph %u): %s\n", bad, tkc_strerror(rc));
    tkc_free_graph(gs[0]);
    tkc_free_graph(gs[1]);
  }
  tkc_destroy(ctx);
  return rc == TKC_OK ? 0 : 1;
}
