"""The oracle's pins must catch plausible mistakes.

Each case copies oracle.c to a temporary directory, plants one mistake (a
dropped term, a wrong sign or index, a transposed operand, a weakened
comparison), builds it, swaps it in for the real library and checks that at
least one pin from test_oracle.py fails.  Nothing here touches the real build
or any GPU."""
import ctypes
import os
import subprocess

import pytest

import oracle
import test_oracle as pins
import test_oracle_nb as nbpins
import test_oracle_harmonic as hpins
import test_oracle_lb as lbpins
import test_oracle_batched as bpins

def _stale_x_mutant():
    """The batched schedule reading x before the step's finished searches are
    merged (the threshold lags one step)."""
    src = open(oracle._SRC).read()
    a = src.index("      /* searches that found nothing new are finished; the others advance */")
    b = src.index("      any = 0;\n", a)
    block = src[a:b]
    x = block.index("      /* x after this step's merges")
    return block, block[x:] + block[:x]


MUTANTS = {
    "bfs_dropped_distance": ("S += dist[w];", "S += dist[w] - (dist[w] > 1);",
                             [pins.test_bfs_equals_floyd_warshall_random]),
    "bfs_level_off_by_one": ("dist[w] = dist[u] + 1;\n        S += dist[w];",
                             "dist[w] = dist[u] + 1 + (u == 0);\n        S += dist[w];",
                             [pins.test_bfs_equals_floyd_warshall_random]),
    "fw_wrong_index": ("if (D[i][m] + D[m][j] < D[i][j]) D[i][j] = D[i][m] + D[m][j];",
                       "if (D[i][m] + D[j][m] < D[i][j]) D[i][j] = D[i][m] + D[j][m];",
                       [lambda: pins.test_bfs_equals_floyd_warshall_exhaustive(4, True)]),
    "order_transposed_operand": ("u128 lhs = (u128)Sa * (u128)((uint64_t)(rb - 1) * (uint64_t)(rb - 1));",
                                 "u128 lhs = (u128)Sa * (u128)((uint64_t)(ra - 1) * (uint64_t)(rb - 1));",
                                 [pins.test_topk_against_fraction_brute_force]),
    "closeness_inverted": ("*closeness = den / num;", "*closeness = num / den;",
                           [pins.test_closeness_against_networkx]),
    "cut_bound_wrong_slope": ("return Sd + (uint64_t)(d + 1) * rem + extra;",
                              "return Sd + (uint64_t)(d + 2) * rem + extra;",
                              [pins.test_cut_bound_invariants]),
    "cut_bound_missing_kink": ("if (kink > lo && kink < hi) cand[nc++] = kink;", "(void)kink;",
                               [pins.test_cut_min_is_minimum_over_whole_interval]),
    "cut_non_strict": ("return lhs > rhs;\n}", "return lhs >= rhs;\n}",
                       [pins.test_bfscut_equals_textbook_small_random]),
    "gamma_wrong_sign_undirected": ("gs += (off[w + 1] - off[w]) - (directed ? 0u : 1u);\n        }\n      }\n    }\n    if (cnt == 0) break;\n    ++d;\n    Sd += (uint64_t)d * cnt;\n    nd += cnt;\n    g = gs;\n  }\n  for",
                                    "gs += (off[w + 1] - off[w]) - (directed ? 0u : 1u) - 1u;\n        }\n      }\n    }\n    if (cnt == 0) break;\n    ++d;\n    Sd += (uint64_t)d * cnt;\n    nd += cnt;\n    g = gs;\n  }\n  for",
                                    [pins.test_cut_bound_invariants]),
    "alpha_too_big": ("A[c] = a + w[c];", "A[c] = a + w[c] + (a > 0);",
                      [pins.test_alpha_omega_bracket_reach_and_exact_on_biggest_scc]),
    "omega_drops_biggest": ("o = o2 + O[big];", "o = o2;",
                            [pins.test_alpha_omega_hand_built_dag]),
    "tree_level2_off": ("cur[s] = sum - deg;", "cur[s] = sum - deg + 1;",
                        [lambda: pins.test_tree_algorithm_matches_bfs(3)]),
    "nb_level2_subtracts_deg_minus_one": ("uint64_t back = (k == 2) ? deg : deg - 1;",
                                          "uint64_t back = deg - 1;",
                                          [lambda: nbpins.test_counts_equal_enumerated_walks(False)]),
    "nb_dropped_backtrack_term": ("Nk[s] = sum - (uint64_t)sub;", "Nk[s] = sum;",
                                  [lambda: nbpins.test_exact_on_trees(0)]),
    "nb_missing_kink": ("if (c1 > a && c1 < o) nb_candidate(", "if (0) nb_candidate(",
                        [lambda: nbpins.test_candidate_minimum_equals_minimum_over_every_reach(40)]),
    "nb_omega_slope_off": ("nb_candidate(P0 + (uint64_t)k * (o - c0), o,", "nb_candidate(P0 + (uint64_t)(k + 1) * (o - c0), o,",
                           [nbpins.test_bound_below_farness_random]),
    "nb_tail_slope_off": ("nb_candidate(P1 + (uint64_t)(k + 1) * (o - c1), o,", "nb_candidate(P1 + (uint64_t)(k + 2) * (o - c1), o,",
                          [lambda: nbpins.test_candidate_minimum_equals_minimum_over_every_reach(2)]),
    "nb_stop_non_strict": ("if (lhs > rhs) break; /* Algorithm 1", "if (lhs >= rhs) break; /* Algorithm 1",
                           [nbpins.test_nbcut_equals_textbook_with_ties]),
    "nb_walks_stop_ignored": ("      if (Nks == 0) {\n        /* no walk", "      if (Nks == 0 && c0 == 1) {\n        /* no walk",
                              [nbpins.test_walks_that_stop_bound_the_reach]),
    "nb_sink_gets_reach_two": ("bS[s] = 0; br[s] = 1; have[s] = 1;", "bS[s] = 0; br[s] = 2; have[s] = 1;",
                               [nbpins.test_out_degree_zero_has_closeness_zero]),
    "harmonic_level_off_by_one": ("    h = h + (double)cnt / (double)d;\n", "    h = h + (double)cnt / (double)(d + (d > 2));\n",
                                  [hpins.test_textbook_within_rounding_of_exact_and_per_level_definition]),
    "harmonic_near_term_too_small": ("double t1 = (double)near / (double)(d + 1);",
                                     "double t1 = (double)near / (double)(d + 2);",
                                     [hpins.test_cut_bounds_hold_and_tighten]),
    "harmonic_ties_by_larger_id": ("  return a->id < b->id;\n}\n\nstatic int cmp_hentry", "  return a->id > b->id;\n}\n\nstatic int cmp_hentry",
                                   [hpins.test_topk_order_and_ties]),
    "harmonic_nb_tail_too_small": ("h_ub[s] = h_ub[s] + (double)(o - c1) / (double)(k + 1);",
                                   "h_ub[s] = h_ub[s] + (double)(o - c1) / (double)(k + 3);",
                                   [hpins.test_nb_upper_bound_holds]),
    "harmonic_nb_last_piece_dropped": ("if (h_ub) h_ub[s] = h_ub[s] + (double)(o - c0) / (double)k;", "(void)0;",
                                       [hpins.test_nb_upper_bound_holds]),
    "lb_drops_source_level": ("  for (uint32_t j = 0; j <= D; ++j) {\n    int64_t diff", "  for (uint32_t j = 1; j <= D; ++j) {\n    int64_t diff",
                              [lbpins.test_level_bound_definition_and_difference_lemma]),
    "lb_directed_uses_both_sides": ("      if (diff <= 1) s += 2 * g[j];\n      else s += g[j] * (uint64_t)diff;",
                                    "      if (ad <= 1) s += 2 * g[j];\n      else s += g[j] * (uint64_t)ad;",
                                    [lbpins.test_vertex_bounds_below_distance_sums]),
    "lb_offset_off_by_one": ("  return s - 2;\n}", "  return s - 1;\n}", [lbpins.test_grid_level_bound_by_hand]),
    "lb_outside_reach_class": ("if (level[w] == UINT32_MAX || comp[w] != comp[v] || w == v) continue;",
                               "if (level[w] == UINT32_MAX || w == v) continue;",
                               [lbpins.test_bfsbound_bounds_only_the_reach_class]),
    "lb_stop_non_strict": ("if (lhs > ((u128)Sx << ORC_NB_FRAC)) break; /* Algorithm 1: the head of Q exceeds x */",
                           "if (lhs >= ((u128)Sx << ORC_NB_FRAC)) break; /* Algorithm 1: the head of Q exceeds x */",
                           [lambda: lbpins.test_bfsbound_equals_textbook_random(False),
                            lambda: lbpins.test_bfsbound_equals_textbook_families(0, False)]),
    "ties_count_skips_kth": ("if (cmp_farness(S[v], r[v], e[kk - 1].S, e[kk - 1].r) == 0) ++t;",
                             "if (cmp_farness(S[v], r[v], e[kk - 1].S, e[kk - 1].r) == 0 && v != e[kk - 1].id) ++t;",
                             [pins.test_topk_against_fraction_brute_force]),
    "farness_rounded_twice": ("*farness = num / den;", "*farness = (double)(n - 1) * ((double)S / den);",
                              [pins.test_farness_doubles_are_single_rounded]),
    "scc_cross_arc_as_back_arc": ("} else if (onstack[w] && index[w] < low[v]) {", "} else if (index[w] < low[v]) {",
                                  [pins.test_scc_by_mutual_reachability]),
    "scc_lowlink_not_propagated": ("if (low[v] < low[u]) low[u] = low[v];", "(void)u;",
                                   [pins.test_scc_by_mutual_reachability]),
    "cut_alpha_not_raised_to_nd": ("  if (lo < nd) lo = nd;\n  if (hi < lo) hi = lo;", "  if (hi < lo) hi = lo;",
                                   [pins.test_cut_min_is_minimum_over_whole_interval,
                                    pins.test_bfscut_equals_textbook_small_random]),
    "cut_min_takes_largest": ("    if (lhs < rhs) { bl = L; br = r; }", "    if (lhs > rhs) { bl = L; br = r; }",
                              [pins.test_cut_min_is_minimum_over_whole_interval]),
    "batched_level0_arcs_dropped": ("        active[s] = 1;\n        c.edges_visited += od;", "        active[s] = 1;",
                                    [lambda: bpins.test_star_counted_by_hand(5)]),
    "batched_no_refill": ("    while (assigned < B && cursor < nq && !stopped) {",
                          "    for (int once = 0; once < 1 && cursor < nq && !stopped; ++once) {",
                          [bpins.test_b1_equals_sequential_bfscut]),
    "batched_undirected_arcs_off": ("arcs[s] = gs[s] + (directed ? 0u : cnt[s]);", "arcs[s] = gs[s];",
                                    [lambda: bpins.test_star_counted_by_hand(5)]),
    "batched_x_read_before_merge": _stale_x_mutant() + ([lambda: bpins.test_star_counted_by_hand(5)],),
    "degree_order_unstable": ("for (uint32_t v = 0; v < n; ++v) order[start[maxd - (off[v + 1] - off[v])]++] = v;",
                              "for (uint32_t v = n; v-- > 0;) order[start[maxd - (off[v + 1] - off[v])]++] = v;",
                              [pins.test_degree_order_matches_lexsort]),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new, checks = MUTANTS[name]
    src = open(oracle._SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    path = tmp_path / "oracle_mut.c"
    path.write_text(src.replace(old, new))
    lib = tmp_path / "liboracle_mut.so"
    subprocess.check_call(["gcc", "-O1", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-o", str(lib),
                           str(path), "-lm"])
    saved = oracle._load()
    oracle._lib = oracle._bind(ctypes.CDLL(str(lib)))
    try:
        caught = False
        for check in checks:
            try:
                check()
            except (AssertionError, RuntimeError):  # a failed pin or an oracle that reports an error
                caught = True
        assert caught, f"planted mistake {name} passed every pin"
    finally:
        oracle._lib = saved
