"""Plant plausible mistakes in the CPU oracle and check the pin suite catches each one.

Every mutant is the oracle's C source with one small textual change (a flipped
comparison, a dropped term, swapped operands), compiled on the CPU into a temporary
library.  A mutant that passes every pin would mean the pins cannot see that kind of
mistake, so the test fails.
"""
import os

import pytest

import pins
from oracle import oracle as O

MUTANTS = {
    # the theta cut becomes exclusive (Abstract: dist <= theta is inclusive)
    "strict_theta_cut": ("            if (nd > bound) continue;\n            if (nd < s->dist[y]) {\n"
                         "                rc = state_reach(s, y, nd);\n                if (rc) break;\n"
                         "            }\n        }\n    }\n    return rc;\n}\n\n/* Shortest distances",
                         "            if (nd >= bound) continue;\n            if (nd < s->dist[y]) {\n"
                         "                rc = state_reach(s, y, nd);\n                if (rc) break;\n"
                         "            }\n        }\n    }\n    return rc;\n}\n\n/* Shortest distances"),
    # parallel edges keep their largest weight instead of the least
    "multi_edge_max": ("if (x->w != y->w) return x->w < y->w ? -1 : 1;",
                       "if (x->w != y->w) return x->w > y->w ? -1 : 1;"),
    # an undirected edge only one way
    "one_way_edges": ("        if (undirected) {\n", "        if (0) {\n"),
    # kCP tie-break (d, v, u) instead of (d, u, v)
    "kcp_tiebreak_vu": ("    if (x->u != y->u) return x->u < y->u ? -1 : 1;\n    if (x->v != y->v) return x->v < y->v ? -1 : 1;\n    return 0;\n}\n\nvoid og_pairs_free",
                        "    if (x->v != y->v) return x->v < y->v ? -1 : 1;\n    if (x->u != y->u) return x->u < y->u ? -1 : 1;\n    return 0;\n}\n\nvoid og_pairs_free"),
    # kCP keeps the worse candidate
    "kcp_keep_worse": ("} else if (trip_less(&c, &h->a[0])) {", "} else if (trip_less(&h->a[0], &c)) {"),
    # kCP tightens its bound before k pairs are held
    "kcp_early_bound": ("    if (kh->len == kh->k && kh->a[0].d < bound) bound = kh->a[0].d;\n    if (shared) {",
                        "    if (kh->len > 0 && kh->a[0].d < bound) bound = kh->a[0].d;\n    if (shared) {"),
    # kCP prunes ties at the bound
    "kcp_prune_ties": ("        if (it.key > bound) break; /* kcp: cut at the bound */",
                       "        if (it.key >= bound && kh->len == kh->k) break; /* kcp: cut at the bound */"),
    # heap pops the larger child: not a min-heap any more
    "heap_wrong_child": ("if (c + 1 < h->len && h->a[c + 1].key < h->a[c].key) c++;",
                         "if (c + 1 < h->len && h->a[c + 1].key > h->a[c].key) c++;"),
    # a relaxation that forgets the arc weight
    "dropped_weight": ("            uint64_t nd = it.key + g->w[e];\n            uint32_t y = g->to[e];\n            if (nd > bound) continue;\n            if (nd < s->dist[y]) {\n                rc = state_reach(s, y, nd);\n                if (rc) break;\n            }\n        }\n    }\n    return rc;\n}\n\n/* Shortest distances",
                       "            uint64_t nd = it.key + 1;\n            uint32_t y = g->to[e];\n            if (nd > bound) continue;\n            if (nd < s->dist[y]) {\n                rc = state_reach(s, y, nd);\n                if (rc) break;\n            }\n        }\n    }\n    return rc;\n}\n\n/* Shortest distances"),
    # the join sorted (v, u)
    "join_sorted_vu": ("        if (l.n) qsort(l.a, l.n, sizeof(og_triple), cmp_uv);\n        uint64_t arcs = out->arcs;",
                       "        if (l.n) qsort(l.a, l.n, sizeof(og_triple), cmp_duv);\n        uint64_t arcs = out->arcs;"),
    # overlap of R and S no longer rejected
    "overlap_accepted": ("        if (S[i] >= n || mark[S[i]]) { free(mark); return OG_EINVAL; }",
                         "        if (S[i] >= n || mark[S[i]] == 2) { free(mark); return OG_EINVAL; }"),
    # emits a pair for every reached node, not only members of S
    "emit_non_members": ("        if (!inS[x] || !s->done[x]) continue;",
                         "        if (!s->done[x]) continue;"),
    # the sparse reset forgets the settled marks: the next source cannot settle them
    "reset_keeps_done": ("        s->dist[s->seen[i]] = OG_INF;\n        s->done[s->seen[i]] = 0;\n",
                         "        s->dist[s->seen[i]] = OG_INF;\n"),
    # the sparse reset forgets the distances: the next source starts from stale ones
    "reset_keeps_dist": ("        s->dist[s->seen[i]] = OG_INF;\n        s->done[s->seen[i]] = 0;\n",
                         "        s->done[s->seen[i]] = 0;\n"),
    # several threads: a chunk's pairs left unsorted before the chunks are laid end to end
    "mt_chunk_unsorted": ("        if (rc == OG_OK && l->n) qsort(l->a, l->n, sizeof(og_triple), cmp_uv);\n", ""),
    # several threads: kCP keeps every thread's k best instead of the k best of them all
    "mt_kcp_no_cut": ("            rc = store_pairs(all.a, all.n < k ? all.n : k, out);",
                      "            rc = store_pairs(all.a, all.n, out);"),
    # points: the meeting of two points along their shared edge forgotten
    "points_no_same_edge": ("                uint64_t gap = q.t > R[i].t ? q.t - R[i].t : R[i].t - q.t;\n                if (gap < d) d = gap;\n",
                            ""),
    # points: the search seeded at the far end with t instead of w - t
    "points_far_seed": ("    const uint64_t sd[2] = {p.t, w - p.t};", "    const uint64_t sd[2] = {p.t, p.t};"),
    # points: an S point reached from its far end at t instead of w - t
    "points_far_offset": ("if (db != OG_INF && db + (wS[j] - q.t) < d) d = db + (wS[j] - q.t);",
                          "if (db != OG_INF && db + q.t < d) d = db + q.t;"),
    # points: on a shared edge named the other way round, the position not mirrored
    "points_unmirrored": ("                uint64_t pos = wS[j] - q.t; /* S[j]'s distance from R[i].a */",
                          "                uint64_t pos = q.t; /* S[j]'s distance from R[i].a */"),
    # Floyd-Warshall with the intermediate loop in the middle
    "fw_loop_order": ("    for (uint32_t m = 0; m < n; m++)\n        for (uint32_t i = 0; i < n; i++) {",
                      "    for (uint32_t i = 0; i < n; i++)\n        for (uint32_t m = 0; m < n; m++) {"),
}


def _run_pins(o):
    failures = []
    for pin in pins.ALL_PINS:
        try:
            pin(o)
        except Exception as e:  # a crash or a wrong answer both count as caught
            failures.append(f"{pin.__name__}: {e}")
    return failures


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    src = open(O.SRC).read()
    old, new = MUTANTS[name]
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    msrc = tmp_path / f"{name}.c"
    msrc.write_text(src.replace(old, new))
    lib = O.build(str(msrc), str(tmp_path / f"lib{name}.so"))
    failures = _run_pins(O.Oracle(lib))
    assert failures, f"mutant {name} passed every pin"


def test_real_oracle_passes_all(oracle):
    assert _run_pins(oracle) == []
