/*
 * rn_oracle.c -- the CPU oracle for the theta-bounded road-network distance join and
 * k-closest-pairs query of Tsatsanifos, "Parallelized Proximity-Based Query Processing
 * Methods for Road Networks" (2016).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call this
 * file: only the tests, the smoke check and the CPU-baseline leg of the benchmark do.
 * It shares no code, header, table or helper with the CUDA engine; the two meet only
 * in the seeded synthetic inputs both are given.
 *
 * What it computes (plain definitions, written out slowly):
 *   dist(u,v)   length of a shortest u->v path under positive integer arc weights
 *               (Section 1, the road-network distance, not the Euclidean one);
 *   join        { (u, v, dist(u,v)) : u in R, v in S, dist(u,v) <= theta }
 *               (Abstract; Section 1; Section 4, the distance predicate theta),
 *               sorted by (u, v);
 *   kCP         the k pairs (u in R, v in S) of least dist, among those with
 *               dist <= theta (Abstract; Section 1; Section 4, "k items within theta"
 *               in Algorithm 2), ties broken by (d, u, v) ascending, so the answer is
 *               unique; fewer than k when fewer pairs exist.
 *
 * Readings taken where the paper is silent or ambiguous:
 *   - the theta cut is inclusive: a path is dropped only when its cost is greater than
 *     theta (Algorithm 4, the "greater than threshold" return; Abstract "<= theta");
 *   - R and S must be disjoint sets of distinct ids (Abstract, "two disjoint sets");
 *     anything else is rejected;
 *   - self-loops are dropped and parallel edges keep their least weight (the paper
 *     does not say; neither changes any distance);
 *   - weights lie in [1, 2^24) and theta in [0, 2^31]; distances are kept in 64 bits
 *     here so no sum can wrap.
 *
 * Points on edges (Section 1: objects moving on an edge are searched from the two ends
 * of their edge, at their distances from those ends): a point on the undirected edge
 * {a, b} at distance t from a; its distance to a node x is the better of
 * t + dist(a, x) and (w - t) + dist(b, x), w the edge's weight; two points on the same
 * edge may also meet along it, at the difference of their positions.
 *
 * Parity pins (tests, run without a GPU): Floyd-Warshall brute force on tiny graphs,
 * closed-form distances on grids, paths and stars, the transpose symmetry of the join
 * on undirected graphs, monotonicity in theta and k, and kCP against its own
 * definition (full join, sort, truncate).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OG_OK 0
#define OG_EINVAL 1
#define OG_ENOMEM 2

#define OG_INF UINT64_MAX
#define OG_WMAX (1u << 24)
#define OG_THETA_MAX (1ull << 31)

/* ------------------------------------------------------------------ graph ---- */

/* Adjacency lists in a flat array: the arcs leaving x are to[off[x] .. off[x+1]). */
typedef struct {
    uint32_t n;
    uint64_t *off;
    uint32_t *to;
    uint32_t *w;
} og_graph;

typedef struct {
    uint32_t a, b, w;
} og_arc;

static int arc_cmp(const void *pa, const void *pb) {
    const og_arc *x = (const og_arc *)pa, *y = (const og_arc *)pb;
    if (x->a != y->a) return x->a < y->a ? -1 : 1;
    if (x->b != y->b) return x->b < y->b ? -1 : 1;
    if (x->w != y->w) return x->w < y->w ? -1 : 1;
    return 0;
}

void og_graph_free(og_graph *g) {
    if (!g) return;
    free(g->off);
    free(g->to);
    free(g->w);
    free(g);
}

/* Build the oracle's graph from an edge list.  undirected != 0 adds both directions.
 * Returns OG_EINVAL for an endpoint >= n or a weight outside [1, 2^24). */
int og_graph_build(uint32_t n, uint64_t m, const uint32_t *src, const uint32_t *dst,
                   const uint32_t *w, int undirected, og_graph **out) {
    *out = NULL;
    uint64_t i;
    for (i = 0; i < m; i++) {
        if (src[i] >= n || dst[i] >= n) return OG_EINVAL;
        if (w[i] < 1 || w[i] >= OG_WMAX) return OG_EINVAL;
    }
    uint64_t cap = undirected ? 2 * m : m;
    og_arc *arcs = (og_arc *)malloc((cap ? cap : 1) * sizeof(og_arc));
    if (!arcs) return OG_ENOMEM;
    uint64_t na = 0;
    for (i = 0; i < m; i++) {
        if (src[i] == dst[i]) continue; /* self-loop: never on a shortest path */
        arcs[na].a = src[i]; arcs[na].b = dst[i]; arcs[na].w = w[i]; na++;
        if (undirected) {
            arcs[na].a = dst[i]; arcs[na].b = src[i]; arcs[na].w = w[i]; na++;
        }
    }
    qsort(arcs, na, sizeof(og_arc), arc_cmp);
    /* keep the first (least-weight) arc of each (a, b) run */
    uint64_t nk = 0;
    for (i = 0; i < na; i++) {
        if (nk > 0 && arcs[nk - 1].a == arcs[i].a && arcs[nk - 1].b == arcs[i].b) continue;
        arcs[nk++] = arcs[i];
    }
    og_graph *g = (og_graph *)calloc(1, sizeof(og_graph));
    if (!g) { free(arcs); return OG_ENOMEM; }
    g->n = n;
    g->off = (uint64_t *)calloc((size_t)n + 1, sizeof(uint64_t));
    g->to = (uint32_t *)malloc((nk ? nk : 1) * sizeof(uint32_t));
    g->w = (uint32_t *)malloc((nk ? nk : 1) * sizeof(uint32_t));
    if (!g->off || !g->to || !g->w) { free(arcs); og_graph_free(g); return OG_ENOMEM; }
    for (i = 0; i < nk; i++) g->off[arcs[i].a + 1]++;
    for (uint32_t x = 0; x < n; x++) g->off[x + 1] += g->off[x];
    for (i = 0; i < nk; i++) { g->to[i] = arcs[i].b; g->w[i] = arcs[i].w; }
    free(arcs);
    *out = g;
    return OG_OK;
}

uint64_t og_graph_arcs(const og_graph *g) { return g->off[g->n]; }

/* Copy the adjacency out (for tests that want to look at it). */
void og_graph_export(const og_graph *g, uint64_t *off, uint32_t *to, uint32_t *w) {
    memcpy(off, g->off, ((size_t)g->n + 1) * sizeof(uint64_t));
    memcpy(to, g->to, g->off[g->n] * sizeof(uint32_t));
    memcpy(w, g->w, g->off[g->n] * sizeof(uint32_t));
}

/* ------------------------------------------------------------ binary heap ---- */

typedef struct {
    uint64_t key;
    uint32_t node;
} og_item;

typedef struct {
    og_item *a;
    uint64_t len, cap;
} og_heap;

static int heap_push(og_heap *h, uint64_t key, uint32_t node) {
    if (h->len == h->cap) {
        uint64_t nc = h->cap ? 2 * h->cap : 64;
        og_item *na = (og_item *)realloc(h->a, nc * sizeof(og_item));
        if (!na) return OG_ENOMEM;
        h->a = na;
        h->cap = nc;
    }
    uint64_t i = h->len++;
    while (i > 0) {
        uint64_t p = (i - 1) / 2;
        if (h->a[p].key <= key) break;
        h->a[i] = h->a[p];
        i = p;
    }
    h->a[i].key = key;
    h->a[i].node = node;
    return OG_OK;
}

static og_item heap_pop(og_heap *h) {
    og_item top = h->a[0];
    og_item last = h->a[--h->len];
    uint64_t i = 0;
    for (;;) {
        uint64_t c = 2 * i + 1;
        if (c >= h->len) break;
        if (c + 1 < h->len && h->a[c + 1].key < h->a[c].key) c++;
        if (last.key <= h->a[c].key) break;
        h->a[i] = h->a[c];
        i = c;
    }
    if (h->len > 0) h->a[i] = last;
    return top;
}

/* --------------------------------------------------------- bounded Dijkstra ---- */

/* Shortest distances from src, bounded: a node is reached only through paths whose
 * every prefix costs <= bound (a path cost above the bound ends the search, as in
 * Algorithm 4).  dist[] receives OG_INF for nodes beyond the bound or unreachable.
 * *arcs (if not NULL) is incremented by the out-degree of every settled node: the
 * arcs a plain per-source search must look at. */
int og_sssp(const og_graph *g, uint32_t src, uint64_t bound, uint64_t *dist, uint64_t *arcs) {
    if (src >= g->n) return OG_EINVAL;
    for (uint32_t x = 0; x < g->n; x++) dist[x] = OG_INF;
    uint8_t *done = (uint8_t *)calloc(g->n, 1);
    og_heap h = {0};
    if (!done) return OG_ENOMEM;
    dist[src] = 0;
    int rc = heap_push(&h, 0, src);
    while (rc == OG_OK && h.len > 0) {
        og_item it = heap_pop(&h);
        if (done[it.node] || it.key != dist[it.node]) continue; /* stale entry */
        if (it.key > bound) break;
        done[it.node] = 1;
        if (arcs) *arcs += g->off[it.node + 1] - g->off[it.node];
        for (uint64_t e = g->off[it.node]; e < g->off[it.node + 1]; e++) {
            uint64_t nd = it.key + g->w[e];
            uint32_t y = g->to[e];
            if (nd > bound) continue;
            if (nd < dist[y]) {
                dist[y] = nd;
                rc = heap_push(&h, nd, y);
                if (rc) break;
            }
        }
    }
    /* nodes that were reached but never settled lie beyond the bound */
    for (uint32_t x = 0; x < g->n; x++)
        if (!done[x]) dist[x] = OG_INF;
    free(done);
    free(h.a);
    return rc;
}

/* ---------------------------------------------------------------- pairs ---- */

typedef struct {
    uint64_t n;
    uint32_t *u;
    uint32_t *v;
    uint64_t *d;
    uint64_t arcs; /* algorithmic arcs: sum of out-degrees of settled nodes */
} og_pairs;

typedef struct {
    uint64_t d;
    uint32_t u, v;
} og_triple;

static int cmp_uv(const void *pa, const void *pb) {
    const og_triple *x = (const og_triple *)pa, *y = (const og_triple *)pb;
    if (x->u != y->u) return x->u < y->u ? -1 : 1;
    if (x->v != y->v) return x->v < y->v ? -1 : 1;
    return 0;
}

static int cmp_duv(const void *pa, const void *pb) {
    const og_triple *x = (const og_triple *)pa, *y = (const og_triple *)pb;
    if (x->d != y->d) return x->d < y->d ? -1 : 1;
    if (x->u != y->u) return x->u < y->u ? -1 : 1;
    if (x->v != y->v) return x->v < y->v ? -1 : 1;
    return 0;
}

void og_pairs_free(og_pairs *p) {
    free(p->u);
    free(p->v);
    free(p->d);
    p->u = NULL; p->v = NULL; p->d = NULL; p->n = 0;
}

static int store_pairs(og_triple *t, uint64_t n, og_pairs *out) {
    out->n = n;
    out->u = (uint32_t *)malloc((n ? n : 1) * sizeof(uint32_t));
    out->v = (uint32_t *)malloc((n ? n : 1) * sizeof(uint32_t));
    out->d = (uint64_t *)malloc((n ? n : 1) * sizeof(uint64_t));
    if (!out->u || !out->v || !out->d) { og_pairs_free(out); return OG_ENOMEM; }
    for (uint64_t i = 0; i < n; i++) { out->u[i] = t[i].u; out->v[i] = t[i].v; out->d[i] = t[i].d; }
    return OG_OK;
}

/* R and S: ids < n, no repeats, no id in both (Abstract: two disjoint sets). */
static int check_sets(uint32_t n, const uint32_t *R, uint32_t nR, const uint32_t *S, uint32_t nS,
                      uint8_t **s_member) {
    uint8_t *mark = (uint8_t *)calloc(n ? n : 1, 1);
    if (!mark) return OG_ENOMEM;
    for (uint32_t i = 0; i < nR; i++) {
        if (R[i] >= n || mark[R[i]]) { free(mark); return OG_EINVAL; }
        mark[R[i]] = 1;
    }
    for (uint32_t i = 0; i < nS; i++) {
        if (S[i] >= n || mark[S[i]]) { free(mark); return OG_EINVAL; }
        mark[S[i]] = 2;
    }
    for (uint32_t x = 0; x < n; x++) mark[x] = (mark[x] == 2);
    *s_member = mark;
    return OG_OK;
}

/* theta-join: one bounded search from every u in R (Section 4, local processing: a
 * best-first search from each element of R that tests every reached node for
 * membership in S), every pair with dist <= theta, sorted by (u, v). */
int og_join(const og_graph *g, const uint32_t *R, uint32_t nR, const uint32_t *S, uint32_t nS,
            uint64_t theta, og_pairs *out) {
    memset(out, 0, sizeof(*out));
    if (theta > OG_THETA_MAX) return OG_EINVAL;
    uint8_t *inS = NULL;
    int rc = check_sets(g->n, R, nR, S, nS, &inS);
    if (rc) return rc;
    uint64_t *dist = (uint64_t *)malloc(((size_t)g->n + 1) * sizeof(uint64_t));
    uint64_t cap = 1024, n = 0;
    og_triple *t = (og_triple *)malloc(cap * sizeof(og_triple));
    if (!dist || !t) { free(dist); free(t); free(inS); return OG_ENOMEM; }
    for (uint32_t i = 0; i < nR && rc == OG_OK; i++) {
        rc = og_sssp(g, R[i], theta, dist, &out->arcs);
        for (uint32_t x = 0; x < g->n && rc == OG_OK; x++) {
            if (!inS[x] || dist[x] == OG_INF) continue;
            if (n == cap) {
                og_triple *nt = (og_triple *)realloc(t, 2 * cap * sizeof(og_triple));
                if (!nt) { rc = OG_ENOMEM; break; }
                t = nt;
                cap *= 2;
            }
            t[n].u = R[i]; t[n].v = x; t[n].d = dist[x]; n++;
        }
    }
    if (rc == OG_OK) {
        qsort(t, n, sizeof(og_triple), cmp_uv);
        uint64_t arcs = out->arcs;
        rc = store_pairs(t, n, out);
        out->arcs = arcs;
    }
    free(t); free(dist); free(inS);
    return rc;
}

/* ------------------------------------------------------------ k-closest pairs ---- */

/* A max-heap of at most k triples ordered by (d, u, v): the root is the worst kept. */
typedef struct {
    og_triple *a;
    uint64_t len, k;
} og_kheap;

static int trip_less(const og_triple *x, const og_triple *y) { return cmp_duv(x, y) < 0; }

static void kheap_sift_down(og_kheap *h, uint64_t i) {
    for (;;) {
        uint64_t c = 2 * i + 1, big = i;
        if (c < h->len && trip_less(&h->a[big], &h->a[c])) big = c;
        if (c + 1 < h->len && trip_less(&h->a[big], &h->a[c + 1])) big = c + 1;
        if (big == i) return;
        og_triple tmp = h->a[i]; h->a[i] = h->a[big]; h->a[big] = tmp;
        i = big;
    }
}

/* Offer a candidate: keep it if fewer than k are held, or if it is better than the
 * worst held, which it then replaces (Section 4: compare against the up to k best and
 * replace the worst, so k items are kept at all times). */
static void kheap_offer(og_kheap *h, og_triple c) {
    if (h->len < h->k) {
        uint64_t i = h->len++;
        while (i > 0) {
            uint64_t p = (i - 1) / 2;
            if (!trip_less(&h->a[p], &c)) break;
            h->a[i] = h->a[p];
            i = p;
        }
        h->a[i] = c;
    } else if (trip_less(&c, &h->a[0])) {
        h->a[0] = c;
        kheap_sift_down(h, 0);
    }
}

/* kCP, the paper's local search with a shrinking bound: from every u in R a
 * best-first search whose bound is min(theta, d of the worst held pair once k pairs are
 * held) (Section 4; the global threshold of Algorithm 3).  A node is dropped only when
 * its cost is greater than the bound, so pairs tied with the k-th survive for the
 * (d, u, v) tie-break.  Result sorted by (d, u, v). */
int og_kcp(const og_graph *g, const uint32_t *R, uint32_t nR, const uint32_t *S, uint32_t nS,
           uint64_t k, uint64_t theta, og_pairs *out) {
    memset(out, 0, sizeof(*out));
    if (theta > OG_THETA_MAX || k == 0) return OG_EINVAL;
    uint8_t *inS = NULL;
    int rc = check_sets(g->n, R, nR, S, nS, &inS);
    if (rc) return rc;
    uint64_t hcap = k < (uint64_t)nR * nS ? k : (uint64_t)nR * nS;
    og_kheap kh = {0};
    kh.k = k;
    kh.a = (og_triple *)malloc((hcap ? hcap : 1) * sizeof(og_triple));
    uint64_t *dist = (uint64_t *)malloc(((size_t)g->n + 1) * sizeof(uint64_t));
    uint8_t *done = (uint8_t *)malloc(g->n ? g->n : 1);
    og_heap h = {0};
    if (!kh.a || !dist || !done) { rc = OG_ENOMEM; goto out; }
    for (uint32_t i = 0; i < nR && rc == OG_OK; i++) {
        uint32_t u = R[i];
        for (uint32_t x = 0; x < g->n; x++) { dist[x] = OG_INF; done[x] = 0; }
        h.len = 0;
        dist[u] = 0;
        rc = heap_push(&h, 0, u);
        while (rc == OG_OK && h.len > 0) {
            og_item it = heap_pop(&h);
            if (done[it.node] || it.key != dist[it.node]) continue;
            uint64_t bound = theta;
            if (kh.len == kh.k && kh.a[0].d < bound) bound = kh.a[0].d;
            if (it.key > bound) break;
            done[it.node] = 1;
            out->arcs += g->off[it.node + 1] - g->off[it.node];
            if (inS[it.node]) {
                og_triple c;
                c.d = it.key; c.u = u; c.v = it.node;
                kheap_offer(&kh, c);
                if (kh.len == kh.k && kh.a[0].d < bound) bound = kh.a[0].d;
            }
            for (uint64_t e = g->off[it.node]; e < g->off[it.node + 1]; e++) {
                uint64_t nd = it.key + g->w[e];
                uint32_t y = g->to[e];
                if (nd > bound) continue;
                if (nd < dist[y]) {
                    dist[y] = nd;
                    rc = heap_push(&h, nd, y);
                    if (rc) break;
                }
            }
        }
    }
    if (rc == OG_OK) {
        qsort(kh.a, kh.len, sizeof(og_triple), cmp_duv);
        uint64_t arcs = out->arcs;
        rc = store_pairs(kh.a, kh.len, out);
        out->arcs = arcs;
    }
out:
    free(kh.a); free(dist); free(done); free(h.a); free(inS);
    return rc;
}

/* kCP straight from its definition: the full theta-join, sorted by (d, u, v), cut to
 * its first k.  Slow; it exists to check og_kcp. */
int og_kcp_bruteforce(const og_graph *g, const uint32_t *R, uint32_t nR, const uint32_t *S,
                      uint32_t nS, uint64_t k, uint64_t theta, og_pairs *out) {
    if (k == 0) { memset(out, 0, sizeof(*out)); return OG_EINVAL; }
    og_pairs all;
    int rc = og_join(g, R, nR, S, nS, theta, &all);
    if (rc) { memset(out, 0, sizeof(*out)); return rc; }
    og_triple *t = (og_triple *)malloc((all.n ? all.n : 1) * sizeof(og_triple));
    if (!t) { og_pairs_free(&all); return OG_ENOMEM; }
    for (uint64_t i = 0; i < all.n; i++) { t[i].u = all.u[i]; t[i].v = all.v[i]; t[i].d = all.d[i]; }
    qsort(t, all.n, sizeof(og_triple), cmp_duv);
    uint64_t keep = all.n < k ? all.n : k;
    uint64_t arcs = all.arcs;
    og_pairs_free(&all);
    rc = store_pairs(t, keep, out);
    out->arcs = arcs;
    free(t);
    return rc;
}

/* ------------------------------------------------------------ Floyd-Warshall ---- */

/* All-pairs shortest distances by Floyd-Warshall, D[i*n + j], OG_INF when no path.
 * Independent of the Dijkstra above: used to pin it on tiny graphs. */
int og_floyd_warshall(const og_graph *g, uint64_t *D) {
    uint32_t n = g->n;
    for (uint64_t i = 0; i < (uint64_t)n * n; i++) D[i] = OG_INF;
    for (uint32_t i = 0; i < n; i++) D[(uint64_t)i * n + i] = 0;
    for (uint32_t x = 0; x < n; x++)
        for (uint64_t e = g->off[x]; e < g->off[x + 1]; e++) {
            uint64_t *c = &D[(uint64_t)x * n + g->to[e]];
            if (g->w[e] < *c) *c = g->w[e];
        }
    for (uint32_t m = 0; m < n; m++)
        for (uint32_t i = 0; i < n; i++) {
            uint64_t dim = D[(uint64_t)i * n + m];
            if (dim == OG_INF) continue;
            for (uint32_t j = 0; j < n; j++) {
                uint64_t dmj = D[(uint64_t)m * n + j];
                if (dmj == OG_INF) continue;
                if (dim + dmj < D[(uint64_t)i * n + j]) D[(uint64_t)i * n + j] = dim + dmj;
            }
        }
    return OG_OK;
}

/* ------------------------------------------------------------ points on edges ---- */

/* A point on the undirected edge {a, b}, at distance t from a, 0 <= t <= w(a, b) (the
 * least weight among parallel a-b edges). */
typedef struct {
    uint32_t a, b, t;
} og_point;

/* The least weight of an arc a -> b, or OG_INF if there is none. */
static uint64_t arc_weight(const og_graph *g, uint32_t a, uint32_t b) {
    uint64_t best = OG_INF;
    for (uint64_t e = g->off[a]; e < g->off[a + 1]; e++)
        if (g->to[e] == b && g->w[e] < best) best = g->w[e];
    return best;
}

static int check_points(const og_graph *g, const og_point *P, uint32_t nP, uint64_t *w) {
    for (uint32_t i = 0; i < nP; i++) {
        if (P[i].a >= g->n || P[i].b >= g->n || P[i].a == P[i].b) return OG_EINVAL;
        uint64_t wab = arc_weight(g, P[i].a, P[i].b), wba = arc_weight(g, P[i].b, P[i].a);
        if (wab == OG_INF || wab != wba || P[i].t > wab) return OG_EINVAL; /* an undirected edge */
        w[i] = wab;
    }
    return OG_OK;
}

/* Bounded search from a point: Dijkstra seeded at a with t and at b with w - t (seeds
 * above the bound are left out), otherwise as og_sssp. */
static int sssp_point(const og_graph *g, og_point p, uint64_t w, uint64_t bound, uint64_t *dist) {
    for (uint32_t x = 0; x < g->n; x++) dist[x] = OG_INF;
    uint8_t *done = (uint8_t *)calloc(g->n, 1);
    og_heap h = {0};
    if (!done) return OG_ENOMEM;
    int rc = OG_OK;
    const uint32_t seed[2] = {p.a, p.b};
    const uint64_t sd[2] = {p.t, w - p.t};
    for (int i = 0; i < 2 && rc == OG_OK; i++) {
        if (sd[i] > bound || sd[i] >= dist[seed[i]]) continue;
        dist[seed[i]] = sd[i];
        rc = heap_push(&h, sd[i], seed[i]);
    }
    while (rc == OG_OK && h.len > 0) {
        og_item it = heap_pop(&h);
        if (done[it.node] || it.key != dist[it.node]) continue;
        if (it.key > bound) break;
        done[it.node] = 1;
        for (uint64_t e = g->off[it.node]; e < g->off[it.node + 1]; e++) {
            uint64_t nd = it.key + g->w[e];
            uint32_t y = g->to[e];
            if (nd > bound) continue;
            if (nd < dist[y]) {
                dist[y] = nd;
                rc = heap_push(&h, nd, y);
                if (rc) break;
            }
        }
    }
    for (uint32_t x = 0; x < g->n; x++)
        if (!done[x]) dist[x] = OG_INF;
    free(done);
    free(h.a);
    return rc;
}

/* theta-join of points: every (i, j), R[i] to S[j] within theta, with its distance,
 * sorted by (i, j).  The distance from R[i] to S[j] on edge {c, e} at s from c is the
 * least of dist(R[i], c) + s and dist(R[i], e) + (w - s), and, when both lie on the
 * same edge, the gap between their positions along it. */
int og_join_points(const og_graph *g, const og_point *R, uint32_t nR, const og_point *S, uint32_t nS,
                   uint64_t theta, og_pairs *out) {
    memset(out, 0, sizeof(*out));
    if (theta > OG_THETA_MAX) return OG_EINVAL;
    uint64_t *wR = (uint64_t *)malloc(((size_t)nR + 1) * sizeof(uint64_t));
    uint64_t *wS = (uint64_t *)malloc(((size_t)nS + 1) * sizeof(uint64_t));
    uint64_t *dist = (uint64_t *)malloc(((size_t)g->n + 1) * sizeof(uint64_t));
    uint64_t cap = 1024, n = 0;
    og_triple *t = (og_triple *)malloc(cap * sizeof(og_triple));
    int rc = (!wR || !wS || !dist || !t) ? OG_ENOMEM : OG_OK;
    if (rc == OG_OK) rc = check_points(g, R, nR, wR);
    if (rc == OG_OK) rc = check_points(g, S, nS, wS);
    for (uint32_t i = 0; i < nR && rc == OG_OK; i++) {
        rc = sssp_point(g, R[i], wR[i], theta, dist);
        for (uint32_t j = 0; j < nS && rc == OG_OK; j++) {
            const og_point q = S[j];
            uint64_t d = OG_INF;
            if (dist[q.a] != OG_INF) d = dist[q.a] + q.t;
            if (dist[q.b] != OG_INF && dist[q.b] + (wS[j] - q.t) < d) d = dist[q.b] + (wS[j] - q.t);
            if (q.a == R[i].a && q.b == R[i].b) {
                uint64_t gap = q.t > R[i].t ? q.t - R[i].t : R[i].t - q.t;
                if (gap < d) d = gap;
            } else if (q.a == R[i].b && q.b == R[i].a) {
                uint64_t pos = wS[j] - q.t; /* S[j]'s distance from R[i].a */
                uint64_t gap = pos > R[i].t ? pos - R[i].t : R[i].t - pos;
                if (gap < d) d = gap;
            }
            if (d > theta) continue;
            if (n == cap) {
                og_triple *nt = (og_triple *)realloc(t, 2 * cap * sizeof(og_triple));
                if (!nt) { rc = OG_ENOMEM; break; }
                t = nt;
                cap *= 2;
            }
            t[n].u = i; t[n].v = j; t[n].d = d; n++;
        }
    }
    if (rc == OG_OK) {
        qsort(t, n, sizeof(og_triple), cmp_uv);
        rc = store_pairs(t, n, out);
    }
    free(t); free(dist); free(wR); free(wS);
    return rc;
}

/* k closest pairs of points within theta, by its definition: the whole join, sorted by
 * (d, i, j), cut to the first k. */
int og_kcp_points(const og_graph *g, const og_point *R, uint32_t nR, const og_point *S, uint32_t nS,
                  uint64_t k, uint64_t theta, og_pairs *out) {
    if (k == 0) return OG_EINVAL;
    og_pairs all;
    int rc = og_join_points(g, R, nR, S, nS, theta, &all);
    memset(out, 0, sizeof(*out));
    if (rc) return rc;
    og_triple *t = (og_triple *)malloc((all.n ? all.n : 1) * sizeof(og_triple));
    if (!t) { og_pairs_free(&all); return OG_ENOMEM; }
    for (uint64_t i = 0; i < all.n; i++) { t[i].u = all.u[i]; t[i].v = all.v[i]; t[i].d = all.d[i]; }
    qsort(t, all.n, sizeof(og_triple), cmp_duv);
    rc = store_pairs(t, all.n < k ? all.n : k, out);
    free(t);
    og_pairs_free(&all);
    return rc;
}
