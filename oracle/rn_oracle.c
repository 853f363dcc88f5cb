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
#include <stdatomic.h>
#include <pthread.h>

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

/* The state of one bounded search, reused from source to source.  At rest dist[] is
 * OG_INF and done[] is 0 for every node; a search lists in seen[] every node it gave a
 * finite distance (each once), and state_clear puts back only those, so a search costs
 * what its ball costs instead of a pass over all n nodes. */
typedef struct {
    uint32_t n;
    uint64_t *dist;
    uint8_t *done;
    uint32_t *seen;
    uint64_t nseen;
    og_heap h;
} og_state;

static void state_free(og_state *s) {
    free(s->dist);
    free(s->done);
    free(s->seen);
    free(s->h.a);
    memset(s, 0, sizeof(*s));
}

static int state_init(og_state *s, uint32_t n) {
    memset(s, 0, sizeof(*s));
    s->n = n;
    s->dist = (uint64_t *)malloc(((size_t)n + 1) * sizeof(uint64_t));
    s->done = (uint8_t *)calloc((size_t)n + 1, 1);
    s->seen = (uint32_t *)malloc(((size_t)n + 1) * sizeof(uint32_t));
    if (!s->dist || !s->done || !s->seen) { state_free(s); return OG_ENOMEM; }
    for (uint32_t x = 0; x < n; x++) s->dist[x] = OG_INF;
    return OG_OK;
}

/* Back to rest: every node the last search reached gets OG_INF and not-done again. */
static void state_clear(og_state *s) {
    for (uint64_t i = 0; i < s->nseen; i++) {
        s->dist[s->seen[i]] = OG_INF;
        s->done[s->seen[i]] = 0;
    }
    s->nseen = 0;
    s->h.len = 0;
}

/* A tentative distance d for node x (smaller than its current one), queued in the heap. */
static int state_reach(og_state *s, uint32_t x, uint64_t d) {
    if (s->dist[x] == OG_INF) s->seen[s->nseen++] = x;
    s->dist[x] = d;
    return heap_push(&s->h, d, x);
}

/* The settled distance of x after a search: OG_INF when x lies beyond the bound or was
 * never reached. */
static uint64_t state_dist(const og_state *s, uint32_t x) { return s->done[x] ? s->dist[x] : OG_INF; }

/* Bounded Dijkstra from nseeds seeds (node seed[i] at distance sd[i]; a seed above the
 * bound is left out): a node is settled only through paths whose every prefix costs
 * <= bound -- a path cost above the bound ends the search, as in Algorithm 4.  The
 * state must be at rest.  *arcs (if not NULL) grows by the out-degree of every settled
 * node: the arcs a plain per-source search must look at. */
static int search_seeds(const og_graph *g, og_state *s, int nseeds, const uint32_t *seed,
                        const uint64_t *sd, uint64_t bound, uint64_t *arcs) {
    int rc = OG_OK;
    for (int i = 0; i < nseeds && rc == OG_OK; i++) {
        if (sd[i] > bound || sd[i] >= s->dist[seed[i]]) continue;
        rc = state_reach(s, seed[i], sd[i]);
    }
    while (rc == OG_OK && s->h.len > 0) {
        og_item it = heap_pop(&s->h);
        if (s->done[it.node] || it.key != s->dist[it.node]) continue; /* stale entry */
        if (it.key > bound) break;
        s->done[it.node] = 1;
        if (arcs) *arcs += g->off[it.node + 1] - g->off[it.node];
        for (uint64_t e = g->off[it.node]; e < g->off[it.node + 1]; e++) {
            uint64_t nd = it.key + g->w[e];
            uint32_t y = g->to[e];
            if (nd > bound) continue;
            if (nd < s->dist[y]) {
                rc = state_reach(s, y, nd);
                if (rc) break;
            }
        }
    }
    return rc;
}

/* Shortest distances from src, bounded as above, into dist[0 .. n): OG_INF for nodes
 * beyond the bound or unreachable. */
int og_sssp(const og_graph *g, uint32_t src, uint64_t bound, uint64_t *dist, uint64_t *arcs) {
    if (src >= g->n) return OG_EINVAL;
    og_state s;
    int rc = state_init(&s, g->n);
    if (rc) return rc;
    const uint64_t zero = 0;
    rc = search_seeds(g, &s, 1, &src, &zero, bound, arcs);
    for (uint32_t x = 0; x < g->n; x++) dist[x] = state_dist(&s, x);
    state_free(&s);
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

/* A growable list of triples. */
typedef struct {
    og_triple *a;
    uint64_t n, cap;
} og_list;

static int list_add(og_list *l, uint32_t u, uint32_t v, uint64_t d) {
    if (l->n == l->cap) {
        uint64_t nc = l->cap ? 2 * l->cap : 1024;
        og_triple *na = (og_triple *)realloc(l->a, nc * sizeof(og_triple));
        if (!na) return OG_ENOMEM;
        l->a = na;
        l->cap = nc;
    }
    l->a[l->n].u = u; l->a[l->n].v = v; l->a[l->n].d = d; l->n++;
    return OG_OK;
}

/* The pairs of one source u: every member of S its search settled (all lie within the
 * bound), appended to l in the order reached. */
static int emit_source(const og_state *s, const uint8_t *inS, uint32_t u, og_list *l) {
    for (uint64_t i = 0; i < s->nseen; i++) {
        uint32_t x = s->seen[i];
        if (!inS[x] || !s->done[x]) continue;
        int rc = list_add(l, u, x, s->dist[x]);
        if (rc) return rc;
    }
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
    og_state s;
    og_list l = {0};
    rc = state_init(&s, g->n);
    const uint64_t zero = 0;
    for (uint32_t i = 0; i < nR && rc == OG_OK; i++) {
        rc = search_seeds(g, &s, 1, &R[i], &zero, theta, &out->arcs);
        if (rc == OG_OK) rc = emit_source(&s, inS, R[i], &l);
        state_clear(&s);
    }
    if (rc == OG_OK) {
        if (l.n) qsort(l.a, l.n, sizeof(og_triple), cmp_uv);
        uint64_t arcs = out->arcs;
        rc = store_pairs(l.a, l.n, out);
        out->arcs = arcs;
    }
    state_free(&s);
    free(l.a); free(inS);
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

/* The bound of kCP's local search: theta, lowered to the d of the worst held pair once k
 * pairs are held (Algorithm 3's global threshold), and to *shared when several threads
 * search (each publishes its own k-th best; any thread's k-th best is an upper bound on
 * the global k-th distance). */
static uint64_t kcp_bound(uint64_t theta, const og_kheap *kh, _Atomic uint64_t *shared) {
    uint64_t bound = theta;
    if (kh->len == kh->k && kh->a[0].d < bound) bound = kh->a[0].d;
    if (shared) {
        uint64_t b = atomic_load_explicit(shared, memory_order_relaxed);
        if (b < bound) bound = b;
    }
    return bound;
}

/* Lower *shared to b (when given). */
static void publish_bound(_Atomic uint64_t *shared, uint64_t b) {
    if (!shared) return;
    uint64_t cur = atomic_load_explicit(shared, memory_order_relaxed);
    while (b < cur && !atomic_compare_exchange_weak_explicit(shared, &cur, b, memory_order_relaxed,
                                                             memory_order_relaxed)) {
    }
}

/* kCP's local search from u (Section 4): best-first, bounded by kcp_bound; every settled
 * member of S is offered to the k best held.  A node is dropped only when its cost is
 * greater than the bound, so pairs tied with the k-th survive for the (d, u, v)
 * tie-break.  The state must be at rest and is left for the caller to clear. */
static int kcp_source(const og_graph *g, og_state *s, const uint8_t *inS, uint32_t u, uint64_t theta,
                      og_kheap *kh, uint64_t *arcs, _Atomic uint64_t *shared) {
    int rc = state_reach(s, u, 0);
    while (rc == OG_OK && s->h.len > 0) {
        og_item it = heap_pop(&s->h);
        if (s->done[it.node] || it.key != s->dist[it.node]) continue;
        uint64_t bound = kcp_bound(theta, kh, shared);
        if (it.key > bound) break; /* kcp: cut at the bound */
        s->done[it.node] = 1;
        *arcs += g->off[it.node + 1] - g->off[it.node];
        if (inS[it.node]) {
            og_triple c;
            c.d = it.key; c.u = u; c.v = it.node;
            kheap_offer(kh, c);
            if (kh->len == kh->k) publish_bound(shared, kh->a[0].d);
            bound = kcp_bound(theta, kh, shared);
        }
        for (uint64_t e = g->off[it.node]; e < g->off[it.node + 1]; e++) {
            uint64_t nd = it.key + g->w[e];
            uint32_t y = g->to[e];
            if (nd > bound) continue;
            if (nd < s->dist[y]) {
                rc = state_reach(s, y, nd);
                if (rc) break;
            }
        }
    }
    return rc;
}

/* kCP, the paper's local search with a shrinking bound: from every u in R a
 * best-first search whose bound is min(theta, d of the worst held pair once k pairs are
 * held) (Section 4; the global threshold of Algorithm 3).  Result sorted by (d, u, v). */
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
    og_state s;
    rc = state_init(&s, g->n);
    if (rc == OG_OK && !kh.a) rc = OG_ENOMEM;
    for (uint32_t i = 0; i < nR && rc == OG_OK; i++) {
        rc = kcp_source(g, &s, inS, R[i], theta, &kh, &out->arcs, NULL);
        state_clear(&s);
    }
    if (rc == OG_OK) {
        if (kh.len) qsort(kh.a, kh.len, sizeof(og_triple), cmp_duv);
        uint64_t arcs = out->arcs;
        rc = store_pairs(kh.a, kh.len, out);
        out->arcs = arcs;
    }
    state_free(&s);
    free(kh.a); free(inS);
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

/* ------------------------------------------------------- all host cores ---- */

/* The same per-source searches on several threads, to time the oracle on every core of
 * a host.  R is taken in increasing id and cut into chunks of consecutive sources; a
 * thread takes the next chunk, searches its sources one after another with a state of
 * its own, and sorts the chunk's pairs by (u, v), so the chunks' lists laid end to end
 * are the join in (u, v) order.  For kCP every thread keeps its own k best and the
 * threads share one bound (see kcp_bound); the k best of all threads' k best are the
 * answer, since every pair of the global k best is among its own thread's k best. */

#define OG_CHUNK 16

static int cmp_u32(const void *pa, const void *pb) {
    uint32_t x = *(const uint32_t *)pa, y = *(const uint32_t *)pb;
    return x < y ? -1 : x > y;
}

typedef struct {
    const og_graph *g;
    const uint32_t *R; /* ascending */
    uint32_t nR;
    const uint8_t *inS;
    uint64_t theta, k;
    _Atomic uint64_t next;  /* next chunk to take */
    _Atomic uint64_t bound; /* kCP: the least k-th best published by any thread */
    _Atomic int rc;
    og_list *chunk;         /* join: per chunk its pairs */
    og_kheap *held;         /* kCP: per thread its k best */
    uint64_t *arcs;         /* per thread */
} og_job;

typedef struct {
    og_job *job;
    uint32_t t;
} og_worker;

static void *join_worker(void *arg) {
    og_worker *w = (og_worker *)arg;
    og_job *j = w->job;
    og_state s;
    int rc = state_init(&s, j->g->n);
    const uint64_t zero = 0, nchunks = ((uint64_t)j->nR + OG_CHUNK - 1) / OG_CHUNK;
    while (rc == OG_OK && atomic_load(&j->rc) == OG_OK) {
        uint64_t c = atomic_fetch_add(&j->next, 1);
        if (c >= nchunks) break;
        og_list *l = &j->chunk[c];
        for (uint64_t i = c * OG_CHUNK; i < (c + 1) * OG_CHUNK && i < j->nR && rc == OG_OK; i++) {
            rc = search_seeds(j->g, &s, 1, &j->R[i], &zero, j->theta, &j->arcs[w->t]);
            if (rc == OG_OK) rc = emit_source(&s, j->inS, j->R[i], l);
            state_clear(&s);
        }
        if (rc == OG_OK && l->n) qsort(l->a, l->n, sizeof(og_triple), cmp_uv);
    }
    state_free(&s);
    if (rc) atomic_store(&j->rc, rc);
    return NULL;
}

static void *kcp_worker(void *arg) {
    og_worker *w = (og_worker *)arg;
    og_job *j = w->job;
    og_state s;
    int rc = state_init(&s, j->g->n);
    const uint64_t nchunks = ((uint64_t)j->nR + OG_CHUNK - 1) / OG_CHUNK;
    while (rc == OG_OK && atomic_load(&j->rc) == OG_OK) {
        uint64_t c = atomic_fetch_add(&j->next, 1);
        if (c >= nchunks) break;
        for (uint64_t i = c * OG_CHUNK; i < (c + 1) * OG_CHUNK && i < j->nR && rc == OG_OK; i++) {
            rc = kcp_source(j->g, &s, j->inS, j->R[i], j->theta, &j->held[w->t], &j->arcs[w->t], &j->bound);
            state_clear(&s);
        }
    }
    state_free(&s);
    if (rc) atomic_store(&j->rc, rc);
    return NULL;
}

/* Run fn on nthreads threads (at least one) over the job. */
static int run_threads(og_job *j, uint32_t nthreads, void *(*fn)(void *)) {
    pthread_t *tid = (pthread_t *)calloc(nthreads, sizeof(pthread_t));
    og_worker *wk = (og_worker *)calloc(nthreads, sizeof(og_worker));
    uint8_t *started = (uint8_t *)calloc(nthreads, 1);
    if (!tid || !wk || !started) { free(tid); free(wk); free(started); return OG_ENOMEM; }
    for (uint32_t t = 0; t < nthreads; t++) {
        wk[t].job = j;
        wk[t].t = t;
        started[t] = pthread_create(&tid[t], NULL, fn, &wk[t]) == 0;
    }
    uint32_t ran = 0;
    for (uint32_t t = 0; t < nthreads; t++)
        if (started[t]) { pthread_join(tid[t], NULL); ran++; }
    if (ran == 0) fn(&wk[0]); /* no thread could be started: run here */
    free(tid); free(wk); free(started);
    return atomic_load(&j->rc);
}

static int job_init(og_job *j, const og_graph *g, const uint32_t *R, uint32_t nR, const uint8_t *inS,
                    uint64_t theta, uint64_t k, uint32_t nthreads, uint32_t **Rsorted) {
    memset(j, 0, sizeof(*j));
    uint32_t *r = (uint32_t *)malloc(((size_t)nR + 1) * sizeof(uint32_t));
    j->arcs = (uint64_t *)calloc(nthreads, sizeof(uint64_t));
    if (!r || !j->arcs) { free(r); free(j->arcs); return OG_ENOMEM; }
    if (nR) memcpy(r, R, (size_t)nR * sizeof(uint32_t));
    qsort(r, nR, sizeof(uint32_t), cmp_u32);
    j->g = g; j->R = r; j->nR = nR; j->inS = inS; j->theta = theta; j->k = k;
    atomic_init(&j->next, 0);
    atomic_init(&j->bound, theta);
    atomic_init(&j->rc, OG_OK);
    *Rsorted = r;
    return OG_OK;
}

/* The theta-join of og_join on nthreads threads: the same pairs in the same order. */
int og_join_mt(const og_graph *g, const uint32_t *R, uint32_t nR, const uint32_t *S, uint32_t nS,
               uint64_t theta, uint32_t nthreads, og_pairs *out) {
    memset(out, 0, sizeof(*out));
    if (theta > OG_THETA_MAX) return OG_EINVAL;
    if (nthreads == 0) nthreads = 1;
    uint8_t *inS = NULL;
    int rc = check_sets(g->n, R, nR, S, nS, &inS);
    if (rc) return rc;
    og_job j;
    uint32_t *r = NULL;
    rc = job_init(&j, g, R, nR, inS, theta, 0, nthreads, &r);
    const uint64_t nchunks = ((uint64_t)nR + OG_CHUNK - 1) / OG_CHUNK;
    if (rc == OG_OK) {
        j.chunk = (og_list *)calloc(nchunks ? nchunks : 1, sizeof(og_list));
        if (!j.chunk) rc = OG_ENOMEM;
    }
    if (rc == OG_OK) rc = run_threads(&j, nthreads, join_worker);
    if (rc == OG_OK) {
        og_list all = {0};
        for (uint64_t c = 0; c < nchunks && rc == OG_OK; c++)
            for (uint64_t i = 0; i < j.chunk[c].n && rc == OG_OK; i++)
                rc = list_add(&all, j.chunk[c].a[i].u, j.chunk[c].a[i].v, j.chunk[c].a[i].d);
        if (rc == OG_OK) rc = store_pairs(all.a, all.n, out);
        for (uint32_t t = 0; t < nthreads; t++) out->arcs += j.arcs[t];
        free(all.a);
    }
    if (j.chunk)
        for (uint64_t c = 0; c < nchunks; c++) free(j.chunk[c].a);
    free(j.chunk); free(j.arcs); free(r); free(inS);
    return rc;
}

/* kCP of og_kcp on nthreads threads: the same k pairs in the same (d, u, v) order. */
int og_kcp_mt(const og_graph *g, const uint32_t *R, uint32_t nR, const uint32_t *S, uint32_t nS,
              uint64_t k, uint64_t theta, uint32_t nthreads, og_pairs *out) {
    memset(out, 0, sizeof(*out));
    if (theta > OG_THETA_MAX || k == 0) return OG_EINVAL;
    if (nthreads == 0) nthreads = 1;
    uint8_t *inS = NULL;
    int rc = check_sets(g->n, R, nR, S, nS, &inS);
    if (rc) return rc;
    og_job j;
    uint32_t *r = NULL;
    rc = job_init(&j, g, R, nR, inS, theta, k, nthreads, &r);
    const uint64_t hcap = k < (uint64_t)nR * nS ? k : (uint64_t)nR * nS;
    if (rc == OG_OK) {
        j.held = (og_kheap *)calloc(nthreads, sizeof(og_kheap));
        if (!j.held) rc = OG_ENOMEM;
        for (uint32_t t = 0; t < nthreads && rc == OG_OK; t++) {
            j.held[t].k = k;
            j.held[t].a = (og_triple *)malloc((hcap ? hcap : 1) * sizeof(og_triple));
            if (!j.held[t].a) rc = OG_ENOMEM;
        }
    }
    if (rc == OG_OK) rc = run_threads(&j, nthreads, kcp_worker);
    if (rc == OG_OK) {
        og_list all = {0};
        for (uint32_t t = 0; t < nthreads && rc == OG_OK; t++)
            for (uint64_t i = 0; i < j.held[t].len && rc == OG_OK; i++)
                rc = list_add(&all, j.held[t].a[i].u, j.held[t].a[i].v, j.held[t].a[i].d);
        if (rc == OG_OK) {
            if (all.n) qsort(all.a, all.n, sizeof(og_triple), cmp_duv);
            rc = store_pairs(all.a, all.n < k ? all.n : k, out);
        }
        for (uint32_t t = 0; t < nthreads; t++) out->arcs += j.arcs[t];
        free(all.a);
    }
    if (j.held)
        for (uint32_t t = 0; t < nthreads; t++) free(j.held[t].a);
    free(j.held); free(j.arcs); free(r); free(inS);
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
 * above the bound are left out), otherwise as og_sssp.  The state must be at rest. */
static int sssp_point(const og_graph *g, og_state *s, og_point p, uint64_t w, uint64_t bound) {
    const uint32_t seed[2] = {p.a, p.b};
    const uint64_t sd[2] = {p.t, w - p.t};
    return search_seeds(g, s, 2, seed, sd, bound, NULL);
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
    uint64_t cap = 1024, n = 0;
    og_triple *t = (og_triple *)malloc(cap * sizeof(og_triple));
    og_state st;
    int rc = (!wR || !wS || !t) ? OG_ENOMEM : state_init(&st, g->n);
    const int have_state = (wR && wS && t && rc == OG_OK);
    if (rc == OG_OK) rc = check_points(g, R, nR, wR);
    if (rc == OG_OK) rc = check_points(g, S, nS, wS);
    for (uint32_t i = 0; i < nR && rc == OG_OK; i++) {
        rc = sssp_point(g, &st, R[i], wR[i], theta);
        for (uint32_t j = 0; j < nS && rc == OG_OK; j++) {
            const og_point q = S[j];
            const uint64_t da = state_dist(&st, q.a), db = state_dist(&st, q.b);
            uint64_t d = OG_INF;
            if (da != OG_INF) d = da + q.t;
            if (db != OG_INF && db + (wS[j] - q.t) < d) d = db + (wS[j] - q.t);
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
        state_clear(&st);
    }
    if (rc == OG_OK) {
        qsort(t, n, sizeof(og_triple), cmp_uv);
        rc = store_pairs(t, n, out);
    }
    if (have_state) state_free(&st);
    free(t); free(wR); free(wS);
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
