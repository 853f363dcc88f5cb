/*
 * rn.h -- C ABI of the GB300 road-network distance-join engine.
 *
 * The engine answers the two queries of Tsatsanifos, "Parallelized Proximity-Based
 * Query Processing Methods for Road Networks" (2016), over a graph it keeps resident
 * in GPU memory:
 *
 *   distance join   all pairs (u in R, v in S) with network distance dist(u,v) <= theta
 *                   (Abstract; Section 1; Section 4, the distance predicate theta);
 *   k closest pairs the k pairs (u in R, v in S) of least network distance, none of
 *                   them farther than theta (Abstract; Section 1; Section 4, where the
 *                   single interface takes both k and theta, Algorithm 2).
 *
 * Conventions shared by every call:
 *   - Node ids are the caller's ids, 0 .. n-1.  R and S are sets: no id twice, and no id
 *     in both (Abstract: two disjoint sets).  Violations return RN_EINVAL.
 *   - Weights are integers in [1, 2^24); distances are exact unsigned integers.
 *   - theta is an integer in [0, 2^31], or RN_INF meaning "no bound", which the engine
 *     treats as 2^31: pairs farther apart than 2^31 are never reported.  A path is cut
 *     only when its cost is greater than theta, so theta itself is included (Algorithm 4
 *     returns when a path cost exceeds the threshold).
 *   - Results are exact and deterministic: a join is sorted by (u, v); k closest pairs
 *     are sorted by (d, u, v), which also breaks ties at the k-th distance.
 *   - Every call returns an rn_status.  No C++ exception crosses this boundary.  On
 *     failure rn_last_error() gives a message for the calling thread.
 *   - Host arrays passed in are read only and may be freed when the call returns.
 *     Results in rn_pairs are host memory owned by the library: free with
 *     rn_pairs_free (page-locked where it could be had, so the copy from the device runs
 *     at the link's speed; freed blocks are kept, up to 1 GiB, for later results; only
 *     the u pointer identifies a result's block, and v and d must not be freed alone).  Results in rn_dpairs are device memory owned by the library:
 *     free with rn_dpairs_free (a struct may be reused across calls; its buffers grow
 *     as needed).
 *   - Queries may be issued from any host thread; those on one device run one at a
 *     time (they share the device's search slab).
 */
#ifndef RN_H
#define RN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RN_OK = 0,
    RN_EINVAL = 1,      /* bad argument: id >= n, repeated id, R and S overlap, theta > 2^31,
                           k = 0, weight outside [1, 2^24), unknown flag */
    RN_ENOMEM = 2,      /* host or device allocation failed */
    RN_ECUDA = 3,       /* a CUDA call failed; rn_last_error() names it */
    RN_ETIMEOUT = 4,    /* a bounded wait ran out (serving) */
    RN_ECANCELLED = 5,  /* the query was cancelled (serving) */
    RN_EBUSY = 6,       /* no admission slot free right now (serving) */
    RN_EINTERNAL = 7,   /* an internal invariant failed (a bug: please report) */
    RN_ENOTIMPL = 8     /* the requested feature is not built */
} rn_status;

#define RN_UNDIRECTED 1u    /* every edge (a, b, w) is also an edge (b, a, w) */
#define RN_REORDER 2u       /* relabel nodes by recursive bisection for locality */
#define RN_INF 0xFFFFFFFFu  /* theta: no bound (treated as RN_THETA_MAX) */
#define RN_THETA_MAX 0x80000000u
#define RN_WEIGHT_LIMIT 0x01000000u /* weights must be < 2^24 */

/* An opaque graph resident in GPU memory. */
typedef struct rn_graph rn_graph;

/* cudaStream_t without the CUDA headers; NULL means the legacy default stream. */
typedef struct CUstream_st *rn_stream;

/* Result pairs in host memory, struct-of-arrays, n entries each. */
typedef struct {
    uint32_t *u;
    uint32_t *v;
    uint32_t *d;
    uint64_t n;
} rn_pairs;

/* Result pairs in device memory, struct-of-arrays; cap = allocated entries. */
typedef struct {
    uint32_t *u;
    uint32_t *v;
    uint32_t *d;
    uint64_t n;
    uint64_t cap;
} rn_dpairs;

/* Engine knobs.  Zero in any field means "choose automatically". */
typedef struct {
    uint32_t tile_width;  /* 1: every source searched by one warp with its ball in a
                             shared-memory map (sources whose ball outgrows the largest
                             warp map, 8192 slots, go to the tile search of width 32);
                             32, 64 or 128: lanes of a slab row, the most sources one
                             thread block searches together; 0: the warp search while the
                             balls met so far, scaled to the query's bound (or, before any
                             search, estimated from it), fit a warp map, else tiles of 32
                             (k closest pairs decides so for each of its radius passes,
                             and takes tiles when the balls at the k-th distance are tiny;
                             a batch plans its instances itself) */
    uint32_t tile_sources;/* sources per tile, <= tile_width; 0 spreads R over whole
                             waves of resident blocks */
    uint32_t delta;       /* bucket width of the delta-stepping search, in weight units;
                             0: 16 median arc weights for the warp search, 4 for tiles */
    uint32_t leaf_size;   /* recursive-bisection leaf size used by RN_REORDER */
    float alpha;          /* smoothing parameter of the bisection (Eq. 1-2), in [0, 1];
                             negative selects the default, 0.5 -- not the 0 of the
                             paper's experiments (Table 1): at 0 the bisection of the
                             road-like graphs is badly unbalanced (slower to build, less
                             compact leaves); the order never changes a result */
    uint32_t map_slots;   /* slots of the first slot map every tile is searched with: 0 or
                             8192 starts with narrow blocks (shared-memory map), 16384 with
                             wide blocks, a larger power of two with a global-memory map of
                             that size (for queries whose balls are known to be large);
                             tiles that overflow are searched again with larger maps */
    uint32_t search_from; /* which set the searches start from (Section 4 searches from
                             each node of R): 0 (RN_FROM_AUTO) the smaller of R and S when
                             the graph was loaded undirected -- distances are symmetric
                             there, so the same pairs come out, (u in R, v in S) as always,
                             from fewer searches -- S when it is at least a fifth smaller,
                             else R; 1 (RN_FROM_R) always R; 2 (RN_FROM_S) always S
                             (RN_EINVAL on a graph not loaded undirected).  Joins, k closest
                             pairs, several joins in one call and batches follow it; points
                             on edges and the hierarchical variant search from R */
} rn_config;

#define RN_FROM_AUTO 0u
#define RN_FROM_R 1u
#define RN_FROM_S 2u

/* An edge list in host memory (library-owned arrays: free with rn_edges_free). */
typedef struct {
    uint32_t n;      /* nodes */
    uint32_t flags;  /* RN_UNDIRECTED | RN_REORDER, as the file asks the graph to be loaded */
    uint64_t m;      /* edges */
    uint32_t *src, *dst, *w;
} rn_edges;

/* Graph facts, filled by rn_graph_info. */
typedef struct {
    uint32_t n;
    uint64_t arcs;          /* directed arcs after cleaning (2 per undirected edge) */
    uint32_t max_degree;
    uint32_t median_weight;
    uint32_t flags;
    double reorder_ms;      /* host time spent on the recursive bisection */
    uint64_t device_bytes;  /* device memory held by the graph and its workspace */
} rn_graph_stats;

/* Counters of the calling thread's last query (rn_last_query_stats). */
typedef struct {
    uint64_t pairs;         /* pairs returned */
    uint64_t tiles;         /* source tiles searched (sources, for the warp search) */
    uint64_t retried_tiles; /* tiles (or sources) searched again with a larger map after an
                               overflow */
    uint64_t scans;         /* slab rows scanned (a node's arcs relaxed for a whole tile) */
    uint32_t tile_width;    /* 1: the warp search ran; else the tile search's width */
    uint32_t tile_sources;  /* sources per tile */
    uint32_t delta;
    uint32_t passes;        /* search passes (k closest pairs widens its radius by passes) */
    uint32_t theta_final;   /* k closest pairs: the k-th distance found, else theta */
    uint32_t launches;      /* kernels the query launched */
    uint32_t blocks_per_sm; /* resident search blocks per SM (occupancy of the first launch) */
    uint64_t slots;         /* sum over tiles of the nodes the tile reached (its union ball) */
    uint64_t slot_arcs;     /* sum over tiles of the arcs leaving those nodes */
    double device_ms;       /* device time of the query, CUDA events on its stream */
    double search_ms;       /* device time of the first search launch (warp or tile search),
                               CUDA events */
    /* search telemetry, summed over blocks: relaxation rounds, queue items over all
       rounds, bucket boundaries, and SM cycles in rounds, boundaries and emission */
    uint64_t rounds, round_items, boundaries;
    uint64_t cycles_rounds, cycles_boundaries, cycles_emission;
    uint64_t cycles_step_a; /* part of cycles_rounds spent taking items and their offsets */
    uint64_t round_arcs;    /* arcs of the scanned items, over all rounds */
    uint64_t max_ball;      /* largest union ball (slots) of a tile that completed */
    double retry_ms;        /* time of the launches that searched overflowed tiles again */
    uint64_t dirty_groups;  /* dirty lane-groups of the scanned items, over all rounds */
    uint64_t slot_lanes;    /* sum over tiles of slots times the tile's lanes (tile_width
                               1: the sum of the sources' balls) */
    uint64_t box_leaf_decided; /* queries in a rectangle: members of R and S kept or dropped
                               by their leaf's bounding rectangle alone */
    uint64_t search_pairs;  /* pairs the search emitted: a join's pairs; k closest pairs: the
                               candidates of the last radius pass, before the selection (the
                               search fields above describe that pass) */
    uint32_t from_s;        /* 1 when the searches started from the nodes of S
                               (rn_config.search_from), 0 from R */
} rn_query_stats;

/*
 * rn_graph_load -- build a graph from an edge list and upload it to the current GPU.
 *   src, dst, w : m edges, host arrays, endpoints < n, weights in [1, 2^24).
 *   flags       : RN_UNDIRECTED and/or RN_REORDER.
 *   xy          : node coordinates, host array of 2 n floats (x, y of node i at 2i,
 *                 2i + 1), finite; may be NULL.  Only queries restricted to a rectangle
 *                 (rn_distance_join_box, rn_kcp_box) read them.
 *   cfg         : may be NULL (defaults).
 * Self-loops are dropped and parallel arcs keep their least weight (neither changes a
 * distance).  With RN_REORDER the nodes are relabelled by the recursive two-seed
 * bisection of Section 3 (Algorithm 1, smoothed by Eq. 1-2) so that every partition of
 * the hierarchy is a contiguous id range; ids seen by the caller never change.  With xy
 * the graph keeps each leaf partition's bounding rectangle (its MBR; without RN_REORDER
 * the leaves are runs of leaf_size consecutive ids).
 * Returns RN_EINVAL for a bad endpoint, weight, coordinate or flag, RN_ENOMEM / RN_ECUDA
 * otherwise.
 */
rn_status rn_graph_load(const uint32_t *src, const uint32_t *dst, const uint32_t *w, uint64_t m,
                        uint32_t n, uint32_t flags, const float *xy, const rn_config *cfg, rn_graph **out);
void rn_graph_free(rn_graph *g);
rn_status rn_graph_info(const rn_graph *g, rn_graph_stats *out);
/*
 * rn_bisection_order -- the relabelling RN_REORDER applies, computed on the host alone
 * (no GPU is touched): order[i] = the original id placed at internal id i, n entries,
 * caller-allocated.  Recursive two-seed bisection (Section 3, Algorithm 1): two
 * clusters grow from two far-apart seeds, each step extending the cluster whose
 * horizon holds the lighter edge, the edge weights smoothed by the relative cluster
 * populations with parameter cfg->alpha (Eq. 1-2); parts of at most cfg->leaf_size
 * nodes (default 512) are leaves.  Same arguments and errors as rn_graph_load.
 */
rn_status rn_bisection_order(const uint32_t *src, const uint32_t *dst, const uint32_t *w, uint64_t m,
                             uint32_t n, uint32_t flags, const rn_config *cfg, uint32_t *order);
/* Copy the relabelling out: perm[orig] = internal id (n entries). */
rn_status rn_graph_permutation(const rn_graph *g, uint32_t *perm);
/* Change a graph's knobs for its later queries; NULL restores the defaults (servers keep
 * the knobs they were made with). */
rn_status rn_graph_set_config(rn_graph *g, const rn_config *cfg);

/*
 * Graph files.  Two formats are read, told apart by their first bytes:
 *   .rng  the engine's binary edge list, little-endian: "RNG1", u32 n, u32 flags,
 *         u64 m, then u32 src[m], u32 dst[m], u32 w[m] (written by rn_graph_write_file);
 *   .gr   DIMACS shortest-path text: "c" comment lines, "p sp n m", then m lines
 *         "a u v w" with 1-based ids, one arc each (flags RN_REORDER).
 * rn_file_read parses a file into host arrays; rn_graph_load_file reads it and loads the
 * graph as rn_graph_load would with the file's flags and default knobs.  RN_EINVAL for a
 * missing, truncated or malformed file (the message names the line or the field).
 */
rn_status rn_file_read(const char *path, rn_edges *out);
void rn_edges_free(rn_edges *e);
rn_status rn_graph_load_file(const char *path, rn_graph **out);
rn_status rn_graph_write_file(const char *path, const uint32_t *src, const uint32_t *dst, const uint32_t *w,
                              uint64_t m, uint32_t n, uint32_t flags);

/*
 * rn_distance_join -- all (u in R, v in S) with dist(u, v) <= theta, sorted by (u, v)
 * (Abstract; Section 4: a threshold theta and no restrictive k).
 *   R, S  : host arrays of nR / nS node ids (sets, disjoint).
 *   out   : filled with library-owned host arrays; free with rn_pairs_free.
 * Synchronous: the pairs are in host memory when it returns.
 */
rn_status rn_distance_join(const rn_graph *g, const uint32_t *R, uint32_t nR, const uint32_t *S,
                           uint32_t nS, uint32_t theta, rn_pairs *out);

/*
 * rn_distance_join_dev -- the same join with inputs and outputs in device memory.
 *   dR, dS : device arrays (caller-owned).  out : library-owned device buffers (see
 *   above); out->n receives the pair count.  All work is ordered on `stream`; the call
 *   returns after the pairs are complete (it reads the pair count back).
 */
rn_status rn_distance_join_dev(const rn_graph *g, const uint32_t *dR, uint32_t nR,
                               const uint32_t *dS, uint32_t nS, uint32_t theta, rn_dpairs *out,
                               rn_stream stream);

/*
 * rn_distance_join_noalloc -- the join of rn_distance_join_dev for callers that cannot
 * let the library allocate device memory: their own allocator has reserved the
 * device, or a cudaFree (which synchronises the whole device) or an allocation that can
 * fail mid-query is not acceptable on their path.  The paper has no counterpart: this
 * is a deployment variant of the same computation.
 *   dR, dS            : device arrays of nR / nS node ids (sets, disjoint).
 *   out_u, out_v, out_d: caller-owned device buffers of out_cap entries each; the pairs
 *                       are written there sorted by (u, v).
 *   n_out             : host; receives the pair count (also when out_cap was too small).
 * It allocates nothing: every scratch buffer lives in one static device array of about
 * 22 MB that every GPU loading the library holds until the process exits.  Limits fixed
 * by that array: at most 2^20 nodes in the graph, 65,536 nodes in R and 2^19 result
 * pairs, and every source tile's search must fit the array's slab; beyond them it
 * returns RN_EINVAL (use rn_distance_join_dev).  The first call on each device finds the
 * array's device address and fills its slab, so make that first call before any stream
 * capture.  All calls share the array and it keeps the last call's contents (each call
 * clears what it needs); calls hold a process-wide lock and return after their GPU
 * work is done, so they do not overlap each other -- any other work that overlapped one
 * of them on the GPU and touched the array would race.
 */
rn_status rn_distance_join_noalloc(const rn_graph *g, const uint32_t *dR, uint32_t nR,
                                   const uint32_t *dS, uint32_t nS, uint32_t theta, uint32_t *out_u,
                                   uint32_t *out_v, uint32_t *out_d, uint64_t out_cap, uint64_t *n_out,
                                   rn_stream stream);

/*
 * rn_kcp -- the k closest pairs (u in R, v in S) with dist(u, v) <= theta, sorted by
 * (d, u, v); fewer than k if fewer pairs lie within theta (Abstract; Section 4,
 * Algorithm 2 "k items within theta"; the global k-th distance of Algorithm 3 bounds
 * every search).  k >= 1.  theta = RN_INF for no distance bound.
 */
rn_status rn_kcp(const rn_graph *g, const uint32_t *R, uint32_t nR, const uint32_t *S,
                 uint32_t nS, uint64_t k, uint32_t theta, rn_pairs *out);
rn_status rn_kcp_dev(const rn_graph *g, const uint32_t *dR, uint32_t nR, const uint32_t *dS,
                     uint32_t nS, uint64_t k, uint32_t theta, rn_dpairs *out, rn_stream stream);

/* ------------------------------------------------- queries in a rectangle ---- */

#define RN_BOX_R 1u /* the rectangle restricts R */
#define RN_BOX_S 2u /* the rectangle restricts S */

/*
 * rn_distance_join_box / rn_kcp_box -- the join (sorted by (u, v)) and k closest pairs
 * (sorted by (d, u, v)) of rn_distance_join / rn_kcp over the members of R (which &
 * RN_BOX_R) and of S (which & RN_BOX_S) whose node lies in the closed rectangle
 * box[0] <= x <= box[2], box[1] <= y <= box[3] of the coordinates given to
 * rn_graph_load; a set the flag leaves out is taken whole.  Geographically constrained
 * queries, Section 2: processing is restricted to the partitions that satisfy the
 * constraint by a comparison with each partition's MBR -- a leaf whose rectangle lies
 * inside the box keeps all its members, one that misses it drops them, and only a leaf
 * on the box's border tests its members one by one.  Distances remain network distances
 * over the whole graph (a path may leave the rectangle).  Host arrays in, library-owned
 * host pairs out.  RN_EINVAL as rn_distance_join / rn_kcp, and for a graph loaded without
 * coordinates, a box with xmin > xmax or ymin > ymax (or a NaN bound), or an unknown flag.
 */
rn_status rn_distance_join_box(const rn_graph *g, const uint32_t *R, uint32_t nR, const uint32_t *S,
                               uint32_t nS, uint32_t theta, const float box[4], uint32_t which, rn_pairs *out);
rn_status rn_kcp_box(const rn_graph *g, const uint32_t *R, uint32_t nR, const uint32_t *S, uint32_t nS,
                     uint64_t k, uint32_t theta, const float box[4], uint32_t which, rn_pairs *out);

/* ------------------------------------------------------ hierarchical variant ---- */

/* Counters of the calling thread's last hierarchical query (rn_last_hier_stats). */
typedef struct {
    uint64_t parts;          /* parts of the hierarchy cut the query used */
    uint64_t max_part;       /* nodes of its largest part */
    uint64_t local_pairs;    /* pairs the local searches found inside their sources' parts */
    uint64_t border_routes;  /* (source, border node) routes of the local searches */
    uint64_t exit_routes;    /* distinct (source, far end of an exit arc) routes */
    uint64_t exit_searches;  /* searches from the far ends of exit arcs */
    uint64_t candidates;     /* pairs through exit arcs before each pair keeps its least distance */
    double local_ms, exit_ms, combine_ms;  /* device time of the three phases (all passes) */
} rn_hier_stats;

/*
 * rn_distance_join_hier / rn_kcp_hier -- the join and k closest pairs of
 * rn_distance_join / rn_kcp (same results, same order, same errors), computed the way of
 * the paper's hierarchical processing (Section 4, Algorithms 2-4) over the partition
 * hierarchy of Algorithm 1: the hierarchy is cut into its coarsest parts of at most
 * part_size nodes (0: its leaves; at least the load's leaf_size, at most 6516);
 * every u in R is searched inside its own part only (local processing), which gives the
 * pairs inside the part and the routes to the part's border nodes; each route is
 * extended over the arcs that leave the part (cross-edges), one search runs from every
 * far end of such an arc and its hits are shared by every u that reaches it (the reuse of
 * the inside routes of Algorithm 4); every pair keeps its least distance.  The search
 * from a far end is not confined to the neighbouring part (the listing's confinement can
 * overstate a distance whose shortest path crosses a border twice), so the result is
 * exact.  k closest pairs grow the radius until the join holds k pairs.  Host arrays in,
 * library-owned host pairs out.  RN_EINVAL also for a part_size outside those limits.
 */
rn_status rn_distance_join_hier(const rn_graph *g, const uint32_t *R, uint32_t nR, const uint32_t *S,
                                uint32_t nS, uint32_t theta, uint32_t part_size, rn_pairs *out);
rn_status rn_kcp_hier(const rn_graph *g, const uint32_t *R, uint32_t nR, const uint32_t *S, uint32_t nS,
                      uint64_t k, uint32_t theta, uint32_t part_size, rn_pairs *out);
rn_status rn_last_hier_stats(rn_hier_stats *out);

/* ---------------------------------------------------------- points on edges ---- */

/* A point on the undirected edge {a, b} at distance t from a (0 <= t <= w, w the edge's
 * weight): an object on the road between two nodes (Section 1: objects moving on edges
 * are searched from the two ends of their edge). */
typedef struct {
    uint32_t a, b, t;
} rn_point;

/*
 * rn_distance_join_points -- the theta-join of points: every (i, j) with the network
 * distance from R[i] to S[j] <= theta, as (u = i, v = j, d), sorted by (u, v).  The
 * distance runs from a point through either end of its edge (or along the edge, for two
 * points on the same edge).  R and S are host arrays of points, which may coincide.
 * RN_EINVAL if a point's {a, b} is not an undirected edge of the graph (both arcs, one
 * weight), a == b, an id is >= n, or t exceeds the edge's weight.  The graph is
 * subdivided at the points for the query (a device copy of the graph plus two arcs per
 * point), then searched as rn_distance_join searches.
 */
rn_status rn_distance_join_points(const rn_graph *g, const rn_point *R, uint32_t nR, const rn_point *S, uint32_t nS,
                                  uint32_t theta, rn_pairs *out);
/* k closest pairs of points within theta, sorted by (d, u, v); u, v index R and S. */
rn_status rn_kcp_points(const rn_graph *g, const rn_point *R, uint32_t nR, const rn_point *S, uint32_t nS,
                        uint64_t k, uint32_t theta, rn_pairs *out);

/* ------------------------------------------------------------------ batches ---- */

/* One theta-join of a batch.  R and S are host arrays and g a loaded graph, read only by
 * rn_batch_create (or rn_join_batch), which copies what it needs: the batch holds no
 * reference to them afterwards.  All graphs of a batch live on the current device. */
typedef struct {
    const rn_graph *g;
    const uint32_t *R;
    uint32_t nR;
    const uint32_t *S;
    uint32_t nS;
    uint32_t theta;
} rn_query;

typedef struct rn_batch rn_batch;

typedef struct {
    uint32_t autotune;  /* 1: before the first run, run the batch under every candidate
                           plan (tile width, bucket width, sources per tile); give each size
                           class of instance (log2 n, log2 |R|, log2 of theta in median arc
                           weights) the candidate with the least SM cycles, and keep that mix
                           if the batch runs faster with it than with the best single
                           candidate; plans are remembered for later batches of the process */
    uint32_t use_graph; /* 1: after the first (eager) run, capture the whole batch in a CUDA
                           graph and replay it on later runs */
} rn_batch_config;

typedef struct {
    uint32_t instances, groups;  /* groups: launches of one plan (search, width or map, shape) */
    uint64_t tiles, retried_tiles, pairs;
    uint32_t eager_runs, graph_runs, launches_per_run;
    uint32_t tuned;              /* 0: not tuned; 1: one candidate plan for every instance;
                                    2: a plan per size class of instance; 3: the plans the
                                    batch had (the default, or a loaded cache's) were the
                                    fastest */
    uint32_t candidates;         /* batch runs the tuning took */
    double device_ms;            /* last run, CUDA events on the batch's stream */
    uint32_t plan_tile_width;    /* tuned = 1: the plan's tile width (1: the warp search) */
    uint32_t plan_delta_mult;    /* tuned = 1: its bucket width in median arc weights */
    uint32_t plan_tile_sources;  /* tuned = 1: its sources per tile (1 for the warp search) */
} rn_batch_stats;

/*
 * rn_batch_create -- upload nq theta-joins (each as rn_distance_join, Section 4) for
 * batched execution.  The graphs are copied into one disjoint union on the device (node
 * ids shifted per instance).  An instance whose ball, estimated from its theta, fits a
 * 2048-slot warp map is searched by the warp search (one source per warp, each source
 * with its instance's theta and bucket width from per-source tables); the others have
 * their sources padded to whole tiles for the tile search.  Every group of one plan
 * (search, tile width or warp map, block shape) is one persistent launch; all pairs are
 * sorted at once, which groups them by instance in (u, v) order.  cfg may be NULL (no autotuning,
 * CUDA graph on).  RN_EINVAL for a bad query (the message names its index), graphs on
 * other devices, or more than 2^32 - 2 nodes or arcs in all; RN_ENOMEM if device memory
 * runs out.
 */
rn_status rn_batch_create(const rn_query *q, uint32_t nq, const rn_batch_config *cfg, rn_batch **out);
/* Run every query of the batch; returns when all pairs are in device memory.  Work is
 * ordered after prior work of `stream` (which may be NULL) and `stream` waits for it. */
rn_status rn_batch_run(rn_batch *b, rn_stream stream);
/* Instance i's pairs of the last run, sorted by (u, v): a library-owned host copy. */
rn_status rn_batch_pairs(const rn_batch *b, uint32_t i, rn_pairs *out);
/* Instance i's pairs of the last run as device pointers owned by the batch (valid until
 * the next rn_batch_run or rn_batch_free). */
rn_status rn_batch_pairs_dev(const rn_batch *b, uint32_t i, const uint32_t **u, const uint32_t **v,
                             const uint32_t **d, uint64_t *n);
rn_status rn_batch_stats_get(const rn_batch *b, rn_batch_stats *out);
/* A batch runs one rn_batch_run at a time; no call on it may overlap rn_batch_free. */
void rn_batch_free(rn_batch *b);
/* The autotuner's plans (per size class: tile width -- 1 for the warp search --, bucket
 * width, sources per tile) to a
 * text file, and back: a loaded file is merged into the process's plans, which later
 * batches use without tuning.  *classes receives how many plans the file held.  RN_EINVAL
 * for a file that cannot be written, opened or parsed. */
rn_status rn_tune_cache_save(const char *path);
rn_status rn_tune_cache_load(const char *path, uint32_t *classes);
/* One call: create a batch (no autotuning), run it once, copy every instance's pairs to
 * outs[0..nq) (free each with rn_pairs_free), free the batch. */
rn_status rn_join_batch(const rn_query *q, uint32_t nq, rn_pairs *outs);

/* ------------------------------------------------------------------ serving ---- */

/* One request to a server: a theta-join (k = 0, as rn_distance_join) or the k closest
 * pairs within theta (k >= 1, as rn_kcp).  R and S are host arrays, copied by
 * rn_serve_submit. */
typedef struct {
    const uint32_t *R;
    uint32_t nR;
    const uint32_t *S;
    uint32_t nS;
    uint32_t theta;
    uint64_t k;
} rn_request;

typedef struct rn_server rn_server;

/*
 * rn_join_many -- several theta-joins over one graph searched together: their sources
 * are laid out one query after another, every tile holds sources of one query and
 * searches with that query's theta against its S, and one sort orders all pairs by
 * (query, u, v).  Small queries then share one launch instead of each leaving most of the
 * GPU idle.  q[i].k must be 0; outs[0..nq) receive each query's pairs sorted by (u, v)
 * (free each with rn_pairs_free).  RN_EINVAL as rn_distance_join, naming the query.
 */
rn_status rn_join_many(const rn_graph *g, const rn_request *q, uint32_t nq, rn_pairs *outs);

/* Zero in any field chooses the default. */
typedef struct {
    uint64_t slab_bytes;  /* the distance-slab arena, the admission budget: a request holds
                             one region of 4 MiB per search block while it runs (default
                             4 GiB) */
    uint32_t workers;     /* requests on the device at once, at most (default 8) */
    uint32_t max_blocks;  /* search blocks (slab regions) of one request, >= 2 (default: the
                             device's SM count) */
} rn_serve_config;

typedef struct {
    uint64_t submitted, completed, failed, pending, running;
    uint64_t cancelled;           /* taken off the queue by rn_serve_cancel */
    uint64_t groups, grouped;     /* searches that served several joins at once, and the
                                     requests they served */
    uint64_t pairs;               /* pairs returned by completed requests */
    uint64_t slab_bytes, slab_bytes_in_use, slab_bytes_peak;
    uint32_t workers, max_running;/* max_running: most requests on the device at once */
    double p50_ms, p99_ms, max_ms, mean_ms;  /* latency, submit to result ready, over the
                                                requests completed since the last reset */
    double mean_queue_ms;         /* submit to admission */
    double busy_s;                /* wall time with at least one request running */
    double span_s;                /* first submit to last completion */
} rn_serve_stats;

/*
 * rn_serve_create -- a server of distance joins and k-closest-pairs requests over one
 * resident graph (the queries of Section 1 and Algorithm 2, answered as by
 * rn_distance_join and rn_kcp).  Requests are admitted first come, first served as soon
 * as a worker and enough contiguous slab regions are free (a request of |R| sources
 * takes min(max_blocks, max(2, ceil(|R| / tile width))) regions); every admitted request
 * runs at once on its own stream with its own slab regions, so requests that arrive
 * while others run overlap with them on the device.  A request's result is the same as
 * the query run alone.  The graph must outlive the server; its own queries (rn_*_join,
 * rn_kcp) may run beside the server's.  RN_EINVAL for bad sizes, RN_ENOMEM when the
 * arena cannot be allocated.
 */
rn_status rn_serve_create(const rn_graph *g, const rn_serve_config *cfg, rn_server **out);
/* (Joins queued one behind another, up to 64 of them and 32,768 sources in all, are
 * admitted together and searched in one launch, as rn_join_many does.) */
/* Queue one request; *ticket identifies it to rn_serve_wait.  RN_EINVAL for a bad
 * request (as rn_distance_join / rn_kcp), found before it is queued. */
rn_status rn_serve_submit(rn_server *s, const rn_request *q, uint64_t *ticket);
/* Wait up to timeout_ms (0: do not wait; 0xFFFFFFFF: no limit) for a request; on
 * success its pairs go to *out (free with rn_pairs_free) and the ticket is spent.
 * RN_ETIMEOUT if it is not done in time (the ticket stays valid); RN_EINVAL for an
 * unknown or spent ticket; otherwise the request's own status. */
rn_status rn_serve_wait(rn_server *s, uint64_t ticket, uint32_t timeout_ms, rn_pairs *out);
/* Take a queued request off the queue: its wait then returns RN_ECANCELLED.  RN_EBUSY
 * if it is already running or finished (it is never interrupted on the device);
 * RN_EINVAL for an unknown ticket. */
rn_status rn_serve_cancel(rn_server *s, uint64_t ticket);
rn_status rn_serve_stats_get(rn_server *s, rn_serve_stats *out);
/* Start a new measurement window: latency samples, counters of completed requests,
 * busy time and span restart (pending and running requests are kept). */
rn_status rn_serve_reset_stats(rn_server *s);
/* Stop the server: running requests finish, queued ones are dropped, uncollected
 * results freed.  No other call on this server may run while it is destroyed. */
void rn_serve_destroy(rn_server *s);

void rn_pairs_free(rn_pairs *p);
void rn_dpairs_free(rn_dpairs *p);

/*
 * rn_set_allocator -- take the library's device memory from the caller's allocator (for
 * instance a framework's caching allocator) instead of cudaMalloc/cudaFree: both
 * functions, or both NULL to go back to cudaMalloc.  alloc(bytes, ctx) returns device
 * memory of the current device, aligned to 256 bytes and ready for use on any stream
 * (the library runs its work on streams of its own), or NULL (RN_ENOMEM); free(ptr, ctx)
 * takes it back.  Every block is returned to the allocator that made it, even after the
 * hook changes; the library frees a block only when none of its work uses it any more.
 * Applies to allocations made after the call, from any thread.  The no-alloc join
 * allocates nothing either way.
 */
typedef void *(*rn_alloc_fn)(size_t bytes, void *ctx);
typedef void (*rn_free_fn)(void *ptr, void *ctx);
rn_status rn_set_allocator(rn_alloc_fn alloc, rn_free_fn free, void *ctx);

/* Per-query stats are also appended as JSON lines to the file named by the environment
 * variable RN_STATS_LOG, when it is set (read once per process). */

/* Message of the calling thread's last failure ("" if none).  Valid until the next call. */
const char *rn_last_error(void);
/* Counters of the calling thread's last successful query. */
rn_status rn_last_query_stats(rn_query_stats *out);
/* Library version string. */
const char *rn_version(void);

#ifdef __cplusplus
}
#endif

#endif /* RN_H */
