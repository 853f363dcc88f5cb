// Internal declarations shared by the host runtime (rn_graph.cpp, rn_api.cpp) and the
// CUDA engine (rn_engine.cu).  Not part of the public ABI (include/rn.h).
#pragma once

#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include <vector_types.h>

#include "rn.h"

#include <nvtx3/nvToolsExt.h>

namespace rn {

// A named NVTX range over a scope (query phases show up by name in Nsight timelines and
// ncu range filters; without a tool attached the calls do nothing).
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};

// Every internal failure is thrown as an Error and turned into an rn_status at the ABI.
struct Error {
    rn_status status;
    std::string msg;
};

[[noreturn]] void fail(rn_status s, const std::string &msg);

// Compressed sparse rows in host memory: the arcs leaving node x are
// (col[e], w[e]) for e in [row_ptr[x], row_ptr[x+1]), sorted by (col, w).
struct HostGraph {
    uint32_t n = 0;
    std::vector<uint32_t> row_ptr;
    std::vector<uint32_t> col;
    std::vector<uint32_t> w;
    uint64_t arcs() const { return col.size(); }
};

// Edge list -> cleaned CSR (self-loops dropped, parallel arcs reduced to least weight).
HostGraph build_csr(uint32_t n, uint64_t m, const uint32_t *src, const uint32_t *dst,
                    const uint32_t *w, bool undirected);

// Recursive two-seed bisection (Algorithm 1 with the smoothing of Eq. 1-2).  Returns
// order[i] = the original id placed at internal id i; every partition of the hierarchy
// occupies a contiguous range of internal ids.  leaf_starts (if given) receives the
// first internal id of every leaf, ascending; parts (if given) every part of the
// hierarchy, root and leaves included, as (first internal id << 32) | size, ascending.
std::vector<uint32_t> bisection_order(const HostGraph &g, uint32_t leaf_size, float alpha, bool symmetric,
                                      std::vector<uint32_t> *leaf_starts = nullptr,
                                      std::vector<uint64_t> *parts = nullptr);

// CSR of g relabelled so that internal id i is original node order[i].
HostGraph relabel(const HostGraph &g, const std::vector<uint32_t> &order);

// The graph as it lives on the device.
struct DeviceGraph {
    uint32_t n = 0;
    uint64_t arcs = 0;
    uint32_t *row_ptr = nullptr;  // n + 1
    uint32_t *adj = nullptr;      // 2 * arcs: (col, w) interleaved, 8-byte aligned
    uint32_t *perm = nullptr;     // original id -> internal id
    uint32_t *iperm = nullptr;    // internal id -> original id
    bool iperm_inverts_perm = true;  // false when output ids are not the input ids (points)
    bool symmetric = false;          // every arc has its reverse with the same weight (undirected)
    // node coordinates (rn_graph_load's xy), or none: per node (x, y) by internal id, and
    // the leaves of the partition -- leaf i holds internal ids [leaf_start[i],
    // leaf_start[i + 1]) -- with their bounding rectangles (xmin, ymin, xmax, ymax)
    float2 *xy = nullptr;
    uint32_t nleaves = 0;
    uint32_t *leaf_start = nullptr;  // nleaves + 1
    float4 *leaf_box = nullptr;      // nleaves
};

struct Workspace;  // device scratch owned by a graph (rn_engine.cu)

struct QueryStats {
    rn_query_stats s{};
};

// Engine entry points (rn_engine.cu).  All device pointers; work ordered on `stream`.
Workspace *workspace_create(const DeviceGraph &g);
void workspace_destroy(Workspace *ws);
uint64_t workspace_bytes(const Workspace *ws);

struct EngineConfig {
    uint32_t tile_width = 0;  // 0: choose; 1: one warp per source; 32, 64, 128: tiles
    uint32_t tile_src = 0;  // sources per tile; 0: spread over whole waves of blocks
    uint32_t delta = 0;     // 0: derive from the weights
    uint32_t map_slots = 0; // first slot map: 0 / 8192 narrow, 16384 wide, larger: global
    uint32_t search_from = 0;  // RN_FROM_AUTO, RN_FROM_R or RN_FROM_S
};

void run_join(const DeviceGraph &g, Workspace *ws, const EngineConfig &cfg, uint32_t median_w,
              const uint32_t *dR, uint32_t nR, const uint32_t *dS, uint32_t nS, uint32_t theta,
              rn_dpairs *out, void *stream, rn_query_stats *stats);

void run_kcp(const DeviceGraph &g, Workspace *ws, const EngineConfig &cfg, uint32_t median_w,
             const uint32_t *dR, uint32_t nR, const uint32_t *dS, uint32_t nS, uint64_t k,
             uint32_t theta, rn_dpairs *out, void *stream, rn_query_stats *stats);

// Several joins over one graph in one search: host arrays of original ids (already
// checked), perm the host original -> internal map; out holds all pairs sorted by
// (query, u, v) and counts[i] query i's number of them.
void run_join_multi(const DeviceGraph &g, Workspace *ws, const EngineConfig &cfg, uint32_t median_w,
                    const std::vector<uint32_t> &perm, const std::vector<const uint32_t *> &R,
                    const std::vector<uint32_t> &nR, const std::vector<const uint32_t *> &S,
                    const std::vector<uint32_t> &nS, const std::vector<uint32_t> &theta, rn_dpairs *out,
                    std::vector<uint64_t> *counts, void *stream, rn_query_stats *stats);

// The join with every scratch buffer in one static device array (no allocation).
void run_join_noalloc(const DeviceGraph &g, uint32_t median_w, const uint32_t *dR, uint32_t nR,
                      const uint32_t *dS, uint32_t nS, uint32_t theta, uint32_t *out_u, uint32_t *out_v,
                      uint32_t *out_d, uint64_t out_cap, uint64_t *n_out, void *stream);

// Batches of joins (rn_engine.cu).
struct Batch;
// graphs[i] with host permutation perms[i] (original -> internal id); R and S host
// arrays already validated.
Batch *batch_create(const std::vector<const DeviceGraph *> &graphs, const std::vector<const std::vector<uint32_t> *> &perms,
                    const std::vector<uint32_t> &median_w, const std::vector<const uint32_t *> &R,
                    const std::vector<uint32_t> &nR, const std::vector<const uint32_t *> &S,
                    const std::vector<uint32_t> &nS, const std::vector<uint32_t> &theta,
                    const std::vector<uint32_t> &search_from);
void batch_tune(Batch *b);
void batch_run(Batch *b, void *stream, bool use_graph);
void batch_pairs_dev(const Batch *b, uint32_t i, const uint32_t **u, const uint32_t **v, const uint32_t **d,
                     uint64_t *n);
const rn_batch_stats &batch_stats(const Batch *b);
void batch_destroy(Batch *b);
void tune_cache_save(const char *path);
uint32_t tune_cache_load(const char *path);

// Workspaces with a slab of their own (servers, rn_engine.cu).
size_t slab_region_bytes();
void workspace_set_slab(Workspace *ws, uint32_t *slab, uint32_t regions);
void workspace_reserve(Workspace *ws, uint32_t max_r, uint64_t max_pairs);

// Graph files (rn_file.cpp): the .rng binary edge list and DIMACS .gr text.
struct EdgeFile {
    uint32_t n = 0, flags = 0;
    std::vector<uint32_t> src, dst, w;
};
void read_edge_file(const char *path, EdgeFile *out);
void write_edge_file(const char *path, uint32_t n, uint64_t m, const uint32_t *src, const uint32_t *dst,
                     const uint32_t *w, uint32_t flags);

// Queries over points on edges (rn_engine.cu): the graph subdivided at the points, then
// the ordinary join (k = 0) or k closest pairs.  perm: host original -> internal ids.
struct PointsState;
void run_points(const DeviceGraph &g, const std::vector<uint32_t> &perm, PointsState **state, const EngineConfig &cfg,
                uint32_t median_w, const rn_point *R, uint32_t nR, const rn_point *S, uint32_t nS, uint64_t k,
                uint32_t theta, rn_dpairs *out, void *stream, rn_query_stats *stats);
void points_destroy(PointsState *ps);

// Request servers (rn_serve.cpp): the graph must outlive its server.
struct Server;
Server *server_create(const rn_graph *g, uint64_t slab_bytes, uint32_t workers, uint32_t max_blocks);
uint64_t server_submit(Server *s, const uint32_t *R, uint32_t nR, const uint32_t *S, uint32_t nS, uint32_t theta,
                       uint64_t k);
// Throws Error(RN_ETIMEOUT) when not done in time, or the request's own error.
void server_wait(Server *s, uint64_t ticket, uint32_t timeout_ms, rn_pairs *out);
void server_cancel(Server *s, uint64_t ticket);
void server_stats(Server *s, rn_serve_stats *out);
void server_reset_stats(Server *s);
void server_destroy(Server *s);

// Device pairs -> library-owned host pairs (rn_pairs_free releases them).
void to_host_pairs(const rn_dpairs &d, rn_pairs *out, void *stream);

void upload_graph(const HostGraph &g, const std::vector<uint32_t> &perm,
                  const std::vector<uint32_t> &iperm, DeviceGraph *out);
// Upload node coordinates (original ids, 2 floats each) and the partition's leaves
// (first internal id of each, ascending) with their bounding rectangles.
void upload_geometry(const float *xy, const std::vector<uint32_t> &order, const std::vector<uint32_t> &leaf_starts,
                     DeviceGraph *out);

// Queries restricted to a rectangle (rn_engine.cu): the members of R (RN_BOX_R in which)
// and of S (RN_BOX_S) outside box = (xmin, ymin, xmax, ymax) are dropped -- a whole leaf
// at a time where its bounding rectangle lies inside or outside the box -- then the
// ordinary join (k = 0) or k closest pairs runs on what is left.
struct BoxState;
struct HierState;
void run_box(const DeviceGraph &g, Workspace *ws, BoxState **state, const EngineConfig &cfg, uint32_t median_w,
             const uint32_t *dR, uint32_t nR, const uint32_t *dS, uint32_t nS, const float *box, uint32_t which,
             uint64_t k, uint32_t theta, rn_dpairs *out, void *stream, rn_query_stats *stats, uint64_t *leaves_whole);
void box_destroy(BoxState *bs);

// The hierarchical variant (rn_engine.cu): searches local to the parts of a cut of the
// partition hierarchy, searches from the far ends of the arcs that leave a part, and
// their combination.  part_start: the first internal id of every part of the cut,
// ascending, the first 0.  R and S: host arrays of original ids (checked); perm the host
// original -> internal map.  k = 0: the join; else k closest pairs.
struct HierState;
void run_hier(const DeviceGraph &g, Workspace *ws, HierState **state, const EngineConfig &cfg, uint32_t median_w,
              const std::vector<uint32_t> &perm, const std::vector<uint32_t> &part_start, const uint32_t *R,
              uint32_t nR, const uint32_t *S, uint32_t nS, uint64_t k, uint32_t theta, rn_dpairs *out, void *stream,
              rn_query_stats *stats, rn_hier_stats *hs);
void hier_destroy(HierState *hs);
void free_graph(DeviceGraph *g);
void dpairs_reserve(rn_dpairs *p, uint64_t cap);
void dpairs_release(rn_dpairs *p);
void copy_to_host(void *dst, const void *src, size_t bytes, void *stream);
void copy_to_device(void *dst, const void *src, size_t bytes, void *stream);
void set_allocator(rn_alloc_fn alloc, rn_free_fn free, void *ctx);
void *device_alloc(size_t bytes);
void device_free(void *p);
void stream_sync(void *stream);

}  // namespace rn

namespace rn {
// Device copies of host R and S and a device result buffer, used by the host-buffer
// entry points of one graph.
struct HostScratch {
    uint32_t *dR = nullptr, *dS = nullptr;
    uint32_t capR = 0, capS = 0;
    rn_dpairs res{};
    void *stream = nullptr;  // cudaStream_t owned by the graph
};
}  // namespace rn

struct rn_graph {
    rn::DeviceGraph dev;
    rn::Workspace *ws = nullptr;
    rn::EngineConfig cfg;
    rn_graph_stats info{};
    std::vector<uint32_t> perm;  // host copy: original -> internal
    std::mutex mu;
    rn::HostScratch hs;
    rn::PointsState *points = nullptr;  // buffers of point queries, grown as needed
    rn::BoxState *box = nullptr;        // buffers of rectangle-restricted queries
    rn::HierState *hier = nullptr;      // buffers of the hierarchical variant
    std::vector<uint64_t> parts;        // the partition hierarchy: (first internal id << 32) | size
    uint32_t leaf_size = 512;
    int device = 0;
};
