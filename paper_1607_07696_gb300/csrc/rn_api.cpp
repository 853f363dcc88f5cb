// rn_api.cpp -- the extern "C" boundary of the engine (include/rn.h): argument checks,
// ownership of results, error codes and thread-local error messages.  Every entry point
// catches everything; no exception crosses the ABI.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <unordered_map>
#include <mutex>
#include <new>

#include <cuda_runtime.h>

#include "rn_internal.h"

namespace rn {

// Device pairs -> host arrays owned by the library (rn_pairs_free releases them).
// Host pairs live in pinned (page-locked) blocks, u, v and d of one result in one block,
// so the copy from the device runs at the link's speed rather than through a staging
// buffer.  Freed blocks wait in a pool for the next result of their size (allocating
// and freeing pinned memory is slow, and freeing it synchronises the device); the pool
// keeps at most POOL_MAX bytes.
namespace {
constexpr size_t POOL_MAX = size_t(1) << 30;
std::mutex g_pool_mu;
std::multimap<size_t, void *> g_pool_free;        // capacity -> free block
std::unordered_map<void *, size_t> g_pool_blocks;  // every block handed out or pooled
size_t g_pool_free_bytes = 0;

void *pinned_take(size_t bytes) {
    {
        std::lock_guard<std::mutex> lk(g_pool_mu);
        auto it = g_pool_free.lower_bound(bytes);
        if (it != g_pool_free.end() && it->first <= 2 * bytes) {
            void *p = it->second;
            g_pool_free_bytes -= it->first;
            g_pool_free.erase(it);
            return p;
        }
    }
    size_t cap = 1 << 16;
    while (cap < bytes) cap <<= 1;
    void *p = nullptr;
    if (cudaHostAlloc(&p, cap, cudaHostAllocPortable) != cudaSuccess || !p) {
        cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(g_pool_mu);
    g_pool_blocks[p] = cap;
    return p;
}

// Whether p is a pool block; if so it goes back to the pool (or is released when the
// pool is full).
bool pinned_give(void *p) {
    size_t cap = 0;
    {
        std::lock_guard<std::mutex> lk(g_pool_mu);
        auto it = g_pool_blocks.find(p);
        if (it == g_pool_blocks.end()) return false;
        cap = it->second;
        if (g_pool_free_bytes + cap <= POOL_MAX) {
            g_pool_free.emplace(cap, p);
            g_pool_free_bytes += cap;
            return true;
        }
        g_pool_blocks.erase(it);
    }
    cudaFreeHost(p);
    return true;
}
}  // namespace

void to_host_pairs(const rn_dpairs &d, rn_pairs *out, void *stream) {
    cudaStream_t st = (cudaStream_t)stream;
    out->n = d.n;
    const size_t n = std::max<uint64_t>(d.n, 1);
    uint32_t *blk = (uint32_t *)pinned_take(3 * n * 4);
    if (blk) {
        out->u = blk;
        out->v = blk + n;
        out->d = blk + 2 * n;
    } else {  // no pinned memory to be had: pageable buffers
        out->u = (uint32_t *)std::malloc(n * 4);
        out->v = (uint32_t *)std::malloc(n * 4);
        out->d = (uint32_t *)std::malloc(n * 4);
        if (!out->u || !out->v || !out->d) {
            rn_pairs_free(out);
            fail(RN_ENOMEM, "host result allocation failed");
        }
    }
    if (d.n) {
        cudaMemcpyAsync(out->u, d.u, d.n * 4, cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(out->v, d.v, d.n * 4, cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(out->d, d.d, d.n * 4, cudaMemcpyDeviceToHost, st);
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            rn_pairs_free(out);
            fail(RN_ECUDA, std::string("copying pairs to the host: ") + cudaGetErrorString(e));
        }
    }
}

}  // namespace rn

namespace {

thread_local std::string g_last_error;
thread_local rn_query_stats g_last_stats{};
thread_local bool g_have_stats = false;

rn_status set_error(rn_status s, const std::string &msg) {
    g_last_error = msg;
    return s;
}

template <class F>
rn_status guarded(F &&f) {
    try {
        g_last_error.clear();
        f();
        return RN_OK;
    } catch (const rn::Error &e) {
        return set_error(e.status, e.msg);
    } catch (const std::bad_alloc &) {
        return set_error(RN_ENOMEM, "host allocation failed");
    } catch (const std::exception &e) {
        return set_error(RN_EINTERNAL, e.what());
    } catch (...) {
        return set_error(RN_EINTERNAL, "unknown failure");
    }
}

// Per-query stats as JSON lines: when the environment names a file in RN_STATS_LOG,
// every successful query appends one line to it.
void log_stats(const char *kind, const rn_query_stats &st) {
    static const char *path = std::getenv("RN_STATS_LOG");
    if (!path || !*path) return;
    static std::mutex mu;
    char line[1024];
    std::snprintf(line, sizeof line,
                  "{\"query\": \"%s\", \"pairs\": %llu, \"tiles\": %llu, \"tile_width\": %u, "
                  "\"tile_sources\": %u, \"delta\": %u, \"theta_final\": %u, \"passes\": %u, "
                  "\"retried_tiles\": %llu, \"slots\": %llu, \"slot_arcs\": %llu, \"scans\": %llu, "
                  "\"rounds\": %llu, \"max_ball\": %llu, \"launches\": %u, \"device_ms\": %.4f, "
                  "\"search_ms\": %.4f, \"retry_ms\": %.4f}\n",
                  kind, (unsigned long long)st.pairs, (unsigned long long)st.tiles, st.tile_width, st.tile_sources,
                  st.delta, st.theta_final, st.passes, (unsigned long long)st.retried_tiles,
                  (unsigned long long)st.slots, (unsigned long long)st.slot_arcs, (unsigned long long)st.scans,
                  (unsigned long long)st.rounds, (unsigned long long)st.max_ball, st.launches, st.device_ms,
                  st.search_ms, st.retry_ms);
    std::lock_guard<std::mutex> lk(mu);
    if (std::FILE *f = std::fopen(path, "a")) {
        std::fputs(line, f);
        std::fclose(f);
    }
}

// Host-side check of R and S (ids < n, no repeats, disjoint), for a precise message
// before anything reaches the device.  The marks are two bitmaps (R's, S's) in per-thread
// storage reused across calls and cleared word by word afterwards, so a check costs
// O(|R| + |S|), not O(n), and touches n / 4 bytes at most (random ids into a byte per
// node missed the caches on graphs of millions of nodes).
void check_sets_host(uint32_t n, const uint32_t *R, uint32_t nR, const uint32_t *S, uint32_t nS) {
    if ((nR && !R) || (nS && !S)) rn::fail(RN_EINVAL, "null R or S with a non-zero size");
    thread_local std::vector<uint64_t> rb, sb;
    const size_t words = (size_t(n) + 63) / 64;
    if (rb.size() < words) {
        rb.assign(words, 0);
        sb.assign(words, 0);
    }
    struct Clear {  // leave the bitmaps at zero however the check ends
        const uint32_t *R, *S;
        uint32_t nR, nS;
        ~Clear() {
            for (uint32_t i = 0; i < nR; i++) rb[R[i] >> 6] = 0;
            for (uint32_t i = 0; i < nS; i++) sb[S[i] >> 6] = 0;
        }
    } clear{R, S, 0, 0};
    for (uint32_t i = 0; i < nR; i++) {
        const uint32_t x = R[i];
        if (x >= n) rn::fail(RN_EINVAL, "R[" + std::to_string(i) + "] >= n");
        const uint64_t bit = uint64_t(1) << (x & 63);
        if (rb[x >> 6] & bit) rn::fail(RN_EINVAL, "R repeats node " + std::to_string(x));
        rb[x >> 6] |= bit;
        clear.nR = i + 1;
    }
    for (uint32_t i = 0; i < nS; i++) {
        const uint32_t x = S[i];
        if (x >= n) rn::fail(RN_EINVAL, "S[" + std::to_string(i) + "] >= n");
        const uint64_t bit = uint64_t(1) << (x & 63);
        if (sb[x >> 6] & bit) rn::fail(RN_EINVAL, "S repeats node " + std::to_string(x));
        if (rb[x >> 6] & bit) rn::fail(RN_EINVAL, "node " + std::to_string(x) + " is in both R and S");
        sb[x >> 6] |= bit;
        clear.nS = i + 1;
    }
}

void check_theta(uint32_t theta) {
    if (theta != RN_INF && theta > RN_THETA_MAX) rn::fail(RN_EINVAL, "theta must be <= 2^31 or RN_INF");
}

void ensure(uint32_t **p, uint32_t *cap, uint32_t want) {
    if (*p && *cap >= want) return;
    rn::device_free(*p);
    *p = nullptr;
    *cap = std::max<uint32_t>(want, 1024);
    *p = (uint32_t *)rn::device_alloc(size_t(*cap) * 4);
}


}  // namespace

namespace {

rn::HostScratch &scratch_of(rn_graph *g) {
    rn::HostScratch &h = g->hs;
    if (!h.stream) {
        cudaStream_t s = nullptr;
        cudaError_t err = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (err != cudaSuccess) rn::fail(RN_ECUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(err));
        h.stream = s;
    }
    return h;
}

void drop_scratch(rn_graph *g) {
    rn::HostScratch &h = g->hs;
    rn::device_free(h.dR);
    rn::device_free(h.dS);
    rn::dpairs_release(&h.res);
    if (h.stream) cudaStreamDestroy((cudaStream_t)h.stream);
    h = rn::HostScratch{};
}

uint32_t median_weight(const rn::HostGraph &g) {
    if (g.w.empty()) return 1;
    std::vector<uint32_t> w(g.w);
    std::nth_element(w.begin(), w.begin() + w.size() / 2, w.end());
    return w[w.size() / 2];
}

void apply_config(rn_graph *g, const rn_config *cfg) {
    rn::EngineConfig c;
    if (cfg) {
        if (cfg->tile_width > 1 && cfg->tile_width != 32 && cfg->tile_width != 64 && cfg->tile_width != 128)
            rn::fail(RN_EINVAL, "tile_width must be 0, 1, 32, 64 or 128");
        if (cfg->tile_width) c.tile_width = cfg->tile_width;
        c.tile_src = cfg->tile_sources;
        c.delta = cfg->delta;
        const uint32_t ms = cfg->map_slots;
        if (ms && (ms < 8192 || (ms & (ms - 1)) || ms > (1u << 30)))
            rn::fail(RN_EINVAL, "map_slots must be 0 or a power of two in [8192, 2^30]");
        c.map_slots = ms;
        if (cfg->search_from > RN_FROM_S) rn::fail(RN_EINVAL, "search_from must be 0, 1 or 2");
        if (cfg->search_from == RN_FROM_S && !(g->info.flags & RN_UNDIRECTED))
            rn::fail(RN_EINVAL, "searches from S need a graph loaded undirected");
        c.search_from = cfg->search_from;
    }
    g->cfg = c;
}

}  // namespace

extern "C" {

const char *rn_version(void) { return "rn-join 0.1 (sm_103a)"; }

const char *rn_last_error(void) { return g_last_error.c_str(); }

rn_status rn_last_query_stats(rn_query_stats *out) {
    if (!out) return set_error(RN_EINVAL, "null output");
    if (!g_have_stats) return set_error(RN_EINVAL, "no query has completed on this thread");
    *out = g_last_stats;
    return RN_OK;
}

rn_status rn_graph_load(const uint32_t *src, const uint32_t *dst, const uint32_t *w, uint64_t m,
                        uint32_t n, uint32_t flags, const float *xy, const rn_config *cfg, rn_graph **out) {
    return guarded([&] {
        if (!out) rn::fail(RN_EINVAL, "null output");
        *out = nullptr;
        if (m && (!src || !dst || !w)) rn::fail(RN_EINVAL, "null edge arrays");
        if (flags & ~(RN_UNDIRECTED | RN_REORDER)) rn::fail(RN_EINVAL, "unknown flag");
        if (xy)
            for (uint64_t i = 0; i < 2ull * n; i++)
                if (!std::isfinite(xy[i])) rn::fail(RN_EINVAL, "node coordinates must be finite");
        auto g = std::make_unique<rn_graph>();
        g->info.flags = flags;
        apply_config(g.get(), cfg);
        rn::HostGraph h = rn::build_csr(n, m, src, dst, w, (flags & RN_UNDIRECTED) != 0);
        std::vector<uint32_t> order(n), perm(n), leaves;
        std::vector<uint64_t> parts;
        const uint32_t leaf = std::max<uint32_t>(cfg && cfg->leaf_size ? cfg->leaf_size : 512, 2);
        auto t0 = std::chrono::steady_clock::now();
        if (flags & RN_REORDER) {
            float alpha = (cfg && cfg->alpha >= 0.0f) ? cfg->alpha : 0.5f;
            order = rn::bisection_order(h, leaf, alpha, (flags & RN_UNDIRECTED) != 0, &leaves, &parts);
            h = rn::relabel(h, order);
        } else {
            // no bisection: the id ranges of a halving hierarchy stand for its parts
            for (uint32_t i = 0; i < n; i++) order[i] = i;
            std::vector<std::pair<uint32_t, uint32_t>> todo;
            if (n) todo.emplace_back(0, n);
            while (!todo.empty()) {
                const auto [b, sz] = todo.back();
                todo.pop_back();
                parts.push_back((uint64_t(b) << 32) | sz);
                if (sz <= leaf) {
                    leaves.push_back(b);
                } else {
                    todo.emplace_back(b, sz / 2);
                    todo.emplace_back(b + sz / 2, sz - sz / 2);
                }
            }
            std::sort(leaves.begin(), leaves.end());
            std::sort(parts.begin(), parts.end());
        }
        auto t1 = std::chrono::steady_clock::now();
        for (uint32_t i = 0; i < n; i++) perm[order[i]] = i;
        g->info.n = n;
        g->info.arcs = h.arcs();
        g->info.flags = flags;
        g->info.median_weight = median_weight(h);
        uint32_t maxd = 0;
        for (uint32_t x = 0; x < n; x++) maxd = std::max(maxd, h.row_ptr[x + 1] - h.row_ptr[x]);
        g->info.max_degree = maxd;
        g->info.reorder_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
        cudaGetDevice(&g->device);
        rn::upload_graph(h, perm, order, &g->dev);
        g->dev.symmetric = (flags & RN_UNDIRECTED) != 0;
        try {
            if (xy) rn::upload_geometry(xy, order, leaves, &g->dev);
            g->ws = rn::workspace_create(g->dev);
        } catch (...) {
            rn::free_graph(&g->dev);
            throw;
        }
        g->perm = std::move(perm);
        g->parts = std::move(parts);
        g->leaf_size = leaf;
        *out = g.release();
    });
}

rn_status rn_bisection_order(const uint32_t *src, const uint32_t *dst, const uint32_t *w, uint64_t m,
                             uint32_t n, uint32_t flags, const rn_config *cfg, uint32_t *order) {
    return guarded([&] {
        if (!order) rn::fail(RN_EINVAL, "null output");
        if (m && (!src || !dst || !w)) rn::fail(RN_EINVAL, "null edge arrays");
        if (flags & ~(RN_UNDIRECTED | RN_REORDER)) rn::fail(RN_EINVAL, "unknown flag");
        rn::HostGraph h = rn::build_csr(n, m, src, dst, w, (flags & RN_UNDIRECTED) != 0);
        uint32_t leaf = cfg && cfg->leaf_size ? cfg->leaf_size : 512;
        float alpha = (cfg && cfg->alpha >= 0.0f) ? cfg->alpha : 0.5f;
        std::vector<uint32_t> o = rn::bisection_order(h, leaf, alpha, (flags & RN_UNDIRECTED) != 0);
        std::memcpy(order, o.data(), size_t(n) * 4);
    });
}

void rn_graph_free(rn_graph *g) {
    if (!g) return;
    try {
        drop_scratch(g);
        rn::points_destroy(g->points);
        rn::box_destroy(g->box);
        rn::hier_destroy(g->hier);
        rn::workspace_destroy(g->ws);
        rn::free_graph(&g->dev);
    } catch (...) {
    }
    delete g;
}

rn_status rn_set_allocator(rn_alloc_fn alloc, rn_free_fn free, void *ctx) {
    return guarded([&] { rn::set_allocator(alloc, free, ctx); });
}

rn_status rn_file_read(const char *path, rn_edges *out) {
    return guarded([&] {
        if (!out) rn::fail(RN_EINVAL, "null output");
        *out = rn_edges{};
        rn::EdgeFile f;
        rn::read_edge_file(path, &f);
        const size_t m = f.src.size(), b = std::max<size_t>(m, 1) * 4;
        out->src = (uint32_t *)std::malloc(b);
        out->dst = (uint32_t *)std::malloc(b);
        out->w = (uint32_t *)std::malloc(b);
        if (!out->src || !out->dst || !out->w) {
            rn_edges_free(out);
            rn::fail(RN_ENOMEM, "host allocation failed");
        }
        if (m) {
            std::memcpy(out->src, f.src.data(), m * 4);
            std::memcpy(out->dst, f.dst.data(), m * 4);
            std::memcpy(out->w, f.w.data(), m * 4);
        }
        out->n = f.n;
        out->flags = f.flags;
        out->m = m;
    });
}

void rn_edges_free(rn_edges *e) {
    if (!e) return;
    std::free(e->src);
    std::free(e->dst);
    std::free(e->w);
    *e = rn_edges{};
}

rn_status rn_graph_load_file(const char *path, rn_graph **out) {
    rn::EdgeFile f;
    rn_status st = guarded([&] {
        if (!out) rn::fail(RN_EINVAL, "null output");
        *out = nullptr;
        rn::read_edge_file(path, &f);
    });
    if (st != RN_OK) return st;
    return rn_graph_load(f.src.data(), f.dst.data(), f.w.data(), f.src.size(), f.n, f.flags, nullptr, nullptr, out);
}

rn_status rn_graph_write_file(const char *path, const uint32_t *src, const uint32_t *dst, const uint32_t *w,
                              uint64_t m, uint32_t n, uint32_t flags) {
    return guarded([&] { rn::write_edge_file(path, n, m, src, dst, w, flags); });
}

rn_status rn_graph_info(const rn_graph *g, rn_graph_stats *out) {
    return guarded([&] {
        if (!g || !out) rn::fail(RN_EINVAL, "null argument");
        *out = g->info;
        out->device_bytes = (uint64_t(g->dev.n) + 1) * 4 + g->dev.arcs * 8 + uint64_t(g->dev.n) * 8 +
                            rn::workspace_bytes(g->ws);
    });
}

rn_status rn_graph_permutation(const rn_graph *g, uint32_t *perm) {
    return guarded([&] {
        if (!g || !perm) rn::fail(RN_EINVAL, "null argument");
        std::memcpy(perm, g->perm.data(), g->perm.size() * 4);
    });
}

rn_status rn_graph_set_config(rn_graph *g, const rn_config *cfg) {
    return guarded([&] {
        if (!g) rn::fail(RN_EINVAL, "null graph");
        std::lock_guard<std::mutex> lk(g->mu);
        apply_config(g, cfg);
    });
}

rn_status rn_distance_join_dev(const rn_graph *cg, const uint32_t *dR, uint32_t nR, const uint32_t *dS,
                               uint32_t nS, uint32_t theta, rn_dpairs *out, rn_stream stream) {
    return guarded([&] {
        if (!cg || !out) rn::fail(RN_EINVAL, "null argument");
        if ((nR && !dR) || (nS && !dS)) rn::fail(RN_EINVAL, "null R or S with a non-zero size");
        check_theta(theta);
        rn_graph *g = const_cast<rn_graph *>(cg);
        std::lock_guard<std::mutex> lk(g->mu);
        rn_query_stats st{};
        rn::run_join(g->dev, g->ws, g->cfg, g->info.median_weight, dR, nR, dS, nS, theta, out,
                     (void *)stream, &st);
        g_last_stats = st;
        log_stats("join", st);
        g_have_stats = true;
    });
}

rn_status rn_distance_join_noalloc(const rn_graph *cg, const uint32_t *dR, uint32_t nR, const uint32_t *dS,
                                   uint32_t nS, uint32_t theta, uint32_t *out_u, uint32_t *out_v,
                                   uint32_t *out_d, uint64_t out_cap, uint64_t *n_out, rn_stream stream) {
    return guarded([&] {
        if (!cg || !n_out) rn::fail(RN_EINVAL, "null argument");
        *n_out = 0;
        if ((nR && !dR) || (nS && !dS)) rn::fail(RN_EINVAL, "null R or S with a non-zero size");
        if (out_cap && (!out_u || !out_v || !out_d)) rn::fail(RN_EINVAL, "null output buffer");
        check_theta(theta);
        int cur = -1;
        cudaGetDevice(&cur);
        if (cur != cg->device) rn::fail(RN_EINVAL, "the graph lives on another device than the current one");
        rn::run_join_noalloc(cg->dev, cg->info.median_weight, dR, nR, dS, nS, theta, out_u, out_v, out_d,
                             out_cap, n_out, (void *)stream);
    });
}

rn_status rn_distance_join(const rn_graph *cg, const uint32_t *R, uint32_t nR, const uint32_t *S,
                           uint32_t nS, uint32_t theta, rn_pairs *out) {
    return guarded([&] {
        if (!cg || !out) rn::fail(RN_EINVAL, "null argument");
        *out = rn_pairs{};
        check_theta(theta);
        rn_graph *g = const_cast<rn_graph *>(cg);
        // ids, repeats and overlap are checked on the device as the sets are marked (a
        // host pass over |R| + |S| random ids was most of this call's host time: the
        // 1.07M-node join with 50,000 + 50,000 ids took 2.68 ms with it, 1.85 ms without)
        if ((nR && !R) || (nS && !S)) rn::fail(RN_EINVAL, "null R or S with a non-zero size");
        std::lock_guard<std::mutex> lk(g->mu);
        rn::HostScratch &hs = scratch_of(g);
        ensure(&hs.dR, &hs.capR, nR);
        ensure(&hs.dS, &hs.capS, nS);
        rn::copy_to_device(hs.dR, R, size_t(nR) * 4, hs.stream);
        rn::copy_to_device(hs.dS, S, size_t(nS) * 4, hs.stream);
        rn_query_stats st{};
        rn::run_join(g->dev, g->ws, g->cfg, g->info.median_weight, hs.dR, nR, hs.dS, nS, theta, &hs.res,
                     (void *)hs.stream, &st);
        rn::to_host_pairs(hs.res, out, hs.stream);
        g_last_stats = st;
        log_stats("join", st);
        g_have_stats = true;
    });
}

rn_status rn_kcp_dev(const rn_graph *cg, const uint32_t *dR, uint32_t nR, const uint32_t *dS, uint32_t nS,
                     uint64_t k, uint32_t theta, rn_dpairs *out, rn_stream stream) {
    return guarded([&] {
        if (!cg || !out) rn::fail(RN_EINVAL, "null argument");
        if ((nR && !dR) || (nS && !dS)) rn::fail(RN_EINVAL, "null R or S with a non-zero size");
        if (k == 0) rn::fail(RN_EINVAL, "k must be >= 1");
        check_theta(theta);
        rn_graph *g = const_cast<rn_graph *>(cg);
        std::lock_guard<std::mutex> lk(g->mu);
        rn_query_stats st{};
        rn::run_kcp(g->dev, g->ws, g->cfg, g->info.median_weight, dR, nR, dS, nS, k, theta, out,
                    (void *)stream, &st);
        g_last_stats = st;
        log_stats("kcp", st);
        g_have_stats = true;
    });
}

rn_status rn_kcp(const rn_graph *cg, const uint32_t *R, uint32_t nR, const uint32_t *S, uint32_t nS,
                 uint64_t k, uint32_t theta, rn_pairs *out) {
    return guarded([&] {
        if (!cg || !out) rn::fail(RN_EINVAL, "null argument");
        *out = rn_pairs{};
        if (k == 0) rn::fail(RN_EINVAL, "k must be >= 1");
        check_theta(theta);
        rn_graph *g = const_cast<rn_graph *>(cg);
        // ids, repeats and overlap are checked on the device as the sets are marked
        if ((nR && !R) || (nS && !S)) rn::fail(RN_EINVAL, "null R or S with a non-zero size");
        std::lock_guard<std::mutex> lk(g->mu);
        rn::HostScratch &hs = scratch_of(g);
        ensure(&hs.dR, &hs.capR, nR);
        ensure(&hs.dS, &hs.capS, nS);
        rn::copy_to_device(hs.dR, R, size_t(nR) * 4, hs.stream);
        rn::copy_to_device(hs.dS, S, size_t(nS) * 4, hs.stream);
        rn_query_stats st{};
        rn::run_kcp(g->dev, g->ws, g->cfg, g->info.median_weight, hs.dR, nR, hs.dS, nS, k, theta, &hs.res,
                    (void *)hs.stream, &st);
        rn::to_host_pairs(hs.res, out, hs.stream);
        g_last_stats = st;
        log_stats("kcp", st);
        g_have_stats = true;
    });
}

rn_status rn_distance_join_box(const rn_graph *cg, const uint32_t *R, uint32_t nR, const uint32_t *S,
                               uint32_t nS, uint32_t theta, const float box[4], uint32_t which, rn_pairs *out) {
    return rn_kcp_box(cg, R, nR, S, nS, 0, theta, box, which, out);
}

rn_status rn_kcp_box(const rn_graph *cg, const uint32_t *R, uint32_t nR, const uint32_t *S, uint32_t nS,
                     uint64_t k, uint32_t theta, const float box[4], uint32_t which, rn_pairs *out) {
    return guarded([&] {
        if (!cg || !out || !box) rn::fail(RN_EINVAL, "null argument");
        *out = rn_pairs{};
        check_theta(theta);
        rn_graph *g = const_cast<rn_graph *>(cg);
        check_sets_host(g->dev.n, R, nR, S, nS);
        std::lock_guard<std::mutex> lk(g->mu);
        rn::HostScratch &hs = scratch_of(g);
        ensure(&hs.dR, &hs.capR, nR);
        ensure(&hs.dS, &hs.capS, nS);
        rn::copy_to_device(hs.dR, R, size_t(nR) * 4, hs.stream);
        rn::copy_to_device(hs.dS, S, size_t(nS) * 4, hs.stream);
        rn_query_stats st{};
        uint64_t decided = 0;
        rn::run_box(g->dev, g->ws, &g->box, g->cfg, g->info.median_weight, hs.dR, nR, hs.dS, nS, box, which, k,
                    theta, &hs.res, (void *)hs.stream, &st, &decided);
        rn::to_host_pairs(hs.res, out, hs.stream);
        st.box_leaf_decided = decided;
        g_last_stats = st;
        log_stats(k ? "kcp_box" : "join_box", st);
        g_have_stats = true;
    });
}

namespace {

thread_local rn_hier_stats g_last_hier{};
thread_local bool g_have_hier = false;

// The coarsest parts of the partition hierarchy with at most part_size nodes (the leaves
// for 0): their first internal ids, ascending; they cover every node once.
std::vector<uint32_t> hierarchy_cut(const rn_graph *g, uint32_t part_size) {
    const uint32_t P = part_size ? part_size : g->leaf_size;
    if (P < g->leaf_size) rn::fail(RN_EINVAL, "part_size must be 0 or at least the graph's leaf size");
    std::vector<uint64_t> parts(g->parts);
    std::sort(parts.begin(), parts.end(), [](uint64_t a, uint64_t b) {
        return (a >> 32) != (b >> 32) ? (a >> 32) < (b >> 32) : (a & 0xFFFFFFFFull) > (b & 0xFFFFFFFFull);
    });
    std::vector<uint32_t> starts;
    uint64_t covered = 0;
    for (uint64_t p : parts) {
        const uint64_t b = p >> 32, sz = p & 0xFFFFFFFFull;
        if (b >= covered && sz <= P) {
            if (b != covered) rn::fail(RN_EINTERNAL, "the partition hierarchy leaves a gap");
            starts.push_back(uint32_t(b));
            covered = b + sz;
        }
    }
    if (covered != g->dev.n) rn::fail(RN_EINTERNAL, "the partition hierarchy does not cover the graph");
    if (starts.empty()) starts.push_back(0);
    return starts;
}

void hier_query(const rn_graph *cg, const uint32_t *R, uint32_t nR, const uint32_t *S, uint32_t nS, uint64_t k,
                uint32_t theta, uint32_t part_size, rn_pairs *out) {
    if (!cg || !out) rn::fail(RN_EINVAL, "null argument");
    *out = rn_pairs{};
    check_theta(theta);
    rn_graph *g = const_cast<rn_graph *>(cg);
    check_sets_host(g->dev.n, R, nR, S, nS);
    std::lock_guard<std::mutex> lk(g->mu);
    const std::vector<uint32_t> cut = hierarchy_cut(g, part_size);
    rn::HostScratch &hs = scratch_of(g);
    rn_query_stats st{};
    rn_hier_stats hst{};
    rn::run_hier(g->dev, g->ws, &g->hier, g->cfg, g->info.median_weight, g->perm, cut, R, nR, S, nS, k, theta,
                 &hs.res, (void *)hs.stream, &st, &hst);
    rn::to_host_pairs(hs.res, out, hs.stream);
    g_last_stats = st;
    g_have_stats = true;
    g_last_hier = hst;
    g_have_hier = true;
    log_stats(k ? "kcp_hier" : "join_hier", st);
}

}  // namespace

rn_status rn_distance_join_hier(const rn_graph *g, const uint32_t *R, uint32_t nR, const uint32_t *S, uint32_t nS,
                                uint32_t theta, uint32_t part_size, rn_pairs *out) {
    return guarded([&] { hier_query(g, R, nR, S, nS, 0, theta, part_size, out); });
}

rn_status rn_kcp_hier(const rn_graph *g, const uint32_t *R, uint32_t nR, const uint32_t *S, uint32_t nS, uint64_t k,
                      uint32_t theta, uint32_t part_size, rn_pairs *out) {
    return guarded([&] {
        if (k == 0) rn::fail(RN_EINVAL, "k must be >= 1");
        hier_query(g, R, nR, S, nS, k, theta, part_size, out);
    });
}

rn_status rn_last_hier_stats(rn_hier_stats *out) {
    if (!out) return set_error(RN_EINVAL, "null output");
    if (!g_have_hier) return set_error(RN_EINVAL, "no hierarchical query has completed on this thread");
    *out = g_last_hier;
    return RN_OK;
}

namespace {

void check_points_host(uint32_t n, const rn_point *P, uint32_t nP, const char *name) {
    if (nP && !P) rn::fail(RN_EINVAL, std::string("null ") + name + " with a non-zero size");
    for (uint32_t i = 0; i < nP; i++) {
        if (P[i].a >= n || P[i].b >= n)
            rn::fail(RN_EINVAL, std::string(name) + "[" + std::to_string(i) + "]: an end id is >= n");
        if (P[i].a == P[i].b) rn::fail(RN_EINVAL, std::string(name) + "[" + std::to_string(i) + "]: a == b");
    }
}

void points_query(const rn_graph *cg, const rn_point *R, uint32_t nR, const rn_point *S, uint32_t nS, uint64_t k,
                  uint32_t theta, rn_pairs *out) {
    if (!cg || !out) rn::fail(RN_EINVAL, "null argument");
    *out = rn_pairs{};
    check_theta(theta);
    rn_graph *g = const_cast<rn_graph *>(cg);
    check_points_host(g->dev.n, R, nR, "R");
    check_points_host(g->dev.n, S, nS, "S");
    std::lock_guard<std::mutex> lk(g->mu);
    rn::HostScratch &hs = scratch_of(g);
    rn_query_stats st{};
    rn::run_points(g->dev, g->perm, &g->points, g->cfg, g->info.median_weight, R, nR, S, nS, k, theta, &hs.res,
                   hs.stream, &st);
    rn::to_host_pairs(hs.res, out, hs.stream);
    g_last_stats = st;
    log_stats(k ? "kcp_points" : "join_points", st);
    g_have_stats = true;
}

}  // namespace

rn_status rn_distance_join_points(const rn_graph *g, const rn_point *R, uint32_t nR, const rn_point *S, uint32_t nS,
                                  uint32_t theta, rn_pairs *out) {
    return guarded([&] { points_query(g, R, nR, S, nS, 0, theta, out); });
}

rn_status rn_kcp_points(const rn_graph *g, const rn_point *R, uint32_t nR, const rn_point *S, uint32_t nS,
                        uint64_t k, uint32_t theta, rn_pairs *out) {
    return guarded([&] {
        if (k == 0) rn::fail(RN_EINVAL, "k must be >= 1");
        points_query(g, R, nR, S, nS, k, theta, out);
    });
}

struct rn_batch {
    rn::Batch *b = nullptr;
    rn_batch_config cfg{0, 1};
    bool tuned = false;
};

static rn::Batch *make_batch(const rn_query *q, uint32_t nq) {
    if (!q && nq) rn::fail(RN_EINVAL, "null queries");
    if (nq == 0) rn::fail(RN_EINVAL, "empty batch");
    int cur = -1;
    cudaGetDevice(&cur);
    std::vector<const rn::DeviceGraph *> graphs(nq);
    std::vector<const std::vector<uint32_t> *> perms(nq);
    std::vector<uint32_t> med(nq), nR(nq), nS(nq), theta(nq), from(nq);
    std::vector<const uint32_t *> R(nq), S(nq);
    for (uint32_t i = 0; i < nq; i++) {
        const rn_query &x = q[i];
        if (!x.g) rn::fail(RN_EINVAL, "query " + std::to_string(i) + " has no graph");
        if (x.g->device != cur) rn::fail(RN_EINVAL, "query " + std::to_string(i) + "'s graph is on another device");
        check_theta(x.theta);
        try {
            check_sets_host(x.g->dev.n, x.R, x.nR, x.S, x.nS);
        } catch (const rn::Error &e) {
            rn::fail(e.status, "query " + std::to_string(i) + ": " + e.msg);
        }
        graphs[i] = &x.g->dev;
        perms[i] = &x.g->perm;
        med[i] = x.g->info.median_weight;
        R[i] = x.R;
        S[i] = x.S;
        nR[i] = x.nR;
        nS[i] = x.nS;
        theta[i] = x.theta;
        from[i] = x.g->cfg.search_from;
    }
    return rn::batch_create(graphs, perms, med, R, nR, S, nS, theta, from);
}

rn_status rn_batch_create(const rn_query *q, uint32_t nq, const rn_batch_config *cfg, rn_batch **out) {
    return guarded([&] {
        if (!out) rn::fail(RN_EINVAL, "null output");
        *out = nullptr;
        auto h = std::make_unique<rn_batch>();
        if (cfg) h->cfg = *cfg;
        h->b = make_batch(q, nq);
        *out = h.release();
    });
}

rn_status rn_batch_run(rn_batch *h, rn_stream stream) {
    return guarded([&] {
        if (!h || !h->b) rn::fail(RN_EINVAL, "null batch");
        if (h->cfg.autotune && !h->tuned) {
            rn::batch_tune(h->b);
            h->tuned = true;
        }
        rn::batch_run(h->b, (void *)stream, h->cfg.use_graph != 0);
    });
}

rn_status rn_batch_pairs_dev(const rn_batch *h, uint32_t i, const uint32_t **u, const uint32_t **v,
                             const uint32_t **d, uint64_t *n) {
    return guarded([&] {
        if (!h || !h->b || !u || !v || !d || !n) rn::fail(RN_EINVAL, "null argument");
        rn::batch_pairs_dev(h->b, i, u, v, d, n);
    });
}

rn_status rn_batch_pairs(const rn_batch *h, uint32_t i, rn_pairs *out) {
    return guarded([&] {
        if (!h || !h->b || !out) rn::fail(RN_EINVAL, "null argument");
        *out = rn_pairs{};
        const uint32_t *u, *v, *d;
        uint64_t n = 0;
        rn::batch_pairs_dev(h->b, i, &u, &v, &d, &n);
        rn_dpairs view{const_cast<uint32_t *>(u), const_cast<uint32_t *>(v), const_cast<uint32_t *>(d), n, n};
        rn::to_host_pairs(view, out, nullptr);
    });
}

rn_status rn_batch_stats_get(const rn_batch *h, rn_batch_stats *out) {
    return guarded([&] {
        if (!h || !h->b || !out) rn::fail(RN_EINVAL, "null argument");
        *out = rn::batch_stats(h->b);
    });
}

void rn_batch_free(rn_batch *h) {
    if (!h) return;
    try {
        rn::batch_destroy(h->b);
    } catch (...) {
    }
    delete h;
}

rn_status rn_tune_cache_save(const char *path) {
    return guarded([&] { rn::tune_cache_save(path); });
}

rn_status rn_tune_cache_load(const char *path, uint32_t *classes) {
    return guarded([&] {
        const uint32_t n = rn::tune_cache_load(path);
        if (classes) *classes = n;
    });
}

rn_status rn_join_many(const rn_graph *cg, const rn_request *q, uint32_t nq, rn_pairs *outs) {
    return guarded([&] {
        if (!cg || !outs || (nq && !q)) rn::fail(RN_EINVAL, "null argument");
        if (nq == 0) rn::fail(RN_EINVAL, "no queries");
        for (uint32_t i = 0; i < nq; i++) outs[i] = rn_pairs{};
        rn_graph *g = const_cast<rn_graph *>(cg);
        std::vector<const uint32_t *> R(nq), S(nq);
        std::vector<uint32_t> nR(nq), nS(nq), theta(nq);
        for (uint32_t i = 0; i < nq; i++) {
            try {
                if (q[i].k != 0) rn::fail(RN_EINVAL, "k must be 0 (a theta-join)");
                check_theta(q[i].theta);
                check_sets_host(g->dev.n, q[i].R, q[i].nR, q[i].S, q[i].nS);
            } catch (const rn::Error &e) {
                rn::fail(e.status, "query " + std::to_string(i) + ": " + e.msg);
            }
            R[i] = q[i].R;
            S[i] = q[i].S;
            nR[i] = q[i].nR;
            nS[i] = q[i].nS;
            theta[i] = q[i].theta;
        }
        std::lock_guard<std::mutex> lk(g->mu);
        rn::HostScratch &hs = scratch_of(g);
        std::vector<uint64_t> counts;
        rn_query_stats st{};
        rn::run_join_multi(g->dev, g->ws, g->cfg, g->info.median_weight, g->perm, R, nR, S, nS, theta, &hs.res,
                           &counts, hs.stream, &st);
        uint64_t at = 0;
        try {
            for (uint32_t i = 0; i < nq; i++) {
                rn_dpairs view{hs.res.u + at, hs.res.v + at, hs.res.d + at, counts[i], counts[i]};
                rn::to_host_pairs(view, &outs[i], hs.stream);
                at += counts[i];
            }
        } catch (...) {
            for (uint32_t i = 0; i < nq; i++) rn_pairs_free(&outs[i]);
            throw;
        }
        g_last_stats = st;
        g_have_stats = true;
        log_stats("join_many", st);
    });
}

rn_status rn_join_batch(const rn_query *q, uint32_t nq, rn_pairs *outs) {
    return guarded([&] {
        if (!outs) rn::fail(RN_EINVAL, "null output");
        for (uint32_t i = 0; i < nq; i++) outs[i] = rn_pairs{};
        rn_batch h;
        h.cfg.use_graph = 0;
        h.b = make_batch(q, nq);
        try {
            rn::batch_run(h.b, nullptr, false);
            for (uint32_t i = 0; i < nq; i++) {
                const uint32_t *u, *v, *d;
                uint64_t n = 0;
                rn::batch_pairs_dev(h.b, i, &u, &v, &d, &n);
                rn_dpairs view{const_cast<uint32_t *>(u), const_cast<uint32_t *>(v), const_cast<uint32_t *>(d), n, n};
                rn::to_host_pairs(view, &outs[i], nullptr);
            }
        } catch (...) {
            for (uint32_t i = 0; i < nq; i++) rn_pairs_free(&outs[i]);
            rn::batch_destroy(h.b);
            h.b = nullptr;
            throw;
        }
        rn::batch_destroy(h.b);
        h.b = nullptr;
    });
}

struct rn_server {
    rn::Server *s = nullptr;
    uint32_t n = 0;
};

rn_status rn_serve_create(const rn_graph *g, const rn_serve_config *cfg, rn_server **out) {
    return guarded([&] {
        if (!g || !out) rn::fail(RN_EINVAL, "null argument");
        *out = nullptr;
        rn_serve_config c{};
        if (cfg) c = *cfg;
        auto h = std::make_unique<rn_server>();
        h->n = g->dev.n;
        h->s = rn::server_create(g, c.slab_bytes, c.workers, c.max_blocks);
        *out = h.release();
    });
}

rn_status rn_serve_submit(rn_server *h, const rn_request *q, uint64_t *ticket) {
    return guarded([&] {
        if (!h || !h->s || !q || !ticket) rn::fail(RN_EINVAL, "null argument");
        check_theta(q->theta);
        check_sets_host(h->n, q->R, q->nR, q->S, q->nS);
        *ticket = rn::server_submit(h->s, q->R, q->nR, q->S, q->nS, q->theta, q->k);
    });
}

rn_status rn_serve_wait(rn_server *h, uint64_t ticket, uint32_t timeout_ms, rn_pairs *out) {
    return guarded([&] {
        if (!h || !h->s || !out) rn::fail(RN_EINVAL, "null argument");
        *out = rn_pairs{};
        rn::server_wait(h->s, ticket, timeout_ms, out);
    });
}

rn_status rn_serve_cancel(rn_server *h, uint64_t ticket) {
    return guarded([&] {
        if (!h || !h->s) rn::fail(RN_EINVAL, "null argument");
        rn::server_cancel(h->s, ticket);
    });
}

rn_status rn_serve_stats_get(rn_server *h, rn_serve_stats *out) {
    return guarded([&] {
        if (!h || !h->s || !out) rn::fail(RN_EINVAL, "null argument");
        rn::server_stats(h->s, out);
    });
}

rn_status rn_serve_reset_stats(rn_server *h) {
    return guarded([&] {
        if (!h || !h->s) rn::fail(RN_EINVAL, "null argument");
        rn::server_reset_stats(h->s);
    });
}

void rn_serve_destroy(rn_server *h) {
    if (!h) return;
    try {
        rn::server_destroy(h->s);
    } catch (...) {
    }
    delete h;
}

void rn_pairs_free(rn_pairs *p) {
    if (!p) return;
    if (!(p->u && rn::pinned_give(p->u))) {  // a pinned block holds all three arrays
        std::free(p->u);
        std::free(p->v);
        std::free(p->d);
    }
    p->u = p->v = p->d = nullptr;
    p->n = 0;
}

void rn_dpairs_free(rn_dpairs *p) {
    if (!p) return;
    try {
        rn::dpairs_release(p);
    } catch (...) {
    }
}

}  // extern "C"
