// Host-side graph ingest: edge list -> cleaned CSR, and the recursive two-seed
// bisection of Section 3 (Algorithm 1, smoothed by Eq. 1-2) used to relabel nodes so
// that every partition of the hierarchy is a contiguous id range.  Source tiles of
// nearby R nodes then search overlapping neighbourhoods, and their slab rows and
// adjacency rows share cache lines.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <memory>
#include <queue>
#include <thread>

#include "rn_internal.h"

namespace rn {

[[noreturn]] void fail(rn_status s, const std::string &msg) { throw Error{s, msg}; }

HostGraph build_csr(uint32_t n, uint64_t m, const uint32_t *src, const uint32_t *dst,
                    const uint32_t *w, bool undirected) {
    if (n == 0) fail(RN_EINVAL, "graph has no nodes");
    for (uint64_t i = 0; i < m; i++) {
        if (src[i] >= n || dst[i] >= n)
            fail(RN_EINVAL, "edge " + std::to_string(i) + " has an endpoint >= n");
        if (w[i] < 1 || w[i] >= RN_WEIGHT_LIMIT)
            fail(RN_EINVAL, "edge " + std::to_string(i) + " has a weight outside [1, 2^24)");
    }
    // bucket arcs by tail (counting sort), self-loops dropped
    std::vector<uint64_t> off(static_cast<size_t>(n) + 1, 0);
    for (uint64_t i = 0; i < m; i++) {
        if (src[i] == dst[i]) continue;
        off[src[i] + 1]++;
        if (undirected) off[dst[i] + 1]++;
    }
    for (uint32_t x = 0; x < n; x++) off[x + 1] += off[x];
    const uint64_t total = off[n];
    std::vector<uint64_t> packed(total);  // (col << 32) | w, sorts as (col, w)
    std::vector<uint64_t> fillp(off.begin(), off.end() - 1);
    for (uint64_t i = 0; i < m; i++) {
        if (src[i] == dst[i]) continue;
        packed[fillp[src[i]]++] = (uint64_t(dst[i]) << 32) | w[i];
        if (undirected) packed[fillp[dst[i]]++] = (uint64_t(src[i]) << 32) | w[i];
    }
    // per row: sort by (col, w) and keep the first arc of each col (least weight)
    HostGraph g;
    g.n = n;
    g.row_ptr.assign(static_cast<size_t>(n) + 1, 0);
    g.col.reserve(total);
    g.w.reserve(total);
    for (uint32_t x = 0; x < n; x++) {
        uint64_t *b = packed.data() + off[x], *e = packed.data() + off[x + 1];
        std::sort(b, e);
        uint32_t last = 0xFFFFFFFFu;
        for (uint64_t *p = b; p < e; p++) {
            uint32_t c = uint32_t(*p >> 32);
            if (c == last) continue;
            last = c;
            g.col.push_back(c);
            g.w.push_back(uint32_t(*p & 0xFFFFFFFFu));
        }
        if (g.col.size() >= 0xFFFFFFFFull) fail(RN_EINVAL, "more than 2^32 - 1 arcs");
        g.row_ptr[x + 1] = uint32_t(g.col.size());
    }
    return g;
}

namespace {

// One recursive bisection job.  Parts are disjoint node sets, so the per-node arrays
// below are written by at most one job at a time.
struct Bisector {
    const HostGraph &g;
    uint32_t leaf;
    float alpha;
    // part label of each node; read across parts (a neighbour's label), so atomic
    std::unique_ptr<std::atomic<uint32_t>[]> label;
    std::vector<uint32_t> stamp;  // BFS visit stamps
    std::vector<uint8_t> side;    // 0 unassigned, 1 left cluster, 2 right cluster
    std::vector<uint32_t> order;  // output: internal id -> original id
    std::mutex leaves_mu;
    std::vector<uint32_t> leaves;  // output: first internal id of every leaf (any order)
    std::vector<uint64_t> parts;   // output: every part of the hierarchy, (first id << 32) | size
    std::atomic<uint32_t> next_label{1};
    std::atomic<uint32_t> next_stamp{1};

    Bisector(const HostGraph &g_, uint32_t leaf_, float alpha_)
        : g(g_), leaf(leaf_), alpha(alpha_), label(new std::atomic<uint32_t>[g_.n]),
          stamp(g_.n, 0), side(g_.n, 0), order(g_.n, 0) {
        for (uint32_t x = 0; x < g.n; x++) label[x].store(0, std::memory_order_relaxed);
    }

    // Breadth-first search inside the part from s; returns the visit order.
    void bfs(uint32_t s, uint32_t lbl, std::vector<uint32_t> &vis) {
        uint32_t st = next_stamp.fetch_add(1);
        vis.clear();
        vis.push_back(s);
        stamp[s] = st;
        for (size_t h = 0; h < vis.size(); h++) {
            uint32_t x = vis[h];
            for (uint32_t e = g.row_ptr[x]; e < g.row_ptr[x + 1]; e++) {
                uint32_t y = g.col[e];
                if (label[y].load(std::memory_order_relaxed) != lbl || stamp[y] == st) continue;
                stamp[y] = st;
                vis.push_back(y);
            }
        }
    }

    // Eq. (1)-(2): expand the left cluster when its smoothed top weight is not larger
    // than the right one's (ties go left).
    bool left_first(uint32_t w1, uint32_t w2, uint64_t v1, uint64_t v2) const {
        if (alpha == 0.0f) return w1 <= w2;
        long double a = alpha;
        long double l = (long double)w1 * v1 * (a * v1 + v2);
        long double r = (long double)w2 * v2 * (v1 + a * v2);
        return l <= r;
    }

    // Horizon edge: weight, discovery sequence number (equal weights are taken in the
    // order they were found, which keeps growth breadth-first among ties), head node.
    struct Arc {
        uint32_t w;
        uint64_t seq;
        uint32_t to;
        bool operator>(const Arc &o) const { return w != o.w ? w > o.w : seq > o.seq; }
    };
    using MinHeap = std::priority_queue<Arc, std::vector<Arc>, std::greater<Arc>>;

    void push_arcs(MinHeap &h, uint32_t x, uint32_t lbl, uint64_t &seq) {
        for (uint32_t e = g.row_ptr[x]; e < g.row_ptr[x + 1]; e++) {
            uint32_t y = g.col[e];
            if (label[y].load(std::memory_order_relaxed) == lbl && side[y] == 0) h.push(Arc{g.w[e], seq++, y});
        }
    }

    // Algorithm 1 on a connected part: grow a left cluster from a and a right cluster
    // from b, each step taking the cluster whose horizon holds the lighter edge.
    void grow(const std::vector<uint32_t> &part, uint32_t lbl, uint32_t a, uint32_t b,
              std::vector<uint32_t> &L, std::vector<uint32_t> &R) {
        for (uint32_t x : part) side[x] = 0;
        MinHeap hl, hr;
        uint64_t seq = 0;
        side[a] = 1;
        side[b] = 2;
        L.push_back(a);
        R.push_back(b);
        push_arcs(hl, a, lbl, seq);
        push_arcs(hr, b, lbl, seq);
        while (!hl.empty() || !hr.empty()) {
            bool go_left = hr.empty() ||
                           (!hl.empty() && left_first(hl.top().w, hr.top().w, L.size(), R.size()));
            MinHeap &h = go_left ? hl : hr;
            Arc t = h.top();
            h.pop();
            if (side[t.to] != 0) continue;  // already in a cluster
            side[t.to] = go_left ? 1 : 2;
            (go_left ? L : R).push_back(t.to);
            push_arcs(h, t.to, lbl, seq);
        }
    }

    void run(std::vector<uint32_t> part, uint32_t lbl, uint32_t out_begin, int depth) {
        if (!part.empty()) {
            std::lock_guard<std::mutex> lk(leaves_mu);
            parts.push_back((uint64_t(out_begin) << 32) | part.size());
        }
        if (part.size() <= leaf) {
            // a leaf keeps the order its nodes joined their cluster in (growth from the seed,
            // lightest horizon edge first): neighbours get near ids, so a search ball is a
            // few runs of consecutive ids (spread evenly by the maps' multiplicative hash,
            // and read from neighbouring CSR rows)
            std::copy(part.begin(), part.end(), order.begin() + out_begin);
            if (!part.empty()) {
                std::lock_guard<std::mutex> lk(leaves_mu);
                leaves.push_back(out_begin);
            }
            return;
        }
        std::vector<uint32_t> vis;
        vis.reserve(part.size());
        bfs(part[0], lbl, vis);
        std::vector<uint32_t> L, R;
        if (vis.size() < part.size()) {
            // Disconnected part (Algorithm 1 would leave the other components
            // unassigned): keep components whole and balance the two sides by size.
            std::vector<std::vector<uint32_t>> comps;
            uint32_t st_done = next_stamp.fetch_add(1);
            std::vector<uint32_t> seen;
            for (uint32_t x : part) {
                if (stamp[x] == st_done) continue;
                bfs(x, lbl, seen);  // symmetric graph: the component of x, disjoint from earlier ones
                for (uint32_t y : seen) stamp[y] = st_done;
                comps.push_back(seen);
            }
            std::stable_sort(comps.begin(), comps.end(),
                             [](const auto &p, const auto &q) { return p.size() > q.size(); });
            for (auto &c : comps) {
                std::vector<uint32_t> &dst = L.size() <= R.size() ? L : R;
                dst.insert(dst.end(), c.begin(), c.end());
            }
        } else {
            // seeds: double sweep (farthest in hops from part[0], then farthest from that)
            uint32_t a = vis.back();
            bfs(a, lbl, vis);
            uint32_t b = vis.back();
            L.reserve(part.size());
            R.reserve(part.size());
            grow(part, lbl, a, b, L, R);
        }
        part.clear();
        part.shrink_to_fit();
        uint32_t ll = next_label.fetch_add(1), rl = next_label.fetch_add(1);
        for (uint32_t x : L) label[x].store(ll, std::memory_order_relaxed);
        for (uint32_t x : R) label[x].store(rl, std::memory_order_relaxed);
        uint32_t r_begin = out_begin + uint32_t(L.size());
        if (depth < 6 && L.size() + R.size() > 20000) {
            std::thread t([this, L = std::move(L), ll, out_begin, depth]() mutable {
                run(std::move(L), ll, out_begin, depth + 1);
            });
            run(std::move(R), rl, r_begin, depth + 1);
            t.join();
        } else {
            run(std::move(L), ll, out_begin, depth + 1);
            run(std::move(R), rl, r_begin, depth + 1);
        }
    }
};

}  // namespace

std::vector<uint32_t> bisection_order(const HostGraph &g0, uint32_t leaf_size, float alpha, bool symmetric,
                                      std::vector<uint32_t> *leaf_starts, std::vector<uint64_t> *parts) {
    if (alpha < 0.0f || alpha > 1.0f) fail(RN_EINVAL, "alpha must lie in [0, 1]");
    // The partitioning looks at proximity only, so a directed graph is bisected through
    // its symmetrised form (every arc both ways, least weight kept).
    HostGraph sym;
    if (!symmetric) {
        std::vector<uint32_t> src, dst;
        src.reserve(g0.arcs());
        dst.reserve(g0.arcs());
        for (uint32_t x = 0; x < g0.n; x++)
            for (uint32_t e = g0.row_ptr[x]; e < g0.row_ptr[x + 1]; e++) {
                src.push_back(x);
                dst.push_back(g0.col[e]);
            }
        sym = build_csr(g0.n, src.size(), src.data(), dst.data(), g0.w.data(), true);
    }
    const HostGraph &g = symmetric ? g0 : sym;
    Bisector b(g, std::max<uint32_t>(leaf_size, 2), alpha);
    std::vector<uint32_t> all(g.n);
    for (uint32_t x = 0; x < g.n; x++) all[x] = x;
    b.run(std::move(all), 0, 0, 0);
    if (leaf_starts) {
        *leaf_starts = std::move(b.leaves);
        std::sort(leaf_starts->begin(), leaf_starts->end());
    }
    if (parts) {
        *parts = std::move(b.parts);
        std::sort(parts->begin(), parts->end());
    }
    return std::move(b.order);
}

HostGraph relabel(const HostGraph &g, const std::vector<uint32_t> &order) {
    std::vector<uint32_t> perm(g.n);
    for (uint32_t i = 0; i < g.n; i++) perm[order[i]] = i;
    HostGraph h;
    h.n = g.n;
    h.row_ptr.assign(static_cast<size_t>(g.n) + 1, 0);
    h.col.resize(g.arcs());
    h.w.resize(g.arcs());
    std::vector<uint64_t> tmp;
    uint32_t pos = 0;
    for (uint32_t i = 0; i < g.n; i++) {
        uint32_t x = order[i];
        tmp.clear();
        for (uint32_t e = g.row_ptr[x]; e < g.row_ptr[x + 1]; e++)
            tmp.push_back((uint64_t(perm[g.col[e]]) << 32) | g.w[e]);
        std::sort(tmp.begin(), tmp.end());
        for (uint64_t v : tmp) {
            h.col[pos] = uint32_t(v >> 32);
            h.w[pos] = uint32_t(v & 0xFFFFFFFFu);
            pos++;
        }
        h.row_ptr[i + 1] = pos;
    }
    return h;
}

}  // namespace rn
