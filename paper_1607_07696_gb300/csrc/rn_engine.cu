// rn_engine.cu -- the GPU engine of the theta-bounded many-source road-network join
// and its k-closest-pairs variant (Tsatsanifos 2016: Abstract, Section 4).
//
// The paper runs one best-first search from every u in R and keeps the S nodes it
// reaches within theta (Section 4, local processing).  Here those searches run a tile
// of T sources at a time (T = 32, 64 or 128) in one thread block:
//
//   * a hash map in shared memory assigns every node the tile reaches a slot;
//   * slot h owns row h of a distance slab in global memory (L2-resident), T uint32
//     lanes wide -- lane t is the tentative distance from source t -- so a warp reads
//     or relaxes a whole row with one coalesced 128*T/32-byte access;
//   * the rows are relaxed by delta-stepping: a near queue in shared memory holds the
//     slots whose smallest improved lane lies in the current bucket, and the bucket
//     advances when the queue drains; a slot's arcs are relaxed for all T lanes at
//     once with fire-and-forget atomicMin;
//   * a relaxation is dropped when its cost is greater than the bound (theta, or the
//     k-closest-pairs radius), so costs equal to the bound are kept (Algorithm 4);
//   * when the tile's search ends, every slot whose node is in S emits the lanes within
//     the bound as (u, v, d) through a warp ballot and a block prefix sum, with one
//     global atomicAdd per block;
//   * pairs are put in canonical order by an LSD radix sort.
//
// All arithmetic is on unsigned integers: distances are at most 2^31 and weights are
// below 2^24, so d + w never wraps, and the result is exact.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <unordered_map>

#include "rn_internal.h"

namespace rn {

#define RN_CUDA(x)                                                                        \
    do {                                                                                  \
        cudaError_t e_ = (x);                                                             \
        if (e_ != cudaSuccess) {                                                          \
            cudaGetLastError();                                                           \
            fail(e_ == cudaErrorMemoryAllocation ? RN_ENOMEM : RN_ECUDA,                  \
                 std::string(#x) + ": " + cudaGetErrorString(e_));                        \
        }                                                                                 \
    } while (0)

constexpr uint32_t INF = 0xFFFFFFFFu;
constexpr uint32_t EMPTY = 0xFFFFFFFFu;
constexpr unsigned FULL = 0xFFFFFFFFu;

// ------------------------------------------------------------------ memory ----

// Device memory comes from cudaMalloc, or from the caller's allocator when one is set
// (rn_set_allocator).  Every block made through a hook remembers that hook, so it goes
// back to the allocator that made it even if the hook changes later.  The library frees
// a block only when none of its work still uses it.
namespace {
struct Hook {
    rn_alloc_fn alloc = nullptr;
    rn_free_fn free = nullptr;
    void *ctx = nullptr;
};
std::mutex g_alloc_mu;
Hook g_hook;
std::unordered_map<void *, Hook> g_hooked;
}  // namespace

void set_allocator(rn_alloc_fn alloc, rn_free_fn free, void *ctx) {
    if (!alloc != !free) fail(RN_EINVAL, "give both allocator functions, or neither");
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_hook = Hook{alloc, free, ctx};
}

void *device_alloc(size_t bytes) {
    Hook h;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        h = g_hook;
    }
    if (!bytes) bytes = 16;
    if (!h.alloc) {
        void *p = nullptr;
        RN_CUDA(cudaMalloc(&p, bytes));
        return p;
    }
    void *p = h.alloc(bytes, h.ctx);
    if (!p) fail(RN_ENOMEM, "the allocator hook returned no memory for " + std::to_string(bytes) + " bytes");
    if (reinterpret_cast<uintptr_t>(p) % 256) {
        h.free(p, h.ctx);
        fail(RN_EINVAL, "the allocator hook returned memory not aligned to 256 bytes");
    }
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_hooked[p] = h;
    return p;
}

void device_free(void *p) {
    if (!p) return;
    Hook h;
    bool hooked = false;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        auto it = g_hooked.find(p);
        if (it != g_hooked.end()) {
            h = it->second;
            hooked = true;
            g_hooked.erase(it);
        }
    }
    if (hooked) h.free(p, h.ctx);
    else cudaFree(p);
}

void copy_to_host(void *dst, const void *src, size_t bytes, void *stream) {
    if (!bytes) return;
    RN_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    RN_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
}

void copy_to_device(void *dst, const void *src, size_t bytes, void *stream) {
    if (!bytes) return;
    RN_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, (cudaStream_t)stream));
}

void stream_sync(void *stream) { RN_CUDA(cudaStreamSynchronize((cudaStream_t)stream)); }

void dpairs_reserve(rn_dpairs *p, uint64_t cap) {
    if (p->u && p->cap >= cap) return;
    dpairs_release(p);
    cap = std::max<uint64_t>(cap, 1024);
    p->u = (uint32_t *)device_alloc(cap * 4);
    p->v = (uint32_t *)device_alloc(cap * 4);
    p->d = (uint32_t *)device_alloc(cap * 4);
    p->cap = cap;
}

void dpairs_release(rn_dpairs *p) {
    device_free(p->u);
    device_free(p->v);
    device_free(p->d);
    p->u = p->v = p->d = nullptr;
    p->cap = 0;
    p->n = 0;
}

void upload_graph(const HostGraph &g, const std::vector<uint32_t> &perm,
                  const std::vector<uint32_t> &iperm, DeviceGraph *out) {
    DeviceGraph d;
    d.n = g.n;
    d.arcs = g.arcs();
    try {
        d.row_ptr = (uint32_t *)device_alloc((size_t(g.n) + 1) * 4);
        d.adj = (uint32_t *)device_alloc(std::max<size_t>(d.arcs, 1) * 8);
        d.perm = (uint32_t *)device_alloc(size_t(g.n) * 4);
        d.iperm = (uint32_t *)device_alloc(size_t(g.n) * 4);
        std::vector<uint32_t> adj(2 * d.arcs);
        for (uint64_t e = 0; e < d.arcs; e++) {
            adj[2 * e] = g.col[e];
            adj[2 * e + 1] = g.w[e];
        }
        RN_CUDA(cudaMemcpy(d.row_ptr, g.row_ptr.data(), (size_t(g.n) + 1) * 4, cudaMemcpyHostToDevice));
        if (d.arcs) RN_CUDA(cudaMemcpy(d.adj, adj.data(), d.arcs * 8, cudaMemcpyHostToDevice));
        RN_CUDA(cudaMemcpy(d.perm, perm.data(), size_t(g.n) * 4, cudaMemcpyHostToDevice));
        RN_CUDA(cudaMemcpy(d.iperm, iperm.data(), size_t(g.n) * 4, cudaMemcpyHostToDevice));
        // a copy from pageable memory may still be in flight when cudaMemcpy returns, and
        // queries run on streams that do not wait for the legacy stream
        RN_CUDA(cudaDeviceSynchronize());
    } catch (...) {
        free_graph(&d);
        throw;
    }
    *out = d;
}

void free_graph(DeviceGraph *g) {
    device_free(g->row_ptr);
    device_free(g->adj);
    device_free(g->perm);
    device_free(g->iperm);
    device_free(g->xy);
    device_free(g->leaf_start);
    device_free(g->leaf_box);
    *g = DeviceGraph{};
}

void upload_geometry(const float *xy, const std::vector<uint32_t> &order, const std::vector<uint32_t> &leaf_starts,
                     DeviceGraph *out) {
    const uint32_t n = out->n;
    std::vector<float2> pos(n);
    for (uint32_t i = 0; i < n; i++) pos[i] = make_float2(xy[2 * size_t(order[i])], xy[2 * size_t(order[i]) + 1]);
    std::vector<uint32_t> starts(leaf_starts);
    if (starts.empty() || starts[0] != 0) starts.insert(starts.begin(), 0);
    const uint32_t nl = n ? uint32_t(starts.size()) : 0;
    starts.push_back(n);
    std::vector<float4> box(std::max<uint32_t>(nl, 1));
    for (uint32_t l = 0; l < nl; l++) {
        float4 b = make_float4(INFINITY, INFINITY, -INFINITY, -INFINITY);
        for (uint32_t i = starts[l]; i < starts[l + 1]; i++) {
            b.x = std::min(b.x, pos[i].x);
            b.y = std::min(b.y, pos[i].y);
            b.z = std::max(b.z, pos[i].x);
            b.w = std::max(b.w, pos[i].y);
        }
        box[l] = b;
    }
    out->xy = (float2 *)device_alloc(std::max<size_t>(n, 1) * sizeof(float2));
    out->leaf_start = (uint32_t *)device_alloc(starts.size() * 4);
    out->leaf_box = (float4 *)device_alloc(box.size() * sizeof(float4));
    out->nleaves = nl;
    if (n) RN_CUDA(cudaMemcpy(out->xy, pos.data(), size_t(n) * sizeof(float2), cudaMemcpyHostToDevice));
    RN_CUDA(cudaMemcpy(out->leaf_start, starts.data(), starts.size() * 4, cudaMemcpyHostToDevice));
    RN_CUDA(cudaMemcpy(out->leaf_box, box.data(), box.size() * sizeof(float4), cudaMemcpyHostToDevice));
    RN_CUDA(cudaDeviceSynchronize());  // pageable copies done before any stream reads them
}

// ---------------------------------------------------------------- workspace ----

// Device-resident control block of one query.
struct Control {
    uint32_t err;          // 1: id >= n, 2: repeated id or R/S overlap
    uint32_t r_count;      // R nodes after validation
    uint32_t tile_next;    // work-queue head of the persistent search
    uint32_t n_failed;     // tiles whose slab overflowed
    unsigned long long pairs;
    unsigned long long scans;
    unsigned long long slots;      // sum over tiles of slab rows used
    unsigned long long slot_arcs;  // sum over tiles of arcs leaving the rows' nodes
    // phase counters of the search (thread 0 of every block): rounds, queue items of
    // all rounds, bucket boundaries, and SM cycles spent in rounds, boundaries, emission
    unsigned long long rounds, round_items, boundaries;
    unsigned long long cyc_round, cyc_bound, cyc_emit;
    unsigned long long cyc_stepA, round_arcs;
    unsigned long long dirty_groups;  // dirty lane-groups of the scanned items
    uint32_t max_fill;  // largest union ball (slots) of a completed tile
    uint32_t check[4];  // first failed device-side check: code, index, value
    unsigned long long slot_lanes;  // sum over tiles of slots times the tile's lanes
    uint32_t src_max_ball;          // largest ball of a source the warp search completed
    uint32_t max_seg;               // most pairs one source emitted in the warp search
};

// Record the first failed device-side check (the access it guarded is skipped).
__device__ __forceinline__ void record_check(Control *ctl, uint32_t code, uint32_t index, uint32_t value) {
    if (atomicCAS(&ctl->check[0], 0u, code) == 0u) {
        ctl->check[1] = index;
        ctl->check[2] = value;
    }
}

// Bounds checks of the debug build (-DRN_CHECKS): a failed check records the first bad
// index in the control block (the host reports RN_EINTERNAL) and the access it guards is
// skipped; in the normal build a check is the constant false and compiles away.
#ifdef RN_CHECKS
#define RN_BAD(cond, code, idx, val) (!(cond) && (record_check(a.ctl, (code), uint32_t(idx), uint32_t(val)), true))
#else
#define RN_BAD(cond, code, idx, val) false
#endif

// Two block shapes: NARROW blocks (512 threads, an 8192-slot shared map, two blocks per
// SM) search every tile first; WIDE blocks (1024 threads, a 16384-slot map, one block
// per SM) search again the tiles whose union ball overflowed, and run the global-map
// retries.  A block of THREADS threads keeps two near queues of 2 THREADS entries and
// stages 0.75 THREADS queue items per round step.
constexpr int NARROW = 512, WIDE = 1024;
constexpr uint32_t SMEM_H = 8192;      // slots of the narrow block's map
constexpr uint32_t SMEM_HW = 16384;    // slots of the wide block's map
constexpr int CTAS_PER_SM = 2;         // narrow blocks resident per SM
__host__ __device__ constexpr uint32_t qcap_of(int threads) { return 2u * threads; }
__host__ __device__ constexpr uint32_t icap_of(int threads) { return 3u * threads / 4; }

// Per device: the slab of the persistent search (one region of SMEM_H rows of the widest
// tile per resident narrow block) and the buffer of the global-map retries.  Every graph
// on the device shares them, so queries on one device run one at a time (mu).
struct DeviceShared {
    std::mutex mu;
    uint32_t *slab = nullptr;
    size_t slab_bytes = 0;
    uint32_t slab_ctas = 0;   // narrow-block regions the slab holds
    bool external = false;    // the slab belongs to someone else (a server's arena)
    uint32_t *gretry = nullptr;
    size_t gretry_bytes = 0;
};
static DeviceShared g_shared[64];

struct Workspace {
    uint32_t n = 0, nwords = 0;
    int num_sms = 0;
    uint32_t *used_bits = nullptr, *rbits = nullptr, *sbits = nullptr;
    uint32_t *block_sums = nullptr;
    uint32_t *rsorted = nullptr;
    uint32_t rsorted_cap = 0;
    uint4 *failed = nullptr, *failed2 = nullptr;  // source ranges whose map overflowed, to search again
    uint32_t failed_cap = 0, failed2_cap = 0;
    Control *ctl = nullptr;
    Control *ctl_host = nullptr;  // pinned
    struct DeviceShared *sh = nullptr;  // the device's slab, shared by every graph on it
    uint32_t *kcp = nullptr;     // k closest pairs: histogram, live threshold, select state
    size_t gretry_bytes = 0;
    // raw pairs and radix-sort buffers
    unsigned long long *keyA = nullptr, *keyB = nullptr;
    uint32_t *valA = nullptr, *valB = nullptr;
    uint64_t pair_cap = 0;
    uint32_t *hist = nullptr;
    size_t hist_cap = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, evs0 = nullptr, evs1 = nullptr;
    DeviceShared *own_sh = nullptr;  // a slab of its own (workspace_set_slab), else null
    cudaEvent_t evr = nullptr;  // end of the last retry launch
    float retry_ms = 0;
    // a workspace may own its global-map buffer instead of using the device's
    bool own_gmap_enabled = false, own_gmap_moved = false;
    uint32_t *own_gmap = nullptr;
    size_t own_gmap_bytes = 0;
    // several joins over one graph: per query its first source, bound, S bitmap pointer
    // and pair count, the S bitmaps, and the S ids with their offsets
    uint32_t *mq_first = nullptr, *mq_bound = nullptr, *mq_sbits = nullptr, *mq_sids = nullptr, *mq_soff = nullptr;
    const uint32_t **mq_sptr = nullptr;
    unsigned long long *mq_counts = nullptr;
    uint8_t *mq_swap = nullptr;  // per query: searched from S
    uint64_t mq_cap_q = 0, mq_cap_bits = 0, mq_cap_sids = 0;
    // the largest source ball the last warp search met (or estimated, for sources
    // whose map overflowed) and its bound: predicts the next query's balls
    double ball_max = 0, ball_mean = 0;
    uint32_t ball_theta = 0;
    // warp search: per source its first pair and pair count; whether the last search
    // handed sources to the tile search (their pairs are then not in segments)
    uint2 *seg = nullptr;
    uint32_t seg_cap = 0;
    uint32_t *slist = nullptr;  // the warp search's per-warp lists of S nodes (SRC_LIST_WORDS)
    bool src_tiles = false;
    uint32_t launches = 0;  // kernels launched by the current query
    int blocks_per_sm = 0;  // occupancy of the shared-map search kernel
    uint64_t bytes = 0;
};

static void ws_alloc(Workspace *ws, void **p, size_t bytes) {
    *p = device_alloc(bytes);
    ws->bytes += bytes;
}

Workspace *workspace_create(const DeviceGraph &g) {
    Workspace *ws = new Workspace();
    try {
        int dev = 0;
        RN_CUDA(cudaGetDevice(&dev));
        RN_CUDA(cudaDeviceGetAttribute(&ws->num_sms, cudaDevAttrMultiProcessorCount, dev));
        if (dev < 0 || dev >= 64) fail(RN_EINVAL, "device ordinal out of range");
        ws->sh = &g_shared[dev];
        ws->n = g.n;
        ws->nwords = (g.n + 31) / 32;
        ws_alloc(ws, (void **)&ws->used_bits, size_t(ws->nwords) * 4);
        ws_alloc(ws, (void **)&ws->rbits, size_t(ws->nwords) * 4);
        ws_alloc(ws, (void **)&ws->sbits, size_t(ws->nwords) * 4);
        ws_alloc(ws, (void **)&ws->block_sums, (ws->nwords / 1024 + 2) * 4);
        ws_alloc(ws, (void **)&ws->ctl, sizeof(Control));
        RN_CUDA(cudaMallocHost(&ws->ctl_host, sizeof(Control)));
        RN_CUDA(cudaEventCreate(&ws->ev0));
        RN_CUDA(cudaEventCreate(&ws->ev1));
        RN_CUDA(cudaEventCreate(&ws->evs0));
        RN_CUDA(cudaEventCreate(&ws->evs1));
        RN_CUDA(cudaEventCreate(&ws->evr));
    } catch (...) {
        workspace_destroy(ws);
        throw;
    }
    return ws;
}

void workspace_destroy(Workspace *ws) {
    if (!ws) return;
    device_free(ws->used_bits);
    device_free(ws->rbits);
    device_free(ws->sbits);
    device_free(ws->block_sums);
    device_free(ws->rsorted);
    device_free(ws->failed);
    device_free(ws->failed2);
    device_free(ws->ctl);
    device_free(ws->kcp);
    device_free(ws->keyA);
    device_free(ws->keyB);
    device_free(ws->valA);
    device_free(ws->valB);
    device_free(ws->hist);
    if (ws->ctl_host) cudaFreeHost(ws->ctl_host);
    if (ws->ev0) cudaEventDestroy(ws->ev0);
    if (ws->ev1) cudaEventDestroy(ws->ev1);
    if (ws->evs0) cudaEventDestroy(ws->evs0);
    if (ws->evs1) cudaEventDestroy(ws->evs1);
    if (ws->evr) cudaEventDestroy(ws->evr);
    for (void *p : {(void *)ws->mq_first, (void *)ws->mq_bound, (void *)ws->mq_sbits, (void *)ws->mq_sids,
                    (void *)ws->mq_soff, (void *)ws->mq_sptr, (void *)ws->mq_counts, (void *)ws->mq_swap})
        device_free(p);
    device_free(ws->own_gmap);
    device_free(ws->seg);
    device_free(ws->slist);
    if (ws->own_sh) {
        device_free(ws->own_sh->gretry);
        delete ws->own_sh;
    }
    delete ws;
}

uint64_t workspace_bytes(const Workspace *ws) { return ws ? ws->bytes : 0; }

size_t slab_region_bytes() { return size_t(SMEM_H) * 128 * 4; }

// Give the workspace a slab of its own: `regions` narrow-block regions (at least two,
// so a wide block fits) at `slab`, which the caller owns and keeps every row of at INF
// between queries (the search leaves the rows it used at INF).  Its queries then need
// no device-wide lock and may overlap with other workspaces' queries on the device.
void workspace_set_slab(Workspace *ws, uint32_t *slab, uint32_t regions) {
    if (regions < 2 || !slab) fail(RN_EINVAL, "a workspace slab needs at least two regions");
    if (!ws->own_sh) ws->own_sh = new DeviceShared();
    ws->own_sh->external = true;
    ws->own_sh->slab = slab;
    ws->own_sh->slab_ctas = regions;
    ws->own_sh->slab_bytes = size_t(regions) * slab_region_bytes();
    ws->sh = ws->own_sh;
}

template <class T>
static void grow(Workspace *ws, T **p, uint64_t *cap, uint64_t want, uint64_t elem) {
    if (*p && *cap >= want) return;
    if (*p) {
        device_free(*p);
        ws->bytes -= *cap * elem;
    }
    *p = nullptr;
    uint64_t c = std::max<uint64_t>(want, 1024);
    *p = (T *)device_alloc(c * elem);
    ws->bytes += c * elem;
    *cap = c;
}

// --------------------------------------------------------------- set prep ----

// Mark one set: reject ids >= n and ids already marked (a repeat, or an id of R met
// again in S: the sets must be disjoint), and set the membership bit of the internal
// id.
// set_bits marks internal ids, or original ids with by_orig.
__global__ void k_mark_set(const uint32_t *__restrict__ ids, uint32_t cnt, uint32_t n,
                           const uint32_t *__restrict__ perm, uint32_t *used_bits,
                           uint32_t *set_bits, Control *ctl, bool by_orig) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x) {
        uint32_t id = ids[i];
        if (id >= n) {
            atomicOr(&ctl->err, 1u);
            continue;
        }
        uint32_t bit = 1u << (id & 31);
        uint32_t old = atomicOr(&used_bits[id >> 5], bit);
        if (old & bit) {
            atomicOr(&ctl->err, 2u);
            continue;
        }
        const uint32_t in = by_orig ? id : perm[id];
        atomicOr(&set_bits[in >> 5], 1u << (in & 31));
    }
}

// Set bits per block of 1024 words.
__global__ void k_bits_count(const uint32_t *__restrict__ bits, uint32_t nwords, uint32_t *block_sums) {
    __shared__ uint32_t warp_sum[32];
    uint32_t i = blockIdx.x * 1024 + threadIdx.x;
    uint32_t c = i < nwords ? __popc(bits[i]) : 0;
    c = __reduce_add_sync(FULL, c);
    if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x < 32) {
        uint32_t s = __reduce_add_sync(FULL, warp_sum[threadIdx.x]);
        if (threadIdx.x == 0) block_sums[blockIdx.x] = s;
    }
}

// Write the ids of the set bits in increasing order (R sorted by internal id, so a
// tile holds R nodes of one neighbourhood).  The last block stores the total.
__global__ void k_bits_compact(const uint32_t *__restrict__ bits, uint32_t nwords,
                               const uint32_t *__restrict__ block_sums, uint32_t nblocks,
                               uint32_t *out, Control *ctl) {
    __shared__ uint32_t warp_sum[32];
    __shared__ uint32_t s_base;
    if (threadIdx.x < 32) {
        uint32_t s = 0;
        for (uint32_t b = threadIdx.x; b < blockIdx.x; b += 32) s += block_sums[b];
        s = __reduce_add_sync(FULL, s);
        if (threadIdx.x == 0) {
            s_base = s;
            if (blockIdx.x == nblocks - 1) ctl->r_count = s + block_sums[blockIdx.x];
        }
    }
    uint32_t i = blockIdx.x * 1024 + threadIdx.x;
    uint32_t word = i < nwords ? bits[i] : 0;
    uint32_t c = __popc(word);
    uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = c;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_sum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t v = warp_sum[lane];
        uint32_t x = v;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t t = __shfl_up_sync(FULL, x, o);
            if (lane >= o) x += t;
        }
        warp_sum[lane] = x - v;
    }
    __syncthreads();
    uint32_t pos = s_base + warp_sum[warp] + incl - c;
    while (word) {
        uint32_t b = __ffs(word) - 1;
        word &= word - 1;
        out[pos++] = i * 32 + b;
    }
}

// ------------------------------------------------------------ tile search ----

struct SearchArgs {
    const uint32_t *__restrict__ row_ptr;
    const uint2 *__restrict__ adj;
    const uint32_t *__restrict__ iperm;
    const uint32_t *__restrict__ sbits;
    const uint32_t *__restrict__ src;       // R, internal ids, ascending
    const uint4 *__restrict__ range_list;   // retry: (first source, count, -, -) of each
                                            // range to search, or null: every tile of R
    uint32_t ntiles;                        // entries of range_list, or tiles of R
    uint32_t tile_src;                      // sources per tile (<= T; lanes beyond stay INF)
    uint32_t bound;                         // theta
    uint32_t delta;
    uint32_t *slab;                         // per-block regions of H rows x T lanes
    uint32_t *gmap;                         // global slot maps (2 H words per block), or null
    uint32_t H, hshift, max_fill;
    uint32_t vbits;                         // key = (u << vbits) | v
    uint32_t n_nodes;                       // the graph's nodes and arcs (bounds checks)
    uint64_t n_arcs;
    Control *ctl;
    uint4 *failed;                          // ranges whose slot map overflowed: (first,
                                            // count, bucket end reached, slots filled)
    unsigned long long *out_key;
    uint32_t *out_d;
    uint64_t out_cap;
    // k closest pairs (null for a join): a histogram of the distances of every pair
    // emitted so far (bin = d >> hist_shift, KCP_BINS bins) and the live threshold, the
    // least bin edge below which at least kcp_k pairs lie; each tile searches with
    // min(bound, *theta_live)
    uint32_t *kcp_hist;
    uint32_t *theta_live;
    unsigned long long kcp_k;
    uint32_t hist_shift;
    // batch (null for a single query): the graph is the disjoint union of the batch's
    // graphs and tile t belongs to instance tile_inst[t], searched with bound
    // tile_bound[t] and bucket width tile_delta[t]; nR_fixed (non-zero) gives the
    // number of sources instead of the control block; per-instance pair counts and SM
    // cycles (for the autotuner) are added to inst_pairs / inst_cycles
    const uint32_t *tile_bound;
    const uint32_t *tile_delta;
    const uint32_t *tile_inst;
    uint32_t nR_fixed;
    unsigned long long *inst_pairs;
    unsigned long long *inst_cycles;
    uint32_t *inst_ball;  // per instance: largest union ball of a completed tile
    // several joins over one graph (null for a single query): query i owns the sources
    // src[inst_first[i] .. inst_first[i + 1]), searches with bound inst_bound[i] against
    // the S bitmap inst_sbits[i], and its keys carry i above bit inst_shift
    const uint32_t *inst_first;
    uint32_t inst_count, inst_shift;
    const uint32_t *const *inst_sbits;
    const uint32_t *inst_bound;
    // searches from S (an undirected graph's distances are symmetric): a source is a node
    // of S and its targets are R's, and every pair is written as (target, source) so the
    // keys stay (u in R, v in S); per instance of a batch or query of several joins
    // inst_swap[inst], else swap_uv for all
    uint32_t swap_uv;
    const uint8_t *inst_swap;
    // warp search: seg[si] = (first pair, pair count) of source si, or null
    uint2 *seg;
    // warp search: per resident warp (block * warps per block + warp) a list of MS slots,
    // the S nodes of the current source's ball in the order first scanned
    uint32_t *slist;
    // the hierarchical variant's local searches: source si relaxes only arcs into its
    // part, internal ids [src_range[si].x, src_range[si].y), and records a route
    // (si << 32 | node, distance) to every border node of the part it settles (a node
    // with an arc leaving its part: border_bits) in brd_key / brd_d
    const uint2 *src_range;
    const uint32_t *border_bits;
    unsigned long long *brd_key;
    uint32_t *brd_d;
    uint64_t brd_cap;
    unsigned long long *brd_count;
};

// What a block needs to know about the tile it searches.
struct TileCtx {
    const uint32_t *row_ptr;
    const uint2 *adj;
    const uint32_t *iperm;
    const uint32_t *sbits;
    const uint32_t *src;
    unsigned long long key_prefix;
    uint32_t first, cnt;  // sources src[first .. first + cnt) of this tile (or part of one)
    uint32_t bound, delta, inst;
    uint32_t swap;        // the tile's sources are S nodes: pairs written (target, source)
};

constexpr uint32_t KCP_BINS = 2048;

template <int L>
struct Row {
    uint32_t x[L];
};

// Slot of node y, inserting it if absent, without touching the fill counter: *inserted
// tells the caller, which counts inserts once per warp.  EMPTY when the map is full.
__device__ __forceinline__ uint32_t find_or_insert_nf(uint32_t *hkeys, uint32_t H, uint32_t hshift, uint32_t y,
                                                      bool *inserted) {
    uint32_t h = (y * 0x9E3779B1u) >> hshift;
    volatile uint32_t *vk = hkeys;
    *inserted = false;
    for (uint32_t probe = 0; probe < H; probe++) {
        const uint32_t k = vk[h];
        if (k == y) return h;
        if (k == EMPTY) {
            const uint32_t prev = atomicCAS(&hkeys[h], EMPTY, y);
            if (prev == EMPTY) {
                *inserted = true;
                return h;
            }
            if (prev == y) return h;
        }
        h = (h + 1) & (H - 1);
    }
    return EMPTY;
}

// Warp-aggregated append: every lane with want = true gets a distinct index of the
// queue (one shared atomic per warp).  All 32 lanes must call.
__device__ __forceinline__ void warp_push(bool want, uint32_t value, uint32_t *count, uint32_t *queue,
                                          uint32_t cap) {
    const uint32_t b = __ballot_sync(FULL, want);
    if (!b) return;
    const uint32_t lane = threadIdx.x & 31;
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(count, uint32_t(__popc(b)));
    base = __shfl_sync(FULL, base, 0);
    if (want) {
        const uint32_t qi = base + __popc(b & ((1u << lane) - 1));
        if (qi < cap) queue[qi] = value;
    }
}

template <int L>
__device__ __forceinline__ Row<L> load_row(const uint32_t *p) {
    Row<L> r;
    if constexpr (L == 1) {
        r.x[0] = __ldcg(p);
    } else if constexpr (L == 2) {
        uint2 v = __ldcg(reinterpret_cast<const uint2 *>(p));
        r.x[0] = v.x;
        r.x[1] = v.y;
    } else {
        uint4 v = __ldcg(reinterpret_cast<const uint4 *>(p));
        r.x[0] = v.x;
        r.x[1] = v.y;
        r.x[2] = v.z;
        r.x[3] = v.w;
    }
    return r;
}

template <int L>
__device__ __forceinline__ void store_inf(uint32_t *p) {
    if constexpr (L == 1) {
        __stcg(p, INF);
    } else if constexpr (L == 2) {
        __stcg(reinterpret_cast<uint2 *>(p), make_uint2(INF, INF));
    } else {
        __stcg(reinterpret_cast<uint4 *>(p), make_uint4(INF, INF, INF, INF));
    }
}

__device__ __forceinline__ uint32_t slot_hash(uint32_t y, uint32_t hshift) {
    return (y * 0x9E3779B1u) >> hshift;
}

// Slot of node y in the tile's map, inserting it if absent.  Linear probing; EMPTY when
// the map is full (the tile then fails and is searched again with a larger map).
__device__ __forceinline__ uint32_t find_or_insert(uint32_t *hkeys, uint32_t H, uint32_t hshift,
                                                   uint32_t y, uint32_t *fill, uint32_t max_fill,
                                                   uint32_t *fail_flag) {
    uint32_t h = slot_hash(y, hshift);
    volatile uint32_t *vk = hkeys;
    for (uint32_t probe = 0; probe < H; probe++) {
        uint32_t k = vk[h];
        if (k == y) return h;
        if (k == EMPTY) {
            uint32_t prev = atomicCAS(&hkeys[h], EMPTY, y);
            if (prev == EMPTY) {
                if (atomicAdd(fill, 1u) >= max_fill) *(volatile uint32_t *)fail_flag = 1;
                return h;
            }
            if (prev == y) return h;
        }
        h = (h + 1) & (H - 1);
    }
    *(volatile uint32_t *)fail_flag = 1;
    return EMPTY;
}

// Exclusive prefix sum of v over the block; *total receives the sum.  All threads call;
// warp_buf must hold THREADS / 32 + 1 words, and the caller puts a barrier between this
// call and the next write to warp_buf (the next call, or any other use).
template <int THREADS>
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *warp_buf, uint32_t *total) {
    constexpr int SEARCH_WARPS = THREADS / 32;
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(FULL, x, o);
        if (lane >= uint32_t(o)) x += t;
    }
    if (lane == 31) warp_buf[warp] = x;
    __syncthreads();
    if (warp == 0) {
        const uint32_t w = lane < SEARCH_WARPS ? warp_buf[lane] : 0;
        uint32_t y = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(FULL, y, o);
            if (lane >= uint32_t(o)) y += t;
        }
        if (lane < SEARCH_WARPS) warp_buf[lane] = y - w;
        if (lane == 31) warp_buf[SEARCH_WARPS] = y;  // warp_buf holds SEARCH_WARPS + 1 words
    }
    __syncthreads();
    const uint32_t r = warp_buf[warp] + x - v;
    *total = warp_buf[SEARCH_WARPS];
    return r;
}

// One thread block searches one tile of up to T = 32 L sources at a time (persistent:
// blocks pop tiles from a global counter).  Lane-group j of a slab row holds sources
// j*L .. j*L+L-1.
//
// Per slot h the map keeps, besides its node id hkeys[h]:
//   prio[h]  the least improved-but-unrelaxed distance in the row, INF when clean;
//   dmask[h] which lane-groups of the row improved since the row was last relaxed.
// A relaxation is: atomicMin on the slab (fire and forget), then dmask |= improved
// groups, then prio = min(prio, least improved value) (pushing h on the near queue when
// it becomes dirty inside the current bucket).  A scan takes prio, skips a clean slot,
// takes dmask and reads the dirty groups of the row.  Scans (step A below) and
// relaxations (step B) never overlap: a block barrier separates them, and the barrier
// makes every slab update of step B visible to the block before the next step A reads
// the row.  So every improvement is relaxed at least once after it happened, and a
// rescan relaxes only the groups that changed.
//
// A round relaxes the near queue in block-wide steps of up to ICAP items: one thread per
// item takes its prio and dmask, its CSR offsets and the least dirty value; a block
// prefix sum over the items' degrees lays their arcs out; then one thread per arc loads
// it, finds (or inserts) the head's slot, and relaxes every dirty lane-group of the
// item into that slot.  So a round costs a few memory round trips, not one per arc.
//
// GMAP = false keeps the map in shared memory; GMAP = true keeps it in global memory
// so a tile whose union ball outgrows shared memory can be searched again.
template <int L, bool GMAP, int THREADS>
__global__ void __launch_bounds__(THREADS, (THREADS == NARROW ? CTAS_PER_SM : 1)) k_tile_search(SearchArgs a) {
    constexpr int T = 32 * L;
    constexpr int G = 4 / L;  // lane-groups of one arc relaxed together
    constexpr int SEARCH_THREADS = THREADS;
    constexpr int SEARCH_WARPS = THREADS / 32;
    constexpr uint32_t QCAP = qcap_of(THREADS);
    constexpr uint32_t ICAP = icap_of(THREADS);
    constexpr uint32_t ICAP_POW2 = 1u << (31 - __builtin_clz(ICAP));  // the largest power of two <= ICAP
    extern __shared__ __align__(16) uint32_t smem[];
    uint32_t *hkeys, *qa;
    if constexpr (GMAP) {
        hkeys = a.gmap + size_t(blockIdx.x) * 3 * a.H;
        qa = smem;
    } else {
        hkeys = smem;
        qa = smem + 3 * a.H;
    }
    uint32_t *prio = hkeys + a.H;
    uint32_t *dmask = prio + a.H;
    uint32_t *qb = qa + QCAP;
    uint32_t *it_x = qb + QCAP;        // staged items: slot,
    uint32_t *it_mask = it_x + ICAP;   // dirty groups,
    uint32_t *it_beg = it_mask + ICAP; // first arc,
    uint32_t *it_off = it_beg + ICAP;  // arc offset in the step,
    uint32_t *it_dmin = it_off + ICAP; // least dirty value
    __shared__ uint32_t src_orig[T];
    __shared__ uint32_t s_tile, s_ncur, s_nnext, s_fill, s_fail, s_minp;
    __shared__ uint32_t s_warp[SEARCH_WARPS + 1];
    __shared__ unsigned long long s_base;

    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t *slab = a.slab + size_t(blockIdx.x) * a.H * T;
    __shared__ TileCtx s_cx;
    uint32_t my_scans = 0, my_slots = 0, my_arcs = 0, my_dirty = 0;
    // telemetry, kept by thread 0 in shared memory: rounds, round items, boundaries,
    // round arcs, cycles in step A, step B, boundaries, emission; clock marks
    enum { T_ROUNDS, T_ITEMS, T_BOUNDS, T_ARCS, T_STEPA, T_STEPB, T_BOUND, T_EMIT, T_N };
    __shared__ unsigned long long s_tel[T_N];
    __shared__ long long s_mark, s_tile0;
    if (tid < T_N) s_tel[tid] = 0;
    if (tid == 0) s_mark = clock64();

    if (__ldcg(&a.ctl->err)) return;
    const uint32_t nR1 = a.nR_fixed ? a.nR_fixed : __ldcg(&a.ctl->r_count);  // sources
    const uint32_t all_tiles = (nR1 + a.tile_src - 1) / a.tile_src;
    const uint32_t ntiles = a.range_list ? a.ntiles : all_tiles;


    for (;;) {
        if (tid == 0) s_tile = atomicAdd(&a.ctl->tile_next, 1u);
        for (uint32_t i = tid; i < a.H; i += SEARCH_THREADS) {
            hkeys[i] = EMPTY;
            prio[i] = INF;
            dmask[i] = 0;
        }
        if (tid == 0) {
            s_ncur = 0;
            s_nnext = 0;
            s_fill = 0;
            s_fail = 0;
        }
        if (tid < T) src_orig[tid] = 0;
        __syncthreads();
        const uint32_t ti = s_tile;
        if (ti >= ntiles) break;
        // this block's sources: tile ti, or the ti-th range of a retry (a whole tile or a
        // part of one); the tile it lies in names its per-tile table entries
        uint32_t first, cnt;
        if (a.range_list) {
            const uint4 r = a.range_list[ti];
            first = r.x;
            cnt = r.y;
        } else {
            first = ti * a.tile_src;
            cnt = first < nR1 ? min(a.tile_src, nR1 - first) : 0u;
        }
        if (cnt == 0 || cnt > a.tile_src || first >= nR1 || cnt > nR1 - first) continue;  // never past R
        const uint32_t tile = first / a.tile_src;
        if (tid == 0) {
            TileCtx c;
            c.row_ptr = a.row_ptr;
            c.adj = a.adj;
            c.iperm = a.iperm;
            c.sbits = a.sbits;
            c.src = a.src;
            c.first = first;
            c.cnt = cnt;
            c.bound = a.tile_bound ? a.tile_bound[tile]
                                   : (a.theta_live ? min(a.bound, __ldcg(a.theta_live)) : a.bound);
            c.delta = a.tile_delta ? a.tile_delta[tile] : a.delta;
            c.inst = a.tile_inst ? a.tile_inst[tile] : 0u;
            c.key_prefix = 0;
            if (a.inst_first) {
                // the query whose sources hold this range: the last with inst_first <= first
                uint32_t lo = 0, hi = a.inst_count - 1;
                while (lo < hi) {
                    const uint32_t mid = (lo + hi + 1) >> 1;
                    if (a.inst_first[mid] <= first) lo = mid;
                    else hi = mid - 1;
                }
                c.inst = lo;
                c.bound = a.inst_bound[lo];
                c.sbits = a.inst_sbits[lo];
                c.key_prefix = (unsigned long long)lo << a.inst_shift;
            }
            c.swap = a.inst_swap ? a.inst_swap[c.inst] : a.swap_uv;
            s_cx = c;
            s_tile0 = clock64();
        }
        __syncthreads();
        const uint32_t *row_ptr = s_cx.row_ptr;
        const uint2 *adj = s_cx.adj;
        const uint32_t bound = s_cx.bound;  // this tile's bound, the same for every thread
        const uint64_t delta = s_cx.delta;
        const uint32_t tsz = s_cx.cnt;

        // sources: lane t of every row belongs to R node first + t, at distance 0
        if (tid < tsz) {
            const uint32_t y = s_cx.src[s_cx.first + tid];
            if (!RN_BAD(y < a.n_nodes, 1, s_cx.first + tid, y)) {
                src_orig[tid] = s_cx.iperm[y];
                const uint32_t h = find_or_insert(hkeys, a.H, a.hshift, y, &s_fill, a.max_fill, &s_fail);
                if (!RN_BAD(h < a.H, 2, tid, h)) {
                    __stcg(&slab[size_t(h) * T + tid], 0u);
                    atomicOr(&dmask[h], 1u << (tid / L));
                    prio[h] = 0;
                    qa[atomicAdd(&s_ncur, 1u)] = h;
                }
            }
        }
        uint32_t *qcur = qa, *qnext = qb;
        uint64_t tau = delta;  // end (exclusive) of the current bucket
        if (tau > uint64_t(bound) + 1) tau = uint64_t(bound) + 1;

        for (;;) {
            // ---- rounds of the current bucket: relax the near queue until it drains.
            // Every thread reads the queue count and the fail flag right after the
            // barrier that ends the step writing them (the sources or the collect step
            // here; step B below), so every thread takes the same decision; the count
            // is reset only after the next barrier (the scan's), when all have read it.
            __syncthreads();
            uint32_t ncur = min(s_ncur, QCAP);
            bool stop = s_fail;
            for (;;) {
                if (tid == 0) {
                    const long long t = clock64();
                    s_tel[T_BOUND] += t - s_mark;
                    s_mark = t;
                }
                if (ncur == 0 || stop) break;
                if (tid == 0) {
                    s_tel[T_ROUNDS]++;
                    s_tel[T_ITEMS] += ncur;
                }
                for (uint32_t c0 = 0; c0 < ncur; c0 += ICAP) {
                    const uint32_t nc = min(ICAP, ncur - c0);
                    // -- step A: one thread per queue item
                    uint32_t deg = 0;
                    if (tid < nc) {
                        const uint32_t x = qcur[c0 + tid];
                        uint32_t mask = 0, beg = 0, dmin = INF;
                        const bool bad_x = RN_BAD(x < a.H, 3, c0 + tid, x);
                        const uint32_t p = bad_x ? INF : atomicExch(&prio[x], INF);
                        if (p != INF) mask = atomicExch(&dmask[x], 0u);
                        if (mask && RN_BAD(hkeys[x] < a.n_nodes, 4, x, hkeys[x])) mask = 0;
                        if (mask) {
                            my_scans++;
                            my_dirty += __popc(mask);
                            const uint32_t y0 = hkeys[x];
                            beg = __ldg(&row_ptr[y0]);
                            deg = __ldg(&row_ptr[y0 + 1]) - beg;
                            if (RN_BAD(uint64_t(beg) + deg <= a.n_arcs, 5, y0, beg)) deg = 0;
                            const uint32_t *xrow = slab + size_t(x) * T;
                            uint32_t m = mask;
                            if ((m & (m - 1)) == 0) {  // one dirty lane-group (m != 0 here)
                                const Row<L> r = load_row<L>(xrow + (__ffs(m) - 1) * L);
#pragma unroll
                                for (int q = 0; q < L; q++) dmin = min(dmin, r.x[q]);
                                m = 0;
                            }
                            while (m) {
                                Row<L> r[G];
#pragma unroll
                                for (int k = 0; k < G; k++) {
#pragma unroll
                                    for (int q = 0; q < L; q++) r[k].x[q] = INF;
                                    if (m) {
                                        r[k] = load_row<L>(xrow + (__ffs(m) - 1) * L);
                                        m &= m - 1;
                                    }
                                }
#pragma unroll
                                for (int k = 0; k < G; k++)
#pragma unroll
                                    for (int q = 0; q < L; q++) dmin = min(dmin, r[k].x[q]);
                            }
                            if (dmin > bound) deg = 0;
                        }
                        it_x[tid] = x;
                        it_mask[tid] = mask;
                        it_beg[tid] = beg;
                        it_dmin[tid] = dmin;
                    }
                    uint32_t total;
                    const uint32_t off = block_exclusive_scan<THREADS>(deg, s_warp, &total);
                    if (tid == 0 && c0 == 0) s_nnext = 0;  // every thread has read the last count
                    if (tid < nc) it_off[tid] = off;
                    __syncthreads();
                    if (tid == 0) {
                        const long long t = clock64();
                        s_tel[T_STEPA] += t - s_mark;
                        s_mark = t;
                        s_tel[T_ARCS] += total;
                    }
                    // -- step B: one thread per arc of the staged items, in chunks of 32 arcs
                    // per warp (warp-uniform trip count, so the ballots below see every
                    // lane).  A thread takes its arc's item, head and weight, prunes it
                    // against the item's least dirty value, finds the head's slot, then
                    // relaxes the item's dirty lane-groups into that slot, G at a time.
                    // (One warp per arc across the row, with coalesced row loads, measured
                    // slower: the round is bound by chains of dependent L2 round trips,
                    // which serialising a warp's arcs lengthens.)
                    for (uint32_t c0 = warp * 32; c0 < total; c0 += SEARCH_THREADS) {
                        const uint32_t gi = c0 + lane;
                        uint32_t item = 0, hy = EMPTY, w = 0;
                        bool push = false;
                        if (gi < total) {
                            // the last item whose arcs start at or before gi: a branchless
                            // search by powers of two below ICAP (it_off is non-decreasing)
                            uint32_t lo = 0;
#pragma unroll
                            for (uint32_t step = ICAP_POW2; step; step >>= 1)
                                if (lo + step < nc && it_off[lo + step] <= gi) lo += step;
                            item = lo;
                            const uint32_t ai = it_beg[lo] + (gi - it_off[lo]);
                            if (!RN_BAD(ai < a.n_arcs, 6, gi, ai)) {
                                const uint2 arc = __ldg(&adj[ai]);
                                w = arc.y;
                                if (it_dmin[lo] + w <= bound) hy = arc.x;  // the head node until its slot is known
                                if (hy != EMPTY && RN_BAD(hy < a.n_nodes, 7, ai, hy)) hy = EMPTY;
                            }
                        }
                        bool ins = false;
                        if (hy != EMPTY) {
                            hy = find_or_insert_nf(hkeys, a.H, a.hshift, hy, &ins);
                            if (hy == EMPTY) s_fail = 1;
                            else if (RN_BAD(hy < a.H, 8, gi, hy)) hy = EMPTY;
                        }
                        const uint32_t inserted = __popc(__ballot_sync(FULL, ins));
                        if (lane == 0 && inserted && atomicAdd(&s_fill, inserted) + inserted > a.max_fill)
                            s_fail = 1;
                        if (hy != EMPTY) {
                            const uint32_t *xrow = slab + size_t(it_x[item]) * T;
                            uint32_t *yrow = slab + size_t(hy) * T;
                            uint32_t imask = 0, imin = INF;
                            uint32_t m = it_mask[item];
                            if (m && (m & (m - 1)) == 0) {
                                // one dirty lane-group (the common case): no batching; with
                                // one lane per group its value is the item's least dirty
                                // value, read in step A (a value lowered since marks the row
                                // dirty again, so it is relaxed in a later round)
                                const uint32_t j = __ffs(m) - 1;
                                Row<L> dv;
                                if constexpr (L == 1) dv.x[0] = it_dmin[item];
                                else dv = load_row<L>(xrow + j * L);
                                const Row<L> cv = load_row<L>(yrow + j * L);
#pragma unroll
                                for (int q = 0; q < L; q++) {
                                    const uint32_t d = dv.x[q] + w;
                                    if (dv.x[q] != INF && d <= bound && d < cv.x[q]) {
                                        atomicMin(yrow + j * L + q, d);
                                        imin = min(imin, d);
                                        imask = 1u << j;
                                    }
                                }
                                m = 0;
                            }
                            while (m) {
                                uint32_t jj[G];
                                Row<L> dv[G], cv[G];
#pragma unroll
                                for (int k = 0; k < G; k++) {
                                    jj[k] = m ? uint32_t(__ffs(m) - 1) : 32u;
                                    if (m) m &= m - 1;
                                }
#pragma unroll
                                for (int k = 0; k < G; k++) {
                                    if (jj[k] < 32) {
                                        dv[k] = load_row<L>(xrow + jj[k] * L);
                                        cv[k] = load_row<L>(yrow + jj[k] * L);
                                    }
                                }
#pragma unroll
                                for (int k = 0; k < G; k++) {
                                    if (jj[k] >= 32) continue;
#pragma unroll
                                    for (int q = 0; q < L; q++) {
                                        if (dv[k].x[q] == INF) continue;
                                        const uint32_t d = dv[k].x[q] + w;
                                        if (d <= bound && d < cv[k].x[q]) {
                                            atomicMin(yrow + jj[k] * L + q, d);
                                            imin = min(imin, d);
                                            imask |= 1u << jj[k];
                                        }
                                    }
                                }
                            }
                            if (imask) {
                                atomicOr(&dmask[hy], imask);
                                const uint32_t old = atomicMin(&prio[hy], imin);
                                push = imin < tau && (old == INF || old >= tau);
                            }
                        }
                        warp_push(push, hy, &s_nnext, qnext, QCAP);
                    }
                    __syncthreads();
                    if (tid == 0) {
                        const long long t = clock64();
                        s_tel[T_STEPB] += t - s_mark;
                        s_mark = t;
                    }
                }
                ncur = min(s_nnext, QCAP);  // after step B's closing barrier
                stop = s_fail;
                uint32_t *t = qcur;
                qcur = qnext;
                qnext = t;
            }
            if (stop) break;
            // ---- the near queue is empty: find the smallest pending priority
            if (tid == 0) {
                s_minp = INF;
                s_ncur = 0;  // the collect step counts from zero (read before the barrier above)
                s_tel[T_BOUNDS]++;
            }
            __syncthreads();
            uint32_t mp = INF;
            for (uint32_t h = tid; h < a.H; h += SEARCH_THREADS) mp = min(mp, prio[h]);
            mp = __reduce_min_sync(FULL, mp);
            if (lane == 0 && mp != INF) atomicMin(&s_minp, mp);
            __syncthreads();
            const uint32_t minp = s_minp;
            if (minp == INF) break;  // nothing pending: the tile's search is complete
            if (minp >= tau) {
                tau = (uint64_t(minp) / delta + 1) * delta;
                if (tau > uint64_t(bound) + 1) tau = uint64_t(bound) + 1;
            }
            // ---- collect every pending slot of the (new) bucket into the near queue
            for (uint32_t h = tid; h < a.H; h += SEARCH_THREADS)  // H is a multiple of THREADS
                warp_push(prio[h] < tau, h, &s_ncur, qcur, QCAP);
        }
        __syncthreads();
        if (tid == 0) {
            const long long t = clock64();
            s_tel[T_BOUND] += t - s_mark;
            s_mark = t;
        }

        // ---- emission: every slot of an S node, every lane within the bound.  Warps
        // take 32 consecutive slots at a time and ballot the ones holding S nodes.
        const bool ok = !s_fail;
        const uint32_t lt = (1u << lane) - 1;
        if (ok) {
            uint32_t cnt = 0;
            for (uint32_t c = warp * 32; c < a.H; c += SEARCH_WARPS * 32) {
                const uint32_t yl = hkeys[c + lane];
                const bool in_s = yl != EMPTY && !RN_BAD(yl < a.n_nodes, 9, c + lane, yl) &&
                                  ((__ldg(&s_cx.sbits[yl >> 5]) >> (yl & 31)) & 1u);
                for (uint32_t b = __ballot_sync(FULL, in_s); b; b &= b - 1) {
                    const uint32_t h = c + __ffs(b) - 1;
                    const Row<L> r = load_row<L>(slab + size_t(h) * T + lane * L);
#pragma unroll
                    for (int q = 0; q < L; q++) cnt += __popc(__ballot_sync(FULL, r.x[q] <= bound));
                }
            }
            if (lane == 0) s_warp[warp] = cnt;
            __syncthreads();
            if (tid == 0) {
                uint32_t run = 0;
                for (int w = 0; w < SEARCH_WARPS; w++) {
                    uint32_t c = s_warp[w];
                    s_warp[w] = run;
                    run += c;
                }
                s_base = atomicAdd(&a.ctl->pairs, (unsigned long long)run);
                if (a.inst_pairs) atomicAdd(&a.inst_pairs[s_cx.inst], (unsigned long long)run);
            }
            __syncthreads();
            unsigned long long pos = s_base + s_warp[warp];
            for (uint32_t c = warp * 32; c < a.H; c += SEARCH_WARPS * 32) {
                const uint32_t yl = hkeys[c + lane];
                const bool in_s = yl != EMPTY && !RN_BAD(yl < a.n_nodes, 9, c + lane, yl) &&
                                  ((__ldg(&s_cx.sbits[yl >> 5]) >> (yl & 31)) & 1u);
                for (uint32_t b = __ballot_sync(FULL, in_s); b; b &= b - 1) {
                    const uint32_t src_lane = __ffs(b) - 1;
                    const uint32_t h = c + src_lane;
                    const uint32_t y = __shfl_sync(FULL, yl, src_lane);
                    const Row<L> r = load_row<L>(slab + size_t(h) * T + lane * L);
                    const unsigned long long v = __ldg(&s_cx.iperm[y]);
#pragma unroll
                    for (int q = 0; q < L; q++) {
                        const bool hit = r.x[q] <= bound;
                        const uint32_t bb = __ballot_sync(FULL, hit);
                        if (hit) {
                            const unsigned long long idx = pos + __popc(bb & lt);
                            if (idx < a.out_cap) {
                                const unsigned long long u = src_orig[lane * L + q];
                                a.out_key[idx] = s_cx.key_prefix | (s_cx.swap ? (v << a.vbits) | u : (u << a.vbits) | v);
                                a.out_d[idx] = r.x[q];
                            }
                            if (a.kcp_hist) atomicAdd(&a.kcp_hist[r.x[q] >> a.hist_shift], 1u);
                        }
                        pos += __popc(bb);
                    }
                }
            }
            if (a.kcp_hist) {
                // the tile's pairs are counted: lower the live threshold to the edge of
                // the first bin where the pairs emitted so far reach k (they are exact,
                // distinct pairs, so the k-th distance cannot lie above that edge)
                __syncthreads();
                if (warp == 0) {
                    constexpr uint32_t PER = KCP_BINS / 32;
                    unsigned long long own = 0;
#pragma unroll 8
                    for (uint32_t i = 0; i < PER; i++) own += __ldcg(&a.kcp_hist[lane * PER + i]);
                    unsigned long long incl = own;
                    for (int o = 1; o < 32; o <<= 1) {
                        const unsigned long long t = __shfl_up_sync(FULL, incl, o);
                        if (lane >= uint32_t(o)) incl += t;
                    }
                    const uint32_t reach = __ballot_sync(FULL, incl >= a.kcp_k);
                    if (reach && lane == uint32_t(__ffs(reach) - 1)) {
                        unsigned long long cum = incl - own;
                        for (uint32_t i = 0; i < PER; i++) {
                            cum += __ldcg(&a.kcp_hist[lane * PER + i]);
                            if (cum >= a.kcp_k) {
                                const unsigned long long edge =
                                    ((unsigned long long)(lane * PER + i + 1) << a.hist_shift) - 1;
                                atomicMin(a.theta_live, uint32_t(min(edge, 0xFFFFFFFFull)));
                                break;
                            }
                        }
                    }
                }
            }
        } else if (tid == 0) {
            a.failed[atomicAdd(&a.ctl->n_failed, 1u)] =
                make_uint4(s_cx.first, s_cx.cnt, uint32_t(min(tau, uint64_t(0xFFFFFFFFu))), s_fill);
        }
        // ---- leave the region clean (every row INF) for the next tile
        for (uint32_t c = warp * 32; c < a.H; c += SEARCH_WARPS * 32) {
            const uint32_t yl = hkeys[c + lane];
            const bool used = yl != EMPTY;
            if (ok && used) {
                my_slots++;
                my_arcs += __ldg(&row_ptr[yl + 1]) - __ldg(&row_ptr[yl]);
            }
            for (uint32_t b = __ballot_sync(FULL, used); b; b &= b - 1)
                store_inf<L>(slab + size_t(c + __ffs(b) - 1) * T + lane * L);
        }
        __syncthreads();
        if (tid == 0) {
            const long long t = clock64();
            s_tel[T_EMIT] += t - s_mark;
            s_mark = t;
            // cycles weighted by the block's share of an SM (a wide block holds it alone)
            if (a.inst_cycles)
                atomicAdd(&a.inst_cycles[s_cx.inst], (unsigned long long)(t - s_tile0) * (THREADS / NARROW));
            if (ok) {
                atomicMax(&a.ctl->max_fill, s_fill);
                if (a.inst_ball) atomicMax(&a.inst_ball[s_cx.inst], s_fill);
            }
        }
    }
    my_slots = __reduce_add_sync(FULL, my_slots);
    my_arcs = __reduce_add_sync(FULL, my_arcs);
    my_scans = __reduce_add_sync(FULL, my_scans);
    my_dirty = __reduce_add_sync(FULL, my_dirty);
    if (lane == 0) {
        atomicAdd(&a.ctl->scans, (unsigned long long)my_scans);
        atomicAdd(&a.ctl->dirty_groups, (unsigned long long)my_dirty);
        atomicAdd(&a.ctl->slots, (unsigned long long)my_slots);
        atomicAdd(&a.ctl->slot_lanes, (unsigned long long)my_slots * T);
        atomicAdd(&a.ctl->slot_arcs, (unsigned long long)my_arcs);
    }
    if (tid == 0) {
        atomicAdd(&a.ctl->rounds, s_tel[T_ROUNDS]);
        atomicAdd(&a.ctl->round_items, s_tel[T_ITEMS]);
        atomicAdd(&a.ctl->boundaries, s_tel[T_BOUNDS]);
        atomicAdd(&a.ctl->cyc_round, s_tel[T_STEPA] + s_tel[T_STEPB]);
        atomicAdd(&a.ctl->cyc_stepA, s_tel[T_STEPA]);
        atomicAdd(&a.ctl->round_arcs, s_tel[T_ARCS]);
        atomicAdd(&a.ctl->cyc_bound, s_tel[T_BOUND]);
        atomicAdd(&a.ctl->cyc_emit, s_tel[T_EMIT]);
    }
}

// ----------------------------------------------------------- source search ----
// One warp searches one source at a time (persistent: warps pop sources from the work
// counter).  The source's ball lives in a map of MS slots in shared memory that only this
// warp touches:
//   key[h]   node id (SK_NODE bits) and four flags: SK_SEEN (its arcs were relaxed at
//            least once), SK_IN_S (the node is in S, read at that first scan), SK_DIRTY
//            (its distance improved since its arcs were last relaxed), SK_QUEUED (in the
//            near queue, or claimed for it); SK_EMPTY when free;
//   dist[h]  tentative distance, INF when free.
// Delta-stepping with one lane of distances: a round takes up to 64 near-queue items (two
// per lane), clears their flags and reads their distance and CSR range, lays their arcs
// out with a warp prefix sum, then relaxes 128 arcs at a time (four per lane): every arc
// load, then every first probe, then every atomicMin on dist,
// then on improvements every flag update is issued before the results are used, so their
// latencies overlap; a slot is pushed when it enters the near queue.  When the
// queue drains, one pass over the map takes the least pending distance and collects the
// slots of the next bucket.  There is no block barrier: lanes synchronise with __syncwarp,
// and a round waits on two dependent L2 round trips (CSR offsets, then arcs).
//
// A source whose ball outgrows 7/8 of the map stops and reports (source, bound, bucket end
// reached, slots filled); the host searches it again with a larger map or with the tile
// search.
constexpr uint32_t SK_NODE = 0x0FFFFFFFu;
constexpr uint32_t SK_EMPTY = SK_NODE;
constexpr uint32_t SK_IN_S = 0x10000000u;
constexpr uint32_t SK_SEEN = 0x20000000u;
constexpr uint32_t SK_DIRTY = 0x40000000u;
constexpr uint32_t SK_QUEUED = 0x80000000u;
constexpr uint32_t SRC_BLOCK_SMEM = 73728;  // shared memory of one block: three per SM
constexpr uint32_t SRC_BLOCKS_PER_SM = 3;
constexpr uint32_t SRC_MS_MIN = 1024, SRC_MS_MAX = 8192;
__host__ __device__ constexpr uint32_t log2u(uint32_t x) { return x <= 1 ? 0 : 1 + log2u(x >> 1); }
__host__ __device__ constexpr uint32_t src_qcap(uint32_t ms) { return ms / 8; }
__host__ __device__ constexpr uint32_t src_words(uint32_t ms) { return 2 * ms + 2 * src_qcap(ms); }
__host__ __device__ constexpr uint32_t src_warps(uint32_t ms) { return SRC_BLOCK_SMEM / (4 * src_words(ms)); }
// The warp search's S-node lists in global memory: MS entries per warp, for every warp of
// every resident block (a block of src_warps(MS) warps holds src_warps(MS) * MS = 8192
// entries whatever MS is).
constexpr size_t SRC_LIST_WORDS_PER_BLOCK = 8192;
static_assert(src_warps(1024) * 1024 <= SRC_LIST_WORDS_PER_BLOCK && src_warps(2048) * 2048 <= SRC_LIST_WORDS_PER_BLOCK &&
                  src_warps(4096) * 4096 <= SRC_LIST_WORDS_PER_BLOCK && src_warps(8192) * 8192 <= SRC_LIST_WORDS_PER_BLOCK,
              "S-node lists too small");

// Slot of node y in a warp map of MS slots, probing from slot h on (linear probing) and
// inserting y if absent; EMPTY when the map is full.
template <uint32_t MS>
__device__ __forceinline__ uint32_t src_slot(uint32_t *key, uint32_t y, uint32_t h, bool *inserted) {
    volatile uint32_t *vk = key;
    *inserted = false;
    for (uint32_t probe = 0; probe < MS; probe++) {
        const uint32_t k = vk[h];
        if ((k & SK_NODE) == y) return h;
        if (k == SK_EMPTY) {
            const uint32_t prev = atomicCAS(&key[h], SK_EMPTY, y);
            if (prev == SK_EMPTY) {
                *inserted = true;
                return h;
            }
            if ((prev & SK_NODE) == y) return h;
        }
        h = (h + 1) & (MS - 1);
    }
    return EMPTY;
}

__device__ __forceinline__ unsigned long long warp_sum64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// One warp: the first bin of the k-closest-pairs histogram where the cumulative count
// reaches k, and the live bound lowered to that bin's upper edge.  Each lane sums its 64
// consecutive bins (16 independent vector loads); the lane whose range holds the k-th
// pair reads its bins again to find the bin.
__device__ __forceinline__ void kcp_lower_bound(const SearchArgs &a, uint32_t lane) {
    constexpr uint32_t PER = KCP_BINS / 32;
    const uint4 *h4 = reinterpret_cast<const uint4 *>(a.kcp_hist) + lane * (PER / 4);
    unsigned long long own = 0;
#pragma unroll
    for (uint32_t i = 0; i < PER / 4; i++) {
        const uint4 q = __ldcg(&h4[i]);
        own += (unsigned long long)q.x + q.y + q.z + q.w;
    }
    unsigned long long incl = own;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long t = __shfl_up_sync(FULL, incl, o);
        if (lane >= uint32_t(o)) incl += t;
    }
    const uint32_t reach = __ballot_sync(FULL, incl >= a.kcp_k);
    if (reach && lane == uint32_t(__ffs(reach) - 1)) {
        unsigned long long cum = incl - own;
        uint32_t bin = lane * PER + PER - 1;
        for (uint32_t i = 0; i < PER / 4; i++) {
            const uint4 q = __ldcg(&h4[i]);
            const uint32_t c4[4] = {q.x, q.y, q.z, q.w};
            bool found = false;
#pragma unroll
            for (uint32_t j = 0; j < 4; j++) {
                cum += c4[j];
                if (!found && cum >= a.kcp_k) {
                    bin = lane * PER + 4 * i + j;
                    found = true;
                }
            }
            if (found) break;
        }
        const unsigned long long edge = ((unsigned long long)(bin + 1) << a.hist_shift) - 1;
        atomicMin(a.theta_live, uint32_t(min(edge, 0xFFFFFFFFull)));
    }
}

template <uint32_t MS, bool HIER>
__global__ void __launch_bounds__(src_warps(MS) * 32, SRC_BLOCKS_PER_SM) k_source_search(SearchArgs a) {
    constexpr uint32_t QS = src_qcap(MS);
    constexpr int AP = 4;  // arcs per lane in flight
    extern __shared__ __align__(16) uint32_t smem[];  // (sixteen-byte stores clear the maps)
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1;
    uint32_t *key = smem + warp * src_words(MS);
    uint32_t *dist = key + MS;
    uint32_t *qa = dist + MS, *qb = qa + QS;
    for (uint32_t h = lane; h < MS; h += 32) {
        key[h] = SK_EMPTY;
        dist[h] = INF;
    }
    __syncwarp();
    if (__ldcg(&a.ctl->err)) return;
    const uint32_t nR1 = a.nR_fixed ? a.nR_fixed : __ldcg(&a.ctl->r_count);
    const uint32_t nitems = a.range_list ? a.ntiles : nR1;
    // telemetry, counted per source in 32-bit registers -- per lane: items scanned, their
    // arcs, arcs of first scans; per warp (every lane the same): rounds, bucket boundaries,
    // SM cycles by phase (32-bit clock differences) -- and added to the warp's 64-bit
    // totals in shared memory when the source ends
    enum { W_SCANS, W_ARCS, W_SLOT_ARCS, W_ROUNDS, W_BOUNDS, W_SLOTS, W_CYC_ROUND, W_CYC_BOUND, W_CYC_EMIT, W_N };
    __shared__ unsigned long long s_tel[src_warps(MS)][W_N];
    __shared__ uint32_t s_max[src_warps(MS)][2];  // largest completed ball, most pairs of a source
    if (lane < W_N) s_tel[warp][lane] = 0;
    if (lane < 2) s_max[warp][lane] = 0;
    __syncwarp();
    const bool kcp = a.kcp_hist != nullptr;
    uint32_t *const slist = a.slist + size_t(blockIdx.x * src_warps(MS) + warp) * MS;
    uint32_t t_mark = uint32_t(clock());

    for (;;) {
        uint32_t item = 0;
        if (lane == 0) item = atomicAdd(&a.ctl->tile_next, 1u);
        item = __shfl_sync(FULL, item, 0);
        if (item >= nitems) break;
        const uint32_t si = a.range_list ? a.range_list[item].x : item;
        if (si >= nR1) continue;  // never past R
        uint32_t bound = a.bound;
        const uint32_t *sbits = a.sbits;
        unsigned long long prefix = 0;
        uint32_t inst = 0;
        if (a.inst_first) {
            // the query whose sources hold si: the last with inst_first <= si
            uint32_t lo = 0, hi = a.inst_count - 1;
            while (lo < hi) {
                const uint32_t mid = (lo + hi + 1) >> 1;
                if (a.inst_first[mid] <= si) lo = mid;
                else hi = mid - 1;
            }
            inst = lo;
            bound = a.inst_bound[lo];
            sbits = a.inst_sbits[lo];
            prefix = (unsigned long long)lo << a.inst_shift;
        }
        uint64_t delta = a.delta;
        if (a.tile_bound) {  // a batch: the source's instance, its bound and bucket width
            inst = a.tile_inst[si];
            bound = a.tile_bound[si];
            delta = a.tile_delta[si];
        }
        const bool swap = a.inst_swap ? a.inst_swap[inst] != 0 : a.swap_uv != 0;
        // k closest pairs: the live k-th distance bound (Algorithm 3's global threshold)
        // caps the source's bound, and is read again at every bucket boundary
        if (kcp) bound = min(bound, __ldcg(a.theta_live));
        const uint32_t y0 = a.src[si];
        if (RN_BAD(y0 < a.n_nodes, 11, si, y0)) continue;
        const unsigned long long u = __ldg(&a.iperm[y0]);
        const uint32_t t_source = uint32_t(clock());
        uint32_t part_lo = 0, part_hi = 0xFFFFFFFFu;  // the hierarchical variant: the source's part
        if (HIER) {
            const uint2 r = a.src_range[si];
            part_lo = r.x;
            part_hi = r.y;
        }
        uint32_t n_scans = 0, n_arcs = 0, n_slot_arcs = 0, n_rounds = 0, n_bounds = 0;
        uint32_t cyc_round = 0, cyc_bound = 0;
        uint32_t n_list = 0;  // S nodes of the ball listed so far (every lane the same)
        // the source, at distance 0, is the only item of the near queue
        if (lane == 0) {
            const uint32_t h = (y0 * 0x9E3779B1u) >> (32 - log2u(MS));
            key[h] = y0 | SK_DIRTY | SK_QUEUED;
            dist[h] = 0;
            qa[0] = h;
        }
        __syncwarp();
        uint32_t *qcur = qa, *qnext = qb;
        uint32_t ncur = 1, fill = 1;
        bool fail = false;
        uint64_t tau = delta < uint64_t(bound) + 1 ? delta : uint64_t(bound) + 1;  // end of the bucket

        // collect: least distance m of the dirty slots; those below lim go to the near
        // queue (as many as fit: the rest stay dirty for the next pass), every other
        // slot loses a stale queued flag (one whose push found the queue full)
        auto collect = [&](uint64_t lim, uint32_t *m) {
            uint32_t nq = 0;
#pragma unroll 4
            for (uint32_t c = 0; c < MS; c += 32) {
                const uint32_t h = c + lane;
                const uint32_t k = key[h];
                const bool dirty = (k & SK_DIRTY) != 0;  // SK_EMPTY carries no flag
                const uint32_t d = dirty ? dist[h] : INF;
                *m = min(*m, d);
                const bool take = dirty && d < lim;
                const uint32_t b = __ballot_sync(FULL, take);
                const uint32_t qi = nq + __popc(b & lt);
                const bool queued = take && qi < QS;
                if (queued) qcur[qi] = h;
                nq += __popc(b);
                const uint32_t nk = queued ? (k | SK_QUEUED) : (k & ~SK_QUEUED);
                if (nk != k) key[h] = nk;
            }
            return nq;
        };

        for (;;) {
            // ---- rounds of the current bucket
            while (ncur && !fail) {
                n_rounds++;
                uint32_t nnext = 0;
                for (uint32_t c0 = 0; c0 < ncur && !fail; c0 += 64) {
                    // step A: items c0 + 2 lane and c0 + 2 lane + 1
                    uint32_t beg[2], deg[2], dv[2], fresh_s[2];
#pragma unroll
                    for (int t = 0; t < 2; t++) {
                        const uint32_t j = c0 + 2 * lane + t;
                        beg[t] = 0;
                        deg[t] = 0;
                        dv[t] = INF;
                        fresh_s[t] = EMPTY;  // the slot, when this is an S node's first scan
                        if (j < ncur) {
                            const uint32_t x = qcur[j];
                            if (!RN_BAD(x < MS, 12, j, x)) {
                                const uint32_t k = key[x];
                                const uint32_t y = k & SK_NODE;
                                if (!RN_BAD(y < a.n_nodes, 13, x, y)) {
                                    dv[t] = dist[x];
                                    beg[t] = __ldg(&a.row_ptr[y]);
                                    deg[t] = __ldg(&a.row_ptr[y + 1]) - beg[t];
                                    uint32_t in_s = k & SK_IN_S;
                                    if (!(k & SK_SEEN)) {  // first scan: S membership, arcs
                                        in_s = ((__ldg(&sbits[y >> 5]) >> (y & 31)) & 1u) ? SK_IN_S : 0u;
                                        n_slot_arcs += deg[t];
                                        if (in_s) fresh_s[t] = x;
                                    }
                                    key[x] = y | SK_SEEN | in_s;
                                    if (RN_BAD(uint64_t(beg[t]) + deg[t] <= a.n_arcs, 14, y, beg[t])) deg[t] = 0;
                                    n_scans++;
                                    n_arcs += deg[t];
                                }
                            }
                        }
                    }
                    // S nodes scanned for the first time join the ball's list (each once:
                    // every node within the bound is scanned, so emission reads the list
                    // instead of the whole map)
#pragma unroll
                    for (int t = 0; t < 2; t++) {
                        const uint32_t fb = __ballot_sync(FULL, fresh_s[t] != EMPTY);
                        const uint32_t at = n_list + __popc(fb & lt);
                        if (fresh_s[t] != EMPTY && at < MS) __stcg(&slist[at], fresh_s[t]);
                        n_list = min(n_list + __popc(fb), MS);  // (a ball never fills its map)
                    }
                    const uint32_t mine = deg[0] + deg[1];
                    uint32_t incl = mine;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const uint32_t t = __shfl_up_sync(FULL, incl, o);
                        if (lane >= uint32_t(o)) incl += t;
                    }
                    const uint32_t total = __shfl_sync(FULL, incl, 31);
                    const uint32_t ex = incl - mine;  // first arc of this lane's items
                    __syncwarp();                     // flags cleared before any relaxation
                    // step B: arcs b0 .. b0 + 127, arc g of lane l's items when
                    // ex[l] <= g < ex[l] + deg[l][0] + deg[l][1] (lanes past the items
                    // have ex = total)
                    const uint32_t tau32 = uint32_t(tau);  // <= bound + 1 <= 2^31 + 1
                    for (uint32_t b0 = 0; b0 < total && !fail; b0 += 32 * AP) {
                        uint32_t y[AP], nd[AP];
#pragma unroll
                        for (int k = 0; k < AP; k++) {
                            const uint32_t gi = b0 + 32 * k + lane;
                            uint32_t l = 0;
#pragma unroll
                            for (uint32_t s = 16; s; s >>= 1)
                                if (__shfl_sync(FULL, ex, l + s) <= gi) l += s;
                            const uint32_t o = gi - __shfl_sync(FULL, ex, l);
                            const uint32_t d0 = __shfl_sync(FULL, deg[0], l);
                            const uint32_t bb0 = __shfl_sync(FULL, beg[0], l);
                            const uint32_t bb1 = __shfl_sync(FULL, beg[1], l);
                            const uint32_t v0 = __shfl_sync(FULL, dv[0], l);
                            const uint32_t v1 = __shfl_sync(FULL, dv[1], l);
                            const bool second = o >= d0;
                            const uint32_t ai = second ? bb1 + (o - d0) : bb0 + o;
                            nd[k] = INF;
                            y[k] = 0;
                            if (gi < total && !RN_BAD(ai < a.n_arcs, 15, gi, ai)) {
                                const uint2 arc = __ldg(&a.adj[ai]);
                                y[k] = arc.x;
                                nd[k] = (second ? v1 : v0) + arc.y;  // <= bound + 2^24: no overflow
                                if (HIER && (arc.x < part_lo || arc.x >= part_hi)) nd[k] = INF;  // leaves the part
                            }
                        }
                        // every first probe, then every atomic, of the batch issued back to back
                        // (their latencies overlap instead of adding up arc after arc)
                        uint32_t h[AP], kv[AP];
#pragma unroll
                        for (int k = 0; k < AP; k++) {
                            if (nd[k] <= bound && RN_BAD(y[k] < a.n_nodes, 16, b0 + 32 * k + lane, y[k])) nd[k] = INF;
                            h[k] = (y[k] * 0x9E3779B1u) >> (32 - log2u(MS));
                            kv[k] = nd[k] <= bound ? ((volatile uint32_t *)key)[h[k]] : 0u;
                        }
                        uint32_t ins_count = 0;
                        bool full = false;
#pragma unroll
                        for (int k = 0; k < AP; k++) {
                            bool ins = false;
                            if (nd[k] > bound) {
                                h[k] = EMPTY;
                            } else if ((kv[k] & SK_NODE) != y[k]) {
                                // the home slot holds another node (keys never leave the map
                                // during a search): probe on from the next slot; it was empty:
                                // probe from it (another lane may have taken it since)
                                const uint32_t h0 = kv[k] == SK_EMPTY ? h[k] : (h[k] + 1) & (MS - 1);
                                h[k] = src_slot<MS>(key, y[k], h0, &ins);
                            }
                            ins_count += ins;
                            full |= nd[k] <= bound && h[k] == EMPTY;
                        }
                        fill += __reduce_add_sync(FULL, ins_count);  // once per batch
                        uint32_t old[AP];
#pragma unroll
                        for (int k = 0; k < AP; k++) old[k] = h[k] != EMPTY ? atomicMin(&dist[h[k]], nd[k]) : 0u;
                        uint32_t kf[AP];
#pragma unroll
                        for (int k = 0; k < AP; k++)
                            kf[k] = h[k] != EMPTY && nd[k] < old[k]
                                        ? atomicOr(&key[h[k]], nd[k] < tau32 ? (SK_DIRTY | SK_QUEUED) : SK_DIRTY)
                                        : SK_QUEUED;
#pragma unroll
                        for (int k = 0; k < AP; k++) {
                            const bool push = h[k] != EMPTY && nd[k] < old[k] && nd[k] < tau32 && !(kf[k] & SK_QUEUED);
                            const uint32_t pb = __ballot_sync(FULL, push);
                            if (push) {
                                const uint32_t qi = nnext + __popc(pb & lt);
                                if (qi < QS) qnext[qi] = h[k];
                            }
                            nnext += __popc(pb);
                        }
                        if (__any_sync(FULL, full) || fill > a.max_fill) fail = true;
                    }
                    __syncwarp();  // this step's relaxations before the next step's scans
                }
                ncur = min(nnext, QS);
                uint32_t *t = qcur;
                qcur = qnext;
                qnext = t;
            }
            {
                const uint32_t t = uint32_t(clock());
                cyc_round += t - t_mark;
                t_mark = t;
            }
            if (fail) break;
            // ---- the near queue is empty: the next bucket
            n_bounds++;
            if (kcp) bound = min(bound, __ldcg(a.theta_live));  // the same for every lane
            const uint64_t top = uint64_t(bound) + 1;
            const uint64_t tau2 = tau + delta < top ? tau + delta : top;
            uint32_t m = INF;
            uint32_t nq = collect(tau2, &m);
            m = __reduce_min_sync(FULL, m);
            // nothing pending within the bound: the search is complete (a bound lowered
            // by k closest pairs leaves dirty slots above it, which are never taken)
            if (m == INF || m > bound) break;
            if (m >= tau2) {
                // no pending slot in the next bucket: skip to the one holding m
                const uint64_t t = (uint64_t(m) / delta + 1) * delta;
                tau = t < top ? t : top;
                uint32_t m2 = INF;
                nq = collect(tau, &m2);
            } else {
                tau = tau2;
            }
            ncur = min(nq, QS);
            __syncwarp();
            {
                const uint32_t t = uint32_t(clock());
                cyc_bound += t - t_mark;
                t_mark = t;
            }
        }

        // ---- emission: every slot of an S node (all lie within the bound), then the map
        // is left clean for the next source
        if (!fail) {
            // the ball's S nodes are the list (a join's all lie within the bound; k closest
            // pairs may have lowered the bound below nodes reached before)
            uint32_t cnt = n_list;
            if (kcp) {
                cnt = 0;
                for (uint32_t i = lane; i - lane < n_list; i += 32) {
                    const bool in = i < n_list && dist[__ldcg(&slist[i])] <= bound;
                    cnt += __popc(__ballot_sync(FULL, in));
                }
            }
            if (HIER) {
                // the routes to the part's border nodes (the inside routes that the search
                // from an exit arc's far end continues)
#pragma unroll 4
                for (uint32_t c = 0; c < MS; c += 32) {
                    const uint32_t kk = key[c + lane];
                    const uint32_t yy = kk & SK_NODE;
                    const bool brd = kk != SK_EMPTY && ((__ldg(&a.border_bits[yy >> 5]) >> (yy & 31)) & 1u);
                    const uint32_t bb = __ballot_sync(FULL, brd);
                    if (!bb) continue;
                    unsigned long long at = 0;
                    if (lane == 0) at = atomicAdd(a.brd_count, (unsigned long long)__popc(bb));
                    at = __shfl_sync(FULL, at, 0) + __popc(bb & lt);
                    if (brd && at < a.brd_cap) {
                        a.brd_key[at] = ((unsigned long long)si << 32) | yy;
                        a.brd_d[at] = dist[c + lane];
                    }
                }
            }
            unsigned long long base = 0;
            if (lane == 0 && cnt) {
                base = atomicAdd(&a.ctl->pairs, (unsigned long long)cnt);
                if (a.inst_pairs) atomicAdd(&a.inst_pairs[inst], (unsigned long long)cnt);
            }
            if (lane == 0 && a.seg) a.seg[si] = make_uint2(uint32_t(base), cnt);
            if (lane == 0) s_max[warp][1] = max(s_max[warp][1], cnt);
            base = __shfl_sync(FULL, base, 0);
            // four chunks of 32 list entries at a time, every output-id load issued before
            // the first write (so their latencies overlap)
            unsigned long long pos = base;
            for (uint32_t i0 = 0; i0 < n_list; i0 += 128) {
                uint32_t dd[4], v[4];
                bool ok[4];
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const uint32_t i = i0 + 32 * q + lane;
                    ok[q] = false;
                    dd[q] = 0;
                    v[q] = 0;
                    if (i < n_list) {
                        const uint32_t h = __ldcg(&slist[i]);
                        const uint32_t y = key[h] & SK_NODE;
                        if (!RN_BAD(h < MS && y < a.n_nodes, 17, h, y)) {
                            dd[q] = dist[h];
                            ok[q] = !kcp || dd[q] <= bound;
                            if (ok[q]) v[q] = __ldg(&a.iperm[y]);
                        }
                    }
                }
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const uint32_t b = __ballot_sync(FULL, ok[q]);
                    if (ok[q]) {
                        const unsigned long long idx = pos + __popc(b & lt);
                        if (idx < a.out_cap) {
                            a.out_key[idx] = prefix | (swap ? ((unsigned long long)v[q] << a.vbits) | u
                                                            : (u << a.vbits) | (unsigned long long)v[q]);
                            a.out_d[idx] = dd[q];
                        }
                        if (kcp) atomicAdd(&a.kcp_hist[dd[q] >> a.hist_shift], 1u);
                    }
                    pos += __popc(b);
                }
            }
            __syncwarp();
            // the map back to empty for the next source, sixteen bytes a store
            for (uint32_t h4 = lane; h4 < MS / 4; h4 += 32) {
                reinterpret_cast<uint4 *>(key)[h4] = make_uint4(SK_EMPTY, SK_EMPTY, SK_EMPTY, SK_EMPTY);
                reinterpret_cast<uint4 *>(dist)[h4] = make_uint4(INF, INF, INF, INF);
            }
            if (kcp && cnt) {
                // the source's pairs are counted: once k pairs exist, lower the live bound
                // to the edge of the first histogram bin where the pairs emitted so far
                // reach k (exact, distinct pairs: the k-th distance cannot lie above it).
                // The warp whose pairs reach k does it, then the warp whose pairs cross
                // each further multiple of k/64 (not every source: each lowering reads the
                // whole histogram)
                const unsigned long long emitted = base + cnt;
                const unsigned long long step = a.kcp_k / 64 + 1;
                if (emitted >= a.kcp_k && (base < a.kcp_k || base / step != emitted / step)) kcp_lower_bound(a, lane);
            }
            if (lane == 0) {
                s_tel[warp][W_SLOTS] += fill;
                s_max[warp][0] = max(s_max[warp][0], fill);
                if (a.inst_ball) atomicMax(&a.inst_ball[inst], fill);
            }
        } else {
            if (lane == 0)
                a.failed[atomicAdd(&a.ctl->n_failed, 1u)] =
                    make_uint4(si, bound, uint32_t(tau < 0xFFFFFFFFull ? tau : 0xFFFFFFFFull), fill);
            for (uint32_t h = lane; h < MS; h += 32) {
                key[h] = SK_EMPTY;
                dist[h] = INF;
            }
        }
        __syncwarp();
        const uint32_t t_end = uint32_t(clock());
        n_scans = __reduce_add_sync(FULL, n_scans);
        n_arcs = __reduce_add_sync(FULL, n_arcs);
        n_slot_arcs = __reduce_add_sync(FULL, n_slot_arcs);
        if (lane == 0) {
            unsigned long long *tel = s_tel[warp];
            tel[W_SCANS] += n_scans;
            tel[W_ARCS] += n_arcs;
            tel[W_SLOT_ARCS] += n_slot_arcs;
            tel[W_ROUNDS] += n_rounds;
            tel[W_BOUNDS] += n_bounds;
            tel[W_CYC_ROUND] += cyc_round;
            tel[W_CYC_BOUND] += cyc_bound;
            tel[W_CYC_EMIT] += t_end - t_mark;
            // a batch: the instance's SM cycles, this warp holding one resident warp's
            // share of its SM
            if (a.inst_cycles)
                atomicAdd(&a.inst_cycles[inst],
                          (unsigned long long)(t_end - t_source) / (src_warps(MS) * SRC_BLOCKS_PER_SM));
        }
        t_mark = t_end;
        __syncwarp();
    }
    if (lane == 0) {
        const unsigned long long *tel = s_tel[warp];
        atomicAdd(&a.ctl->scans, tel[W_SCANS]);
        atomicAdd(&a.ctl->dirty_groups, tel[W_SCANS]);
        atomicAdd(&a.ctl->round_items, tel[W_SCANS]);
        atomicAdd(&a.ctl->round_arcs, tel[W_ARCS]);
        atomicAdd(&a.ctl->slot_arcs, tel[W_SLOT_ARCS]);
        atomicAdd(&a.ctl->slots, tel[W_SLOTS]);
        atomicAdd(&a.ctl->slot_lanes, tel[W_SLOTS]);
        atomicAdd(&a.ctl->rounds, tel[W_ROUNDS]);
        atomicAdd(&a.ctl->boundaries, tel[W_BOUNDS]);
        atomicAdd(&a.ctl->cyc_round, tel[W_CYC_ROUND]);
        atomicAdd(&a.ctl->cyc_bound, tel[W_CYC_BOUND]);
        atomicAdd(&a.ctl->cyc_emit, tel[W_CYC_EMIT]);
        atomicMax(&a.ctl->max_fill, s_max[warp][0]);
        atomicMax(&a.ctl->src_max_ball, s_max[warp][0]);
        atomicMax(&a.ctl->max_seg, s_max[warp][1]);
    }
}

// ---------------------------------------------------- cooperative source search ----
// A source whose ball needs a large warp map (4096 or 8192 slots) leaves a lone warp
// with a map that fills a sixth or a third of an SM's shared memory: three to six warps
// per SM, each walking its round's items alone.  Here W warps share one source's map.
// A round is taken in waves of W x 64 items: every warp scans its 64 (flags cleared,
// distance and CSR range read), a block barrier, every warp relaxes the arcs of its
// items, a barrier -- so no warp clears a slot's flags while another relaxes into it,
// and each wave sees the distances of the waves before it, as the warp search's chunks
// do.  Queue pushes, the fill count and the S-node list go through shared atomics;
// bucket boundaries split the map between the warps.  The protocol and the results
// are the warp search's.
template <uint32_t MS, uint32_t W>
__global__ void __launch_bounds__(W * 32, (3 * 8192) / MS) k_source_coop(SearchArgs a) {
    constexpr uint32_t QS = src_qcap(MS);
    constexpr uint32_t NT = W * 32;
    constexpr int AP = 4;
    extern __shared__ __align__(16) uint32_t smem[];
    // block-wide state of the current source, read by every thread after a barrier
    __shared__ uint32_t s_item, s_ncur, s_nnext, s_fill, s_nlist, s_fail, s_bound, s_min, s_nq, s_cnt, s_stop;
    __shared__ unsigned long long s_base;
    __shared__ uint32_t s_wcnt[W];
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t lt = (1u << lane) - 1;
    uint32_t *key = smem, *dist = smem + MS, *qa = dist + MS, *qb = qa + QS;
    for (uint32_t h = tid; h < MS; h += NT) {
        key[h] = SK_EMPTY;
        dist[h] = INF;
    }
    if (tid == 0) s_stop = __ldcg(&a.ctl->err) != 0;
    __syncthreads();
    if (s_stop) return;
    const uint32_t nR1 = a.nR_fixed ? a.nR_fixed : __ldcg(&a.ctl->r_count);
    const uint32_t nitems = a.range_list ? a.ntiles : nR1;
    const bool kcp = a.kcp_hist != nullptr;
    uint32_t *const slist = a.slist + size_t(blockIdx.x) * MS;
    // telemetry: per lane (scans, arcs, arcs of first scans), then per warp at the end;
    // rounds, boundaries, slots and cycles counted by thread 0
    unsigned long long t_scans = 0, t_arcs = 0, t_slot_arcs = 0;
    unsigned long long t_rounds = 0, t_bounds = 0, t_slots = 0, t_cyc_round = 0, t_cyc_bound = 0, t_cyc_emit = 0;
    uint32_t t_max_ball = 0, t_max_seg = 0;

    for (;;) {
        if (tid == 0) s_item = atomicAdd(&a.ctl->tile_next, 1u);
        __syncthreads();
        const uint32_t item = s_item;
        __syncthreads();  // every thread has read s_item
        if (item >= nitems) break;
        const uint32_t si = a.range_list ? a.range_list[item].x : item;
        if (si >= nR1) continue;  // never past R (the same for every thread)
        uint32_t bound = a.bound;
        const uint32_t *sbits = a.sbits;
        unsigned long long prefix = 0;
        uint32_t inst = 0;
        if (a.inst_first) {
            uint32_t lo = 0, hi = a.inst_count - 1;
            while (lo < hi) {
                const uint32_t mid = (lo + hi + 1) >> 1;
                if (a.inst_first[mid] <= si) lo = mid;
                else hi = mid - 1;
            }
            inst = lo;
            bound = a.inst_bound[lo];
            sbits = a.inst_sbits[lo];
            prefix = (unsigned long long)lo << a.inst_shift;
        }
        uint64_t delta = a.delta;
        if (a.tile_bound) {
            inst = a.tile_inst[si];
            bound = a.tile_bound[si];
            delta = a.tile_delta[si];
        }
        const bool swap = a.inst_swap ? a.inst_swap[inst] != 0 : a.swap_uv != 0;
        const uint32_t y0 = a.src[si];
        if (y0 >= a.n_nodes) {  // (the same for every thread)
            if (tid == 0) record_check(a.ctl, 11, si, y0);
            continue;
        }
        const unsigned long long u = __ldg(&a.iperm[y0]);
        const uint32_t t_source = uint32_t(clock());
        uint32_t t_mark = t_source;
        if (tid == 0) {
            const uint32_t h = (y0 * 0x9E3779B1u) >> (32 - log2u(MS));
            key[h] = y0 | SK_DIRTY | SK_QUEUED;
            dist[h] = 0;
            qa[0] = h;
            s_ncur = 1;
            s_nnext = 0;
            s_fill = 1;
            s_nlist = 0;
            s_fail = 0;
            s_bound = kcp ? min(bound, __ldcg(a.theta_live)) : bound;
        }
        __syncthreads();
        bound = s_bound;  // the k-closest-pairs live bound, read once for the whole block
        uint32_t *qcur = qa, *qnext = qb;
        uint64_t tau = delta < uint64_t(bound) + 1 ? delta : uint64_t(bound) + 1;

        // the dirty slots below lim go to the near queue (as many as fit), every other slot
        // loses a stale queued flag; the least dirty distance goes to s_min.  The callers
        // reset s_nq and s_min and hold a barrier before and after.
        auto collect = [&](uint64_t lim) {
            uint32_t m = INF;
            for (uint32_t h = tid; h < MS; h += NT) {
                const uint32_t k = key[h];
                const bool dirty = (k & SK_DIRTY) != 0;
                const uint32_t d = dirty ? dist[h] : INF;
                m = min(m, d);
                const bool take = dirty && d < lim;
                const uint32_t b = __ballot_sync(FULL, take);
                uint32_t qb0 = 0;
                if (lane == 0 && b) qb0 = atomicAdd(&s_nq, uint32_t(__popc(b)));
                const uint32_t qi = __shfl_sync(FULL, qb0, 0) + __popc(b & lt);
                const bool queued = take && qi < QS;
                if (queued) qcur[qi] = h;
                const uint32_t nk = queued ? (k | SK_QUEUED) : (k & ~SK_QUEUED);
                if (nk != k) key[h] = nk;
            }
            m = __reduce_min_sync(FULL, m);
            if (lane == 0) atomicMin(&s_min, m);
        };

        for (;;) {
            // ---- rounds of the current bucket
            for (;;) {
                const uint32_t ncur = s_ncur;
                if (!ncur || s_fail) break;  // (read after a barrier: the same for every thread)
                t_rounds++;
                const uint32_t tau32 = uint32_t(tau);
                for (uint32_t w0 = 0; w0 < ncur; w0 += W * 64) {
                    // phase A: the wave's items split evenly between the warps (a round
                    // of 72 items gives each of four warps 18, not the first warp 64):
                    // this warp's are j0 + 2 lane + t below j1
                    const uint32_t cw = min(ncur - w0, W * 64), per = (cw + W - 1) / W;
                    const uint32_t j0 = w0 + min(cw, warp * per), j1 = w0 + min(cw, (warp + 1) * per);
                    uint32_t beg[2], deg[2], dv[2], fresh_s[2];
#pragma unroll
                    for (int t = 0; t < 2; t++) {
                        const uint32_t j = j0 + 2 * lane + t;
                        beg[t] = 0;
                        deg[t] = 0;
                        dv[t] = INF;
                        fresh_s[t] = EMPTY;
                        if (j < j1) {
                            const uint32_t x = qcur[j];
                            if (!RN_BAD(x < MS, 12, j, x)) {
                                const uint32_t k = key[x];
                                const uint32_t y = k & SK_NODE;
                                if (!RN_BAD(y < a.n_nodes, 13, x, y)) {
                                    dv[t] = dist[x];
                                    beg[t] = __ldg(&a.row_ptr[y]);
                                    deg[t] = __ldg(&a.row_ptr[y + 1]) - beg[t];
                                    uint32_t in_s = k & SK_IN_S;
                                    if (!(k & SK_SEEN)) {
                                        in_s = ((__ldg(&sbits[y >> 5]) >> (y & 31)) & 1u) ? SK_IN_S : 0u;
                                        t_slot_arcs += deg[t];
                                        if (in_s) fresh_s[t] = x;
                                    }
                                    key[x] = y | SK_SEEN | in_s;
                                    if (RN_BAD(uint64_t(beg[t]) + deg[t] <= a.n_arcs, 14, y, beg[t])) deg[t] = 0;
                                    t_scans++;
                                    t_arcs += deg[t];
                                }
                            }
                        }
                    }
#pragma unroll
                    for (int t = 0; t < 2; t++) {
                        const uint32_t fb = __ballot_sync(FULL, fresh_s[t] != EMPTY);
                        if (fb) {
                            uint32_t lb = 0;
                            if (lane == 0) lb = atomicAdd(&s_nlist, uint32_t(__popc(fb)));
                            const uint32_t at = __shfl_sync(FULL, lb, 0) + __popc(fb & lt);
                            if (fresh_s[t] != EMPTY && at < MS) __stcg(&slist[at], fresh_s[t]);
                        }
                    }
                    __syncthreads();  // every warp's items scanned before any relaxation
                    // phase B: the arcs of this warp's items, 128 at a time
                    const uint32_t mine = deg[0] + deg[1];
                    uint32_t incl = mine;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const uint32_t t = __shfl_up_sync(FULL, incl, o);
                        if (lane >= uint32_t(o)) incl += t;
                    }
                    const uint32_t total = __shfl_sync(FULL, incl, 31);
                    const uint32_t ex = incl - mine;
                    bool wfail = false;
                    for (uint32_t b0 = 0; b0 < total && !wfail; b0 += 32 * AP) {
                        uint32_t y[AP], nd[AP];
#pragma unroll
                        for (int k = 0; k < AP; k++) {
                            const uint32_t gi = b0 + 32 * k + lane;
                            uint32_t l = 0;
#pragma unroll
                            for (uint32_t s = 16; s; s >>= 1)
                                if (__shfl_sync(FULL, ex, l + s) <= gi) l += s;
                            const uint32_t o = gi - __shfl_sync(FULL, ex, l);
                            const uint32_t d0 = __shfl_sync(FULL, deg[0], l);
                            const uint32_t bb0 = __shfl_sync(FULL, beg[0], l);
                            const uint32_t bb1 = __shfl_sync(FULL, beg[1], l);
                            const uint32_t v0 = __shfl_sync(FULL, dv[0], l);
                            const uint32_t v1 = __shfl_sync(FULL, dv[1], l);
                            const bool second = o >= d0;
                            const uint32_t ai = second ? bb1 + (o - d0) : bb0 + o;
                            nd[k] = INF;
                            y[k] = 0;
                            if (gi < total && !RN_BAD(ai < a.n_arcs, 15, gi, ai)) {
                                const uint2 arc = __ldg(&a.adj[ai]);
                                y[k] = arc.x;
                                nd[k] = (second ? v1 : v0) + arc.y;
                            }
                        }
                        uint32_t h[AP], kv[AP];
#pragma unroll
                        for (int k = 0; k < AP; k++) {
                            if (nd[k] <= bound && RN_BAD(y[k] < a.n_nodes, 16, b0 + 32 * k + lane, y[k])) nd[k] = INF;
                            h[k] = (y[k] * 0x9E3779B1u) >> (32 - log2u(MS));
                            kv[k] = nd[k] <= bound ? ((volatile uint32_t *)key)[h[k]] : 0u;
                        }
                        uint32_t ins_count = 0;
                        bool full = false;
#pragma unroll
                        for (int k = 0; k < AP; k++) {
                            bool ins = false;
                            if (nd[k] > bound) {
                                h[k] = EMPTY;
                            } else if ((kv[k] & SK_NODE) != y[k]) {
                                const uint32_t h0 = kv[k] == SK_EMPTY ? h[k] : (h[k] + 1) & (MS - 1);
                                h[k] = src_slot<MS>(key, y[k], h0, &ins);
                            }
                            ins_count += ins;
                            full |= nd[k] <= bound && h[k] == EMPTY;
                        }
                        const uint32_t ins_tot = __reduce_add_sync(FULL, ins_count);
                        uint32_t fnow = 0;
                        if (lane == 0) fnow = ins_tot ? atomicAdd(&s_fill, ins_tot) + ins_tot : *(volatile uint32_t *)&s_fill;
                        fnow = __shfl_sync(FULL, fnow, 0);
                        uint32_t old[AP];
#pragma unroll
                        for (int k = 0; k < AP; k++) old[k] = h[k] != EMPTY ? atomicMin(&dist[h[k]], nd[k]) : 0u;
                        uint32_t kf[AP];
#pragma unroll
                        for (int k = 0; k < AP; k++)
                            kf[k] = h[k] != EMPTY && nd[k] < old[k]
                                        ? atomicOr(&key[h[k]], nd[k] < tau32 ? (SK_DIRTY | SK_QUEUED) : SK_DIRTY)
                                        : SK_QUEUED;
#pragma unroll
                        for (int k = 0; k < AP; k++) {
                            const bool push = h[k] != EMPTY && nd[k] < old[k] && nd[k] < tau32 && !(kf[k] & SK_QUEUED);
                            const uint32_t pb = __ballot_sync(FULL, push);
                            if (pb) {
                                uint32_t pbase = 0;
                                if (lane == 0) pbase = atomicAdd(&s_nnext, uint32_t(__popc(pb)));
                                const uint32_t qi = __shfl_sync(FULL, pbase, 0) + __popc(pb & lt);
                                if (push && qi < QS) qnext[qi] = h[k];
                            }
                        }
                        if (__any_sync(FULL, full) || fnow > a.max_fill) {
                            wfail = true;
                            if (lane == 0) s_fail = 1;
                        }
                    }
                    __syncthreads();  // this wave's relaxations before the next wave's scans
                }
                if (tid == 0) {
                    s_ncur = min(s_nnext, QS);
                    s_nnext = 0;
                }
                uint32_t *t = qcur;
                qcur = qnext;
                qnext = t;
                __syncthreads();
            }
            {
                const uint32_t t = uint32_t(clock());
                t_cyc_round += t - t_mark;
                t_mark = t;
            }
            if (s_fail) break;
            // ---- the near queue is empty: the next bucket
            t_bounds++;
            if (tid == 0) {
                if (kcp) s_bound = min(s_bound, __ldcg(a.theta_live));
                s_nq = 0;
                s_min = INF;
            }
            __syncthreads();
            bound = s_bound;
            const uint64_t top = uint64_t(bound) + 1;
            const uint64_t tau2 = tau + delta < top ? tau + delta : top;
            collect(tau2);
            __syncthreads();
            const uint32_t m = s_min;
            uint32_t nq = s_nq;
            if (m == INF || m > bound) break;
            if (m >= tau2) {
                const uint64_t t = (uint64_t(m) / delta + 1) * delta;
                tau = t < top ? t : top;
                __syncthreads();  // every thread has read s_nq and s_min
                if (tid == 0) {
                    s_nq = 0;
                    s_min = INF;
                }
                __syncthreads();
                collect(tau);
                __syncthreads();
                nq = s_nq;
            } else {
                tau = tau2;
            }
            __syncthreads();  // every thread has read the boundary's results
            if (tid == 0) s_ncur = min(nq, QS);
            __syncthreads();
            {
                const uint32_t t = uint32_t(clock());
                t_cyc_bound += t - t_mark;
                t_mark = t;
            }
        }
        __syncthreads();  // the last boundary's (or round's) reads of shared state are done

        const uint32_t fill = s_fill;
        if (!s_fail) {
            const uint32_t n_list = min(s_nlist, MS);
            // the pairs: the listed S nodes (k closest pairs: those within the lowered bound);
            // warp w writes list entries [w per, (w + 1) per)
            const uint32_t per = (n_list + W - 1) / W;
            const uint32_t lo = min(n_list, warp * per), hi = min(n_list, lo + per);
            uint32_t wc = hi - lo;
            if (kcp) {
                wc = 0;
                for (uint32_t i = lo + lane; i - lane < hi; i += 32) {
                    const bool in = i < hi && dist[__ldcg(&slist[i]) & (MS - 1)] <= bound;
                    wc += __popc(__ballot_sync(FULL, in));
                }
            }
            if (lane == 0) s_wcnt[warp] = wc;
            __syncthreads();
            uint32_t cnt = 0, before = 0;
#pragma unroll
            for (uint32_t w = 0; w < W; w++) {
                if (w < warp) before += s_wcnt[w];
                cnt += s_wcnt[w];
            }
            if (tid == 0) {
                unsigned long long b = 0;
                if (cnt) {
                    b = atomicAdd(&a.ctl->pairs, (unsigned long long)cnt);
                    if (a.inst_pairs) atomicAdd(&a.inst_pairs[inst], (unsigned long long)cnt);
                }
                s_base = b;
                if (a.seg) a.seg[si] = make_uint2(uint32_t(b), cnt);
                t_max_seg = max(t_max_seg, cnt);
            }
            __syncthreads();
            unsigned long long pos = s_base + before;
            for (uint32_t i0 = lo; i0 < hi; i0 += 32) {
                const uint32_t i = i0 + lane;
                bool ok = false;
                uint32_t dd = 0, v = 0;
                if (i < hi) {
                    const uint32_t h = __ldcg(&slist[i]);
                    const uint32_t y = key[h & (MS - 1)] & SK_NODE;
                    if (!RN_BAD(h < MS && y < a.n_nodes, 17, h, y)) {
                        dd = dist[h & (MS - 1)];
                        ok = !kcp || dd <= bound;
                        if (ok) v = __ldg(&a.iperm[y]);
                    }
                }
                const uint32_t b = __ballot_sync(FULL, ok);
                if (ok) {
                    const unsigned long long idx = pos + __popc(b & lt);
                    if (idx < a.out_cap) {
                        a.out_key[idx] = prefix | (swap ? ((unsigned long long)v << a.vbits) | u
                                                        : (u << a.vbits) | (unsigned long long)v);
                        a.out_d[idx] = dd;
                    }
                    if (kcp) atomicAdd(&a.kcp_hist[dd >> a.hist_shift], 1u);
                }
                pos += __popc(b);
            }
            __syncthreads();  // the list and the map read before the map is cleared
            for (uint32_t h4 = tid; h4 < MS / 4; h4 += NT) {
                reinterpret_cast<uint4 *>(key)[h4] = make_uint4(SK_EMPTY, SK_EMPTY, SK_EMPTY, SK_EMPTY);
                reinterpret_cast<uint4 *>(dist)[h4] = make_uint4(INF, INF, INF, INF);
            }
            if (kcp && cnt && warp == 0) {
                const unsigned long long emitted = s_base + cnt;
                const unsigned long long step = a.kcp_k / 64 + 1;
                if (emitted >= a.kcp_k && (s_base < a.kcp_k || s_base / step != emitted / step)) kcp_lower_bound(a, lane);
            }
            if (tid == 0) {
                t_slots += fill;
                t_max_ball = max(t_max_ball, fill);
                if (a.inst_ball) atomicMax(&a.inst_ball[inst], fill);
            }
        } else {
            if (tid == 0)
                a.failed[atomicAdd(&a.ctl->n_failed, 1u)] =
                    make_uint4(si, bound, uint32_t(tau < 0xFFFFFFFFull ? tau : 0xFFFFFFFFull), fill);
            for (uint32_t h = tid; h < MS; h += NT) {
                key[h] = SK_EMPTY;
                dist[h] = INF;
            }
        }
        __syncthreads();  // the map is empty before the next source
        const uint32_t t_end = uint32_t(clock());
        t_cyc_emit += t_end - t_mark;
        if (tid == 0 && a.inst_cycles)
            atomicAdd(&a.inst_cycles[inst], (unsigned long long)(t_end - t_source) / ((3 * 8192) / MS));
    }
    // telemetry: lane sums per warp, the rest from thread 0
    const unsigned long long ws_ = warp_sum64(t_scans), wa_ = warp_sum64(t_arcs), wsa_ = warp_sum64(t_slot_arcs);
    if (lane == 0) {
        atomicAdd(&a.ctl->scans, ws_);
        atomicAdd(&a.ctl->dirty_groups, ws_);
        atomicAdd(&a.ctl->round_items, ws_);
        atomicAdd(&a.ctl->round_arcs, wa_);
        atomicAdd(&a.ctl->slot_arcs, wsa_);
    }
    if (tid == 0) {
        atomicAdd(&a.ctl->slots, t_slots);
        atomicAdd(&a.ctl->slot_lanes, t_slots);
        atomicAdd(&a.ctl->rounds, t_rounds);
        atomicAdd(&a.ctl->boundaries, t_bounds);
        atomicAdd(&a.ctl->cyc_round, t_cyc_round);
        atomicAdd(&a.ctl->cyc_bound, t_cyc_bound);
        atomicAdd(&a.ctl->cyc_emit, t_cyc_emit);
        atomicMax(&a.ctl->max_fill, t_max_ball);
        atomicMax(&a.ctl->src_max_ball, t_max_ball);
        atomicMax(&a.ctl->max_seg, t_max_seg);
    }
}

// ------------------------------------------------- order without a sort ----
// The warp search writes every source's pairs contiguously (seg[si] = first pair, count);
// with the sources in increasing original id, the (u, v) order is the sources' segments
// one after another, each sorted by v.  So a join's canonical order (Section 4's result
// sorted by (u, v)) needs a scan of the counts and one placement pass, in which a warp
// sorts one segment of up to 256 pairs in registers (bitonic network) and writes it.

__global__ void k_seg_counts(const uint2 *__restrict__ seg, uint32_t n, uint32_t *cnt) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) cnt[i] = seg[i].y;
}

// Ascending bitonic sort of the warp's 32 E values, element lane * E + e in x[e].
template <int E>
__device__ __forceinline__ void warp_bitonic(unsigned long long (&x)[E], uint32_t lane) {
#pragma unroll
    for (uint32_t k = 2; k <= 32u * E; k <<= 1) {
#pragma unroll
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
            if (j >= uint32_t(E)) {  // partner in lane ^ (j / E), same register
                const uint32_t lj = j / E;
                const bool lower = (lane & lj) == 0;
#pragma unroll
                for (int e = 0; e < E; e++) {
                    const unsigned long long p = __shfl_xor_sync(FULL, x[e], lj);
                    const bool up = ((lane * E + e) & k) == 0;
                    x[e] = (lower == up) ? (x[e] < p ? x[e] : p) : (x[e] < p ? p : x[e]);
                }
            } else {  // partner in this lane, register e ^ j
#pragma unroll
                for (int e = 0; e < E; e++) {
                    if ((e & j) == 0) {
                        const bool up = ((lane * E + e) & k) == 0;
                        const unsigned long long lo = x[e], hi = x[e ^ j];
                        if ((lo > hi) == up) {
                            x[e] = hi;
                            x[e ^ j] = lo;
                        }
                    }
                }
            }
        }
    }
}

template <int E>
__device__ __forceinline__ void place_segment(uint32_t lane, uint32_t base, uint32_t cnt, uint32_t o, uint32_t u,
                                              const unsigned long long *__restrict__ key,
                                              const uint32_t *__restrict__ val, unsigned long long vmask,
                                              uint32_t *out_u, uint32_t *out_v, uint32_t *out_d,
                                              unsigned long long *out_key, uint32_t *out_val) {
    unsigned long long x[E];
#pragma unroll
    for (int e = 0; e < E; e++) {
        const uint32_t i = lane * E + e;
        x[e] = i < cnt ? ((key[base + i] & vmask) << 32) | val[base + i] : ~0ull;  // v, then d
    }
    warp_bitonic<E>(x, lane);
    if (out_key) {  // records (key, distance) for a sort that follows
        const unsigned long long khi = key[base] & ~vmask;
#pragma unroll
        for (int e = 0; e < E; e++) {
            const uint32_t i = lane * E + e;
            if (i < cnt) {
                out_key[o + i] = khi | (x[e] >> 32);
                out_val[o + i] = uint32_t(x[e]);
            }
        }
        return;
    }
#pragma unroll
    for (int e = 0; e < E; e++) {
        const uint32_t i = lane * E + e;
        if (i < cnt) {
            out_u[o + i] = u;
            out_v[o + i] = uint32_t(x[e] >> 32);
            out_d[o + i] = uint32_t(x[e]);
        }
    }
}

// One warp per source: its segment, sorted by v, at its offset off[si] of the result
// (u, v, d arrays; or, when out_key is given, (key, d) records).
__global__ void k_place(const uint2 *__restrict__ seg, const uint32_t *__restrict__ off, uint32_t n,
                        const unsigned long long *__restrict__ key, const uint32_t *__restrict__ val, uint32_t vbits,
                        uint32_t umask, uint32_t *out_u, uint32_t *out_v, uint32_t *out_d,
                        unsigned long long *out_key = nullptr, uint32_t *out_val = nullptr) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t warps = gridDim.x * (blockDim.x / 32);
    const unsigned long long vmask = (1ull << vbits) - 1;
    for (uint32_t si = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); si < n; si += warps) {
        const uint2 sg = seg[si];
        const uint32_t cnt = sg.y;
        if (!cnt) continue;
        const uint32_t u = uint32_t(key[sg.x] >> vbits) & umask;
        const uint32_t o = off[si];
        if (cnt <= 32) place_segment<1>(lane, sg.x, cnt, o, u, key, val, vmask, out_u, out_v, out_d, out_key, out_val);
        else if (cnt <= 64) place_segment<2>(lane, sg.x, cnt, o, u, key, val, vmask, out_u, out_v, out_d, out_key, out_val);
        else if (cnt <= 128) place_segment<4>(lane, sg.x, cnt, o, u, key, val, vmask, out_u, out_v, out_d, out_key, out_val);
        else place_segment<8>(lane, sg.x, cnt, o, u, key, val, vmask, out_u, out_v, out_d, out_key, out_val);
    }
}

// Replace the original ids of list[0, min(cap, r_count)) by internal ids.
__global__ void k_to_internal(uint32_t *list, uint32_t cap, const uint32_t *__restrict__ perm,
                              const Control *__restrict__ ctl) {
    const uint32_t n = min(cap, ctl->r_count);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) list[i] = perm[list[i]];
}

constexpr uint32_t PLACE_MAX = 256;  // longest segment k_place sorts

// ------------------------------------------------------------- radix sort ----
// LSD radix sort of (64-bit key, 32-bit value) records, 8 bits per pass.  Stable within
// a pass: a block's 2048 records are ranked warp by warp and round by round.

constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ROUNDS = 8;
constexpr int RS_TILE = RS_THREADS * RS_ROUNDS;

__device__ __forceinline__ uint32_t rs_digit(unsigned long long k, uint32_t v, int shift) {
    // shift < 64: bits of the key; shift >= 64: bits of the value
    return shift < 64 ? uint32_t(k >> shift) & 0xFFu : (v >> (shift - 64)) & 0xFFu;
}

__global__ void k_rs_hist(const unsigned long long *__restrict__ keys, const uint32_t *__restrict__ vals,
                          uint64_t n, int shift, uint32_t *hist, uint32_t nblocks) {
    __shared__ uint32_t cnt[256];
    for (int i = threadIdx.x; i < 256; i += RS_THREADS) cnt[i] = 0;
    __syncthreads();
    const uint64_t base = uint64_t(blockIdx.x) * RS_TILE;
    for (int r = 0; r < RS_ROUNDS; r++) {
        const uint64_t i = base + uint64_t(r) * RS_THREADS + threadIdx.x;
        if (i < n) atomicAdd(&cnt[rs_digit(keys[i], vals[i], shift)], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += RS_THREADS) hist[uint64_t(d) * nblocks + blockIdx.x] = cnt[d];
}

// Exclusive scan of hist[0..total) in place, one block of 1024 threads: each warp owns a
// contiguous chunk; it sums the chunk with coalesced loads, the block scans the 32 warp
// sums, then each warp rewrites its chunk 32 entries at a time with a warp scan.
__global__ void k_rs_scan(uint32_t *hist, uint32_t total) {
    __shared__ uint32_t warp_sum[32];
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t chunk = ((total + 31) / 32 + 31) & ~31u;  // multiple of 32
    const uint32_t lo = min(total, warp * chunk), hi = min(total, lo + chunk);
    uint32_t s = 0;
#pragma unroll 8
    for (uint32_t i = lo + lane; i < hi; i += 32) s += hist[i];
    s = __reduce_add_sync(FULL, s);
    if (lane == 0) warp_sum[warp] = s;
    __syncthreads();
    if (warp == 0) {
        const uint32_t v = warp_sum[lane];
        uint32_t x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(FULL, x, o);
            if (lane >= uint32_t(o)) x += t;
        }
        warp_sum[lane] = x - v;
    }
    __syncthreads();
    uint32_t carry = warp_sum[warp];
    for (uint32_t i = lo; i < hi; i += 32) {
        const uint32_t v = i + lane < hi ? hist[i + lane] : 0;
        uint32_t x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(FULL, x, o);
            if (lane >= uint32_t(o)) x += t;
        }
        if (i + lane < hi) hist[i + lane] = carry + x - v;
        carry += __shfl_sync(FULL, x, 31);
    }
}

// Large histograms are scanned by many blocks: each block scans a chunk of SCAN_CHUNK
// entries in place and leaves the chunk's total, one block scans the totals, and every
// chunk adds its offset.  A histogram buffer of n entries holds the chunk totals after
// them (hist_words gives the size).
constexpr uint32_t SCAN_CHUNK = 8192;  // 1024 threads x 8 entries
__host__ __device__ constexpr uint64_t hist_words(uint64_t entries) {
    return entries + (entries + SCAN_CHUNK - 1) / SCAN_CHUNK + 64;
}

__global__ void __launch_bounds__(1024) k_scan_chunks(uint32_t *a, uint32_t total, uint32_t *sums) {
    __shared__ uint32_t warp_sum[32];
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t base = blockIdx.x * SCAN_CHUNK + threadIdx.x * 8;
    uint32_t v[8], s = 0;
#pragma unroll
    for (int k = 0; k < 8; k++) {
        v[k] = base + k < total ? a[base + k] : 0u;
        s += v[k];
    }
    uint32_t x = s;  // inclusive scan of the threads' sums over the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(FULL, x, o);
        if (lane >= uint32_t(o)) x += t;
    }
    if (lane == 31) warp_sum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        const uint32_t wv = warp_sum[lane];
        uint32_t y = wv;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(FULL, y, o);
            if (lane >= uint32_t(o)) y += t;
        }
        warp_sum[lane] = y - wv;
    }
    __syncthreads();
    uint32_t run = warp_sum[warp] + x - s;
#pragma unroll
    for (int k = 0; k < 8; k++) {
        if (base + k < total) a[base + k] = run;
        run += v[k];
    }
    if (threadIdx.x == 1023) sums[blockIdx.x] = run;
}

__global__ void __launch_bounds__(1024) k_scan_add(uint32_t *a, uint32_t total, const uint32_t *__restrict__ sums) {
    const uint32_t add = sums[blockIdx.x];
    const uint32_t base = blockIdx.x * SCAN_CHUNK + threadIdx.x * 8;
#pragma unroll
    for (int k = 0; k < 8; k++)
        if (base + k < total) a[base + k] += add;
}

// Exclusive scan of hist[0, total) in place; hist holds hist_words(total) entries.
// Returns the kernels launched.
static uint32_t scan_hist(uint32_t *hist, uint32_t total, cudaStream_t st) {
    if (total <= 2 * SCAN_CHUNK) {
        k_rs_scan<<<1, 1024, 0, st>>>(hist, total);
        return 1;
    }
    const uint32_t nb = (total + SCAN_CHUNK - 1) / SCAN_CHUNK;
    uint32_t *sums = hist + total;
    k_scan_chunks<<<nb, 1024, 0, st>>>(hist, total, sums);
    k_rs_scan<<<1, 1024, 0, st>>>(sums, nb);
    k_scan_add<<<nb, 1024, 0, st>>>(hist, total, sums);
    return 3;
}

// Scatter pass.  With out_u != null the pass is the last one of a join sort and writes
// the struct-of-arrays result (u = key >> vbits, v = key & mask, d = value) directly.
__global__ void k_rs_scatter(const unsigned long long *__restrict__ kin, const uint32_t *__restrict__ vin,
                             unsigned long long *kout, uint32_t *vout, uint64_t n, int shift,
                             const uint32_t *__restrict__ hist, uint32_t nblocks, uint32_t *out_u,
                             uint32_t *out_v, uint32_t *out_d, uint32_t vbits, uint32_t umask = 0xFFFFFFFFu) {
    __shared__ uint32_t wcnt[RS_WARPS][256];
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < RS_WARPS * 256; i += RS_THREADS) (&wcnt[0][0])[i] = 0;
    __syncthreads();
    const uint64_t base = uint64_t(blockIdx.x) * RS_TILE + uint64_t(warp) * (RS_ROUNDS * 32);
    unsigned long long k[RS_ROUNDS];
    uint32_t v[RS_ROUNDS], dg[RS_ROUNDS], rank[RS_ROUNDS];
    const uint32_t lt = (1u << lane) - 1;
#pragma unroll
    for (int r = 0; r < RS_ROUNDS; r++) {
        const uint64_t i = base + uint64_t(r) * 32 + lane;
        const bool valid = i < n;
        k[r] = valid ? kin[i] : 0ull;
        v[r] = valid ? vin[i] : 0u;
        dg[r] = valid ? rs_digit(k[r], v[r], shift) : 256u;
        const uint32_t peers = __match_any_sync(FULL, dg[r]);
        const uint32_t before = valid ? wcnt[warp][dg[r]] : 0u;
        __syncwarp();
        rank[r] = before + __popc(peers & lt);
        if (valid && (peers & lt) == 0) wcnt[warp][dg[r]] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += RS_THREADS) {
        uint32_t run = 0;
        for (int w = 0; w < RS_WARPS; w++) {
            const uint32_t c = wcnt[w][d];
            wcnt[w][d] = run;
            run += c;
        }
    }
    __syncthreads();
    const unsigned long long vmask = (1ull << vbits) - 1;
#pragma unroll
    for (int r = 0; r < RS_ROUNDS; r++) {
        if (dg[r] == 256u) continue;
        const uint64_t pos = uint64_t(hist[uint64_t(dg[r]) * nblocks + blockIdx.x]) + wcnt[warp][dg[r]] + rank[r];
        if (out_u) {
            out_u[pos] = uint32_t(k[r] >> vbits) & umask;
            out_v[pos] = uint32_t(k[r] & vmask);
            out_d[pos] = v[r];
        } else {
            kout[pos] = k[r];
            vout[pos] = v[r];
        }
    }
}

// Sort n (key, value) records by the listed digit shifts (least significant first; a
// shift >= 64 takes the value's bits), passing between (k0, v0) and (k1, v1); returns the
// pair of buffers that holds the sorted records.
static std::pair<unsigned long long *, uint32_t *> sort_kv(Workspace *ws, unsigned long long *k0, uint32_t *v0,
                                                           unsigned long long *k1, uint32_t *v1, uint64_t n,
                                                           const std::vector<int> &shifts, cudaStream_t st) {
    if (n == 0) return {k0, v0};
    if (n > 0xFFFFFFFFull) fail(RN_EINVAL, "more than 2^32 - 1 records to sort");
    const uint32_t nblocks = uint32_t((n + RS_TILE - 1) / RS_TILE);
    grow(ws, &ws->hist, &ws->hist_cap, hist_words(uint64_t(nblocks) * 256), 4);
    for (int sh : shifts) {
        k_rs_hist<<<nblocks, RS_THREADS, 0, st>>>(k0, v0, n, sh, ws->hist, nblocks);
        ws->launches += scan_hist(ws->hist, nblocks * 256, st) + 2;
        k_rs_scatter<<<nblocks, RS_THREADS, 0, st>>>(k0, v0, k1, v1, n, sh, ws->hist, nblocks, nullptr, nullptr,
                                                     nullptr, 32);
        std::swap(k0, k1);
        std::swap(v0, v1);
    }
    RN_CUDA(cudaGetLastError());
    return {k0, v0};
}

// Sort n records in (keyA, valA) by the listed digit shifts (least significant first);
// the last pass writes the struct-of-arrays result into out.
static void radix_sort_to_pairs(Workspace *ws, uint64_t n, const std::vector<int> &shifts,
                                uint32_t vbits, rn_dpairs *out, cudaStream_t st, uint32_t umask = 0xFFFFFFFFu) {
    if (n == 0) return;
    if (n > 0xFFFFFFFFull) fail(RN_EINVAL, "more than 2^32 - 1 result pairs");
    const uint32_t nblocks = uint32_t((n + RS_TILE - 1) / RS_TILE);
    grow(ws, &ws->hist, &ws->hist_cap, hist_words(uint64_t(nblocks) * 256), 4);
    unsigned long long *ki = ws->keyA, *ko = ws->keyB;
    uint32_t *vi = ws->valA, *vo = ws->valB;
    for (size_t p = 0; p < shifts.size(); p++) {
        const bool last = p + 1 == shifts.size();
        k_rs_hist<<<nblocks, RS_THREADS, 0, st>>>(ki, vi, n, shifts[p], ws->hist, nblocks);
        ws->launches += scan_hist(ws->hist, nblocks * 256, st) - 1;
        k_rs_scatter<<<nblocks, RS_THREADS, 0, st>>>(ki, vi, ko, vo, n, shifts[p], ws->hist, nblocks,
                                                     last ? out->u : nullptr, last ? out->v : nullptr,
                                                     last ? out->d : nullptr, vbits, umask);
        std::swap(ki, ko);
        std::swap(vi, vo);
        ws->launches += 3;
    }
    RN_CUDA(cudaGetLastError());
}

// ------------------------------------------------------------ orchestration ----

static uint32_t bits_for(uint32_t n) {
    uint32_t b = 1;
    while (b < 32 && (1ull << b) < n) b++;
    return b;
}

// Dynamic shared memory of a search block: the slot map (node, prio, dmask) unless it
// lives in global memory, the two near queues and the staged items.
static size_t search_smem(uint32_t H, bool gmap, int threads) {
    return (gmap ? 0 : size_t(H) * 12) + size_t(qcap_of(threads)) * 8 + size_t(icap_of(threads)) * 20;
}

// A kernel's attributes (its dynamic shared-memory limit, the carveout) belong to the
// device that was current when they were set, so every kernel sets them once per device.
constexpr int MAX_DEVICES = 64;
static int attr_device() {
    int d = 0;
    RN_CUDA(cudaGetDevice(&d));
    if (d < 0 || d >= MAX_DEVICES) fail(RN_EINVAL, "device ordinal out of range");
    return d;
}

template <int L, bool GMAP, int THREADS>
static void launch_search(const SearchArgs &a, uint32_t grid, cudaStream_t st) {
    const size_t smem = search_smem(a.H, GMAP, THREADS);
    static std::once_flag once[MAX_DEVICES];
    std::call_once(once[attr_device()], [&] {
        RN_CUDA(cudaFuncSetAttribute(k_tile_search<L, GMAP, THREADS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     int(search_smem(THREADS == NARROW ? SMEM_H : SMEM_HW, GMAP, THREADS))));
        RN_CUDA(cudaFuncSetAttribute(k_tile_search<L, GMAP, THREADS>,
                                     cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    });
    k_tile_search<L, GMAP, THREADS><<<grid, THREADS, smem, st>>>(a);
    RN_CUDA(cudaGetLastError());
}

template <int L>
static int search_occupancy() {
    int b = 0;
    RN_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_tile_search<L, false, NARROW>, NARROW,
                                                          search_smem(SMEM_H, false, NARROW)));
    return b;
}

enum class Shape { Narrow, Wide, WideGlobal };

static void search(uint32_t T, Shape shape, const SearchArgs &a, uint32_t grid, cudaStream_t st) {
    const int L = int(T / 32);
    if (T != 32 && T != 64 && T != 128) fail(RN_EINVAL, "tile width must be 32, 64 or 128");
    switch (shape) {
        case Shape::Narrow:
            if (L == 1) launch_search<1, false, NARROW>(a, grid, st);
            else if (L == 2) launch_search<2, false, NARROW>(a, grid, st);
            else launch_search<4, false, NARROW>(a, grid, st);
            break;
        case Shape::Wide:
            if (L == 1) launch_search<1, false, WIDE>(a, grid, st);
            else if (L == 2) launch_search<2, false, WIDE>(a, grid, st);
            else launch_search<4, false, WIDE>(a, grid, st);
            break;
        case Shape::WideGlobal:
            if (L == 1) launch_search<1, true, WIDE>(a, grid, st);
            else if (L == 2) launch_search<2, true, WIDE>(a, grid, st);
            else launch_search<4, true, WIDE>(a, grid, st);
            break;
    }
}

static Control read_control(Workspace *ws, cudaStream_t st) {
    RN_CUDA(cudaMemcpyAsync(ws->ctl_host, ws->ctl, sizeof(Control), cudaMemcpyDeviceToHost, st));
    RN_CUDA(cudaStreamSynchronize(st));
    return *ws->ctl_host;
}

// Slots of the first map of a search: 8192 (narrow blocks, shared memory), 16384 (wide
// blocks, shared memory) or a larger power of two (global memory), never more than the
// largest map the graph can need.
static uint64_t first_map(uint32_t want, uint64_t hcap) {
    if (want <= SMEM_H) return SMEM_H;
    uint64_t H = 1;
    while (H < want) H <<= 1;
    H = std::min<uint64_t>(H, hcap);
    return H <= SMEM_HW ? SMEM_HW : H;
}

// One launch with global-memory slot maps of H slots over n tiles (tile_list, or all).
// The maps and slab regions come from the device's retry buffer, or from the
// workspace's own buffer when it has one (a batch, whose captured CUDA graph must keep
// its addresses).
static void launch_gmap(const DeviceGraph &g, Workspace *ws, uint32_t T, SearchArgs r, uint64_t H, uint32_t n,
                        cudaStream_t st) {
    (void)g;
    const size_t per_block = (3 * H + H * T) * 4;
    const size_t budget = size_t(8) << 30;
    const uint32_t rgrid = uint32_t(std::max<size_t>(
        1, std::min<size_t>({size_t(n), size_t(ws->num_sms), size_t(ws->sh->slab_ctas), budget / per_block})));
    uint32_t **buf = ws->own_gmap_enabled ? &ws->own_gmap : &ws->sh->gretry;
    size_t *bytes = ws->own_gmap_enabled ? &ws->own_gmap_bytes : &ws->sh->gretry_bytes;
    if (*bytes < per_block * rgrid) {
        // grow with room to spare: freeing device memory synchronises the whole device
        const size_t want = std::max(per_block * rgrid, std::min(*bytes * 2, budget));
        device_free(*buf);
        *buf = nullptr;
        *bytes = 0;
        *buf = (uint32_t *)device_alloc(want);
        *bytes = want;
        ws->own_gmap_moved = true;
    }
    RN_CUDA(cudaMemsetAsync(*buf, 0xFF, per_block * rgrid, st));  // rows INF
    r.gmap = *buf;
    r.slab = *buf + size_t(rgrid) * 3 * H;
    r.H = uint32_t(H);
    r.hshift = 32 - bits_for(uint32_t(H));
    r.max_fill = uint32_t(H * 7 / 8);
    search(T, Shape::WideGlobal, r, rgrid, st);
}

// Search every tile with the first map (by default narrow blocks: 8192-slot shared
// maps, two per SM), then search again the source ranges whose union ball overflowed.
// An overflowed range reports the bucket end tau it reached and its fill; in a road
// network a ball grows about as the square of its radius, so its whole union ball is
// estimated as fill * (bound / tau)^2.  A range whose sources lie far apart in the
// locality order (balls nearly disjoint: a sparse R on a large graph) is cut once into
// as many parts as that estimate asks, each searched again with the same shared map.
// A range of nearby sources (overlapping balls, which cutting would not shrink), and
// every part that still overflows, goes to the map its estimate fits (wide blocks with
// 16384-slot shared maps, else a global map), growing four times on each further
// overflow.  The map never needs more than the next power of two >= 2n slots, where it
// cannot overflow.
constexpr uint32_t SPARSE_GAP = 2048;  // mean internal-id gap of sources with disjoint balls

static void ensure_ranges(uint4 **p, uint32_t *cap, uint32_t want) {
    if (*p && *cap >= want) return;
    device_free(*p);
    *p = nullptr;
    *cap = std::max<uint32_t>(want, 1024);
    *p = (uint4 *)device_alloc(size_t(*cap) * 16);
}

static std::vector<uint4> read_ranges(const uint4 *d, uint32_t n, cudaStream_t st) {
    std::vector<uint4> h(n);
    if (n) {
        RN_CUDA(cudaMemcpyAsync(h.data(), d, size_t(n) * 16, cudaMemcpyDeviceToHost, st));
        RN_CUDA(cudaStreamSynchronize(st));
    }
    return h;
}

// Slots a map needs for an estimated ball: room to spare below its 7/8 fill limit.
static uint64_t map_for(uint64_t ball, uint64_t hcap) {
    const uint64_t need = ball + ball / 7 + ball / 4 + 1;
    if (need <= SMEM_H) return SMEM_H;
    if (need <= SMEM_HW) return SMEM_HW;
    uint64_t H = SMEM_HW * 2;
    while (H < need && H < hcap) H <<= 1;
    return std::min(H, hcap);
}

static Control search_all(const DeviceGraph &g, Workspace *ws, uint32_t T, SearchArgs a,
                          uint32_t ntiles, cudaStream_t st, uint64_t *retried, uint32_t map_slots = 0,
                          bool split = true, const std::vector<uint4> *first_ranges = nullptr,
                          bool timed = true) {
    // narrow blocks: one slab region each; wide blocks: two regions each
    const uint32_t grid_max = ws->sh->slab_ctas;
    const uint32_t grid_wide = std::max<uint32_t>(1, std::min<uint32_t>(grid_max / 2, uint32_t(ws->num_sms)));
    a.slab = ws->sh->slab;
    a.n_nodes = g.n;
    a.n_arcs = g.arcs;
    if (ntiles && (!a.src || !a.slab || !a.sbits || !a.out_key || !a.out_d || !a.row_ptr || !a.adj || !a.ctl ||
                   !ws->failed || !ws->failed2))
        fail(RN_EINTERNAL, "tile search without its buffers");
    uint64_t hcap = 1;
    while (hcap < 2ull * g.n) hcap <<= 1;
    const uint64_t H0 = first_map(map_slots, hcap);
    a.gmap = nullptr;
    a.range_list = nullptr;
    a.ntiles = ntiles;
    if (first_ranges) {
        // the first launch searches the given source ranges instead of the tiles of R
        ntiles = uint32_t(first_ranges->size());
        ensure_ranges(&ws->failed, &ws->failed_cap, std::max<uint32_t>(ntiles, 1));
        ensure_ranges(&ws->failed2, &ws->failed2_cap, std::max<uint32_t>(ntiles, 1));
        if (ntiles)
            RN_CUDA(cudaMemcpyAsync(ws->failed2, first_ranges->data(), size_t(ntiles) * 16, cudaMemcpyHostToDevice, st));
        a.range_list = ws->failed2;
        a.ntiles = ntiles;
    }
    a.failed = ws->failed;
    auto set_shared = [](SearchArgs &x, uint32_t h) {
        x.gmap = nullptr;
        x.H = h;
        x.hshift = 32 - bits_for(h);
        x.max_fill = h * 7 / 8;
    };
    // one launch over n ranges (or every tile) with a map of h slots
    auto launch = [&](SearchArgs &x, uint64_t h, uint32_t n) {
        if (h == SMEM_H) {
            set_shared(x, SMEM_H);
            search(T, Shape::Narrow, x, std::max<uint32_t>(1, std::min(n, grid_max)), st);
        } else if (h == SMEM_HW) {
            set_shared(x, SMEM_HW);
            search(T, Shape::Wide, x, std::max<uint32_t>(1, std::min(n, grid_wide)), st);
        } else {
            launch_gmap(g, ws, T, x, h, n, st);
        }
        ws->launches++;
    };
    if (timed) RN_CUDA(cudaEventRecord(ws->evs0, st));
    if (ntiles) {
        launch(a, H0, ntiles);
        if (timed)
            ws->blocks_per_sm = H0 > SMEM_H ? 1 : T == 32 ? search_occupancy<1>() : T == 64 ? search_occupancy<2>() : search_occupancy<4>();
    }
    if (timed) RN_CUDA(cudaEventRecord(ws->evs1, st));
    Control c = read_control(ws, st);
    if (timed) ws->retry_ms = 0;
    if (!c.n_failed || c.err) return c;
    // relaunch `ranges` with a map of h slots; the ranges that overflow again come back
    auto relaunch = [&](const std::vector<uint4> &ranges, uint64_t h) {
        const uint32_t n = uint32_t(ranges.size());
        ensure_ranges(&ws->failed, &ws->failed_cap, n);
        ensure_ranges(&ws->failed2, &ws->failed2_cap, n);
        RN_CUDA(cudaMemcpyAsync(ws->failed2, ranges.data(), size_t(n) * 16, cudaMemcpyHostToDevice, st));
        RN_CUDA(cudaMemsetAsync(&ws->ctl->tile_next, 0, 8, st));  // tile_next, n_failed
        SearchArgs r = a;
        r.range_list = ws->failed2;
        r.ntiles = n;
        r.failed = ws->failed;
        launch(r, h, n);
        *retried += n;
        RN_CUDA(cudaEventRecord(ws->evr, st));
        c = read_control(ws, st);
        float ms = 0;
        RN_CUDA(cudaEventElapsedTime(&ms, ws->evs1, ws->evr));
        ws->retry_ms = ms;
        return c.err ? std::vector<uint4>() : read_ranges(ws->failed, c.n_failed, st);
    };
    // estimated union ball of an overflowed range (at least what it filled, at most n)
    auto estimate = [&](const uint4 &f) {
        const double r = double(a.bound) / double(std::max<uint32_t>(f.z, 1));
        const double e = double(std::max<uint32_t>(f.w, 1)) * std::min(r * r, 1e12);
        return uint64_t(std::min<double>(std::max<double>(e, f.w), double(g.n)));
    };
    std::vector<uint4> over = read_ranges(ws->failed, c.n_failed, st);
    // ranges waiting for a larger map, by the map size they go to next
    std::map<uint64_t, std::vector<uint4>> grow;
    auto to_grow = [&](const uint4 &f, uint64_t failed_at) {
        const uint64_t h = std::max(map_for(estimate(f), hcap), failed_at == SMEM_H ? uint64_t(SMEM_HW)
                                                                                     : std::min(failed_at * 4, hcap));
        if (failed_at >= hcap) fail(RN_EINTERNAL, "slot map overflowed at its largest size");
        grow[h].push_back(make_uint4(f.x, f.y, 0, 0));
    };
    if (split && H0 <= SMEM_HW) {
        // the sources of the overflowed ranges, to see how far apart they lie
        std::vector<uint32_t> src(std::max<uint32_t>(a.nR_fixed ? a.nR_fixed : c.r_count, 1));
        RN_CUDA(cudaMemcpyAsync(src.data(), a.src, src.size() * 4, cudaMemcpyDeviceToHost, st));
        RN_CUDA(cudaStreamSynchronize(st));
        // parts go to wide blocks, sized to fill about 60% of their map: sources of one
        // tile cost little more than one (its rounds are bound by latency, not by the
        // sources it carries), so fewer, fuller parts beat many small ones
        const double room = double(SMEM_HW) * 7 / 8 * 0.6;
        std::vector<uint4> parts;
        for (const uint4 &f : over) {
            const bool sparse = f.y >= 2 && f.x + f.y <= src.size() &&
                                double(src[f.x + f.y - 1] - src[f.x]) / double(f.y - 1) >= SPARSE_GAP;
            const uint32_t np = sparse ? uint32_t(std::min<double>(f.y, std::ceil(double(estimate(f)) / room))) : 1;
            if (np < 2) {
                to_grow(f, H0);
                continue;
            }
            const uint32_t part = (f.y + np - 1) / np;
            for (uint32_t j = 0; j * part < f.y; j++)
                parts.push_back(make_uint4(f.x + j * part, std::min(part, f.y - j * part), 0, 0));
        }
        if (!parts.empty()) {
            const uint64_t hp = std::max<uint64_t>(H0, std::min<uint64_t>(SMEM_HW, hcap));
            for (const uint4 &f : relaunch(parts, hp)) to_grow(f, hp);
            if (c.err) return c;
        }
    } else {
        for (const uint4 &f : over) to_grow(f, H0);
    }
    while (!grow.empty()) {
        const uint64_t h = grow.begin()->first;
        std::vector<uint4> ranges;
        ranges.swap(grow.begin()->second);
        grow.erase(grow.begin());
        for (const uint4 &f : relaunch(ranges, h)) to_grow(f, h);
        if (c.err) return c;
    }
    return c;
}

// ---------------------------------------------------- source search, host side ----

template <uint32_t MS, bool HIER = false>
static void launch_source(const SearchArgs &a, uint32_t grid, cudaStream_t st) {
    constexpr uint32_t smem = src_warps(MS) * src_words(MS) * 4;
    static std::once_flag once[MAX_DEVICES];
    std::call_once(once[attr_device()], [&] {
        RN_CUDA(cudaFuncSetAttribute(k_source_search<MS, HIER>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
        RN_CUDA(cudaFuncSetAttribute(k_source_search<MS, HIER>, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    });
    k_source_search<MS, HIER><<<grid, src_warps(MS) * 32, smem, st>>>(a);
    RN_CUDA(cudaGetLastError());
}

// The cooperative search for sources whose maps have 4096 or 8192 slots: coop_warps(MS)
// warps per source (0: the warp search), as many blocks per SM as the warp search has
// warps with maps of that size (6 or 3).  Measured on the 6M-node serving stream: four
// warps per source on both sizes took its requests' device time from 4.06 to 2.78 s,
// eight on the 8192-slot maps to 2.54 s; two on 2048-slot maps slowed the 264k-node join.
__host__ __device__ constexpr uint32_t coop_warps(uint32_t ms) { return ms == 4096 ? 4 : ms == 8192 ? 8 : 0; }
template <uint32_t MS>
static void launch_coop(const SearchArgs &a, uint32_t grid, cudaStream_t st) {
    constexpr uint32_t W = coop_warps(MS), smem = src_words(MS) * 4;
    static std::once_flag once[MAX_DEVICES];
    std::call_once(once[attr_device()], [&] {
        RN_CUDA(cudaFuncSetAttribute(k_source_coop<MS, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
        RN_CUDA(cudaFuncSetAttribute(k_source_coop<MS, W>, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    });
    k_source_coop<MS, W><<<grid, W * 32, smem, st>>>(a);
    RN_CUDA(cudaGetLastError());
}

template <uint32_t MS>
static int source_occupancy() {
    int b = 0;
    RN_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_source_search<MS, false>, src_warps(MS) * 32,
                                                          src_warps(MS) * src_words(MS) * 4));
    return b;
}

// Resident warp-search blocks per SM with maps of ms slots (after the first launch set
// the kernel's shared-memory limit).
template <uint32_t MS>
static int coop_occupancy() {
    if constexpr (coop_warps(MS) == 0) {
        return source_occupancy<MS>();
    } else {
        int b = 0;
        RN_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_source_coop<MS, coop_warps(MS)>, coop_warps(MS) * 32,
                                                              src_words(MS) * 4));
        return b;
    }
}

static int source_blocks_per_sm(uint32_t ms) {
    switch (ms) {
        case 1024: return coop_occupancy<1024>();
        case 2048: return coop_occupancy<2048>();
        case 4096: return coop_occupancy<4096>();
        default: return coop_occupancy<8192>();
    }
}

static uint32_t *ensure_slist(Workspace *ws) {
    if (!ws->slist) {
        const size_t words = size_t(ws->num_sms) * SRC_BLOCKS_PER_SM * SRC_LIST_WORDS_PER_BLOCK;
        ws->slist = (uint32_t *)device_alloc(words * 4);
        ws->bytes += words * 4;
    }
    return ws->slist;
}

// One warp-search launch over `items` sources with maps of ms slots: a block per
// src_warps sources up to three blocks per SM of the device.  The warp search uses no slab,
// so a server's request is not held to the slab regions it was given (those serve its
// tile fallback): its blocks share the SMs with the other requests' as they free up.
static void source_launch(uint32_t ms, SearchArgs a, uint32_t items, Workspace *ws, cudaStream_t st,
                          bool hier = false) {
    a.H = ms;
    a.hshift = 32 - log2u(ms);
    a.max_fill = ms * 7 / 8;
    a.gmap = nullptr;
    a.slist = ensure_slist(ws);
    if (coop_warps(ms) && !hier) {
        // a block per source (its list: MS entries at blockIdx.x MS, within the lists of
        // the warp search's resident blocks)
        const uint32_t per_sm = (3 * 8192) / ms;
        const uint32_t grid = std::max<uint32_t>(1, std::min<uint32_t>(items, uint32_t(ws->num_sms) * per_sm));
        switch (ms) {
            case 1024: if constexpr (coop_warps(1024) != 0) launch_coop<1024>(a, grid, st); break;
            case 2048: if constexpr (coop_warps(2048) != 0) launch_coop<2048>(a, grid, st); break;
            case 4096: if constexpr (coop_warps(4096) != 0) launch_coop<4096>(a, grid, st); break;
            case 8192: if constexpr (coop_warps(8192) != 0) launch_coop<8192>(a, grid, st); break;
            default: fail(RN_EINTERNAL, "cooperative map size must be 1024 .. 8192");
        }
        ws->launches++;
        return;
    }
    const uint32_t per_block = src_warps(ms);
    const uint32_t resident = std::max<uint32_t>(1, uint32_t(ws->num_sms) * SRC_BLOCKS_PER_SM);
    const uint32_t grid = std::max<uint32_t>(1, std::min<uint32_t>((items + per_block - 1) / per_block, resident));
    switch (ms * 2 + (hier ? 1 : 0)) {
        case 2048: launch_source<1024>(a, grid, st); break;
        case 4096: launch_source<2048>(a, grid, st); break;
        case 8192: launch_source<4096>(a, grid, st); break;
        case 16384: launch_source<8192>(a, grid, st); break;
        case 2049: launch_source<1024, true>(a, grid, st); break;
        case 4097: launch_source<2048, true>(a, grid, st); break;
        case 8193: launch_source<4096, true>(a, grid, st); break;
        case 16385: launch_source<8192, true>(a, grid, st); break;
        default: fail(RN_EINTERNAL, "warp map size must be 1024 .. 8192");
    }
    ws->launches++;
}

// Slots a warp map of ms slots is expected to hold with room to spare below its 7/8 limit.
static double src_fit(uint32_t ms) { return double(ms) * 7 / 8 / 1.1; }

// The largest source ball expected at bound theta from the last warp search on this
// workspace (balls grow about as the square of the radius), 0 when there was none.
static double predicted_ball(const Workspace *ws, uint32_t theta) {
    if (!ws->ball_theta) return 0;
    const double r = double(theta) / double(ws->ball_theta);
    return double(ws->ball_max) * r * r;
}

// The ball of a source at bound theta on a graph with no search behind it yet: on a
// planar road network the nodes within theta are about those within theta / w_med hops,
// and a lattice holds 2 r^2 nodes within r hops; never more than the graph.
static double first_ball_estimate(const DeviceGraph &g, uint32_t theta, uint32_t median_w) {
    const double r = double(theta) / double(std::max<uint32_t>(median_w, 1));
    return std::min(2.0 * r * r, double(g.n));
}

// Whether a join runs the warp-per-source search: always for tile width 1, never for
// 32, 64 or 128 or an explicit first map; by default while the balls seen on this
// workspace, scaled to this bound, fit the largest warp map (with no search behind the
// workspace yet, while the ball estimated from the bound does).
static bool use_source_search(const DeviceGraph &g, const Workspace *ws, const EngineConfig &cfg, uint32_t theta,
                              uint32_t median_w) {
    if (g.n >= SK_NODE) return false;
    if (cfg.tile_width == 1) return true;
    if (cfg.tile_width || cfg.map_slots) return false;
    const double ball = ws->ball_theta ? predicted_ball(ws, theta) : first_ball_estimate(g, theta, median_w);
    return ball <= src_fit(SRC_MS_MAX);
}

// First warp map: the smallest whose 7/8 holds 1.3 times the predicted mean ball and
// nearly the predicted largest (up to 15% over: the few sources that overflow are searched
// again with a larger map, while a smaller map fits twice as many warps on an SM).  With
// no history: the smallest map that fits the ball estimated from the bound (`first`, the
// largest ball a lattice would give: k closest pairs, whose searches teach the workspace
// nothing), else 2048 slots (a join's first search, which its measured balls then size).
static uint32_t source_first_map(const Workspace *ws, uint32_t theta, double first = 0) {
    const double b = predicted_ball(ws, theta);
    if (b <= 0) {
        if (first <= 0) return 2048;
        for (uint32_t ms = SRC_MS_MIN; ms <= SRC_MS_MAX; ms *= 2)
            if (first <= src_fit(ms)) return ms;
        return SRC_MS_MAX;
    }
    const double r = double(theta) / double(ws->ball_theta);
    const double mean = ws->ball_mean * r * r;
    for (uint32_t ms = SRC_MS_MIN; ms <= SRC_MS_MAX; ms *= 2) {
        const double room = double(ms) * 7 / 8;
        if (mean > 0 ? (mean * 1.3 <= room && b <= room * 1.15) : b <= src_fit(ms)) return ms;
    }
    return SRC_MS_MAX;
}

// Search sources 0 .. nsrc-1 with warp maps of ms0 slots, then the sources whose ball
// overflowed: with the smallest warp map their estimated ball fits (fill * (bound /
// tau)^2, as for tiles), and past the largest warp map with the tile search of width T,
// as ranges of consecutive sources of one query (inst_first: the first source of every
// query, empty for a single query).  Remembers the largest and the mean ball seen, for
// the next query's choice of path and map.
static Control source_search_all(const DeviceGraph &g, Workspace *ws, SearchArgs a, uint32_t nsrc, uint32_t ms0,
                                 uint32_t T, uint32_t theta, const std::vector<uint32_t> &inst_first,
                                 cudaStream_t st, uint64_t *retried, bool learn_balls = true) {
    a.n_nodes = g.n;
    a.n_arcs = g.arcs;
    a.range_list = nullptr;
    a.ntiles = nsrc;
    if (nsrc && (!a.src || (!a.sbits && !a.inst_sbits) || !a.out_key || !a.out_d || !a.row_ptr || !a.adj || !a.ctl))
        fail(RN_EINTERNAL, "source search without its buffers");
    ensure_ranges(&ws->failed, &ws->failed_cap, std::max<uint32_t>(nsrc, 1));
    ensure_ranges(&ws->failed2, &ws->failed2_cap, std::max<uint32_t>(nsrc, 1));
    a.failed = ws->failed;
    RN_CUDA(cudaEventRecord(ws->evs0, st));
    if (nsrc) source_launch(ms0, a, nsrc, ws, st);
    RN_CUDA(cudaEventRecord(ws->evs1, st));
    Control c = read_control(ws, st);
    ws->retry_ms = 0;
    ws->src_tiles = false;
    ws->blocks_per_sm = nsrc ? source_blocks_per_sm(ms0) : 0;
    double ball = c.src_max_ball;
    // mean ball of the sources the first pass completed (0 when none did)
    const double mean = nsrc > c.n_failed ? double(c.slots) / double(nsrc - c.n_failed) : 0.0;
    auto learn = [&] {
        // (k closest pairs lowers its bound as it goes: its balls say nothing of theta)
        if (learn_balls && nsrc && ball >= 64) {  // a handful of nodes says little about the growth
            ws->ball_theta = std::max<uint32_t>(theta, 1);
            ws->ball_max = ball;
            ws->ball_mean = mean;
        }
    };
    if (!c.n_failed || c.err || c.check[0]) {
        learn();
        return c;
    }
    auto estimate = [&](const uint4 &f) {
        const double r = double(f.y) / double(std::max<uint32_t>(f.z, 1));
        const double e = double(std::max<uint32_t>(f.w, 1)) * std::min(r * r, 1e12);
        return std::min<double>(std::max<double>(e, f.w), double(g.n));
    };
    std::map<uint32_t, std::vector<uint4>> grow;  // warp map -> its sources (index, 0, 0, 0)
    std::vector<uint4> to_tiles;
    double tile_est = 0;
    auto route = [&](const uint4 &f, uint32_t failed_at) {
        const double e = estimate(f);
        ball = std::max(ball, e);
        uint32_t ms = failed_at * 2;
        while (ms <= SRC_MS_MAX && e > src_fit(ms)) ms *= 2;
        if (ms <= SRC_MS_MAX) {
            grow[ms].push_back(make_uint4(f.x, 0, 0, 0));
        } else {
            to_tiles.push_back(f);
            tile_est = std::max(tile_est, e);
        }
    };
    for (const uint4 &f : read_ranges(ws->failed, c.n_failed, st)) route(f, ms0);
    while (!grow.empty()) {
        const uint32_t ms = grow.begin()->first;
        std::vector<uint4> items;
        items.swap(grow.begin()->second);
        grow.erase(grow.begin());
        const uint32_t n = uint32_t(items.size());
        RN_CUDA(cudaMemcpyAsync(ws->failed2, items.data(), size_t(n) * 16, cudaMemcpyHostToDevice, st));
        RN_CUDA(cudaMemsetAsync(&ws->ctl->tile_next, 0, 8, st));  // tile_next, n_failed
        SearchArgs r = a;
        r.range_list = ws->failed2;
        r.ntiles = n;
        source_launch(ms, r, n, ws, st);
        *retried += n;
        c = read_control(ws, st);
        if (c.err || c.check[0]) return c;
        ball = std::max<double>(ball, c.src_max_ball);
        for (const uint4 &f : read_ranges(ws->failed, c.n_failed, st)) route(f, ms);
    }
    ws->src_tiles = !to_tiles.empty();
    if (!to_tiles.empty()) {
        // consecutive sources of one query become ranges of up to T sources each
        std::sort(to_tiles.begin(), to_tiles.end(), [](const uint4 &x, const uint4 &y) { return x.x < y.x; });
        auto query_of = [&](uint32_t si) {
            return inst_first.empty()
                       ? 0u
                       : uint32_t(std::upper_bound(inst_first.begin(), inst_first.end(), si) - inst_first.begin());
        };
        // (a batch's tables hold one entry per source: its sources go one per tile)
        const bool per_source = a.tile_bound != nullptr;
        std::vector<uint4> ranges;
        for (const uint4 &f : to_tiles) {
            if (!ranges.empty() && !per_source) {
                uint4 &b = ranges.back();
                if (b.x + b.y == f.x && b.y < T && query_of(b.x) == query_of(f.x)) {
                    b.y++;
                    continue;
                }
            }
            ranges.push_back(make_uint4(f.x, 1, 0, 0));
        }
        RN_CUDA(cudaMemsetAsync(&ws->ctl->tile_next, 0, 8, st));
        SearchArgs t = a;
        t.tile_src = per_source ? 1 : T;
        uint64_t want = uint64_t(tile_est) * 2;  // the union of a few neighbours' balls
        c = search_all(g, ws, T, t, 0, st, retried, uint32_t(std::min<uint64_t>(want, 1u << 30)), true, &ranges,
                       false);
        *retried += ranges.size();
    }
    RN_CUDA(cudaEventRecord(ws->evr, st));
    RN_CUDA(cudaEventSynchronize(ws->evr));
    float ms = 0;
    RN_CUDA(cudaEventElapsedTime(&ms, ws->evs1, ws->evr));
    ws->retry_ms = ms;
    learn();
    return c;
}

// Per-source segments of the warp search for nsrc sources, cleared on the stream.
static uint2 *ensure_segments(Workspace *ws, uint32_t nsrc, cudaStream_t st) {
    if (!ws->seg || ws->seg_cap < nsrc) {
        device_free(ws->seg);
        ws->seg = nullptr;
        ws->seg_cap = std::max<uint32_t>(nsrc, 1024);
        ws->seg = (uint2 *)device_alloc(size_t(ws->seg_cap) * 8);
    }
    if (nsrc) RN_CUDA(cudaMemsetAsync(ws->seg, 0, size_t(nsrc) * 8, st));
    return ws->seg;
}

// Whether the pairs of the last warp search can be ordered by placement (every source's
// pairs in one segment of at most PLACE_MAX, all written).
static bool can_place(const Workspace *ws, const Control &c) {
    return !ws->src_tiles && c.max_seg <= PLACE_MAX && c.pairs <= ws->pair_cap && c.pairs < 0xFFFFFFFFull;
}

// The canonical order by placement: offsets from the segments' counts (source order is
// the output order), then one warp per segment; with no `out`, into the workspace's
// (keyA, valA) records instead, in (u, v) order.
static void place_pairs(Workspace *ws, uint32_t nsrc, uint32_t vbits, uint32_t umask, rn_dpairs *out,
                        cudaStream_t st) {
    if (!nsrc) return;
    grow(ws, &ws->hist, &ws->hist_cap, hist_words(nsrc), 4);
    const uint32_t nb = std::min<uint32_t>((nsrc + 255) / 256, 4096);
    k_seg_counts<<<nb, 256, 0, st>>>(ws->seg, nsrc, ws->hist);
    ws->launches += 1 + scan_hist(ws->hist, nsrc, st);
    k_place<<<std::min<uint32_t>((nsrc + 7) / 8, 8192), 256, 0, st>>>(
        ws->seg, ws->hist, nsrc, ws->keyA, ws->valA, vbits, umask, out ? out->u : nullptr, out ? out->v : nullptr,
        out ? out->d : nullptr, out ? nullptr : ws->keyB, out ? nullptr : ws->valB);
    ws->launches++;
    RN_CUDA(cudaGetLastError());
    if (!out) {  // the placed records become the radix sort's input
        std::swap(ws->keyA, ws->keyB);
        std::swap(ws->valA, ws->valB);
    }
}

// Bucket width unless configured: four median arc weights for the tile search, sixteen
// for the warp search.  Wider buckets mean fewer rounds and bucket boundaries at the price
// of some relaxations redone inside a bucket; a warp's boundary is a pass over its whole
// map, so the warp search gains from wider buckets (measured on road-like graphs: 4, 8,
// 16, 32 medians gave 1.51, 1.43, 1.42, 1.55 ms on the 264k join and 3.31, 2.82, 2.69,
// 2.64 ms on the 1.07M one).
static uint32_t choose_delta(const EngineConfig &cfg, uint32_t median_w, bool by_source = false) {
    if (cfg.delta) return cfg.delta;
    const uint64_t d = uint64_t(by_source ? 16 : 4) * median_w;
    return uint32_t(std::max<uint64_t>(1, std::min<uint64_t>(d, RN_THETA_MAX)));
}

static void ensure_u32(uint32_t **p, uint32_t *cap, uint32_t want) {
    if (*p && *cap >= want) return;
    device_free(*p);
    *p = nullptr;
    *cap = std::max<uint32_t>(want, 1024);
    *p = (uint32_t *)device_alloc(size_t(*cap) * 4);
}

static void ensure_pairs(Workspace *ws, uint64_t want) {
    if (ws->pair_cap >= want && ws->keyA) return;
    want = std::max<uint64_t>(want, 1 << 16);
    for (void **p : {(void **)&ws->keyA, (void **)&ws->keyB, (void **)&ws->valA, (void **)&ws->valB}) {
        device_free(*p);
        *p = nullptr;
    }
    ws->bytes -= ws->pair_cap * 24;
    ws->pair_cap = 0;
    ws->keyA = (unsigned long long *)device_alloc(want * 8);
    ws->keyB = (unsigned long long *)device_alloc(want * 8);
    ws->valA = (uint32_t *)device_alloc(want * 4);
    ws->valB = (uint32_t *)device_alloc(want * 4);
    ws->pair_cap = want;
    ws->bytes += want * 24;
}

static void ensure_slab(Workspace *ws) {
    const uint32_t grid_max = uint32_t(ws->num_sms) * CTAS_PER_SM;
    DeviceShared *sh = ws->sh;
    if (sh->external) {
        if (!sh->slab || sh->slab_ctas < 2) fail(RN_EINTERNAL, "workspace slab not set");
        return;
    }
    if (sh->slab && sh->slab_ctas >= grid_max) return;
    device_free(sh->slab);
    sh->slab = nullptr;
    sh->slab_bytes = size_t(SMEM_H) * 128 * 4 * grid_max;  // rows of the widest tile
    sh->slab = (uint32_t *)device_alloc(sh->slab_bytes);
    RN_CUDA(cudaMemset(sh->slab, 0xFF, sh->slab_bytes));  // every row INF
    RN_CUDA(cudaDeviceSynchronize());  // before any search on a stream of its own
    sh->slab_ctas = grid_max;
}

// Grow the workspace's buffers now for queries of up to max_r sources and max_pairs
// pairs (raw pairs and their sort), so such queries allocate and free nothing later:
// freeing device memory synchronises the whole device, which would stall every other
// stream's work.
void workspace_reserve(Workspace *ws, uint32_t max_r, uint64_t max_pairs) {
    ensure_u32(&ws->rsorted, &ws->rsorted_cap, std::max<uint32_t>(max_r, 1));
    ensure_ranges(&ws->failed, &ws->failed_cap, std::max<uint32_t>(max_r, 1));
    ensure_ranges(&ws->failed2, &ws->failed2_cap, std::max<uint32_t>(max_r, 1));
    ensure_pairs(ws, max_pairs);
    grow(ws, &ws->hist, &ws->hist_cap, hist_words((max_pairs + RS_TILE - 1) / RS_TILE * 256), 4);
    ensure_slist(ws);
    if (!ws->seg || ws->seg_cap < max_r) {  // the warp search's per-source segments
        device_free(ws->seg);
        ws->seg = nullptr;
        ws->seg_cap = std::max<uint32_t>(max_r, 1024);
        ws->seg = (uint2 *)device_alloc(size_t(ws->seg_cap) * 8);
    }
}

// a2: validate R and S on the device, build the S membership bitmap and the list of R
// nodes in increasing internal id (so consecutive sources are graph neighbours).
// by_orig: R in increasing original id instead (each source alone, so the order of
// sources need not follow the graph; it is the output order).
static void prep_sets(const DeviceGraph &g, Workspace *ws, const uint32_t *dR, uint32_t nR,
                      const uint32_t *dS, uint32_t nS, cudaStream_t st, bool by_orig = false) {
    RN_CUDA(cudaMemsetAsync(ws->used_bits, 0, size_t(ws->nwords) * 4, st));
    RN_CUDA(cudaMemsetAsync(ws->rbits, 0, size_t(ws->nwords) * 4, st));
    RN_CUDA(cudaMemsetAsync(ws->sbits, 0, size_t(ws->nwords) * 4, st));
    RN_CUDA(cudaMemsetAsync(ws->ctl, 0, sizeof(Control), st));
    if (nR)
        k_mark_set<<<std::min<uint32_t>((nR + 255) / 256, 4096), 256, 0, st>>>(dR, nR, g.n, g.perm, ws->used_bits,
                                                                               ws->rbits, ws->ctl, by_orig);
    if (nS)
        k_mark_set<<<std::min<uint32_t>((nS + 255) / 256, 4096), 256, 0, st>>>(dS, nS, g.n, g.perm, ws->used_bits,
                                                                               ws->sbits, ws->ctl, false);
    ensure_u32(&ws->rsorted, &ws->rsorted_cap, std::max<uint32_t>(nR, 1));
    const uint32_t nblocks = (ws->nwords + 1023) / 1024;
    k_bits_count<<<nblocks, 1024, 0, st>>>(ws->rbits, ws->nwords, ws->block_sums);
    k_bits_compact<<<nblocks, 1024, 0, st>>>(ws->rbits, ws->nwords, ws->block_sums, nblocks, ws->rsorted, ws->ctl);
    ws->launches += (nR ? 1 : 0) + (nS ? 1 : 0) + 2;
    if (by_orig && nR) {
        k_to_internal<<<std::min<uint32_t>((nR + 255) / 256, 4096), 256, 0, st>>>(ws->rsorted, nR, g.perm, ws->ctl);
        ws->launches++;
    }
    RN_CUDA(cudaGetLastError());
}

static void check_control(const Control &c) {
    if (c.check[0])
        fail(RN_EINTERNAL, "device check " + std::to_string(c.check[0]) + " failed at index " +
                               std::to_string(c.check[1]) + " (value " + std::to_string(c.check[2]) + ")");
    if (c.err & 1u) fail(RN_EINVAL, "a node id of R or S is >= n");
    if (c.err & 2u) fail(RN_EINVAL, "R or S repeats an id, or R and S overlap");
}

// Whether a query's searches start from S.  The paper searches from every node of R; on
// an undirected graph d(u, v) = d(v, u), so searching from S instead finds the same pairs
// (written back as (u in R, v in S)) with |S| searches instead of |R|.  By default that
// is done when S is at least a fifth smaller than R (below that the saving does not pay
// for losing the warp search's placement order).
static bool search_from_s(const DeviceGraph &g, const EngineConfig &cfg, uint64_t nR, uint64_t nS) {
    if (cfg.search_from == RN_FROM_R) return false;
    if (cfg.search_from == RN_FROM_S) {
        if (!g.symmetric) fail(RN_EINVAL, "searches from S need a graph loaded undirected");
        return true;
    }
    return g.symmetric && nS * 5 < nR * 4;
}

void run_join(const DeviceGraph &g, Workspace *ws, const EngineConfig &cfg, uint32_t median_w,
              const uint32_t *dR, uint32_t nR, const uint32_t *dS, uint32_t nS, uint32_t theta,
              rn_dpairs *out, void *stream, rn_query_stats *stats) {
    cudaStream_t st = (cudaStream_t)stream;
    if (theta == RN_INF) theta = RN_THETA_MAX;
    if (theta > RN_THETA_MAX) fail(RN_EINVAL, "theta must be <= 2^31 or RN_INF");
    const uint32_t T = cfg.tile_width > 1 ? cfg.tile_width : 32;  // the tile search's width
    if (T != 32 && T != 64 && T != 128) fail(RN_EINVAL, "tile width must be 1, 32, 64 or 128");
    std::lock_guard<std::mutex> device_lock(ws->sh->mu);
    Range range("rn.join");
    *stats = rn_query_stats{};
    const bool from_s = search_from_s(g, cfg, nR, nS);
    if (from_s) {  // S's nodes are the sources, R's the targets (below, "R" is the sources)
        std::swap(dR, dS);
        std::swap(nR, nS);
    }
    stats->from_s = from_s;
    const bool by_source = use_source_search(g, ws, cfg, theta, median_w);
    // the warp search's segments give the output order when sources run in output order
    // (and are R's: a segment of an S source holds one v and many u)
    const bool place = by_source && g.iperm_inverts_perm && !from_s;
    const uint32_t delta = choose_delta(cfg, median_w, by_source);
    stats->tile_width = by_source ? 1 : T;
    stats->delta = delta;
    stats->theta_final = theta;
    ws->launches = 0;
    RN_CUDA(cudaEventRecord(ws->ev0, st));

    prep_sets(g, ws, dR, nR, dS, nS, st, place);
    // sources per tile: as many as fit a row, but spread so the tiles fill the resident
    // blocks in whole waves (a last wave of a few tiles would double the search time)
    ensure_slab(ws);
    const uint32_t grid_max = ws->sh->slab_ctas;  // resident narrow blocks the slab serves
    uint32_t tile_src = T;
    if (nR) {
        const uint64_t waves = (uint64_t(nR) + uint64_t(T) * grid_max - 1) / (uint64_t(T) * grid_max);
        tile_src = uint32_t(std::min<uint64_t>(T, (nR + waves * grid_max - 1) / (waves * grid_max)));
        if (cfg.tile_src) tile_src = std::min(cfg.tile_src, T);
    }
    if (by_source) tile_src = 1;
    const uint32_t ntiles = (nR + tile_src - 1) / tile_src;
    ensure_ranges(&ws->failed, &ws->failed_cap, std::max<uint32_t>(ntiles, 1));
    ensure_ranges(&ws->failed2, &ws->failed2_cap, std::max<uint32_t>(ntiles, 1));
    ensure_pairs(ws, std::max<uint64_t>(ws->pair_cap, uint64_t(nR) * 64));
    const uint32_t ms0 = by_source ? source_first_map(ws, theta) : 0;

    const uint32_t vbits = bits_for(g.n);
    SearchArgs a{};
    a.row_ptr = g.row_ptr;
    a.adj = reinterpret_cast<const uint2 *>(g.adj);
    a.iperm = g.iperm;
    a.sbits = ws->sbits;
    a.src = ws->rsorted;
    a.bound = theta;
    a.delta = delta;
    a.slab = ws->sh->slab;
    a.vbits = vbits;
    a.tile_src = tile_src;
    a.ctl = ws->ctl;
    a.out_key = ws->keyA;
    a.out_d = ws->valA;
    a.out_cap = ws->pair_cap;
    a.seg = place ? ensure_segments(ws, nR, st) : nullptr;
    a.swap_uv = from_s;
    uint64_t retried = 0;
    const std::vector<uint32_t> one_query;
    auto search_pass = [&] {
        return by_source ? source_search_all(g, ws, a, nR, ms0, T, theta, one_query, st, &retried)
                         : search_all(g, ws, T, a, ntiles, st, &retried, cfg.map_slots);
    };
    Control c;
    {
        Range r("rn.search");
        c = search_pass();
    }
    check_control(c);
    if (c.pairs > ws->pair_cap) {
        // the pair buffer was too small: grow it and search again (same result)
        ensure_pairs(ws, c.pairs + c.pairs / 8);
        prep_sets(g, ws, dR, nR, dS, nS, st, place);
        a.src = ws->rsorted;
        a.out_key = ws->keyA;
        a.out_d = ws->valA;
        a.out_cap = ws->pair_cap;
        a.seg = place ? ensure_segments(ws, nR, st) : nullptr;
        c = search_pass();
        check_control(c);
        if (c.pairs > ws->pair_cap) fail(RN_EINTERNAL, "pair count changed between passes");
    }
    const uint64_t np = c.pairs;

    // a5: canonical order by (u, v), written straight into the caller's buffers: by
    // placing the warp search's per-source segments, else by a radix sort of all pairs
    Range rsort("rn.sort");
    dpairs_reserve(out, np);
    if (place && can_place(ws, c)) {
        place_pairs(ws, nR, vbits, 0xFFFFFFFFu, out, st);
    } else {
        std::vector<int> shifts;
        for (uint32_t sh = 0; sh < 2 * vbits; sh += 8) shifts.push_back(int(sh));
        radix_sort_to_pairs(ws, np, shifts, vbits, out, st);
    }
    out->n = np;
    RN_CUDA(cudaEventRecord(ws->ev1, st));
    RN_CUDA(cudaEventSynchronize(ws->ev1));
    float ms = 0, sms = 0;
    RN_CUDA(cudaEventElapsedTime(&ms, ws->ev0, ws->ev1));
    RN_CUDA(cudaEventElapsedTime(&sms, ws->evs0, ws->evs1));
    stats->pairs = np;
    stats->tiles = ntiles;
    stats->tile_sources = tile_src;
    stats->retried_tiles = retried;
    stats->scans = c.scans;
    stats->slots = c.slots;
    stats->slot_arcs = c.slot_arcs;
    stats->passes = 1;
    stats->launches = ws->launches;
    stats->blocks_per_sm = uint32_t(ws->blocks_per_sm);
    stats->device_ms = ms;
    stats->search_ms = sms;
    stats->rounds = c.rounds;
    stats->round_items = c.round_items;
    stats->boundaries = c.boundaries;
    stats->cycles_rounds = c.cyc_round;
    stats->cycles_boundaries = c.cyc_bound;
    stats->cycles_emission = c.cyc_emit;
    stats->cycles_step_a = c.cyc_stepA;
    stats->round_arcs = c.round_arcs;
    stats->max_ball = c.max_fill;
    stats->dirty_groups = c.dirty_groups;
    stats->retry_ms = ws->retry_ms;
    stats->slot_lanes = c.slot_lanes;
    stats->search_pairs = np;
}

// ------------------------------------------------ several joins, one graph ----
// Several theta-joins over the same graph searched together (the server's micro-batches
// of small requests, rn_join_many): their sources are laid out one query after another,
// every tile is a range of one query's sources, and a tile takes its query's bound, S
// bitmap and key prefix (the query index above the (u, v) bits).  One sort then orders
// all pairs by (query, u, v), and the per-query counts cut the result.

// Set the S bit of every id of every query: ids[soff[i] .. soff[i+1]) belong to query i.
__global__ void k_set_bits_multi(const uint32_t *__restrict__ ids, const uint32_t *__restrict__ soff, uint32_t nq,
                                 uint32_t total, const uint32_t *__restrict__ perm, uint32_t *bits, uint32_t nwords) {
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < total; j += gridDim.x * blockDim.x) {
        uint32_t lo = 0, hi = nq - 1;
        while (lo < hi) {
            const uint32_t mid = (lo + hi + 1) >> 1;
            if (soff[mid] <= j) lo = mid;
            else hi = mid - 1;
        }
        const uint32_t x = perm[ids[j]];
        atomicOr(&bits[size_t(lo) * nwords + (x >> 5)], 1u << (x & 31));
    }
}

void run_join_multi(const DeviceGraph &g, Workspace *ws, const EngineConfig &cfg, uint32_t median_w,
                    const std::vector<uint32_t> &perm, const std::vector<const uint32_t *> &R,
                    const std::vector<uint32_t> &nR, const std::vector<const uint32_t *> &S,
                    const std::vector<uint32_t> &nS, const std::vector<uint32_t> &theta, rn_dpairs *out,
                    std::vector<uint64_t> *counts, void *stream, rn_query_stats *stats) {
    cudaStream_t st = (cudaStream_t)stream;
    const uint32_t nq = uint32_t(R.size());
    if (nq == 0) fail(RN_EINVAL, "no queries");
    const uint32_t T = cfg.tile_width > 1 ? cfg.tile_width : 32;  // the tile search's width
    if (T != 32 && T != 64 && T != 128) fail(RN_EINVAL, "tile width must be 1, 32, 64 or 128");
    const uint32_t vbits = bits_for(g.n), qbits = bits_for(nq);
    if (2 * vbits + qbits > 64) fail(RN_EINVAL, "too many queries for this graph in one search");
    std::lock_guard<std::mutex> device_lock(ws->sh->mu);
    Range range("rn.join_many");
    *stats = rn_query_stats{};
    uint32_t max_bound = 0;
    for (uint32_t t : theta) max_bound = std::max(max_bound, std::min(t, RN_THETA_MAX));
    const bool by_source = use_source_search(g, ws, cfg, max_bound, median_w);
    const uint32_t delta = choose_delta(cfg, median_w, by_source);
    stats->tile_width = by_source ? 1 : T;
    stats->delta = delta;
    ws->launches = 0;
    RN_CUDA(cudaEventRecord(ws->ev0, st));
    // the sources: every query's R (or, searched from S, its S) in internal ids, ascending,
    // one query after another
    std::vector<uint32_t> src, first(nq + 1, 0), bound(nq), soff(nq + 1, 0), sids, nsrc(nq);
    std::vector<uint8_t> swp(nq, 0);
    bool any_swap = false;
    for (uint32_t i = 0; i < nq; i++) {
        const bool sw = search_from_s(g, cfg, nR[i], nS[i]);
        swp[i] = sw;
        any_swap |= sw;
        const uint32_t *Ri = sw ? S[i] : R[i], *Si = sw ? R[i] : S[i];
        nsrc[i] = sw ? nS[i] : nR[i];
        const uint32_t nt = sw ? nR[i] : nS[i];
        first[i] = uint32_t(src.size());
        const size_t b = src.size();
        if (by_source && g.iperm_inverts_perm) {
            // each source alone: in increasing original id, the output order
            std::vector<uint32_t> r(Ri, Ri + nsrc[i]);
            std::sort(r.begin(), r.end());
            for (uint32_t x : r) src.push_back(perm[x]);
        } else {
            for (uint32_t j = 0; j < nsrc[i]; j++) src.push_back(perm[Ri[j]]);
            std::sort(src.begin() + b, src.end());  // graph neighbours share tiles
        }
        bound[i] = theta[i] == RN_INF ? RN_THETA_MAX : theta[i];
        if (bound[i] > RN_THETA_MAX) fail(RN_EINVAL, "theta must be <= 2^31 or RN_INF");
        soff[i] = uint32_t(sids.size());
        sids.insert(sids.end(), Si, Si + nt);
        if (src.size() >= 0xFFFFFFFFull || sids.size() >= 0xFFFFFFFFull) fail(RN_EINVAL, "too many sources or targets");
    }
    first[nq] = uint32_t(src.size());
    soff[nq] = uint32_t(sids.size());
    const uint32_t total = uint32_t(src.size());
    ensure_slab(ws);
    // sources per tile: spread over whole waves of the slab's blocks, as for one query
    const uint32_t grid_max = ws->sh->slab_ctas;
    uint32_t tile_src = T;
    if (total) {
        const uint64_t waves = (uint64_t(total) + uint64_t(T) * grid_max - 1) / (uint64_t(T) * grid_max);
        tile_src = uint32_t(std::min<uint64_t>(T, (total + waves * grid_max - 1) / (waves * grid_max)));
        if (cfg.tile_src) tile_src = std::min(cfg.tile_src, T);
    }
    if (by_source) tile_src = 1;
    const uint32_t ms0 = by_source ? source_first_map(ws, max_bound) : 0;
    std::vector<uint4> ranges;
    for (uint32_t i = 0; i < nq; i++)
        for (uint32_t j = 0; j < nsrc[i]; j += tile_src)
            ranges.push_back(make_uint4(first[i] + j, std::min(tile_src, nsrc[i] - j), 0, 0));
    // device copies
    ensure_u32(&ws->rsorted, &ws->rsorted_cap, std::max<uint32_t>(total, 1));
    if (ws->mq_cap_q < nq + 1) {
        for (void **p : {(void **)&ws->mq_first, (void **)&ws->mq_bound, (void **)&ws->mq_soff, (void **)&ws->mq_sptr,
                         (void **)&ws->mq_counts, (void **)&ws->mq_swap}) {
            device_free(*p);
            *p = nullptr;
        }
        ws->mq_cap_q = std::max<uint64_t>(nq + 1, 64);
        ws->mq_swap = (uint8_t *)device_alloc(ws->mq_cap_q);
        ws->mq_first = (uint32_t *)device_alloc(ws->mq_cap_q * 4);
        ws->mq_bound = (uint32_t *)device_alloc(ws->mq_cap_q * 4);
        ws->mq_soff = (uint32_t *)device_alloc(ws->mq_cap_q * 4);
        ws->mq_sptr = (const uint32_t **)device_alloc(ws->mq_cap_q * 8);
        ws->mq_counts = (unsigned long long *)device_alloc(ws->mq_cap_q * 8);
    }
    const uint64_t bits_words = uint64_t(nq) * ws->nwords;
    if (ws->mq_cap_bits < bits_words) {
        device_free(ws->mq_sbits);
        ws->mq_sbits = nullptr;
        ws->mq_cap_bits = bits_words + bits_words / 2;
        ws->mq_sbits = (uint32_t *)device_alloc(ws->mq_cap_bits * 4);
    }
    if (ws->mq_cap_sids < std::max<size_t>(sids.size(), 1)) {
        device_free(ws->mq_sids);
        ws->mq_sids = nullptr;
        ws->mq_cap_sids = std::max<uint64_t>(sids.size() + sids.size() / 2, 1024);
        ws->mq_sids = (uint32_t *)device_alloc(ws->mq_cap_sids * 4);
    }
    std::vector<const uint32_t *> sptr(nq);
    for (uint32_t i = 0; i < nq; i++) sptr[i] = ws->mq_sbits + size_t(i) * ws->nwords;
    if (total) RN_CUDA(cudaMemcpyAsync(ws->rsorted, src.data(), size_t(total) * 4, cudaMemcpyHostToDevice, st));
    RN_CUDA(cudaMemcpyAsync(ws->mq_first, first.data(), size_t(nq + 1) * 4, cudaMemcpyHostToDevice, st));
    RN_CUDA(cudaMemcpyAsync(ws->mq_bound, bound.data(), size_t(nq) * 4, cudaMemcpyHostToDevice, st));
    RN_CUDA(cudaMemcpyAsync(ws->mq_soff, soff.data(), size_t(nq + 1) * 4, cudaMemcpyHostToDevice, st));
    RN_CUDA(cudaMemcpyAsync(ws->mq_sptr, sptr.data(), size_t(nq) * 8, cudaMemcpyHostToDevice, st));
    if (any_swap) RN_CUDA(cudaMemcpyAsync(ws->mq_swap, swp.data(), nq, cudaMemcpyHostToDevice, st));
    if (!sids.empty())
        RN_CUDA(cudaMemcpyAsync(ws->mq_sids, sids.data(), sids.size() * 4, cudaMemcpyHostToDevice, st));
    RN_CUDA(cudaMemsetAsync(ws->mq_sbits, 0, bits_words * 4, st));
    RN_CUDA(cudaMemsetAsync(ws->mq_counts, 0, size_t(nq) * 8, st));
    RN_CUDA(cudaMemsetAsync(ws->ctl, 0, sizeof(Control), st));
    if (!sids.empty()) {
        k_set_bits_multi<<<std::min<uint32_t>((uint32_t(sids.size()) + 255) / 256, 4096), 256, 0, st>>>(
            ws->mq_sids, ws->mq_soff, nq, uint32_t(sids.size()), g.perm, ws->mq_sbits, ws->nwords);
        ws->launches++;
        RN_CUDA(cudaGetLastError());
    }
    ensure_pairs(ws, std::max<uint64_t>(ws->pair_cap, uint64_t(total) * 64));
    SearchArgs a{};
    a.row_ptr = g.row_ptr;
    a.adj = reinterpret_cast<const uint2 *>(g.adj);
    a.iperm = g.iperm;
    a.sbits = ws->mq_sbits;  // every tile replaces it by its query's bitmap
    a.src = ws->rsorted;
    a.bound = RN_THETA_MAX;
    a.delta = delta;
    a.vbits = vbits;
    a.tile_src = tile_src;
    a.nR_fixed = total;
    a.ctl = ws->ctl;
    a.out_key = ws->keyA;
    a.out_d = ws->valA;
    a.out_cap = ws->pair_cap;
    a.inst_pairs = ws->mq_counts;
    a.inst_first = ws->mq_first;
    a.inst_count = nq;
    a.inst_shift = 2 * vbits;
    a.inst_sbits = ws->mq_sptr;
    a.inst_bound = ws->mq_bound;
    a.inst_swap = any_swap ? ws->mq_swap : nullptr;
    stats->from_s = any_swap;
    const bool place = by_source && g.iperm_inverts_perm && !any_swap;
    a.seg = place ? ensure_segments(ws, total, st) : nullptr;
    uint64_t retried = 0;
    auto search_pass = [&] {
        return by_source ? source_search_all(g, ws, a, total, ms0, T, max_bound, first, st, &retried)
                         : search_all(g, ws, T, a, 0, st, &retried, cfg.map_slots, true, &ranges);
    };
    Control c = search_pass();
    check_control(c);
    if (c.pairs > ws->pair_cap) {
        // the pair buffer was too small: grow it and search again (same result)
        ensure_pairs(ws, c.pairs + c.pairs / 8);
        RN_CUDA(cudaMemsetAsync(ws->mq_counts, 0, size_t(nq) * 8, st));
        RN_CUDA(cudaMemsetAsync(ws->ctl, 0, sizeof(Control), st));
        a.out_key = ws->keyA;
        a.out_d = ws->valA;
        a.out_cap = ws->pair_cap;
        a.seg = place ? ensure_segments(ws, total, st) : nullptr;
        c = search_pass();
        check_control(c);
        if (c.pairs > ws->pair_cap) fail(RN_EINTERNAL, "pair count changed between passes");
    }
    std::vector<unsigned long long> cnt(nq);
    RN_CUDA(cudaMemcpyAsync(cnt.data(), ws->mq_counts, size_t(nq) * 8, cudaMemcpyDeviceToHost, st));
    RN_CUDA(cudaStreamSynchronize(st));
    counts->assign(cnt.begin(), cnt.end());
    uint64_t sum = 0;
    for (uint64_t x : *counts) sum += x;
    if (sum != c.pairs) fail(RN_EINTERNAL, "per-query pair counts do not add up");
    const uint64_t np = c.pairs;
    Range rsort("rn.sort");
    dpairs_reserve(out, np);
    const uint32_t umask = vbits >= 32 ? 0xFFFFFFFFu : (1u << vbits) - 1;
    if (place && can_place(ws, c)) {
        place_pairs(ws, total, vbits, umask, out, st);  // sources in (query, u) order
    } else {
        std::vector<int> shifts;
        for (uint32_t sh = 0; sh < 2 * vbits + qbits; sh += 8) shifts.push_back(int(sh));
        radix_sort_to_pairs(ws, np, shifts, vbits, out, st, umask);
    }
    out->n = np;
    RN_CUDA(cudaEventRecord(ws->ev1, st));
    RN_CUDA(cudaEventSynchronize(ws->ev1));
    float ms = 0, sms = 0;
    RN_CUDA(cudaEventElapsedTime(&ms, ws->ev0, ws->ev1));
    RN_CUDA(cudaEventElapsedTime(&sms, ws->evs0, ws->evs1));
    stats->pairs = np;
    stats->tiles = ranges.size();
    stats->tile_sources = tile_src;
    stats->retried_tiles = retried;
    stats->slots = c.slots;
    stats->slot_arcs = c.slot_arcs;
    stats->scans = c.scans;
    stats->passes = 1;
    stats->launches = ws->launches;
    stats->device_ms = ms;
    stats->search_ms = sms;
    stats->retry_ms = ws->retry_ms;
    stats->rounds = c.rounds;
    stats->max_ball = c.max_fill;
    stats->slot_lanes = c.slot_lanes;
}

// ------------------------------------------------- join without allocation ----
// The entry point rn_distance_join_noalloc runs the same join through the same kernels,
// but takes every scratch buffer from one statically sized device array instead of
// allocating: for callers that cannot let the library allocate device memory (their
// own allocator owns the device, a cudaFree would synchronise the whole device in a
// latency-critical path, or a failed allocation in the middle of a query is not
// acceptable).  Its limits are fixed at build time (below); every GPU that loads the
// library holds the array (about 22 MB) until the process exits.

constexpr uint32_t NA_MAX_N = 1u << 20;       // nodes of the graph
constexpr uint32_t NA_MAX_R = 1u << 16;       // |R|
constexpr uint32_t NA_MAX_PAIRS = 1u << 19;   // result pairs
constexpr uint32_t NA_BLOCKS = 8;             // narrow search blocks (slab regions)
constexpr size_t NA_ALIGN = 64;               // sub-arrays start on 256-byte boundaries
constexpr size_t na_round(size_t w) { return (w + NA_ALIGN - 1) / NA_ALIGN * NA_ALIGN; }
constexpr size_t NA_CTL = 0;
constexpr size_t NA_BITS = NA_CTL + na_round(sizeof(Control) / 4 + 1);
constexpr size_t NA_NWORDS = NA_MAX_N / 32;
constexpr size_t NA_BSUMS = NA_BITS + 3 * na_round(NA_NWORDS);
constexpr size_t NA_RSORT = NA_BSUMS + na_round(NA_NWORDS / 1024 + 2);
constexpr size_t NA_FAIL = NA_RSORT + na_round(NA_MAX_R);
constexpr size_t NA_KEYS = NA_FAIL + 2 * na_round(NA_MAX_R);
constexpr size_t NA_VALS = NA_KEYS + 2 * na_round(2 * size_t(NA_MAX_PAIRS));
constexpr size_t NA_HIST = NA_VALS + 2 * na_round(NA_MAX_PAIRS);
constexpr size_t NA_SLAB = NA_HIST + na_round(size_t(256) * (NA_MAX_PAIRS / RS_TILE + 1));
constexpr size_t NA_WORDS = NA_SLAB + size_t(NA_BLOCKS) * SMEM_H * 32;

static __device__ __align__(256) uint32_t g_noalloc_scratch[NA_WORDS];

namespace {
std::mutex g_na_mu;       // one call at a time in this process
uint32_t *g_na_ptr[64];   // device address of the scratch array, per device
}  // namespace

// Once per device, with that device current: the array's device address (host code
// sees only a host-side stand-in for the symbol) and a first fill of the slab rows
// with INF.
static uint32_t *noalloc_scratch(int dev) {
    if (dev < 0 || dev >= 64) fail(RN_EINVAL, "device ordinal out of range for the no-alloc join");
    if (!g_na_ptr[dev]) {
        void *p = nullptr;
        RN_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        RN_CUDA(cudaMemset(static_cast<uint32_t *>(p) + NA_SLAB, 0xFF, size_t(NA_BLOCKS) * SMEM_H * 32 * 4));
        RN_CUDA(cudaDeviceSynchronize());
        g_na_ptr[dev] = static_cast<uint32_t *>(p);
    }
    return g_na_ptr[dev];
}

void run_join_noalloc(const DeviceGraph &g, uint32_t median_w, const uint32_t *dR, uint32_t nR,
                      const uint32_t *dS, uint32_t nS, uint32_t theta, uint32_t *out_u, uint32_t *out_v,
                      uint32_t *out_d, uint64_t out_cap, uint64_t *n_out, void *stream) {
    cudaStream_t st = (cudaStream_t)stream;
    if (theta == RN_INF) theta = RN_THETA_MAX;
    if (theta > RN_THETA_MAX) fail(RN_EINVAL, "theta must be <= 2^31 or RN_INF");
    if (g.n > NA_MAX_N) fail(RN_EINVAL, "the no-alloc join takes graphs of at most 2^20 nodes");
    if (nR > NA_MAX_R) fail(RN_EINVAL, "the no-alloc join takes at most 65536 R nodes");
    std::lock_guard<std::mutex> lk(g_na_mu);
    int dev = 0;
    RN_CUDA(cudaGetDevice(&dev));
    uint32_t *base = noalloc_scratch(dev);
    Control *ctl = reinterpret_cast<Control *>(base + NA_CTL);
    uint32_t *used_bits = base + NA_BITS, *rbits = used_bits + na_round(NA_NWORDS),
             *sbits = rbits + na_round(NA_NWORDS);
    uint32_t *bsums = base + NA_BSUMS, *rsorted = base + NA_RSORT;
    // the failed-range lists: NA_MAX_R words, NA_MAX_R / 4 ranges each (a launch has at
    // most 2048 tiles)
    uint4 *failed = reinterpret_cast<uint4 *>(base + NA_FAIL);
    uint4 *failed2 = reinterpret_cast<uint4 *>(base + NA_FAIL + na_round(NA_MAX_R));
    unsigned long long *keyA = reinterpret_cast<unsigned long long *>(base + NA_KEYS);
    unsigned long long *keyB = reinterpret_cast<unsigned long long *>(base + NA_KEYS + na_round(2 * size_t(NA_MAX_PAIRS)));
    uint32_t *valA = base + NA_VALS, *valB = valA + na_round(NA_MAX_PAIRS);
    uint32_t *hist = base + NA_HIST;
    uint32_t *slab = base + NA_SLAB;
    const uint32_t nwords = (g.n + 31) / 32;
    const uint32_t nblocks = (nwords + 1023) / 1024;

    // the array keeps the previous call's contents: clear what must start at zero, and
    // put the slab rows back to INF (a previous call may have stopped half-way)
    RN_CUDA(cudaMemsetAsync(ctl, 0, sizeof(Control), st));
    RN_CUDA(cudaMemsetAsync(used_bits, 0, size_t(nwords) * 4, st));
    RN_CUDA(cudaMemsetAsync(rbits, 0, size_t(nwords) * 4, st));
    RN_CUDA(cudaMemsetAsync(sbits, 0, size_t(nwords) * 4, st));
    RN_CUDA(cudaMemsetAsync(slab, 0xFF, size_t(NA_BLOCKS) * SMEM_H * 32 * 4, st));
    if (nR)
        k_mark_set<<<std::min<uint32_t>((nR + 255) / 256, 4096), 256, 0, st>>>(dR, nR, g.n, g.perm, used_bits, rbits, ctl, false);
    if (nS)
        k_mark_set<<<std::min<uint32_t>((nS + 255) / 256, 4096), 256, 0, st>>>(dS, nS, g.n, g.perm, used_bits, sbits, ctl, false);
    k_bits_count<<<nblocks, 1024, 0, st>>>(rbits, nwords, bsums);
    k_bits_compact<<<nblocks, 1024, 0, st>>>(rbits, nwords, bsums, nblocks, rsorted, ctl);
    RN_CUDA(cudaGetLastError());

    constexpr uint32_t T = 32;
    const uint32_t tile_src = std::max<uint32_t>(1, std::min<uint32_t>(T, (nR + NA_BLOCKS - 1) / NA_BLOCKS));
    const uint32_t ntiles = (nR + tile_src - 1) / tile_src;
    const uint32_t vbits = bits_for(g.n);
    SearchArgs a{};
    a.row_ptr = g.row_ptr;
    a.adj = reinterpret_cast<const uint2 *>(g.adj);
    a.iperm = g.iperm;
    a.sbits = sbits;
    a.src = rsorted;
    a.bound = theta;
    a.delta = std::max<uint32_t>(1, 4 * median_w);
    a.slab = slab;
    a.vbits = vbits;
    a.tile_src = tile_src;
    a.ctl = ctl;
    a.out_key = keyA;
    a.out_d = valA;
    a.out_cap = NA_MAX_PAIRS;
    a.ntiles = ntiles;
    a.H = SMEM_H;
    a.hshift = 32 - bits_for(SMEM_H);
    a.max_fill = SMEM_H * 7 / 8;
    a.failed = failed;
    a.n_nodes = g.n;
    a.n_arcs = g.arcs;
    if (ntiles) search(T, Shape::Narrow, a, std::min(ntiles, NA_BLOCKS), st);
    Control c;
    RN_CUDA(cudaMemcpyAsync(&c, ctl, sizeof(Control), cudaMemcpyDeviceToHost, st));
    RN_CUDA(cudaStreamSynchronize(st));
    if (c.n_failed && !c.err) {
        // wide blocks: the slab holds NA_BLOCKS / 2 regions of SMEM_HW rows
        RN_CUDA(cudaMemsetAsync(&ctl->tile_next, 0, 8, st));
        SearchArgs r = a;
        r.range_list = failed;
        r.ntiles = c.n_failed;
        r.failed = failed2;
        r.H = SMEM_HW;
        r.hshift = 32 - bits_for(SMEM_HW);
        r.max_fill = SMEM_HW * 7 / 8;
        search(T, Shape::Wide, r, std::min<uint32_t>(c.n_failed, NA_BLOCKS / 2), st);
        RN_CUDA(cudaMemcpyAsync(&c, ctl, sizeof(Control), cudaMemcpyDeviceToHost, st));
        RN_CUDA(cudaStreamSynchronize(st));
        if (c.n_failed) fail(RN_EINVAL, "a tile's search outgrew the no-alloc slab: use rn_distance_join_dev");
    }
    if (c.err & 1u) fail(RN_EINVAL, "a node id of R or S is >= n");
    if (c.err & 2u) fail(RN_EINVAL, "R or S repeats an id, or R and S overlap");
    *n_out = c.pairs;
    if (c.pairs > NA_MAX_PAIRS) fail(RN_EINVAL, "the join has more than 2^19 pairs, the no-alloc limit");
    if (c.pairs > out_cap) fail(RN_EINVAL, "the output buffers hold fewer entries than the join's pairs");
    if (c.pairs) {
        const uint64_t np = c.pairs;
        const uint32_t rb = uint32_t((np + RS_TILE - 1) / RS_TILE);
        unsigned long long *ki = keyA, *ko = keyB;
        uint32_t *vi = valA, *vo = valB;
        for (uint32_t sh = 0; sh < 2 * vbits; sh += 8) {
            const bool last = sh + 8 >= 2 * vbits;
            k_rs_hist<<<rb, RS_THREADS, 0, st>>>(ki, vi, np, int(sh), hist, rb);
            k_rs_scan<<<1, 1024, 0, st>>>(hist, rb * 256);
            k_rs_scatter<<<rb, RS_THREADS, 0, st>>>(ki, vi, ko, vo, np, int(sh), hist, rb, last ? out_u : nullptr,
                                                    last ? out_v : nullptr, last ? out_d : nullptr, vbits);
            std::swap(ki, ko);
            std::swap(vi, vo);
        }
        RN_CUDA(cudaGetLastError());
        RN_CUDA(cudaStreamSynchronize(st));
    }
}

// ---------------------------------------------------------- k closest pairs ----
// The answer is the first k of all pairs within theta in (d, u, v) order (Abstract;
// Section 4; Algorithm 2 takes both k and theta).  The search runs in radius passes:
// pass i searches every tile with bound tau_i, and inside a pass a global threshold --
// the least histogram edge below which k exact pairs have been emitted (Algorithm 3's
// global k-th distance) -- tightens the bound of every later tile.  A pass that ends
// with fewer than k pairs was searched with tau_i everywhere, so its pairs are all the
// pairs within tau_i: the next pass widens tau by the planar growth of the pair count
// (pairs ~ tau^2).  Once k pairs exist, every pair with d <= the k-th distance is in
// the candidates; a device radix select finds that distance, it is broadcast through
// device memory to a compaction, and the survivors are sorted by (d, u, v).

struct SelState {
    uint32_t prefix;         // digits of the k-th value chosen so far
    uint32_t pad;
    unsigned long long krem; // rank of the k-th value among the candidates still matching
};

__global__ void k_set_u32(uint32_t *p, uint32_t v) { *p = v; }

__global__ void k_sel_init(SelState *st, unsigned long long k) {
    st->prefix = 0;
    st->krem = k;
}

// Histogram of one 11/11/10-bit digit of the candidates whose higher digits equal the
// prefix chosen so far.
__global__ void k_sel_hist(const uint32_t *__restrict__ vals, uint64_t n, int shift, uint32_t nbits, uint32_t himask,
                           const SelState *st, uint32_t *hist) {
    __shared__ uint32_t h[2048];
    for (uint32_t i = threadIdx.x; i < 2048; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const uint32_t prefix = st->prefix;
    const uint32_t dmask = (1u << nbits) - 1;
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += uint64_t(gridDim.x) * blockDim.x) {
        const uint32_t v = vals[i];
        if ((v & himask) == prefix) atomicAdd(&h[(v >> shift) & dmask], 1u);
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < (1u << nbits); i += blockDim.x)
        if (h[i]) atomicAdd(&hist[i], h[i]);
}

// One warp: the digit whose bin holds the krem-th candidate; clears the histogram.
__global__ void k_sel_pick(uint32_t *hist, uint32_t nbits, int shift, SelState *st) {
    const uint32_t lane = threadIdx.x;
    const uint32_t nb = 1u << nbits, per = nb / 32;
    unsigned long long own = 0;
    for (uint32_t i = 0; i < per; i++) own += hist[lane * per + i];
    unsigned long long incl = own;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long t = __shfl_up_sync(FULL, incl, o);
        if (lane >= uint32_t(o)) incl += t;
    }
    const unsigned long long krem = st->krem;
    const uint32_t reach = __ballot_sync(FULL, incl >= krem);
    const uint32_t who = reach ? uint32_t(__ffs(reach) - 1) : 31u;
    if (lane == who) {
        unsigned long long cum = incl - own;
        uint32_t b = lane * per + per - 1;
        for (uint32_t i = 0; i < per; i++) {
            const uint32_t c = hist[lane * per + i];
            if (cum + c >= krem) {
                b = lane * per + i;
                break;
            }
            cum += c;
        }
        st->prefix |= b << shift;
        st->krem = krem - cum;
    }
    __syncwarp();
    for (uint32_t i = lane; i < nb; i += 32) hist[i] = 0;
}

// Keep the candidates with d <= the selected threshold (ties included).
__global__ void k_compact_le(const unsigned long long *__restrict__ kin, const uint32_t *__restrict__ vin,
                             uint64_t n, const SelState *st, unsigned long long *kout, uint32_t *vout,
                             unsigned long long *count) {
    const uint32_t theta = st->prefix;
    const uint32_t lane = threadIdx.x & 31;
    for (uint64_t base = (uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) & ~31ull; base < n;
         base += uint64_t(gridDim.x) * blockDim.x) {
        const uint64_t i = base + lane;
        const bool keep = i < n && vin[i] <= theta;
        const uint32_t b = __ballot_sync(FULL, keep);
        if (!b) continue;
        unsigned long long pos = 0;
        if (lane == 0) pos = atomicAdd(count, (unsigned long long)__popc(b));
        pos = __shfl_sync(FULL, pos, 0);
        if (keep) {
            const unsigned long long at = pos + __popc(b & ((1u << lane) - 1));
            kout[at] = kin[i];
            vout[at] = vin[i];
        }
    }
}

void run_kcp(const DeviceGraph &g, Workspace *ws, const EngineConfig &cfg, uint32_t median_w, const uint32_t *dR,
             uint32_t nR, const uint32_t *dS, uint32_t nS, uint64_t k, uint32_t theta, rn_dpairs *out, void *stream,
             rn_query_stats *stats) {
    cudaStream_t st = (cudaStream_t)stream;
    if (k == 0) fail(RN_EINVAL, "k must be >= 1");
    if (theta == RN_INF) theta = RN_THETA_MAX;
    if (theta > RN_THETA_MAX) fail(RN_EINVAL, "theta must be <= 2^31 or RN_INF");
    const uint32_t T = cfg.tile_width > 1 ? cfg.tile_width : 32;
    if (T != 32 && T != 64 && T != 128) fail(RN_EINVAL, "tile width must be 1, 32, 64 or 128");
    std::lock_guard<std::mutex> device_lock(ws->sh->mu);
    Range range("rn.kcp");
    *stats = rn_query_stats{};
    const bool from_s = search_from_s(g, cfg, nR, nS);
    if (from_s) {  // S's nodes are the sources, R's the targets (below, "R" is the sources)
        std::swap(dR, dS);
        std::swap(nR, nS);
    }
    stats->from_s = from_s;
    ws->launches = 0;
    RN_CUDA(cudaEventRecord(ws->ev0, st));

    ensure_slab(ws);
    const uint32_t grid_max = ws->sh->slab_ctas;  // resident narrow blocks the slab serves
    uint32_t tile_src = T;
    if (nR) {
        const uint64_t waves = (uint64_t(nR) + uint64_t(T) * grid_max - 1) / (uint64_t(T) * grid_max);
        tile_src = uint32_t(std::min<uint64_t>(T, (nR + waves * grid_max - 1) / (waves * grid_max)));
        if (cfg.tile_src) tile_src = std::min(cfg.tile_src, T);
    }
    const uint32_t ntiles = (nR + tile_src - 1) / tile_src;
    ensure_ranges(&ws->failed, &ws->failed_cap, std::max<uint32_t>(std::max(ntiles, nR), 1));
    ensure_ranges(&ws->failed2, &ws->failed2_cap, std::max<uint32_t>(std::max(ntiles, nR), 1));
    ensure_pairs(ws, std::max<uint64_t>(ws->pair_cap, std::min<uint64_t>(k + (k >> 2) + 4096, uint64_t(nR) * 64 + 4096)));
    if (!ws->kcp) {
        ws->kcp = (uint32_t *)device_alloc((KCP_BINS + 16) * 4 + sizeof(SelState));
        ws->bytes += (KCP_BINS + 16) * 4 + sizeof(SelState);
    }
    uint32_t *hist = ws->kcp, *theta_live = ws->kcp + KCP_BINS;
    SelState *sel = reinterpret_cast<SelState *>(ws->kcp + KCP_BINS + 16);

    const uint32_t vbits = bits_for(g.n);
    SearchArgs a{};
    a.row_ptr = g.row_ptr;
    a.adj = reinterpret_cast<const uint2 *>(g.adj);
    a.iperm = g.iperm;
    a.sbits = ws->sbits;
    a.slab = ws->sh->slab;
    a.vbits = vbits;
    a.ctl = ws->ctl;
    a.kcp_hist = hist;
    a.theta_live = theta_live;
    a.kcp_k = k;
    a.swap_uv = from_s;
    // a source's ball at the k-th distance holds about (k / |R|) (n / |S|) nodes (each
    // source's share of the k pairs, one S node per n / |S| nodes): a warp's map passes at
    // bucket boundaries and emission do not pay for balls of a few dozen nodes, which the
    // tile search shares between the sources of a tile
    const double kth_ball = nR && nS ? double(k) / nR * (double(g.n) / nS) : 0.0;
    const bool warp_ok = cfg.tile_width == 1 || kth_ball >= 64.0;
    // the first radius: where about 1.25 k pairs are expected, the balls growing as the
    // workspace's last warp search measured them (mean ball at its bound, times the
    // squared radius ratio) or, with none behind it, as a lattice's 2 (r / w_med)^2; a
    // radius too small costs a second pass, one too large only candidates the live
    // bound soon stops collecting
    uint64_t tau = theta;
    if (kth_ball > 0) {
        const double need = 1.25 * kth_ball;  // nodes per ball
        const double r = ws->ball_theta && ws->ball_mean > 0
                             ? double(ws->ball_theta) * std::sqrt(need / ws->ball_mean)
                             : double(std::max<uint32_t>(median_w, 1)) * std::sqrt(need / 2.0);
        tau = std::min<uint64_t>(theta, std::max<uint64_t>(uint64_t(std::min(r, 4e9)), std::max<uint32_t>(median_w, 1)));
    }
    uint64_t retried = 0;
    uint32_t passes = 0;
    Control c{};
    unsigned long long scans = 0;
    bool any_tiles = false, last_by_source = false;
    for (;;) {
        // every pass takes the warp search while the balls at tau fit a warp map
        const bool by_source = warp_ok && use_source_search(g, ws, cfg, uint32_t(tau), median_w);
        const uint32_t delta = choose_delta(cfg, median_w, by_source);
        // the warp search takes R in output order and records each source's segment
        const bool place = by_source && g.iperm_inverts_perm && !from_s;
        prep_sets(g, ws, dR, nR, dS, nS, st, place);
        a.src = ws->rsorted;  // prep_sets may have (re)allocated the R list
        a.seg = place ? ensure_segments(ws, nR, st) : nullptr;
        last_by_source = place;
        RN_CUDA(cudaMemsetAsync(hist, 0, KCP_BINS * 4, st));
        k_set_u32<<<1, 1, 0, st>>>(theta_live, uint32_t(tau));
        ws->launches++;
        uint32_t shift = 0;
        while ((tau >> shift) >= KCP_BINS) shift++;
        a.bound = uint32_t(tau);
        a.delta = delta;
        a.hist_shift = shift;
        a.out_key = ws->keyA;
        a.out_d = ws->valA;
        a.out_cap = ws->pair_cap;
        if (by_source) {
            a.tile_src = 1;
            c = source_search_all(g, ws, a, nR,
                                  source_first_map(ws, uint32_t(tau), first_ball_estimate(g, uint32_t(tau), median_w)), T,
                                  uint32_t(tau), {}, st,
                                  &retried, false);
        } else {
            a.tile_src = tile_src;
            c = search_all(g, ws, T, a, ntiles, st, &retried, cfg.map_slots);
        }
        any_tiles |= !by_source;
        check_control(c);
        if (c.pairs > ws->pair_cap) {  // the candidate buffer was too small: same pass again
            ensure_pairs(ws, c.pairs + c.pairs / 4);
            continue;
        }
        passes++;
        scans += c.scans;
        stats->delta = delta;
        if (c.pairs >= k || tau >= theta) break;
        // widen: pairs grow about as tau^2 on a road network
        double f = c.pairs ? std::sqrt(double(k) / double(c.pairs)) * 1.25 : 4.0;
        f = std::max(f, 1.5);
        tau = std::min<uint64_t>(theta, uint64_t(double(tau) * f) + 1);
    }
    stats->tile_width = any_tiles ? T : 1;
    const Control cs = c;  // the last search pass (the one the selection takes its pairs from)
    const uint64_t m = c.pairs;
    uint64_t kept = m;
    uint32_t theta_k = uint32_t(tau);
    const bool placed = last_by_source && m && can_place(ws, cs);
    if (placed) {
        // the warp search's segments placed in (u, v) order, then a stable LSD sort of all
        // candidates by distance alone: (d, u, v) order, of which the first k are the answer
        // (no selection: three distance passes instead of the (u, v) digits' six)
        place_pairs(ws, nR, vbits, 0xFFFFFFFFu, nullptr, st);
        dpairs_reserve(out, m);
        std::vector<int> shifts;
        const uint32_t dbits = bits_for(uint32_t(std::min<uint64_t>(tau, RN_THETA_MAX)) + 1);
        for (uint32_t sh = 0; sh < dbits; sh += 8) shifts.push_back(64 + int(sh));
        radix_sort_to_pairs(ws, m, shifts, vbits, out, st);
        out->n = std::min<uint64_t>(k, m);
        if (m >= k) RN_CUDA(cudaMemcpyAsync(&theta_k, out->d + (k - 1), 4, cudaMemcpyDeviceToHost, st));
    } else if (m > k) {
        // device radix select of the k-th distance (11 + 11 + 10 bits), then broadcast
        // through device memory to the compaction
        k_sel_init<<<1, 1, 0, st>>>(sel, k);
        RN_CUDA(cudaMemsetAsync(hist, 0, KCP_BINS * 4, st));
        const uint32_t grid = std::min<uint64_t>((m + 255) / 256, uint64_t(ws->num_sms) * 8);
        const int shifts[3] = {21, 10, 0};
        const uint32_t nbits[3] = {11, 11, 10};
        const uint32_t himask[3] = {0u, 0xFFE00000u, 0xFFFFFC00u};
        for (int r = 0; r < 3; r++) {
            k_sel_hist<<<grid, 256, 0, st>>>(ws->valA, m, shifts[r], nbits[r], himask[r], sel, hist);
            k_sel_pick<<<1, 32, 0, st>>>(hist, nbits[r], shifts[r], sel);
        }
        RN_CUDA(cudaMemsetAsync(&ws->ctl->pairs, 0, 8, st));
        k_compact_le<<<grid, 256, 0, st>>>(ws->keyA, ws->valA, m, sel, ws->keyB, ws->valB, &ws->ctl->pairs);
        ws->launches += 1 + 6 + 1;
        RN_CUDA(cudaGetLastError());
        SelState hs{};
        RN_CUDA(cudaMemcpyAsync(&hs, sel, sizeof(hs), cudaMemcpyDeviceToHost, st));
        c = read_control(ws, st);
        kept = c.pairs;
        theta_k = hs.prefix;
        std::swap(ws->keyA, ws->keyB);
        std::swap(ws->valA, ws->valB);
    }
    if (!placed) {
        // canonical (d, u, v) order: (u, v) digits first, then the distance digits
        dpairs_reserve(out, kept);
        std::vector<int> shifts;
        for (uint32_t sh = 0; sh < 2 * vbits; sh += 8) shifts.push_back(int(sh));
        const uint32_t dbits = bits_for(theta_k + 1);
        for (uint32_t sh = 0; sh < dbits; sh += 8) shifts.push_back(64 + int(sh));
        radix_sort_to_pairs(ws, kept, shifts, vbits, out, st);
        out->n = std::min<uint64_t>(k, kept);
    }
    RN_CUDA(cudaEventRecord(ws->ev1, st));
    RN_CUDA(cudaEventSynchronize(ws->ev1));
    float ms = 0, sms = 0;
    RN_CUDA(cudaEventElapsedTime(&ms, ws->ev0, ws->ev1));
    RN_CUDA(cudaEventElapsedTime(&sms, ws->evs0, ws->evs1));
    stats->pairs = out->n;
    stats->tiles = ntiles;
    stats->tile_sources = tile_src;
    stats->retried_tiles = retried;
    stats->scans = scans;
    stats->passes = passes;
    stats->theta_final = m >= k ? theta_k : uint32_t(tau);
    stats->launches = ws->launches;
    stats->blocks_per_sm = uint32_t(ws->blocks_per_sm);
    stats->device_ms = ms;
    stats->search_ms = sms;
    stats->search_pairs = m;
    stats->slots = cs.slots;
    stats->slot_arcs = cs.slot_arcs;
    stats->slot_lanes = cs.slot_lanes;
    stats->rounds = cs.rounds;
    stats->round_items = cs.round_items;
    stats->boundaries = cs.boundaries;
    stats->round_arcs = cs.round_arcs;
    stats->max_ball = cs.max_fill;
    stats->cycles_rounds = cs.cyc_round;
    stats->cycles_boundaries = cs.cyc_bound;
    stats->cycles_emission = cs.cyc_emit;
}

// ------------------------------------------------------------ points on edges ----
// Joins and k closest pairs of points that lie on edges (objects moving on the road
// network, searched from the two ends of their edge: Section 1).  The query runs the
// ordinary engine over the graph subdivided at its points: every point becomes a node,
// and every edge {p, q} that carries points becomes a chain p - o_1 - ... - o_k - q with
// links of the positions' differences (a point at an end, or two points at one
// position, give links of weight 0).  The subdivided graph is built on the device for
// each query: a copy of the graph's arrays, the two arcs p->q and q->p turned into the
// chain's first and last links, and two arcs per point node; the point nodes' output
// ids are their indices in R and S.  R's points are numbered in the order of their
// edges' internal ids, so a tile's sources lie near each other.

// For each undirected edge {p, q} (p < q, internal ids): the positions of the arcs
// p->q and q->p in adj and their weights, EMPTY where there is no such arc.
__global__ void k_edge_find(const uint32_t *__restrict__ row_ptr, const uint2 *__restrict__ adj,
                            const uint2 *__restrict__ keys, uint32_t nkeys, uint4 *out) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nkeys; i += gridDim.x * blockDim.x) {
        const uint2 k = keys[i];
        uint4 r = make_uint4(EMPTY, EMPTY, EMPTY, EMPTY);
        for (uint32_t e = row_ptr[k.x]; e < row_ptr[k.x + 1]; e++)
            if (adj[e].x == k.y && (r.x == EMPTY || adj[e].y < r.z)) {
                r.x = e;
                r.z = adj[e].y;
            }
        for (uint32_t e = row_ptr[k.y]; e < row_ptr[k.y + 1]; e++)
            if (adj[e].x == k.x && (r.y == EMPTY || adj[e].y < r.w)) {
                r.y = e;
                r.w = adj[e].y;
            }
        out[i] = r;
    }
}

// adj[pos] = (target, weight) for every patch (pos, target, weight).
__global__ void k_patch_arcs(uint2 *adj, const uint4 *__restrict__ patches, uint32_t n, uint64_t arcs) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint4 pt = patches[i];
        if (pt.x < arcs) adj[pt.x] = make_uint2(pt.y, pt.z);
    }
}

struct PointsState {
    DeviceGraph aug;
    uint64_t cap_nodes = 0, cap_arcs = 0;
    Workspace *ws = nullptr;  // bitmaps sized for cap_nodes
    uint32_t *ids = nullptr;  // R ids then S ids (the point nodes)
    uint32_t cap_ids = 0;
    uint2 *keys = nullptr;
    uint4 *found = nullptr, *patches = nullptr;
    uint32_t cap_keys = 0;
};

void points_destroy(PointsState *ps) {
    if (!ps) return;
    for (void *p : {(void *)ps->aug.row_ptr, (void *)ps->aug.adj, (void *)ps->aug.perm, (void *)ps->aug.iperm,
                    (void *)ps->ids, (void *)ps->keys, (void *)ps->found, (void *)ps->patches})
        device_free(p);
    workspace_destroy(ps->ws);
    delete ps;
}

// Build the subdivided graph for the points in ps->aug (grow-only buffers).
static void points_graph(const DeviceGraph &g, const std::vector<uint32_t> &perm, const rn_point *R, uint32_t nR,
                         const rn_point *S, uint32_t nS, PointsState *ps, cudaStream_t st) {
    const uint32_t np = nR + nS;
    const uint64_t n_aug = uint64_t(g.n) + np, arcs_aug = g.arcs + 2ull * np;
    if (n_aug >= 0xFFFFFFFFull || arcs_aug >= 0xFFFFFFFFull) fail(RN_EINVAL, "too many points for this graph");
    struct P {
        uint32_t p, q, pos_raw, from_p, idx;  // edge {p < q}; t from a; a == p?; index in R ++ S
    };
    std::vector<P> pts(np);
    for (uint32_t i = 0; i < np; i++) {
        const rn_point &x = i < nR ? R[i] : S[i - nR];
        const uint32_t a = perm[x.a], b = perm[x.b];
        pts[i] = {std::min(a, b), std::max(a, b), x.t, a < b ? 1u : 0u, i};
    }
    // the distinct edges, and their arcs on the device
    std::vector<uint32_t> order(np);
    for (uint32_t i = 0; i < np; i++) order[i] = i;
    std::sort(order.begin(), order.end(), [&](uint32_t x, uint32_t y) {
        return pts[x].p != pts[y].p ? pts[x].p < pts[y].p : pts[x].q != pts[y].q ? pts[x].q < pts[y].q : x < y;
    });
    std::vector<uint2> keys;
    std::vector<uint32_t> key_of(np);
    for (uint32_t j = 0; j < np; j++) {
        const P &x = pts[order[j]];
        if (keys.empty() || keys.back().x != x.p || keys.back().y != x.q) keys.push_back(make_uint2(x.p, x.q));
        key_of[order[j]] = uint32_t(keys.size() - 1);
    }
    const uint32_t nk = uint32_t(keys.size());
    if (ps->cap_keys < std::max<uint32_t>(nk, 1)) {
        for (void **q : {(void **)&ps->keys, (void **)&ps->found, (void **)&ps->patches}) {
            device_free(*q);
            *q = nullptr;
        }
        ps->cap_keys = std::max<uint32_t>(nk, 1024);
        ps->keys = (uint2 *)device_alloc(size_t(ps->cap_keys) * 8);
        ps->found = (uint4 *)device_alloc(size_t(ps->cap_keys) * 16);
        ps->patches = (uint4 *)device_alloc(size_t(ps->cap_keys) * 2 * 16);
    }
    std::vector<uint4> found(nk);
    if (nk) {
        RN_CUDA(cudaMemcpyAsync(ps->keys, keys.data(), size_t(nk) * 8, cudaMemcpyHostToDevice, st));
        k_edge_find<<<std::min<uint32_t>((nk + 255) / 256, 1024), 256, 0, st>>>(
            g.row_ptr, reinterpret_cast<const uint2 *>(g.adj), ps->keys, nk, ps->found);
        RN_CUDA(cudaGetLastError());
        RN_CUDA(cudaMemcpyAsync(found.data(), ps->found, size_t(nk) * 16, cudaMemcpyDeviceToHost, st));
        RN_CUDA(cudaStreamSynchronize(st));
    }
    // positions from p, checked against the edge
    std::vector<uint32_t> pos(np);
    for (uint32_t i = 0; i < np; i++) {
        const uint4 f = found[key_of[i]];
        const rn_point &x = i < nR ? R[i] : S[i - nR];
        const std::string who = (i < nR ? "R[" + std::to_string(i) : "S[" + std::to_string(i - nR)) + "]";
        if (f.x == EMPTY || f.y == EMPTY || f.z != f.w)
            fail(RN_EINVAL, who + ": {" + std::to_string(x.a) + ", " + std::to_string(x.b) + "} is not an undirected edge");
        if (pts[i].pos_raw > f.z) fail(RN_EINVAL, who + ": t is longer than its edge");
        pos[i] = pts[i].from_p ? pts[i].pos_raw : f.z - pts[i].pos_raw;
    }
    // node ids: R points in the order of their edges (locality), then S points
    std::vector<uint32_t> node(np), rank_ids(np);
    {
        uint32_t nextR = 0, nextS = 0;
        for (uint32_t j = 0; j < np; j++) {
            const uint32_t i = order[j];
            if (i < nR) node[i] = g.n + nextR++;
        }
        for (uint32_t i = nR; i < np; i++) node[i] = g.n + nR + nextS++;
        for (uint32_t i = 0; i < np; i++) rank_ids[node[i] - g.n] = i < nR ? i : i - nR;
    }
    // chains: per edge, its points by position (then index), links between neighbours
    std::vector<uint32_t> tail(2 * size_t(np) * 2);  // object rows: (col, w) x 2 per point node
    std::vector<uint4> patches;
    patches.reserve(2 * size_t(nk));
    std::sort(order.begin(), order.end(), [&](uint32_t x, uint32_t y) {
        if (key_of[x] != key_of[y]) return key_of[x] < key_of[y];
        return pos[x] != pos[y] ? pos[x] < pos[y] : x < y;
    });
    for (uint32_t j = 0; j < np;) {
        uint32_t e = j;
        while (e < np && key_of[order[e]] == key_of[order[j]]) e++;
        const uint32_t k = key_of[order[j]];
        const uint4 f = found[k];
        const uint32_t p = keys[k].x, q = keys[k].y, w = f.z;
        for (uint32_t c = j; c < e; c++) {
            const uint32_t i = order[c], me = node[i] - g.n;
            const uint32_t prev = c == j ? p : node[order[c - 1]], prev_pos = c == j ? 0 : pos[order[c - 1]];
            const uint32_t next = c + 1 == e ? q : node[order[c + 1]], next_pos = c + 1 == e ? w : pos[order[c + 1]];
            tail[4 * size_t(me) + 0] = prev;
            tail[4 * size_t(me) + 1] = pos[i] - prev_pos;
            tail[4 * size_t(me) + 2] = next;
            tail[4 * size_t(me) + 3] = next_pos - pos[i];
        }
        patches.push_back(make_uint4(f.x, node[order[j]], pos[order[j]], 0));            // p -> o_1
        patches.push_back(make_uint4(f.y, node[order[e - 1]], w - pos[order[e - 1]], 0));  // q -> o_k
        j = e;
    }
    // the subdivided graph's arrays
    if (ps->cap_nodes < n_aug || ps->cap_arcs < arcs_aug) {
        for (void **q : {(void **)&ps->aug.row_ptr, (void **)&ps->aug.adj, (void **)&ps->aug.perm, (void **)&ps->aug.iperm}) {
            device_free(*q);
            *q = nullptr;
        }
        ps->cap_nodes = n_aug + n_aug / 4;
        ps->cap_arcs = arcs_aug + arcs_aug / 4;
        ps->aug.row_ptr = (uint32_t *)device_alloc((ps->cap_nodes + 1) * 4);
        ps->aug.adj = (uint32_t *)device_alloc(ps->cap_arcs * 8);
        ps->aug.perm = (uint32_t *)device_alloc(ps->cap_nodes * 4);
        ps->aug.iperm = (uint32_t *)device_alloc(ps->cap_nodes * 4);
        workspace_destroy(ps->ws);
        ps->ws = nullptr;
        DeviceGraph capg{};
        capg.n = uint32_t(ps->cap_nodes);
        ps->ws = workspace_create(capg);
    }
    ps->aug.n = uint32_t(n_aug);
    ps->aug.arcs = arcs_aug;
    std::vector<uint32_t> rp_tail(np), perm_tail(np);
    for (uint32_t i = 0; i < np; i++) {
        rp_tail[i] = uint32_t(g.arcs + 2ull * (i + 1));  // row_ptr[n + 1 + i]
        perm_tail[i] = g.n + i;                          // the point nodes are named by themselves
    }
    RN_CUDA(cudaMemcpyAsync(ps->aug.row_ptr, g.row_ptr, (size_t(g.n) + 1) * 4, cudaMemcpyDeviceToDevice, st));
    RN_CUDA(cudaMemcpyAsync(ps->aug.adj, g.adj, g.arcs * 8, cudaMemcpyDeviceToDevice, st));
    ps->aug.iperm_inverts_perm = false;  // a point node's output id is its index in R or S
    RN_CUDA(cudaMemcpyAsync(ps->aug.perm, g.perm, size_t(g.n) * 4, cudaMemcpyDeviceToDevice, st));
    RN_CUDA(cudaMemcpyAsync(ps->aug.iperm, g.iperm, size_t(g.n) * 4, cudaMemcpyDeviceToDevice, st));
    if (np) {
        RN_CUDA(cudaMemcpyAsync(ps->aug.row_ptr + g.n + 1, rp_tail.data(), size_t(np) * 4, cudaMemcpyHostToDevice, st));
        RN_CUDA(cudaMemcpyAsync(ps->aug.adj + 2 * g.arcs, tail.data(), size_t(np) * 16, cudaMemcpyHostToDevice, st));
        RN_CUDA(cudaMemcpyAsync(ps->aug.perm + g.n, perm_tail.data(), size_t(np) * 4, cudaMemcpyHostToDevice, st));
        RN_CUDA(cudaMemcpyAsync(ps->aug.iperm + g.n, rank_ids.data(), size_t(np) * 4, cudaMemcpyHostToDevice, st));
        RN_CUDA(cudaMemcpyAsync(ps->patches, patches.data(), patches.size() * 16, cudaMemcpyHostToDevice, st));
        k_patch_arcs<<<std::min<uint32_t>((uint32_t(patches.size()) + 255) / 256, 1024), 256, 0, st>>>(
            reinterpret_cast<uint2 *>(ps->aug.adj), ps->patches, uint32_t(patches.size()), g.arcs);
        RN_CUDA(cudaGetLastError());
    }
    // the query's sets: the point nodes
    if (ps->cap_ids < std::max<uint32_t>(np, 1)) {
        device_free(ps->ids);
        ps->ids = nullptr;
        ps->cap_ids = std::max<uint32_t>(np, 1024);
        ps->ids = (uint32_t *)device_alloc(size_t(ps->cap_ids) * 4);
    }
    if (np) RN_CUDA(cudaMemcpyAsync(ps->ids, perm_tail.data(), size_t(np) * 4, cudaMemcpyHostToDevice, st));
    RN_CUDA(cudaStreamSynchronize(st));  // the host vectors above are temporaries
}

void run_points(const DeviceGraph &g, const std::vector<uint32_t> &perm, PointsState **state, const EngineConfig &cfg,
                uint32_t median_w, const rn_point *R, uint32_t nR, const rn_point *S, uint32_t nS, uint64_t k,
                uint32_t theta, rn_dpairs *out, void *stream, rn_query_stats *stats) {
    if (!*state) *state = new PointsState();
    PointsState *ps = *state;
    cudaStream_t st = (cudaStream_t)stream;
    {
        Range r("rn.points.subdivide");
        points_graph(g, perm, R, nR, S, nS, ps, st);
    }
    EngineConfig pc = cfg;
    pc.search_from = RN_FROM_R;  // the points' searches start from R's points
    if (k == 0)
        run_join(ps->aug, ps->ws, pc, median_w, ps->ids, nR, ps->ids + nR, nS, theta, out, stream, stats);
    else
        run_kcp(ps->aug, ps->ws, pc, median_w, ps->ids, nR, ps->ids + nR, nS, k, theta, out, stream, stats);
}

// ----------------------------------------------------- queries in a rectangle ----
// Geographically constrained queries (Section 2: processing is restricted to the
// partitions that satisfy the constraint, by a comparison with each partition's MBR).
// A member of R or S belongs to the query when its node lies in the closed rectangle
// box = (xmin, ymin, xmax, ymax).  The members are filtered on the device leaf by leaf:
// a leaf whose bounding rectangle lies inside the box keeps all its members, one that
// misses the box drops them, and only a leaf that straddles the box's border tests each
// member's own coordinates.  Distances are still network distances over the whole graph
// (a path may leave the rectangle); only the sets are restricted.

struct BoxState {
    uint32_t *ids = nullptr;     // R survivors, then S survivors
    uint32_t cap = 0;
    unsigned long long *counts = nullptr;  // R kept, S kept, members decided by a whole leaf
    unsigned long long *counts_host = nullptr;  // pinned
};

void box_destroy(BoxState *bs) {
    if (!bs) return;
    device_free(bs->ids);
    device_free(bs->counts);
    if (bs->counts_host) cudaFreeHost(bs->counts_host);
    delete bs;
}

// Keep the ids (original node ids) whose node lies in the box, appending them to out
// (order not kept: the query's preparation sorts its sets); counts[slot] gets the
// survivors and counts[2] the members decided by their leaf's rectangle alone.  An id
// >= n is kept, for the query's own validation to reject.
__global__ void k_box_filter(const uint32_t *__restrict__ ids, uint32_t cnt, uint32_t n,
                             const uint32_t *__restrict__ perm, const uint32_t *__restrict__ leaf_start,
                             uint32_t nleaves, const float4 *__restrict__ leaf_box, const float2 *__restrict__ xy,
                             float4 box, uint32_t *out, unsigned long long *counts, uint32_t slot) {
    const uint32_t lane = threadIdx.x & 31;
    for (uint32_t base = (blockIdx.x * blockDim.x + threadIdx.x) & ~31u; base < cnt; base += gridDim.x * blockDim.x) {
        const uint32_t i = base + lane;
        bool keep = false, whole = false;
        if (i < cnt) {
            const uint32_t id = ids[i];
            if (id >= n) {
                keep = true;
            } else {
                const uint32_t x = perm[id];
                // the leaf holding x: the last leaf starting at or before x
                uint32_t lo = 0, hi = nleaves - 1;
                while (lo < hi) {
                    const uint32_t mid = (lo + hi + 1) >> 1;
                    if (leaf_start[mid] <= x) lo = mid;
                    else hi = mid - 1;
                }
                const float4 b = leaf_box[lo];
                if (b.x >= box.x && b.z <= box.z && b.y >= box.y && b.w <= box.w) {
                    keep = whole = true;  // the leaf lies inside the box
                } else if (b.z < box.x || b.x > box.z || b.w < box.y || b.y > box.w) {
                    whole = true;  // the leaf misses the box
                } else {
                    const float2 q = xy[x];
                    keep = q.x >= box.x && q.x <= box.z && q.y >= box.y && q.y <= box.w;
                }
            }
        }
        const uint32_t kb = __ballot_sync(FULL, keep);
        const uint32_t wb = __ballot_sync(FULL, whole);
        uint32_t at = 0;
        if (lane == 0) {
            if (kb) at = uint32_t(atomicAdd(&counts[slot], (unsigned long long)__popc(kb)));
            if (wb) atomicAdd(&counts[2], (unsigned long long)__popc(wb));
        }
        at = __shfl_sync(FULL, at, 0);
        if (keep) out[at + __popc(kb & ((1u << lane) - 1))] = ids[i];
    }
}

void run_box(const DeviceGraph &g, Workspace *ws, BoxState **state, const EngineConfig &cfg, uint32_t median_w,
             const uint32_t *dR, uint32_t nR, const uint32_t *dS, uint32_t nS, const float *box, uint32_t which,
             uint64_t k, uint32_t theta, rn_dpairs *out, void *stream, rn_query_stats *stats, uint64_t *leaves_whole) {
    cudaStream_t st = (cudaStream_t)stream;
    if (!g.xy || !g.leaf_box) fail(RN_EINVAL, "the graph was loaded without node coordinates");
    if (!(box[0] <= box[2] && box[1] <= box[3])) fail(RN_EINVAL, "the box must have xmin <= xmax and ymin <= ymax");
    if (which & ~uint32_t(RN_BOX_R | RN_BOX_S)) fail(RN_EINVAL, "unknown box flag");
    if (!*state) *state = new BoxState();
    BoxState *bs = *state;
    if (!bs->counts) {
        bs->counts = (unsigned long long *)device_alloc(4 * 8);
        RN_CUDA(cudaMallocHost(&bs->counts_host, 4 * 8));
    }
    const uint64_t want = uint64_t(nR) + nS;
    if (bs->cap < want) {
        device_free(bs->ids);
        bs->ids = nullptr;
        bs->cap = uint32_t(std::min<uint64_t>(std::max<uint64_t>(want + want / 4, 1024), 0xFFFFFFFFull));
        bs->ids = (uint32_t *)device_alloc(size_t(bs->cap) * 4);
    }
    uint32_t *oR = bs->ids, *oS = bs->ids + nR;
    const float4 b4 = make_float4(box[0], box[1], box[2], box[3]);
    RN_CUDA(cudaMemsetAsync(bs->counts, 0, 4 * 8, st));
    // a set the box does not restrict is copied whole
    if (nR) {
        if (which & RN_BOX_R)
            k_box_filter<<<std::min<uint32_t>((nR + 255) / 256, 4096), 256, 0, st>>>(
                dR, nR, g.n, g.perm, g.leaf_start, g.nleaves, g.leaf_box, g.xy, b4, oR, bs->counts, 0);
        else
            RN_CUDA(cudaMemcpyAsync(oR, dR, size_t(nR) * 4, cudaMemcpyDeviceToDevice, st));
    }
    if (nS) {
        if (which & RN_BOX_S)
            k_box_filter<<<std::min<uint32_t>((nS + 255) / 256, 4096), 256, 0, st>>>(
                dS, nS, g.n, g.perm, g.leaf_start, g.nleaves, g.leaf_box, g.xy, b4, oS, bs->counts, 1);
        else
            RN_CUDA(cudaMemcpyAsync(oS, dS, size_t(nS) * 4, cudaMemcpyDeviceToDevice, st));
    }
    RN_CUDA(cudaGetLastError());
    RN_CUDA(cudaMemcpyAsync(bs->counts_host, bs->counts, 4 * 8, cudaMemcpyDeviceToHost, st));
    RN_CUDA(cudaStreamSynchronize(st));
    const uint32_t kR = (which & RN_BOX_R) ? uint32_t(bs->counts_host[0]) : nR;
    const uint32_t kS = (which & RN_BOX_S) ? uint32_t(bs->counts_host[1]) : nS;
    *leaves_whole = bs->counts_host[2];
    if (k) run_kcp(g, ws, cfg, median_w, oR, kR, oS, kS, k, theta, out, stream, stats);
    else run_join(g, ws, cfg, median_w, oR, kR, oS, kS, theta, out, stream, stats);
}

// ------------------------------------------------------ hierarchical variant ----
// The paper's hierarchical processing (Section 4; Algorithms 2-4) on the GPU.  The graph's
// partition hierarchy (Algorithm 1) is cut into parts of at most a given size (the
// granularity the paper chooses by its degree of parallelism); then
//   1. local processing: from every u in R a search confined to u's own part (no arc that
//      leaves the part is relaxed), which gives the pairs inside the part and the routes
//      from u to the part's border nodes ("inside routes": a border node has an arc that
//      leaves its part);
//   2. cross-edge expansion: each route (u, b, d) is extended over every arc b -> f that
//      leaves u's part, giving (u, f, d + w); for every far end f one search runs (bounded
//      by theta less the least such offset), and its S-hits are shared by every u that
//      reaches f -- the reuse of the inside routes that Algorithm 4 makes;
//   3. combination: every (u, f, off) with every hit (f, y, e) of f gives the candidate
//      (u, y, off + e) within theta, and each pair keeps its least distance, merged with
//      the local pairs (Algorithm 3 merging the partial results).
// Exactness (a reading: the listing expands a cross-edge only inside the sibling partition,
// which can overstate a distance whose shortest path crosses a border more than once):
// here the search from f is not confined.  A shortest u -> y path either stays in u's part,
// or leaves it a first time over some arc b -> f; its part before that arc lies inside the
// part, so its length is at least d_part(u, b) + w(b, f) + d(f, y), which is a u -> y walk;
// the least candidate is therefore dist(u, y).  k closest pairs take the join within a
// radius grown until it holds k pairs (radius passes), then the first k in (d, u, v) order.

struct HierState {
    std::vector<uint32_t> cut;      // part starts the border bitmap below was built for
    cudaEvent_t ev[2] = {nullptr, nullptr};
    uint32_t *part_start = nullptr, *border = nullptr;
    uint32_t cap_parts = 0, cap_border = 0;
    struct Buf {
        void *p = nullptr;
        size_t bytes = 0;
    };
    std::map<std::string, Buf> bufs;
    unsigned long long *count = nullptr, *count_host = nullptr;  // 4 device counters, pinned copy
    template <class T>
    T *get(const char *name, uint64_t n) {
        Buf &b = bufs[name];
        const size_t want = std::max<size_t>(size_t(n) * sizeof(T), 256);
        if (b.bytes < want) {
            device_free(b.p);
            b.p = nullptr;
            b.bytes = 0;
            b.p = device_alloc(want + want / 4);
            b.bytes = want + want / 4;
        }
        return static_cast<T *>(b.p);
    }
};

void hier_destroy(HierState *h) {
    if (!h) return;
    device_free(h->part_start);
    device_free(h->border);
    for (auto &kv : h->bufs) device_free(kv.second.p);
    device_free(h->count);
    if (h->count_host) cudaFreeHost(h->count_host);
    for (cudaEvent_t e : h->ev)
        if (e) cudaEventDestroy(e);
    delete h;
}

// The part of internal id x: the last part starting at or before it.
__device__ __forceinline__ uint32_t part_of(const uint32_t *__restrict__ start, uint32_t nparts, uint32_t x) {
    uint32_t lo = 0, hi = nparts - 1;
    while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (start[mid] <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Border bitmap: node x is a border node when one of its arcs leaves its part.
__global__ void k_border_bits(const uint32_t *__restrict__ row_ptr, const uint2 *__restrict__ adj, uint32_t n,
                              const uint32_t *__restrict__ start, uint32_t nparts, uint32_t *bits) {
    for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x) {
        const uint32_t p = part_of(start, nparts, x);
        const uint32_t lo = start[p], hi = p + 1 < nparts ? start[p + 1] : n;
        bool out = false;
        for (uint32_t e = row_ptr[x]; e < row_ptr[x + 1] && !out; e++) {
            const uint32_t y = adj[e].x;
            out = y < lo || y >= hi;
        }
        if (out) atomicOr(&bits[x >> 5], 1u << (x & 31));
    }
}

// Extend every inside route (si << 32 | b, d) over the arcs b -> f that leave source si's
// part: exit routes (orig(f) << 32 | si, d + w) within theta.  Warp-aggregated appends.
__global__ void k_exit_expand(const unsigned long long *__restrict__ brd_key, const uint32_t *__restrict__ brd_d,
                              uint64_t nb, const uint2 *__restrict__ src_range, const uint32_t *__restrict__ row_ptr,
                              const uint2 *__restrict__ adj, const uint32_t *__restrict__ iperm, uint32_t theta,
                              unsigned long long *ex_key, uint32_t *ex_d, uint64_t cap, unsigned long long *count) {
    const uint32_t lane = threadIdx.x & 31;
    for (uint64_t base = (uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) & ~31ull; base < nb;
         base += uint64_t(gridDim.x) * blockDim.x) {
        const uint64_t i = base + lane;
        uint32_t si = 0, x = 0, d = 0, e0 = 0, e1 = 0, c = 0;
        uint2 r = make_uint2(0, 0);
        if (i < nb) {
            const unsigned long long kk = brd_key[i];
            si = uint32_t(kk >> 32);
            x = uint32_t(kk);
            d = brd_d[i];
            r = src_range[si];
            e0 = row_ptr[x];
            e1 = row_ptr[x + 1];
            for (uint32_t e = e0; e < e1; e++) {
                const uint2 a = adj[e];
                c += (a.x < r.x || a.x >= r.y) && uint64_t(d) + a.y <= theta;
            }
        }
        uint32_t incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(FULL, incl, o);
            if (lane >= uint32_t(o)) incl += t;
        }
        unsigned long long at = 0;
        if (lane == 31 && incl) at = atomicAdd(count, (unsigned long long)incl);
        at = __shfl_sync(FULL, at, 31) + (incl - c);
        for (uint32_t e = e0; e < e1 && c; e++) {
            const uint2 a = adj[e];
            if ((a.x < r.x || a.x >= r.y) && uint64_t(d) + a.y <= theta) {
                if (at < cap) {
                    ex_key[at] = ((unsigned long long)iperm[a.x] << 32) | si;
                    ex_d[at] = d + a.y;
                }
                at++;
            }
        }
    }
}

// Flags over records sorted by key: keep[i] = first of its key, head[i] = first of its
// key's upper 32 bits (its far end f).
__global__ void k_exit_flags(const unsigned long long *__restrict__ key, uint64_t m, uint32_t *keep, uint32_t *head) {
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < m; i += uint64_t(gridDim.x) * blockDim.x) {
        const unsigned long long k = key[i];
        const bool first = i == 0 || key[i - 1] != k;
        keep[i] = first;
        head[i] = first && (i == 0 || (key[i - 1] >> 32) != (k >> 32));
    }
}

// Compact the kept exit routes (each (f, si) with its least offset: records sorted by key
// then offset) into (j << 32 | si, off), j the index of far end f in f_list; f_list[j] =
// orig(f), fmin[j] = its least offset (fmin starts at INF).
__global__ void k_exit_compact(const unsigned long long *__restrict__ key, const uint32_t *__restrict__ d, uint64_t m,
                               const uint32_t *__restrict__ keep, const uint32_t *__restrict__ keep_at,
                               const uint32_t *__restrict__ head, const uint32_t *__restrict__ head_at,
                               unsigned long long *e_key, uint32_t *e_off, uint32_t *f_list, uint32_t *fmin) {
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < m; i += uint64_t(gridDim.x) * blockDim.x) {
        if (!keep[i]) continue;
        const unsigned long long k = key[i];
        const uint32_t j = head_at[i] + head[i] - 1;
        if (head[i]) f_list[j] = uint32_t(k >> 32);
        e_key[keep_at[i]] = ((unsigned long long)j << 32) | uint32_t(k);
        e_off[keep_at[i]] = d[i];
        atomicMin(&fmin[j], d[i]);
    }
}

// Sources of the searches from the far ends: internal ids and per-source tables.
__global__ void k_exit_sources(const uint32_t *__restrict__ f_list, const uint32_t *__restrict__ fmin, uint32_t nf,
                               const uint32_t *__restrict__ perm, uint32_t theta, uint32_t delta, uint32_t *src,
                               uint32_t *tb, uint32_t *td, uint32_t *ti) {
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < nf; j += gridDim.x * blockDim.x) {
        src[j] = perm[f_list[j]];
        tb[j] = theta - min(fmin[j], theta);
        td[j] = delta;
        ti[j] = 0;
    }
}

// The hits of far end j: the run of sorted hit keys (orig(f) << vbits | v) with f_list[j].
__global__ void k_hit_ranges(const unsigned long long *__restrict__ hkey, uint64_t nh,
                             const uint32_t *__restrict__ f_list, uint32_t nf, uint32_t vbits, uint2 *range) {
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < nf; j += gridDim.x * blockDim.x) {
        const unsigned long long lo_key = (unsigned long long)f_list[j] << vbits;
        const unsigned long long hi_key = (unsigned long long)(f_list[j] + 1ull) << vbits;
        uint64_t a = 0, b = nh;
        while (a < b) {
            const uint64_t mid = (a + b) >> 1;
            if (hkey[mid] < lo_key) a = mid + 1;
            else b = mid;
        }
        uint64_t c = a, e = nh;
        while (c < e) {
            const uint64_t mid = (c + e) >> 1;
            if (hkey[mid] < hi_key) c = mid + 1;
            else e = mid;
        }
        range[j] = make_uint2(uint32_t(a), uint32_t(c));
    }
}

// Candidates: exit route (j << 32 | si, off) with every hit (f_j, v, e) of its far end,
// (orig(u_si) << vbits | v, off + e) when within theta.  A warp per exit route.
__global__ void k_hier_combine(const unsigned long long *__restrict__ e_key, const uint32_t *__restrict__ e_off,
                               uint64_t ne, const uint2 *__restrict__ range, const unsigned long long *__restrict__ hkey,
                               const uint32_t *__restrict__ hd, const uint32_t *__restrict__ src,
                               const uint32_t *__restrict__ iperm, uint32_t theta, uint32_t vbits,
                               unsigned long long *c_key, uint32_t *c_d, uint64_t cap, unsigned long long *count) {
    const uint32_t lane = threadIdx.x & 31, lt = (1u << lane) - 1;
    const uint64_t warps = uint64_t(gridDim.x) * (blockDim.x / 32);
    const unsigned long long vmask = (1ull << vbits) - 1;
    for (uint64_t i = uint64_t(blockIdx.x) * (blockDim.x / 32) + (threadIdx.x >> 5); i < ne; i += warps) {
        const unsigned long long ek = e_key[i];
        const uint32_t j = uint32_t(ek >> 32), si = uint32_t(ek), off = e_off[i];
        const uint2 r = range[j];
        const unsigned long long u = (unsigned long long)iperm[src[si]] << vbits;
        for (uint32_t h0 = r.x; h0 < r.y; h0 += 32) {
            const uint32_t h = h0 + lane;
            const bool ok = h < r.y && uint64_t(off) + hd[h] <= theta;
            const uint32_t b = __ballot_sync(FULL, ok);
            if (!b) continue;
            unsigned long long at = 0;
            if (lane == 0) at = atomicAdd(count, (unsigned long long)__popc(b));
            at = __shfl_sync(FULL, at, 0) + __popc(b & lt);
            if (ok && at < cap) {
                c_key[at] = u | (hkey[h] & vmask);
                c_d[at] = off + hd[h];
            }
        }
    }
}

// Flags of the first record of every key (records sorted by key, then distance).
__global__ void k_first_of_key(const unsigned long long *__restrict__ key, uint64_t m, uint32_t *first) {
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < m; i += uint64_t(gridDim.x) * blockDim.x)
        first[i] = i == 0 || key[i - 1] != key[i];
}

// The first (least-distance) record of every key, compacted in key order.
__global__ void k_first_compact(const unsigned long long *__restrict__ key, const uint32_t *__restrict__ d, uint64_t m,
                                const uint32_t *__restrict__ first, const uint32_t *__restrict__ at,
                                unsigned long long *okey, uint32_t *od) {
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < m; i += uint64_t(gridDim.x) * blockDim.x) {
        if (!first[i]) continue;
        okey[at[i]] = key[i];
        od[at[i]] = d[i];
    }
}

// Records (key, d) to struct-of-arrays pairs (u = key >> vbits, v = the low bits, d).
__global__ void k_split_pairs(const unsigned long long *__restrict__ key, const uint32_t *__restrict__ d, uint64_t n,
                              uint32_t vbits, uint32_t *u, uint32_t *v, uint32_t *dd) {
    const unsigned long long vmask = (1ull << vbits) - 1;
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += uint64_t(gridDim.x) * blockDim.x) {
        u[i] = uint32_t(key[i] >> vbits);
        v[i] = uint32_t(key[i] & vmask);
        dd[i] = d[i];
    }
}

namespace {

uint32_t grid_of(const Workspace *ws, uint64_t n, uint32_t per = 256) {
    return uint32_t(std::max<uint64_t>(1, std::min<uint64_t>((n + per - 1) / per, uint64_t(ws->num_sms) * 16)));
}

// Digit shifts of a radix sort over the key bits [lo, hi) and then the value bits [0, vhi)
// (least significant first: values sort first when given first).
void add_shifts(std::vector<int> *sh, uint32_t lo, uint32_t hi, int offset = 0) {
    for (uint32_t b = lo; b < hi; b += 8) sh->push_back(offset + int(b));
}

}  // namespace


void run_hier(const DeviceGraph &g, Workspace *ws, HierState **state, const EngineConfig &cfg, uint32_t median_w,
              const std::vector<uint32_t> &perm, const std::vector<uint32_t> &part_start, const uint32_t *R,
              uint32_t nR, const uint32_t *S, uint32_t nS, uint64_t k, uint32_t theta, rn_dpairs *out, void *stream,
              rn_query_stats *stats, rn_hier_stats *hs) {
    cudaStream_t st = (cudaStream_t)stream;
    if (theta == RN_INF) theta = RN_THETA_MAX;
    if (theta > RN_THETA_MAX) fail(RN_EINVAL, "theta must be <= 2^31 or RN_INF");
    if (g.n >= SK_NODE) fail(RN_EINVAL, "the hierarchical variant takes graphs of fewer than 2^28 nodes");
    if (part_start.empty() || part_start[0] != 0) fail(RN_EINTERNAL, "hierarchy cut does not start at node 0");
    const uint32_t nparts = uint32_t(part_start.size());
    uint32_t max_part = 0;
    for (uint32_t p = 0; p < nparts; p++)
        max_part = std::max(max_part, (p + 1 < nparts ? part_start[p + 1] : g.n) - part_start[p]);
    // a local search never leaves its part: a warp map holding the largest part never overflows
    uint32_t map_slots = 0;
    for (uint32_t m = SRC_MS_MIN; m <= SRC_MS_MAX && !map_slots; m *= 2)
        if (double(max_part) <= src_fit(m)) map_slots = m;
    if (!map_slots) fail(RN_EINVAL, "the hierarchical variant takes parts of at most 6516 nodes");
    std::lock_guard<std::mutex> device_lock(ws->sh->mu);
    Range range("rn.hier");
    *stats = rn_query_stats{};
    *hs = rn_hier_stats{};
    hs->parts = nparts;
    ws->launches = 0;
    if (!*state) *state = new HierState();
    HierState *h = *state;
    if (!h->count) {
        h->count = (unsigned long long *)device_alloc(4 * 8);
        RN_CUDA(cudaMallocHost(&h->count_host, 4 * 8));
        RN_CUDA(cudaEventCreate(&h->ev[0]));
        RN_CUDA(cudaEventCreate(&h->ev[1]));
    }
    RN_CUDA(cudaEventRecord(ws->ev0, st));
    auto counts = [&] {
        RN_CUDA(cudaMemcpyAsync(h->count_host, h->count, 4 * 8, cudaMemcpyDeviceToHost, st));
        RN_CUDA(cudaStreamSynchronize(st));
    };
    double phase_ms[3] = {0, 0, 0};
    auto mark = [&] { RN_CUDA(cudaEventRecord(h->ev[0], st)); };
    auto lap = [&](int p) {
        RN_CUDA(cudaEventRecord(h->ev[1], st));
        RN_CUDA(cudaEventSynchronize(h->ev[1]));
        float t = 0;
        RN_CUDA(cudaEventElapsedTime(&t, h->ev[0], h->ev[1]));
        phase_ms[p] += t;
    };
    // the border bitmap of this cut of the hierarchy (kept for the next query)
    if (h->cut != part_start) {
        const uint32_t nw = (g.n + 31) / 32;
        if (h->cap_parts < nparts) {
            device_free(h->part_start);
            h->part_start = nullptr;
            h->part_start = (uint32_t *)device_alloc(size_t(nparts) * 4);
            h->cap_parts = nparts;
        }
        if (h->cap_border < std::max<uint32_t>(nw, 1)) {
            device_free(h->border);
            h->border = nullptr;
            h->border = (uint32_t *)device_alloc(std::max<size_t>(nw, 1) * 4);
            h->cap_border = std::max<uint32_t>(nw, 1);
        }
        RN_CUDA(cudaMemcpyAsync(h->part_start, part_start.data(), size_t(nparts) * 4, cudaMemcpyHostToDevice, st));
        RN_CUDA(cudaMemsetAsync(h->border, 0, std::max<size_t>(nw, 1) * 4, st));
        if (g.n)
            k_border_bits<<<grid_of(ws, g.n), 256, 0, st>>>(g.row_ptr, reinterpret_cast<const uint2 *>(g.adj), g.n,
                                                            h->part_start, nparts, h->border);
        RN_CUDA(cudaGetLastError());
        RN_CUDA(cudaStreamSynchronize(st));  // part_start is the caller's host vector
        h->cut = part_start;
        ws->launches++;
    }
    // sources: R in internal ids, ascending, each with its part's id range
    std::vector<uint32_t> src(nR);
    for (uint32_t j = 0; j < nR; j++) src[j] = perm[R[j]];
    std::sort(src.begin(), src.end());
    std::vector<uint2> rng(nR);
    for (uint32_t j = 0; j < nR; j++) {
        const uint32_t p = uint32_t(std::upper_bound(part_start.begin(), part_start.end(), src[j]) - part_start.begin()) - 1;
        rng[j] = make_uint2(part_start[p], p + 1 < nparts ? part_start[p + 1] : g.n);
    }
    uint32_t *d_src = h->get<uint32_t>("src", nR);
    uint2 *d_rng = h->get<uint2>("range", nR);
    uint32_t *dR = h->get<uint32_t>("R", nR), *dS = h->get<uint32_t>("S", nS);
    if (nR) {
        RN_CUDA(cudaMemcpyAsync(d_src, src.data(), size_t(nR) * 4, cudaMemcpyHostToDevice, st));
        RN_CUDA(cudaMemcpyAsync(d_rng, rng.data(), size_t(nR) * 8, cudaMemcpyHostToDevice, st));
        RN_CUDA(cudaMemcpyAsync(dR, R, size_t(nR) * 4, cudaMemcpyHostToDevice, st));
    }
    if (nS) RN_CUDA(cudaMemcpyAsync(dS, S, size_t(nS) * 4, cudaMemcpyHostToDevice, st));
    prep_sets(g, ws, dR, nR, dS, nS, st);  // validation and the S bitmap
    check_control(read_control(ws, st));   // (host vectors above are copied by now)
    ensure_ranges(&ws->failed, &ws->failed_cap, std::max<uint32_t>(nR, 1));
    ensure_ranges(&ws->failed2, &ws->failed2_cap, std::max<uint32_t>(nR, 1));
    const uint32_t vbits = bits_for(g.n);
    const uint32_t delta = choose_delta(cfg, median_w, true);
    uint64_t retried = 0;

    // The join within bound bnd: every pair's least distance, sorted by (u, v), as records
    // (orig(u) << vbits | orig(v), d) in (*ok, *od).
    auto join_at = [&](uint32_t bnd, unsigned long long **ok, uint32_t **od) -> uint64_t {
        const int dbits = int(bits_for(uint32_t(std::min<uint64_t>(bnd + 1ull, 0xFFFFFFFFull))));
        // 1. local searches: pairs inside each source's part, routes to its border nodes
        mark();
        ensure_pairs(ws, std::max<uint64_t>(ws->pair_cap, uint64_t(nR) * 64));
        uint64_t brd_cap = std::max<uint64_t>(uint64_t(nR) * 64, 1 << 16);
        Control c{};
        unsigned long long *brd_key = nullptr;
        uint32_t *brd_d = nullptr;
        for (;;) {
            brd_key = h->get<unsigned long long>("brd_key", brd_cap);
            brd_d = h->get<uint32_t>("brd_d", brd_cap);
            RN_CUDA(cudaMemsetAsync(ws->ctl, 0, sizeof(Control), st));
            RN_CUDA(cudaMemsetAsync(h->count, 0, 4 * 8, st));
            SearchArgs a{};
            a.row_ptr = g.row_ptr;
            a.adj = reinterpret_cast<const uint2 *>(g.adj);
            a.iperm = g.iperm;
            a.sbits = ws->sbits;
            a.src = d_src;
            a.bound = bnd;
            a.delta = delta;
            a.vbits = vbits;
            a.ctl = ws->ctl;
            a.out_key = ws->keyA;
            a.out_d = ws->valA;
            a.out_cap = ws->pair_cap;
            a.nR_fixed = nR;
            a.ntiles = nR;
            a.n_nodes = g.n;
            a.n_arcs = g.arcs;
            a.failed = ws->failed;
            a.src_range = d_rng;
            a.border_bits = h->border;
            a.brd_key = brd_key;
            a.brd_d = brd_d;
            a.brd_cap = brd_cap;
            a.brd_count = h->count;
            if (nR) source_launch(map_slots, a, nR, ws, st, true);
            c = read_control(ws, st);
            counts();
            check_control(c);
            if (c.n_failed) fail(RN_EINTERNAL, "a local search outgrew a map that holds its part");
            if (c.pairs > ws->pair_cap) {
                ensure_pairs(ws, c.pairs + c.pairs / 4);
                continue;
            }
            if (h->count_host[0] > brd_cap) {
                brd_cap = h->count_host[0] + h->count_host[0] / 4;
                continue;
            }
            break;
        }
        const uint64_t local = c.pairs, nb = h->count_host[0];
        lap(0);
        mark();
        // 2. exit routes (orig(f) << 32 | si, off); each (f, si) keeps its least offset
        uint64_t ex_cap = std::max<uint64_t>(nb * 3, 1 << 16), nx = 0;
        unsigned long long *xk = nullptr;
        uint32_t *xd = nullptr;
        for (;;) {
            xk = h->get<unsigned long long>("ex_key", ex_cap);
            xd = h->get<uint32_t>("ex_d", ex_cap);
            RN_CUDA(cudaMemsetAsync(h->count, 0, 4 * 8, st));
            if (nb) {
                k_exit_expand<<<grid_of(ws, nb), 256, 0, st>>>(brd_key, brd_d, nb, d_rng, g.row_ptr,
                                                               reinterpret_cast<const uint2 *>(g.adj), g.iperm, bnd,
                                                               xk, xd, ex_cap, h->count);
                ws->launches++;
            }
            RN_CUDA(cudaGetLastError());
            counts();
            nx = h->count_host[0];
            if (nx <= ex_cap) break;
            ex_cap = nx + nx / 4;
        }
        unsigned long long *xk2 = h->get<unsigned long long>("ex_key2", nx);
        uint32_t *xd2 = h->get<uint32_t>("ex_d2", nx);
        std::vector<int> sh;
        add_shifts(&sh, 0, uint32_t(dbits), 64);                      // offset
        add_shifts(&sh, 0, bits_for(std::max<uint32_t>(nR, 2)));      // si
        add_shifts(&sh, 32, 32 + vbits);                              // orig(f)
        const auto xs = sort_kv(ws, xk, xd, xk2, xd2, nx, sh, st);
        uint32_t *keep = h->get<uint32_t>("keep", nx + 1), *keep_at = h->get<uint32_t>("keep_at", hist_words(nx + 1));
        uint32_t *head = h->get<uint32_t>("head", nx + 1), *head_at = h->get<uint32_t>("head_at", hist_words(nx + 1));
        uint32_t ne = 0, nf = 0;
        if (nx) {
            k_exit_flags<<<grid_of(ws, nx), 256, 0, st>>>(xs.first, nx, keep, head);
            RN_CUDA(cudaMemsetAsync(keep + nx, 0, 4, st));
            RN_CUDA(cudaMemsetAsync(head + nx, 0, 4, st));
            RN_CUDA(cudaMemcpyAsync(keep_at, keep, (nx + 1) * 4, cudaMemcpyDeviceToDevice, st));
            RN_CUDA(cudaMemcpyAsync(head_at, head, (nx + 1) * 4, cudaMemcpyDeviceToDevice, st));
            ws->launches += 1 + scan_hist(keep_at, uint32_t(nx + 1), st) + scan_hist(head_at, uint32_t(nx + 1), st);
            uint32_t *tot = reinterpret_cast<uint32_t *>(h->count_host);
            RN_CUDA(cudaMemcpyAsync(&tot[0], keep_at + nx, 4, cudaMemcpyDeviceToHost, st));
            RN_CUDA(cudaMemcpyAsync(&tot[1], head_at + nx, 4, cudaMemcpyDeviceToHost, st));
            RN_CUDA(cudaStreamSynchronize(st));
            ne = tot[0];
            nf = tot[1];
        }
        unsigned long long *ek = h->get<unsigned long long>("e_key", ne);
        uint32_t *eo = h->get<uint32_t>("e_off", ne), *f_list = h->get<uint32_t>("f_list", nf);
        uint32_t *fmin = h->get<uint32_t>("fmin", nf);
        if (nx) {
            RN_CUDA(cudaMemsetAsync(fmin, 0xFF, size_t(std::max<uint32_t>(nf, 1)) * 4, st));
            k_exit_compact<<<grid_of(ws, nx), 256, 0, st>>>(xs.first, xs.second, nx, keep, keep_at, head, head_at, ek,
                                                            eo, f_list, fmin);
            ws->launches++;
            RN_CUDA(cudaGetLastError());
        }
        // 3. one unconfined search from every far end f, bounded by theta less its least
        // offset (source_search_all: larger maps, then tiles, for balls that outgrow a map)
        uint32_t *fsrc = h->get<uint32_t>("f_src", nf), *tb = h->get<uint32_t>("f_tb", nf);
        uint32_t *td = h->get<uint32_t>("f_td", nf), *ti = h->get<uint32_t>("f_ti", nf);
        if (nf) {
            k_exit_sources<<<grid_of(ws, nf), 256, 0, st>>>(f_list, fmin, nf, g.perm, bnd, delta, fsrc, tb, td, ti);
            ws->launches++;
        }
        uint64_t hit_cap = std::max<uint64_t>(uint64_t(nf) * 32, 1 << 16), nh = 0;
        unsigned long long *hk = nullptr;
        uint32_t *hd = nullptr;
        if (nf) ensure_slab(ws);  // the tile fallback of balls that outgrow a warp map
        for (;;) {
            hk = h->get<unsigned long long>("hit_key", hit_cap);
            hd = h->get<uint32_t>("hit_d", hit_cap);
            RN_CUDA(cudaMemsetAsync(ws->ctl, 0, sizeof(Control), st));
            SearchArgs a{};
            a.row_ptr = g.row_ptr;
            a.adj = reinterpret_cast<const uint2 *>(g.adj);
            a.iperm = g.iperm;
            a.sbits = ws->sbits;
            a.src = fsrc;
            a.bound = bnd;
            a.delta = delta;
            a.vbits = vbits;
            a.ctl = ws->ctl;
            a.out_key = hk;
            a.out_d = hd;
            a.out_cap = hit_cap;
            a.nR_fixed = nf;
            a.tile_bound = tb;
            a.tile_delta = td;
            a.tile_inst = ti;
            a.slab = ws->sh->slab;
            const Control cc =
                source_search_all(g, ws, a, nf, source_first_map(ws, bnd), 32, bnd, {}, st, &retried, false);
            check_control(cc);
            if (cc.pairs > hit_cap) {
                hit_cap = cc.pairs + cc.pairs / 4;
                continue;
            }
            nh = cc.pairs;
            break;
        }
        unsigned long long *hk2 = h->get<unsigned long long>("hit_key2", nh);
        uint32_t *hd2 = h->get<uint32_t>("hit_d2", nh);
        sh.clear();
        add_shifts(&sh, 0, 2 * vbits);
        const auto hsrt = sort_kv(ws, hk, hd, hk2, hd2, nh, sh, st);
        uint2 *fr = h->get<uint2>("f_range", nf);
        if (nf) {
            k_hit_ranges<<<grid_of(ws, nf), 256, 0, st>>>(hsrt.first, nh, f_list, nf, vbits, fr);
            ws->launches++;
        }
        lap(1);
        mark();
        // 4. candidates through the exit arcs after the local pairs, then every pair's least
        // distance (records sorted by (u, v) and distance; the first of each (u, v) kept)
        uint64_t cap = std::max<uint64_t>(local + nh * 2, 1 << 16), m = 0;
        unsigned long long *mk0 = nullptr;
        uint32_t *md0 = nullptr;
        for (;;) {
            mk0 = h->get<unsigned long long>("m_key", cap);
            md0 = h->get<uint32_t>("m_d", cap);
            if (local > cap) {
                cap = local + local / 4;
                continue;
            }
            h->count_host[0] = local;
            RN_CUDA(cudaMemcpyAsync(h->count, h->count_host, 8, cudaMemcpyHostToDevice, st));
            if (local) {
                RN_CUDA(cudaMemcpyAsync(mk0, ws->keyA, local * 8, cudaMemcpyDeviceToDevice, st));
                RN_CUDA(cudaMemcpyAsync(md0, ws->valA, local * 4, cudaMemcpyDeviceToDevice, st));
            }
            if (ne) {
                k_hier_combine<<<grid_of(ws, uint64_t(ne) * 32), 256, 0, st>>>(ek, eo, ne, fr, hsrt.first, hsrt.second,
                                                                               d_src, g.iperm, bnd, vbits, mk0, md0,
                                                                               cap, h->count);
                ws->launches++;
            }
            RN_CUDA(cudaGetLastError());
            counts();
            m = h->count_host[0];
            if (m <= cap) break;
            cap = m + m / 4;
        }
        unsigned long long *mk1 = h->get<unsigned long long>("m_key2", m);
        uint32_t *md1 = h->get<uint32_t>("m_d2", m);
        sh.clear();
        add_shifts(&sh, 0, uint32_t(dbits), 64);  // distance
        add_shifts(&sh, 0, 2 * vbits);           // (u, v)
        const auto msrt = sort_kv(ws, mk0, md0, mk1, md1, m, sh, st);
        uint32_t *first = h->get<uint32_t>("first", m + 1), *first_at = h->get<uint32_t>("first_at", hist_words(m + 1));
        unsigned long long *uk = h->get<unsigned long long>("u_key", m);
        uint32_t *ud = h->get<uint32_t>("u_d", m);
        uint64_t nu = 0;
        if (m) {
            k_first_of_key<<<grid_of(ws, m), 256, 0, st>>>(msrt.first, m, first);
            RN_CUDA(cudaMemsetAsync(first + m, 0, 4, st));
            RN_CUDA(cudaMemcpyAsync(first_at, first, (m + 1) * 4, cudaMemcpyDeviceToDevice, st));
            ws->launches += 2 + scan_hist(first_at, uint32_t(m + 1), st);
            k_first_compact<<<grid_of(ws, m), 256, 0, st>>>(msrt.first, msrt.second, m, first, first_at, uk, ud);
            uint32_t *tot = reinterpret_cast<uint32_t *>(h->count_host);
            RN_CUDA(cudaMemcpyAsync(&tot[0], first_at + m, 4, cudaMemcpyDeviceToHost, st));
            RN_CUDA(cudaStreamSynchronize(st));
            nu = tot[0];
            RN_CUDA(cudaGetLastError());
        }
        lap(2);
        hs->local_pairs = local;
        hs->border_routes = nb;
        hs->exit_routes = ne;
        hs->exit_searches = nf;
        hs->candidates = m - local;
        *ok = uk;
        *od = ud;
        return nu;
    };

    unsigned long long *rk = nullptr;
    uint32_t *rd = nullptr;
    uint64_t np = 0;
    uint32_t passes = 0;
    if (k == 0) {
        np = join_at(theta, &rk, &rd);
        passes = 1;
    } else {
        // k closest pairs: the join within a radius grown until it holds k pairs (pairs
        // grow about as the square of the radius on a road network), then the first k by
        // (d, u, v)
        uint64_t tau = std::min<uint64_t>(theta, std::max<uint32_t>(delta, 1));
        for (;;) {
            np = join_at(uint32_t(tau), &rk, &rd);
            passes++;
            if (np >= k || tau >= theta) break;
            double f = np ? std::sqrt(double(k) / double(np)) * 1.25 : 4.0;
            tau = std::min<uint64_t>(theta, uint64_t(double(tau) * std::max(f, 1.5)) + 1);
        }
        unsigned long long *sk = h->get<unsigned long long>("k_key", np);
        uint32_t *sd = h->get<uint32_t>("k_d", np);
        std::vector<int> sh;
        add_shifts(&sh, 0, 2 * vbits);                                     // (u, v)
        add_shifts(&sh, 0, bits_for(uint32_t(std::min<uint64_t>(tau + 1, 0xFFFFFFFFull))), 64);  // distance
        const auto ks = sort_kv(ws, rk, rd, sk, sd, np, sh, st);
        rk = ks.first;
        rd = ks.second;
        np = std::min<uint64_t>(np, k);
    }
    dpairs_reserve(out, np);
    if (np) {
        k_split_pairs<<<grid_of(ws, np), 256, 0, st>>>(rk, rd, np, vbits, out->u, out->v, out->d);
        ws->launches++;
        RN_CUDA(cudaGetLastError());
    }
    out->n = np;
    RN_CUDA(cudaEventRecord(ws->ev1, st));
    RN_CUDA(cudaEventSynchronize(ws->ev1));
    float ms = 0;
    RN_CUDA(cudaEventElapsedTime(&ms, ws->ev0, ws->ev1));
    stats->pairs = np;
    stats->tile_width = 1;
    stats->delta = delta;
    stats->passes = passes;
    stats->theta_final = theta;
    stats->launches = ws->launches;
    stats->device_ms = ms;
    stats->retried_tiles = retried;
    hs->local_ms = phase_ms[0];
    hs->exit_ms = phase_ms[1];
    hs->combine_ms = phase_ms[2];
    hs->max_part = max_part;
}

// ------------------------------------------------------------------- batch ----
// Many independent theta-joins (their own graphs, sets and thetas) searched by one
// persistent launch per (tile width, first map, sources per tile) group.  The batch's
// graphs are copied into one disjoint union (node ids and arc positions shifted per
// instance, plus one isolated pad node), so the search runs exactly as for a single
// query on that graph: every instance's R list, in internal ids, is padded with the pad
// node to whole tiles, and per-tile tables give each tile its instance's theta, bucket
// width and index.  Pairs are sorted by (u, v) in union ids, which puts every instance's
// pairs together in (u, v) order; a last kernel shifts them back to the instance's ids.
//
// The first map of an instance's tiles follows the largest union ball its tiles reached
// in an earlier run (a shared-memory map when it fits, else a global map of the right
// size), so tiles whose balls are known to be large are not first searched with maps
// they overflow.  Once a run needs no retry, the whole run (clears, searches, sort) is
// captured in a CUDA graph and replayed; a replay that does not reproduce the counts
// falls back to an eager run.  An autotuner picks, per size class of instance, the tile
// width, the bucket width and the sources per tile from per-instance SM cycles measured
// in the kernel.

// Copy one instance's graph into the union: nodes shifted by node_off, arcs by arc_off.
__global__ void k_union_graph(const uint32_t *__restrict__ row_ptr, const uint2 *__restrict__ adj,
                              const uint32_t *__restrict__ iperm, uint32_t n, uint32_t arcs, uint32_t node_off,
                              uint32_t arc_off, uint32_t *u_row_ptr, uint2 *u_adj, uint32_t *u_iperm) {
    const uint32_t m = max(n, arcs);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        if (i < n) {
            u_row_ptr[node_off + i] = row_ptr[i] + arc_off;
            u_iperm[node_off + i] = iperm[i] + node_off;
        }
        if (i < arcs) {
            const uint2 e = adj[i];
            u_adj[arc_off + i] = make_uint2(e.x + node_off, e.y);
        }
    }
}

// Shift every pair back to its instance's ids: pair p belongs to the instance i with
// pair_off[i] <= p < pair_off[i+1].
__global__ void k_localize(uint32_t *u, uint32_t *v, uint64_t n, const unsigned long long *__restrict__ pair_off,
                           const uint32_t *__restrict__ node_off, uint32_t nq) {
    for (uint64_t p = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; p < n; p += uint64_t(gridDim.x) * blockDim.x) {
        uint32_t lo = 0, hi = nq - 1;
        while (lo < hi) {
            const uint32_t mid = (lo + hi + 1) >> 1;
            if (pair_off[mid] <= p) lo = mid;
            else hi = mid - 1;
        }
        u[p] -= node_off[lo];
        v[p] -= node_off[lo];
    }
}

namespace {

struct BatchPlan {
    uint32_t T = 32;          // 1: the warp search; 32, 64, 128: tiles of that width
    uint32_t delta_mult = 4;  // bucket width in median arc weights
    uint32_t src_div = 1;     // sources per tile = T / src_div
};

constexpr BatchPlan WARP_PLAN{1, 16, 1}, TILE_PLAN{32, 4, 1};
// Instances whose balls outgrow the warp maps: tiles of 8 sources.  Their balls span much
// of their graph, so a tile's search is long and runs mostly alone; more, narrower tiles
// spread an instance over more SMs and shorten the batch's tail (batch512: 129 -> 87 ms
// with the warp search for the rest).
constexpr BatchPlan BIG_PLAN{32, 4, 4};

// Sources per tile of a plan (one for the warp search).
uint32_t plan_tile_src(const BatchPlan &p) { return std::max<uint32_t>(1, p.T / p.src_div); }

// The smallest warp map whose 7/8 holds a ball of `ball` nodes with room to spare, or 0
// when even the largest does not.
uint32_t warp_map_for_ball(double ball) {
    for (uint32_t ms = SRC_MS_MIN; ms <= SRC_MS_MAX; ms *= 2)
        if (ball <= src_fit(ms)) return ms;
    return 0;
}

// Size class of an instance for the autotuner: log2 of its node count, of |R| and of
// theta in median arc weights (the hop radius of a search, which sets its ball).
uint32_t size_class(uint32_t n, uint32_t nR, uint32_t theta, uint32_t median_w) {
    const uint64_t hops = uint64_t(theta) / std::max<uint32_t>(1, median_w);
    return (bits_for(n) << 16) | (bits_for(std::max<uint32_t>(nR, 1)) << 8) |
           bits_for(uint32_t(std::min<uint64_t>(hops + 1, 1u << 20)));
}

// First map for tiles whose union ball reached `ball` slots: the narrow shared map
// while it holds the ball with some room, then the wide one, then a global map.
uint32_t map_for_ball(uint32_t ball) {
    const uint64_t need = uint64_t(ball) * 8 / 7 + uint64_t(ball) / 8 + 1;
    if (need <= SMEM_H) return SMEM_H;
    if (need <= SMEM_HW) return SMEM_HW;
    uint64_t H = SMEM_HW * 2;
    while (H < need) H <<= 1;
    return uint32_t(std::min<uint64_t>(H, 1u << 30));
}

std::mutex g_tune_mu;
std::map<uint32_t, BatchPlan> g_tune_cache;  // size class -> tuned plan, for the process

}  // namespace

// The tuned plans as text, one "class T delta_mult src_div" line per size class (class =
// log2 n << 16 | log2 |R| << 8 | log2 hops), after a "rn-tune 1" line.
void tune_cache_save(const char *path) {
    if (!path) fail(RN_EINVAL, "null path");
    std::string text = "rn-tune 1\n";
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        for (const auto &kv : g_tune_cache)
            text += std::to_string(kv.first) + " " + std::to_string(kv.second.T) + " " +
                    std::to_string(kv.second.delta_mult) + " " + std::to_string(kv.second.src_div) + "\n";
    }
    std::FILE *f = std::fopen(path, "w");
    if (!f) fail(RN_EINVAL, std::string(path) + ": cannot create");
    const bool ok = std::fputs(text.c_str(), f) >= 0;
    if ((std::fclose(f) != 0) || !ok) fail(RN_EINVAL, std::string(path) + ": write failed");
}

// Merge the plans of a saved cache into the process's (later batches use them).
uint32_t tune_cache_load(const char *path) {
    if (!path) fail(RN_EINVAL, "null path");
    std::FILE *f = std::fopen(path, "r");
    if (!f) fail(RN_EINVAL, std::string(path) + ": cannot open");
    std::map<uint32_t, BatchPlan> plans;
    char line[256];
    int lineno = 0;
    bool ok = true;
    std::string why;
    while (ok && std::fgets(line, sizeof line, f)) {
        lineno++;
        if (lineno == 1) {
            ok = std::strncmp(line, "rn-tune 1", 9) == 0;
            why = "not a tune cache";
            continue;
        }
        unsigned long cls = 0, T = 0, dm = 0, sd = 0;
        if (std::sscanf(line, "%lu %lu %lu %lu", &cls, &T, &dm, &sd) != 4 || (T != 1 && T != 32 && T != 64 && T != 128) ||
            dm < 1 || dm > 1024 || sd < 1 || sd > T || cls > 0xFFFFFFFFul) {
            ok = false;
            why = "line " + std::to_string(lineno) + " is not 'class T delta_mult src_div'";
            break;
        }
        plans[uint32_t(cls)] = BatchPlan{uint32_t(T), uint32_t(dm), uint32_t(sd)};
    }
    std::fclose(f);
    if (!ok || lineno == 0) fail(RN_EINVAL, std::string(path) + ": " + (lineno ? why : "empty file"));
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (const auto &kv : plans) g_tune_cache[kv.first] = kv.second;
    return uint32_t(plans.size());
}

struct Batch {
    int device = 0;
    uint32_t nq = 0, n_u = 0, pad = 0, vbits = 1;
    uint64_t arcs_u = 0;
    std::vector<uint32_t> n, nR, theta, median_w, cls, node_off;  // nR: the instance's sources
    std::vector<std::vector<uint32_t>> rint;  // per instance: its sources in union internal ids, ascending
    std::vector<BatchPlan> plan;
    std::vector<uint32_t> map;       // per instance: slots of the first map
    std::vector<uint32_t> ball;      // per instance: largest union ball seen under plan[i].T
    std::vector<uint32_t> ball_T;    // the tile width ball[i] was measured with (0: none)
    std::vector<double> tile_cost;   // per instance: SM cycles of one of its tiles, last run
    bool costs_known = false;        // tile_cost holds measurements (else a size proxy)
    bool laid_out_by_cost = false;   // the layout used measured costs
    DeviceGraph ug;  // the union graph (row_ptr, adj, iperm)
    uint32_t *sbits = nullptr, *node_off_d = nullptr, *inst_ball = nullptr;
    uint8_t *inst_swap = nullptr;  // per instance: searched from S (null when none is)
    Workspace *ws = nullptr;  // control block, retry lists, global maps, events of the batch
    cudaStream_t stream = nullptr;
    unsigned long long *inst_pairs = nullptr, *inst_cycles = nullptr, *pair_off_d = nullptr;
    struct Group {
        uint32_t T = 32, map = SMEM_H, tile_src = 32, nsrc = 0, tiles = 0;
        uint32_t *src = nullptr, *tbound = nullptr, *tdelta = nullptr, *tinst = nullptr;
    };
    std::vector<Group> groups;
    uint64_t pair_cap = 0;
    unsigned long long *keyA = nullptr, *keyB = nullptr;
    uint32_t *valA = nullptr, *valB = nullptr, *hist = nullptr;
    size_t hist_cap = 0;
    uint32_t *out_u = nullptr, *out_v = nullptr, *out_d = nullptr;
    uint64_t out_cap = 0;
    std::vector<uint64_t> cnt, off;  // per instance: pairs and their first index
    uint64_t total = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint64_t exec_pairs = 0;
    rn_batch_stats stats{};
};

static void batch_drop_graph(Batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

static void batch_free_groups(Batch *b) {
    for (auto &g : b->groups)
        for (void *p : {(void *)g.src, (void *)g.tbound, (void *)g.tdelta, (void *)g.tinst}) device_free(p);
    b->groups.clear();
}

void batch_destroy(Batch *b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    batch_drop_graph(b);
    batch_free_groups(b);
    for (void *p : {(void *)b->sbits, (void *)b->inst_swap, (void *)b->node_off_d, (void *)b->inst_ball, (void *)b->inst_pairs,
                    (void *)b->inst_cycles, (void *)b->pair_off_d, (void *)b->keyA, (void *)b->keyB,
                    (void *)b->valA, (void *)b->valB, (void *)b->hist, (void *)b->out_u, (void *)b->out_v,
                    (void *)b->out_d, (void *)b->ug.row_ptr, (void *)b->ug.adj, (void *)b->ug.iperm})
        device_free(p);
    if (b->stream) cudaStreamDestroy(b->stream);
    workspace_destroy(b->ws);
    delete b;
}

template <class T>
static T *upload_vec(const std::vector<T> &v) {
    T *p = (T *)device_alloc(std::max<size_t>(v.size(), 1) * sizeof(T));
    if (!v.empty()) RN_CUDA(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return p;
}

// First maps from the balls measured under each instance's current tile width: for the
// warp search the smallest warp map its largest source ball fits (an instance whose balls
// outgrow the largest warp map moves to tiles), for tiles the map of its largest union
// ball.
static bool batch_adapt_maps(Batch *b) {
    bool changed = false;
    for (uint32_t i = 0; i < b->nq; i++) {
        const bool measured = b->ball_T[i] == b->plan[i].T;
        if (b->plan[i].T == 1 && measured && !warp_map_for_ball(b->ball[i])) {
            b->plan[i] = BIG_PLAN;
            changed = true;
        }
        uint32_t m;
        if (b->plan[i].T == 1) m = measured ? warp_map_for_ball(b->ball[i]) : 2048;
        else m = b->ball_T[i] == b->plan[i].T ? map_for_ball(b->ball[i]) : SMEM_H;
        if (m != b->map[i]) changed = true;
        b->map[i] = m;
    }
    return changed;
}

// Group the instances by (tile width, first map, sources per tile) and upload each
// group's padded source list and per-tile tables.
static void batch_layout(Batch *b) {
    batch_drop_graph(b);
    batch_free_groups(b);
    std::map<std::tuple<uint32_t, uint32_t, uint32_t>, std::vector<uint32_t>> by;
    for (uint32_t i = 0; i < b->nq; i++)
        by[std::make_tuple(b->plan[i].T, b->map[i], b->plan[i].src_div)].push_back(i);
    // longest tiles first, in every group and across groups (the persistent blocks then
    // end together instead of waiting on a few long tiles popped last)
    std::vector<std::pair<double, std::vector<uint32_t>>> order;
    for (auto &kv : by) {
        auto &v = kv.second;
        std::stable_sort(v.begin(), v.end(), [&](uint32_t x, uint32_t y) { return b->tile_cost[x] > b->tile_cost[y]; });
        order.emplace_back(b->tile_cost[v.front()], v);
    }
    std::stable_sort(order.begin(), order.end(), [](const auto &x, const auto &y) { return x.first > y.first; });
    uint64_t tiles = 0;
    for (auto &ov : order) {
        const auto &first = ov.second.front();
        const std::pair<std::tuple<uint32_t, uint32_t, uint32_t>, std::vector<uint32_t>> kv{
            std::make_tuple(b->plan[first].T, b->map[first], b->plan[first].src_div), ov.second};
        Batch::Group g;
        g.T = std::get<0>(kv.first);
        g.map = std::get<1>(kv.first);
        g.tile_src = plan_tile_src(b->plan[first]);
        std::vector<uint32_t> src, tb, td, ti;
        for (uint32_t i : kv.second) {
            const auto &r = b->rint[i];
            const uint32_t nt = uint32_t((r.size() + g.tile_src - 1) / g.tile_src);
            src.insert(src.end(), r.begin(), r.end());
            src.resize(src.size() + size_t(nt) * g.tile_src - r.size(), b->pad);  // pad to whole tiles
            const uint32_t delta = std::max<uint32_t>(1, b->plan[i].delta_mult * b->median_w[i]);
            for (uint32_t t = 0; t < nt; t++) {
                tb.push_back(b->theta[i]);
                td.push_back(delta);
                ti.push_back(i);
            }
        }
        if (src.size() > 0xFFFFFFFFull) fail(RN_EINVAL, "batch too large: more than 2^32 - 1 sources");
        // every tile lies inside one instance and every source inside the union
        if (src.size() != size_t(tb.size()) * g.tile_src || td.size() != tb.size() || ti.size() != tb.size())
            fail(RN_EINTERNAL, "batch layout: tile tables do not match the source list");
        for (uint32_t x : src)
            if (x >= b->n_u) fail(RN_EINTERNAL, "batch layout: source outside the union graph");
        g.nsrc = uint32_t(src.size());
        g.tiles = uint32_t(tb.size());
        g.src = upload_vec(src);
        g.tbound = upload_vec(tb);
        g.tdelta = upload_vec(td);
        g.tinst = upload_vec(ti);
        tiles += g.tiles;
        b->groups.push_back(g);
    }
    RN_CUDA(cudaDeviceSynchronize());  // the batch's stream does not wait for these copies
    ensure_ranges(&b->ws->failed, &b->ws->failed_cap, uint32_t(std::max<uint64_t>(tiles, 1)));
    ensure_ranges(&b->ws->failed2, &b->ws->failed2_cap, uint32_t(std::max<uint64_t>(tiles, 1)));
    b->stats.tiles = tiles;
    b->stats.groups = uint32_t(b->groups.size());
}

static void batch_reserve_pairs(Batch *b, uint64_t want) {
    if (b->pair_cap >= want) return;
    want = std::max<uint64_t>(want, 1 << 16);
    for (void **p : {(void **)&b->keyA, (void **)&b->keyB, (void **)&b->valA, (void **)&b->valB}) {
        device_free(*p);
        *p = nullptr;
    }
    b->pair_cap = 0;
    b->keyA = (unsigned long long *)device_alloc(want * 8);
    b->keyB = (unsigned long long *)device_alloc(want * 8);
    b->valA = (uint32_t *)device_alloc(want * 4);
    b->valB = (uint32_t *)device_alloc(want * 4);
    b->pair_cap = want;
    batch_drop_graph(b);
}

static SearchArgs batch_args(Batch *b, const Batch::Group &g) {
    SearchArgs a{};
    a.row_ptr = b->ug.row_ptr;
    a.adj = reinterpret_cast<const uint2 *>(b->ug.adj);
    a.iperm = b->ug.iperm;
    a.sbits = b->sbits;
    a.src = g.src;
    a.tile_src = g.tile_src;
    a.nR_fixed = g.nsrc;
    a.tile_bound = g.tbound;
    a.tile_delta = g.tdelta;
    a.tile_inst = g.tinst;
    a.inst_pairs = b->inst_pairs;
    a.inst_cycles = b->inst_cycles;
    a.inst_ball = b->inst_ball;
    a.inst_swap = b->inst_swap;
    a.vbits = b->vbits;
    a.ctl = b->ws->ctl;
    a.out_key = b->keyA;
    a.out_d = b->valA;
    a.out_cap = b->pair_cap;
    return a;
}

static void batch_clear(Batch *b, cudaStream_t st) {
    RN_CUDA(cudaMemsetAsync(b->ws->ctl, 0, sizeof(Control), st));
    RN_CUDA(cudaMemsetAsync(b->inst_pairs, 0, size_t(b->nq) * 8, st));
    RN_CUDA(cudaMemsetAsync(b->inst_cycles, 0, size_t(b->nq) * 8, st));
    RN_CUDA(cudaMemsetAsync(b->inst_ball, 0, size_t(b->nq) * 4, st));
}

// Sort `total` pairs by (u, v) into the result arrays and shift them to instance ids.
static void batch_finish(Batch *b, uint64_t total, cudaStream_t st) {
    if (!total) return;
    if (total > 0xFFFFFFFFull) fail(RN_EINVAL, "more than 2^32 - 1 result pairs in the batch");
    const uint32_t nblocks = uint32_t((total + RS_TILE - 1) / RS_TILE);
    unsigned long long *ki = b->keyA, *ko = b->keyB;
    uint32_t *vi = b->valA, *vo = b->valB;
    for (uint32_t sh = 0; sh < 2 * b->vbits; sh += 8) {
        const bool last = sh + 8 >= 2 * b->vbits;
        k_rs_hist<<<nblocks, RS_THREADS, 0, st>>>(ki, vi, total, int(sh), b->hist, nblocks);
        scan_hist(b->hist, nblocks * 256, st);
        k_rs_scatter<<<nblocks, RS_THREADS, 0, st>>>(ki, vi, ko, vo, total, int(sh), b->hist, nblocks,
                                                     last ? b->out_u : nullptr, last ? b->out_v : nullptr,
                                                     last ? b->out_d : nullptr, b->vbits);
        std::swap(ki, ko);
        std::swap(vi, vo);
    }
    const uint32_t grid = uint32_t(std::min<uint64_t>((total + 255) / 256, uint64_t(b->ws->num_sms) * 8));
    k_localize<<<grid, 256, 0, st>>>(b->out_u, b->out_v, total, b->pair_off_d, b->node_off_d, b->nq);
    RN_CUDA(cudaGetLastError());
}

// Per-instance pair counts and offsets, and the balls of the run.
static void batch_counts(Batch *b, cudaStream_t st) {
    std::vector<unsigned long long> c(b->nq), cyc(b->nq);
    std::vector<uint32_t> ball(b->nq);
    RN_CUDA(cudaMemcpyAsync(c.data(), b->inst_pairs, size_t(b->nq) * 8, cudaMemcpyDeviceToHost, st));
    RN_CUDA(cudaMemcpyAsync(cyc.data(), b->inst_cycles, size_t(b->nq) * 8, cudaMemcpyDeviceToHost, st));
    RN_CUDA(cudaMemcpyAsync(ball.data(), b->inst_ball, size_t(b->nq) * 4, cudaMemcpyDeviceToHost, st));
    RN_CUDA(cudaStreamSynchronize(st));
    for (uint32_t i = 0; i < b->nq; i++) {
        const uint32_t ts = plan_tile_src(b->plan[i]);
        const uint32_t nt = (b->nR[i] + ts - 1) / ts;
        b->tile_cost[i] = nt ? double(cyc[i]) / nt : 0.0;
    }
    b->costs_known = true;
    b->cnt.assign(c.begin(), c.end());
    b->off.assign(b->nq + 1, 0);
    for (uint32_t i = 0; i < b->nq; i++) {
        b->off[i + 1] = b->off[i] + b->cnt[i];
        if (b->ball_T[i] != b->plan[i].T) {
            b->ball_T[i] = b->plan[i].T;
            b->ball[i] = 0;
        }
        b->ball[i] = std::max(b->ball[i], ball[i]);
    }
}

// The first launch of one group (the capturable part of its search).
static void batch_launch_group(Batch *b, const Batch::Group &g, cudaStream_t st) {
    if (!g.tiles) return;
    SearchArgs a = batch_args(b, g);
    a.slab = b->ws->sh->slab;
    a.failed = b->ws->failed;
    a.ntiles = g.tiles;
    a.n_nodes = b->ug.n;
    a.n_arcs = b->ug.arcs;
    if (g.T == 1) {  // the warp search: one source per tile, a warp map of g.map slots
        source_launch(g.map, a, g.nsrc, b->ws, st);
        return;
    }
    if (g.map > SMEM_HW) {
        launch_gmap(b->ug, b->ws, g.T, a, g.map, g.tiles, st);
        return;
    }
    a.H = g.map;
    a.hshift = 32 - bits_for(g.map);
    a.max_fill = g.map * 7 / 8;
    const uint32_t grid_max = uint32_t(b->ws->num_sms) * CTAS_PER_SM;
    if (g.map == SMEM_H) search(g.T, Shape::Narrow, a, std::max<uint32_t>(1, std::min(g.tiles, grid_max)), st);
    else search(g.T, Shape::Wide, a, std::max<uint32_t>(1, std::min(g.tiles, uint32_t(b->ws->num_sms))), st);
}

// A full run with host checks between steps: retries of overflowed tiles, growth of
// the pair buffer.  Returns the number of retried tiles.
static uint64_t batch_run_eager(Batch *b, cudaStream_t st) {
    b->ws->own_gmap_moved = false;
    for (;;) {
        batch_clear(b, st);
        uint64_t retried = 0;
        Control c{};
        for (const auto &g : b->groups) {
            RN_CUDA(cudaMemsetAsync(&b->ws->ctl->tile_next, 0, 8, st));  // tile_next, n_failed
            if (g.T == 1)
                c = source_search_all(b->ug, b->ws, batch_args(b, g), g.nsrc, g.map, TILE_PLAN.T, RN_THETA_MAX, {},
                                      st, &retried, false);
            else
                c = search_all(b->ug, b->ws, g.T, batch_args(b, g), g.tiles, st, &retried, g.map, false);
            check_control(c);
        }
        b->stats.retried_tiles = retried;
        if (c.pairs > b->pair_cap) {
            batch_reserve_pairs(b, c.pairs + c.pairs / 8);
            continue;
        }
        b->total = c.pairs;
        batch_counts(b, st);
        if (b->off[b->nq] != b->total) fail(RN_EINTERNAL, "batch pair counts do not add up");
        if (b->out_cap < b->total) {
            for (void **p : {(void **)&b->out_u, (void **)&b->out_v, (void **)&b->out_d}) {
                device_free(*p);
                *p = nullptr;
            }
            b->out_cap = std::max<uint64_t>(b->total, 1024);
            b->out_u = (uint32_t *)device_alloc(b->out_cap * 4);
            b->out_v = (uint32_t *)device_alloc(b->out_cap * 4);
            b->out_d = (uint32_t *)device_alloc(b->out_cap * 4);
            batch_drop_graph(b);
        }
        const uint32_t nblocks = uint32_t((b->total + RS_TILE - 1) / RS_TILE);
        if (b->hist_cap < hist_words(uint64_t(nblocks) * 256)) {
            device_free(b->hist);
            b->hist = nullptr;
            b->hist_cap = hist_words(uint64_t(nblocks) * 256);
            b->hist = (uint32_t *)device_alloc(b->hist_cap * 4);
            batch_drop_graph(b);
        }
        if (b->ws->own_gmap_moved) batch_drop_graph(b);
        std::vector<unsigned long long> po(b->off.begin(), b->off.end());
        RN_CUDA(cudaMemcpyAsync(b->pair_off_d, po.data(), po.size() * 8, cudaMemcpyHostToDevice, st));
        batch_finish(b, b->total, st);
        RN_CUDA(cudaStreamSynchronize(st));  // po is a host temporary
        b->stats.eager_runs++;
        return retried;
    }
}

// The capturable sequence: clears, one launch per group, sort and shift.
static void batch_record(Batch *b, cudaStream_t st) {
    batch_clear(b, st);
    for (const auto &g : b->groups) {
        RN_CUDA(cudaMemsetAsync(&b->ws->ctl->tile_next, 0, 8, st));
        batch_launch_group(b, g, st);
    }
    batch_finish(b, b->exec_pairs, st);
}

// One run: a graph replay when the last eager run needed no retries, else eager.  An
// eager run with retries sets the instances' first maps from the balls it measured.
void batch_run(Batch *b, void *user_stream, bool use_graph) {
    std::lock_guard<std::mutex> device_lock(b->ws->sh->mu);
    Range range("rn.batch.run");
    cudaStream_t st = b->stream;
    if (user_stream) {
        RN_CUDA(cudaEventRecord(b->ws->ev0, (cudaStream_t)user_stream));
        RN_CUDA(cudaStreamWaitEvent(st, b->ws->ev0, 0));
    }
    ensure_slab(b->ws);
    RN_CUDA(cudaEventRecord(b->ws->ev0, st));
    bool done = false;
    if (use_graph && b->exec) {
        RN_CUDA(cudaGraphLaunch(b->exec, st));
        const Control c = read_control(b->ws, st);
        b->stats.graph_runs++;
        if (!c.err && !c.n_failed && c.pairs == b->exec_pairs) {
            b->total = c.pairs;
            done = true;
        } else {
            batch_drop_graph(b);  // the replay did not reproduce the eager run: run eagerly
        }
    }
    if (!done) {
        b->ws->launches = 0;
        const uint64_t retried = batch_run_eager(b, st);
        const uint32_t passes = (2 * b->vbits + 7) / 8;
        const uint64_t entries = (b->total + RS_TILE - 1) / RS_TILE * 256;
        b->stats.launches_per_run = b->ws->launches + passes * (entries <= 2 * SCAN_CHUNK ? 3 : 5) + 1;
        if (retried || !b->laid_out_by_cost) {
            // the next run starts with fitting maps and the measured tile order
            batch_adapt_maps(b);
            batch_layout(b);
            b->laid_out_by_cost = true;
        } else if (use_graph && !b->exec) {
            b->exec_pairs = b->total;
            ensure_slist(b->ws);  // allocates nothing inside the capture
            RN_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            try {
                batch_record(b, st);
            } catch (...) {
                cudaGraph_t g = nullptr;
                cudaStreamEndCapture(st, &g);
                if (g) cudaGraphDestroy(g);
                throw;
            }
            RN_CUDA(cudaStreamEndCapture(st, &b->graph));
            RN_CUDA(cudaGraphInstantiate(&b->exec, b->graph, 0));
        }
    }
    RN_CUDA(cudaEventRecord(b->ws->ev1, st));
    RN_CUDA(cudaEventSynchronize(b->ws->ev1));
    float ms = 0;
    RN_CUDA(cudaEventElapsedTime(&ms, b->ws->ev0, b->ws->ev1));
    b->stats.device_ms = ms;
    b->stats.pairs = b->total;
    if (user_stream) {
        RN_CUDA(cudaEventRecord(b->ws->ev1, st));
        RN_CUDA(cudaStreamWaitEvent((cudaStream_t)user_stream, b->ws->ev1, 0));
    }
}

// Autotuner.  Every candidate plan (tile width, bucket width, sources per tile) is run
// on the whole batch, each instance with first maps fitted to its measured balls and
// tiles ordered longest first; the run's wall time and every instance's SM cycles
// (weighted by the share of an SM its blocks hold) are recorded.  Each size class then
// takes the candidate with the least cycles; that mixed plan is kept if the batch runs
// faster with it than with the best single candidate, else the best single candidate
// is.  The default plan is a candidate, so tuning never loses to it on the batch it
// was tuned on.  The chosen plan of each size class is remembered for the process.
static double batch_time_eager(Batch *b) {
    batch_adapt_maps(b);
    batch_layout(b);
    if (batch_run_eager(b, b->stream)) {  // overflowed: refit the maps, run again
        batch_adapt_maps(b);
        batch_layout(b);
        batch_run_eager(b, b->stream);
    }
    batch_layout(b);  // measured tile order
    const auto t0 = std::chrono::steady_clock::now();
    batch_run_eager(b, b->stream);
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

void batch_tune(Batch *b) {
    Range range("rn.batch.tune");
    static const BatchPlan cands[] = {
        {1, 16, 1}, {1, 8, 1}, {1, 32, 1}, {32, 4, 1}, {32, 8, 1}, {32, 4, 2}, {32, 4, 4}, {32, 8, 4}, {64, 4, 1}, {128, 4, 1},
    };
    const size_t nc = sizeof(cands) / sizeof(cands[0]);
    std::map<uint32_t, std::vector<double>> cost;  // class -> cycles per candidate
    std::vector<double> wall(nc);
    std::vector<BatchPlan> mixed(b->nq);
    const std::vector<BatchPlan> initial = b->plan;  // the default (or cached) plans
    double wall_mixed = 0, wall_initial = 0;
    {
        std::lock_guard<std::mutex> device_lock(b->ws->sh->mu);
        ensure_slab(b->ws);
        wall_initial = batch_time_eager(b);
        for (size_t c = 0; c < nc; c++) {
            for (uint32_t i = 0; i < b->nq; i++) b->plan[i] = cands[c];
            wall[c] = batch_time_eager(b);
            std::vector<unsigned long long> cyc(b->nq);
            RN_CUDA(cudaMemcpy(cyc.data(), b->inst_cycles, size_t(b->nq) * 8, cudaMemcpyDeviceToHost));
            for (uint32_t i = 0; i < b->nq; i++) {
                auto &v = cost[b->cls[i]];
                if (v.empty()) v.assign(nc, 0.0);
                v[c] += double(cyc[i]);
            }
        }
        std::map<uint32_t, size_t> pick;
        for (auto &kv : cost) {
            size_t best = 0;
            for (size_t c = 1; c < nc; c++)
                if (kv.second[c] < kv.second[best]) best = c;
            pick[kv.first] = best;
        }
        for (uint32_t i = 0; i < b->nq; i++) mixed[i] = b->plan[i] = cands[pick[b->cls[i]]];
        wall_mixed = batch_time_eager(b);
    }
    const size_t best = size_t(std::min_element(wall.begin(), wall.end()) - wall.begin());
    // the fastest of: the plans the batch had, the best single candidate, the per-class mix
    const int pick = wall_initial <= std::min(wall_mixed, wall[best]) ? 3 : (wall_mixed < wall[best] ? 2 : 1);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        for (uint32_t i = 0; i < b->nq; i++) {
            b->plan[i] = pick == 3 ? initial[i] : pick == 2 ? mixed[i] : cands[best];
            g_tune_cache[b->cls[i]] = b->plan[i];
        }
    }
    batch_adapt_maps(b);
    batch_layout(b);
    b->laid_out_by_cost = false;  // costs of the chosen plan are measured by the next run
    b->stats.tuned = uint32_t(pick);
    b->stats.plan_tile_width = pick == 1 ? cands[best].T : 0;
    b->stats.plan_delta_mult = pick == 1 ? cands[best].delta_mult : 0;
    b->stats.plan_tile_sources = pick == 1 ? plan_tile_src(cands[best]) : 0;
    b->stats.candidates = uint32_t(nc + 2);
}

Batch *batch_create(const std::vector<const DeviceGraph *> &graphs, const std::vector<const std::vector<uint32_t> *> &perms,
                    const std::vector<uint32_t> &median_w, const std::vector<const uint32_t *> &R,
                    const std::vector<uint32_t> &nR, const std::vector<const uint32_t *> &S,
                    const std::vector<uint32_t> &nS, const std::vector<uint32_t> &theta,
                    const std::vector<uint32_t> &search_from) {
    Batch *b = new Batch();
    try {
        b->nq = uint32_t(graphs.size());
        RN_CUDA(cudaGetDevice(&b->device));
        // each instance searches from its smaller set on an undirected graph (as a single
        // join does): its sources and its target bitmap swap roles
        std::vector<uint8_t> swp(b->nq, 0);
        bool any_swap = false;
        b->nR.resize(b->nq);
        for (uint32_t i = 0; i < b->nq; i++) {
            EngineConfig ec;
            ec.search_from = search_from.empty() ? 0u : search_from[i];
            swp[i] = search_from_s(*graphs[i], ec, nR[i], nS[i]);
            any_swap |= swp[i] != 0;
            b->nR[i] = swp[i] ? nS[i] : nR[i];
        }
        b->median_w = median_w;
        b->n.resize(b->nq);
        b->theta.resize(b->nq);
        b->cls.resize(b->nq);
        b->node_off.assign(b->nq + 1, 0);
        b->plan.assign(b->nq, BIG_PLAN);
        b->map.assign(b->nq, SMEM_H);
        b->ball.assign(b->nq, 0);
        b->ball_T.assign(b->nq, 0);
        b->tile_cost.resize(b->nq);
        for (uint32_t i = 0; i < b->nq; i++) b->tile_cost[i] = double(graphs[i]->n);  // until measured
        uint64_t nsum = 0, asum = 0;
        for (uint32_t i = 0; i < b->nq; i++) {
            b->n[i] = graphs[i]->n;
            b->theta[i] = theta[i] == RN_INF ? RN_THETA_MAX : theta[i];
            if (b->theta[i] > RN_THETA_MAX) fail(RN_EINVAL, "theta must be <= 2^31 or RN_INF");
            b->cls[i] = size_class(b->n[i], b->nR[i], b->theta[i], median_w[i]);
            // the default plan: the warp search while the ball estimated from the bound
            // fits a 2048-slot warp map (a dozen warps per SM or more), else tiles, whose
            // sources share their searches' passes
            if (graphs[i]->n < SK_NODE && first_ball_estimate(*graphs[i], b->theta[i], median_w[i]) <= src_fit(2048))
                b->plan[i] = WARP_PLAN;
            b->node_off[i] = uint32_t(nsum);
            nsum += graphs[i]->n;
            asum += graphs[i]->arcs;
            if (nsum + 1 >= 0xFFFFFFFFull || asum >= 0xFFFFFFFFull)
                fail(RN_EINVAL, "batch too large: more than 2^32 - 2 nodes or arcs in all");
        }
        b->node_off[b->nq] = uint32_t(nsum);
        b->pad = uint32_t(nsum);
        b->n_u = uint32_t(nsum + 1);
        b->arcs_u = asum;
        b->vbits = bits_for(b->n_u);
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            for (uint32_t i = 0; i < b->nq; i++) {
                auto it = g_tune_cache.find(b->cls[i]);
                if (it != g_tune_cache.end()) b->plan[i] = it->second;
            }
        }
        DeviceGraph capg{};
        capg.n = b->n_u;
        b->ws = workspace_create(capg);
        b->ws->own_gmap_enabled = true;
        RN_CUDA(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
        // the union graph
        b->ug.n = b->n_u;
        b->ug.arcs = asum;
        b->ug.row_ptr = (uint32_t *)device_alloc((size_t(b->n_u) + 1) * 4);
        b->ug.adj = (uint32_t *)device_alloc(std::max<uint64_t>(asum, 1) * 8);
        b->ug.iperm = (uint32_t *)device_alloc(size_t(b->n_u) * 4);
        uint64_t aoff = 0;
        for (uint32_t i = 0; i < b->nq; i++) {
            const DeviceGraph &g = *graphs[i];
            const uint32_t m = std::max<uint32_t>(g.n, uint32_t(g.arcs));
            const uint32_t grid = std::max<uint32_t>(1, std::min<uint32_t>((m + 255) / 256, 1024));
            k_union_graph<<<grid, 256, 0, b->stream>>>(g.row_ptr, reinterpret_cast<const uint2 *>(g.adj), g.iperm, g.n,
                                                        uint32_t(g.arcs), b->node_off[i], uint32_t(aoff), b->ug.row_ptr,
                                                        reinterpret_cast<uint2 *>(b->ug.adj), b->ug.iperm);
            aoff += g.arcs;
        }
        RN_CUDA(cudaGetLastError());
        const uint32_t tail_rp[2] = {uint32_t(asum), uint32_t(asum)};  // the pad node: no arcs
        RN_CUDA(cudaMemcpyAsync(b->ug.row_ptr + b->pad, tail_rp, 8, cudaMemcpyHostToDevice, b->stream));
        RN_CUDA(cudaMemcpyAsync(b->ug.iperm + b->pad, &b->pad, 4, cudaMemcpyHostToDevice, b->stream));
        RN_CUDA(cudaStreamSynchronize(b->stream));
        // sets, in union internal ids: R lists (sorted, per instance) and the S bitmap
        std::vector<uint32_t> sb((b->n_u + 31) / 32, 0);
        b->rint.resize(b->nq);
        for (uint32_t i = 0; i < b->nq; i++) {
            const std::vector<uint32_t> &perm = *perms[i];
            const uint32_t *src = swp[i] ? S[i] : R[i], *tgt = swp[i] ? R[i] : S[i];
            const uint32_t ntgt = swp[i] ? nR[i] : nS[i];
            auto &r = b->rint[i];
            r.resize(b->nR[i]);
            for (uint32_t j = 0; j < b->nR[i]; j++) r[j] = perm[src[j]] + b->node_off[i];
            std::sort(r.begin(), r.end());
            for (uint32_t j = 0; j < ntgt; j++) {
                const uint32_t x = perm[tgt[j]] + b->node_off[i];
                sb[x >> 5] |= 1u << (x & 31);
            }
        }
        b->sbits = upload_vec(sb);
        if (any_swap) b->inst_swap = upload_vec(swp);
        b->node_off_d = upload_vec(b->node_off);
        b->inst_pairs = (unsigned long long *)device_alloc(size_t(b->nq) * 8);
        b->inst_cycles = (unsigned long long *)device_alloc(size_t(b->nq) * 8);
        b->inst_ball = (uint32_t *)device_alloc(size_t(b->nq) * 4);
        b->pair_off_d = (unsigned long long *)device_alloc((size_t(b->nq) + 1) * 8);
        uint64_t totR = 0;
        for (uint32_t x : b->nR) totR += x;
        batch_reserve_pairs(b, std::max<uint64_t>(totR * 64, 1 << 16));
        b->stats.instances = b->nq;
        if (b->n_u >= SK_NODE)  // the warp search keys nodes in 28 bits
            for (auto &p : b->plan)
                if (p.T == 1) p = TILE_PLAN;
        batch_adapt_maps(b);
        batch_layout(b);
    } catch (...) {
        batch_destroy(b);
        throw;
    }
    return b;
}

void batch_pairs_dev(const Batch *b, uint32_t i, const uint32_t **u, const uint32_t **v, const uint32_t **d,
                     uint64_t *n) {
    if (i >= b->nq) fail(RN_EINVAL, "instance index out of range");
    if (b->cnt.empty()) fail(RN_EINVAL, "the batch has not run yet");
    *n = b->cnt[i];
    *u = b->out_u + b->off[i];
    *v = b->out_v + b->off[i];
    *d = b->out_d + b->off[i];
}

const rn_batch_stats &batch_stats(const Batch *b) { return b->stats; }

}  // namespace rn
