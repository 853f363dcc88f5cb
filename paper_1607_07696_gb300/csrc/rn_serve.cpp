// rn_serve.cpp -- serving distance joins and k-closest-pairs requests over one resident
// graph with continuous batching.
//
// A server owns an arena of distance-slab regions (the admission budget) and a pool of
// worker threads, each with its own engine workspace and CUDA stream.  Requests queue
// first come, first served; the head of the queue is admitted as soon as a worker is
// idle and enough contiguous slab regions are free.  An admitted request runs the
// engine's whole query (set preparation, tile search, emission, sort; for k closest
// pairs the radius passes and the select) on its worker's stream, with a search grid of
// as many blocks as it holds regions, so the kernels of every running request share the
// device: a request that arrives while others run starts at once if it fits, and its
// work overlaps theirs.  No kernel waits on another or on the host; the overlap comes
// from independent streams only.  A request's result does not depend on what else runs:
// it is computed by the same kernels on its own buffers.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <thread>
#include <unordered_map>

#include <cuda_runtime.h>

#include "rn_internal.h"

namespace rn {

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Request {
    uint64_t ticket = 0;
    std::vector<uint32_t> R, S;
    uint32_t theta = 0;
    uint64_t k = 0;
    uint32_t units = 0, unit_off = 0;
    Clock::time_point t_submit, t_admit, t_done;
    bool done = false;
    rn_status status = RN_OK;
    std::string err;
    rn_pairs out{};
};

struct Worker {
    Workspace *ws = nullptr;
    cudaStream_t stream = nullptr;
    uint32_t *dR = nullptr, *dS = nullptr;
    uint32_t capR = 0, capS = 0;
    rn_dpairs res{};
    std::thread th;
};

void check(cudaError_t e, const char *what) {
    if (e != cudaSuccess)
        fail(e == cudaErrorMemoryAllocation ? RN_ENOMEM : RN_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

void ensure_u32(uint32_t **p, uint32_t *cap, uint32_t want) {
    if (*p && *cap >= want) return;
    device_free(*p);
    *p = nullptr;
    *cap = std::max<uint32_t>(want, 4096);
    *p = (uint32_t *)device_alloc(size_t(*cap) * 4);
}

}  // namespace

struct Server {
    const rn_graph *g = nullptr;
    EngineConfig cfg;  // the graph's knobs when the server was made (a later change does not race)
    int device = 0;
    uint32_t tile_width = 32, max_blocks = 64;
    uint32_t *arena = nullptr;
    uint32_t units_total = 0;
    size_t unit_words = 0;
    std::vector<uint8_t> unit_busy;
    std::vector<Worker> workers;

    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Request>> pending;
    std::unordered_map<uint64_t, std::shared_ptr<Request>> reqs;
    uint64_t next_ticket = 1;
    bool stop = false;

    // statistics of the current window
    uint64_t submitted = 0, completed = 0, failed = 0, cancelled = 0, pairs = 0;
    uint64_t groups = 0, grouped = 0;  // searches that served several requests, and those requests
    uint32_t running = 0, max_running = 0, units_in_use = 0, units_peak = 0;
    std::vector<double> latency_ms;
    double queue_ms = 0, busy_s = 0;
    bool have_first = false;
    Clock::time_point first_submit, last_done, busy_since;

    // First fit of n contiguous free regions; false if none.
    bool fit(uint32_t n, uint32_t *off) const {
        uint32_t run = 0;
        for (uint32_t i = 0; i < units_total; i++) {
            run = unit_busy[i] ? 0 : run + 1;
            if (run == n) {
                *off = i + 1 - n;
                return true;
            }
        }
        return false;
    }

    void loop(Worker *w);
    void execute(Worker *w, Request *q);
    void execute_group(Worker *w, std::vector<std::shared_ptr<Request>> &grp, uint32_t units, uint32_t off);
};

void Server::execute(Worker *w, Request *q) {
    Range range(q->k ? "rn.serve.kcp" : "rn.serve.join");
    const rn_graph *G = g;
    workspace_set_slab(w->ws, arena + size_t(q->unit_off) * unit_words, q->units);
    const uint32_t nR = uint32_t(q->R.size()), nS = uint32_t(q->S.size());
    ensure_u32(&w->dR, &w->capR, std::max<uint32_t>(nR, 1));
    ensure_u32(&w->dS, &w->capS, std::max<uint32_t>(nS, 1));
    if (nR) copy_to_device(w->dR, q->R.data(), size_t(nR) * 4, w->stream);
    if (nS) copy_to_device(w->dS, q->S.data(), size_t(nS) * 4, w->stream);
    rn_query_stats st{};
    if (q->k == 0)
        run_join(G->dev, w->ws, cfg, G->info.median_weight, w->dR, nR, w->dS, nS, q->theta, &w->res, w->stream,
                 &st);
    else
        run_kcp(G->dev, w->ws, cfg, G->info.median_weight, w->dR, nR, w->dS, nS, q->k, q->theta, &w->res,
                w->stream, &st);
    to_host_pairs(w->res, &q->out, w->stream);
}

// Joins queued one behind another are taken together, up to MB_MAX of them and
// MB_MAX_SOURCES sources in all (the sources a worker's buffers are reserved for), and
// searched in one launch (continuous batching: requests that arrive while others run are
// admitted into the next free slot as a group).
constexpr uint32_t MB_MAX = 64, MB_MAX_SOURCES = 1u << 15;

void Server::execute_group(Worker *w, std::vector<std::shared_ptr<Request>> &grp, uint32_t units, uint32_t off) {
    Range range("rn.serve.join_many");
    const rn_graph *G = g;
    workspace_set_slab(w->ws, arena + size_t(off) * unit_words, units);
    const uint32_t nq = uint32_t(grp.size());
    std::vector<const uint32_t *> R(nq), S(nq);
    std::vector<uint32_t> nR(nq), nS(nq), theta(nq);
    for (uint32_t i = 0; i < nq; i++) {
        R[i] = grp[i]->R.data();
        S[i] = grp[i]->S.data();
        nR[i] = uint32_t(grp[i]->R.size());
        nS[i] = uint32_t(grp[i]->S.size());
        theta[i] = grp[i]->theta;
    }
    std::vector<uint64_t> counts;
    rn_query_stats st{};
    run_join_multi(G->dev, w->ws, cfg, G->info.median_weight, G->perm, R, nR, S, nS, theta, &w->res, &counts,
                   w->stream, &st);
    uint64_t at = 0;
    for (uint32_t i = 0; i < nq; i++) {
        rn_dpairs view{w->res.u + at, w->res.v + at, w->res.d + at, counts[i], counts[i]};
        to_host_pairs(view, &grp[i]->out, w->stream);
        at += counts[i];
    }
}

void Server::loop(Worker *w) {
    cudaSetDevice(device);  // the current device is per host thread
    for (;;) {
        std::vector<std::shared_ptr<Request>> grp;
        uint32_t units = 0, off = 0;
        {
            std::unique_lock<std::mutex> lk(mu);
            cv_work.wait(lk, [&] { return stop || (!pending.empty() && fit(pending.front()->units, &off)); });
            if (stop) return;
            grp.push_back(pending.front());
            pending.pop_front();
            units = grp[0]->units;
            auto join = [](const Request &r) { return r.k == 0; };
            if (join(*grp[0])) {
                // the joins right behind it join the group while their sources and regions fit
                uint64_t sources = grp[0]->R.size();
                while (grp.size() < MB_MAX && !pending.empty() && join(*pending.front())) {
                    const uint64_t more = sources + pending.front()->R.size();
                    if (more > MB_MAX_SOURCES) break;
                    const uint32_t want = std::min<uint32_t>(max_blocks, std::max<uint64_t>(2, (more + tile_width - 1) / tile_width));
                    uint32_t at = 0;
                    if (want > units && !fit(want, &at)) break;
                    if (want > units) {
                        units = want;
                        off = at;
                    }
                    sources = more;
                    grp.push_back(pending.front());
                    pending.pop_front();
                }
            }
            for (auto &q : grp) {
                q->unit_off = off;
                q->t_admit = Clock::now();
            }
            for (uint32_t i = 0; i < units; i++) unit_busy[off + i] = 1;
            units_in_use += units;
            units_peak = std::max(units_peak, units_in_use);
            if (running == 0) busy_since = grp[0]->t_admit;
            running += uint32_t(grp.size());
            max_running = std::max(max_running, running);
            if (grp.size() > 1) groups++, grouped += grp.size();
        }
        rn_status status = RN_OK;
        std::string err;
        try {
            if (grp.size() == 1) execute(w, grp[0].get());
            else execute_group(w, grp, units, off);
        } catch (const Error &e) {
            status = e.status;
            err = e.msg;
        } catch (const std::bad_alloc &) {
            status = RN_ENOMEM;
            err = "host allocation failed";
        } catch (const std::exception &e) {
            status = RN_EINTERNAL;
            err = e.what();
        }
        {
            std::lock_guard<std::mutex> lk(mu);
            for (uint32_t i = 0; i < units; i++) unit_busy[off + i] = 0;
            units_in_use -= units;
            const Clock::time_point now = Clock::now();
            for (auto &q : grp) {
                if (status != RN_OK) {
                    rn_pairs_free(&q->out);
                    q->status = status;
                    q->err = err;
                }
                q->t_done = now;
                q->done = true;
                if (q->status == RN_OK) {
                    completed++;
                    pairs += q->out.n;
                    latency_ms.push_back(ms_between(q->t_submit, q->t_done));
                    queue_ms += ms_between(q->t_submit, q->t_admit);
                } else {
                    failed++;
                }
            }
            running -= uint32_t(grp.size());
            if (running == 0) busy_s += ms_between(busy_since, now) / 1e3;
            last_done = now;
        }
        cv_done.notify_all();
        cv_work.notify_all();
    }
}

Server *server_create(const rn_graph *g, uint64_t slab_bytes, uint32_t workers, uint32_t max_blocks) {
    auto s = std::make_unique<Server>();
    s->g = g;
    {
        std::lock_guard<std::mutex> lk(const_cast<rn_graph *>(g)->mu);
        s->cfg = g->cfg;
    }
    s->device = g->device;
    check(cudaSetDevice(g->device), "cudaSetDevice");
    s->tile_width = s->cfg.tile_width > 1 ? s->cfg.tile_width : 32;
    int sms = 0;
    check(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device), "cudaDeviceGetAttribute");
    // by default a request may spread over one block per SM: its sources then sit a few to
    // a tile, whose union balls fit the shared maps, and a few requests still share the GPU
    s->max_blocks = max_blocks ? max_blocks : uint32_t(std::max(sms, 2));
    if (s->max_blocks < 2) fail(RN_EINVAL, "max_blocks must be >= 2");
    const uint32_t nworkers = workers ? workers : 8;
    if (nworkers > 256) fail(RN_EINVAL, "at most 256 workers");
    const size_t region = slab_region_bytes();
    const uint64_t bytes = slab_bytes ? slab_bytes : (uint64_t(4) << 30);
    s->units_total = uint32_t(std::min<uint64_t>(bytes / region, 1u << 20));
    if (s->units_total < s->max_blocks)
        fail(RN_EINVAL, "slab_bytes must hold max_blocks regions of " + std::to_string(region) + " bytes");
    s->unit_words = region / 4;
    s->unit_busy.assign(s->units_total, 0);
    s->arena = (uint32_t *)device_alloc(size_t(s->units_total) * region);
    check(cudaMemset(s->arena, 0xFF, size_t(s->units_total) * region), "cudaMemset");  // every row INF
    check(cudaDeviceSynchronize(), "cudaDeviceSynchronize");  // before any worker's stream uses it
    s->workers.resize(nworkers);
    try {
        for (auto &w : s->workers) {
            w.ws = workspace_create(g->dev);
            // requests up to 32768 sources and 2^22 pairs then allocate nothing
            workspace_reserve(w.ws, 1u << 15, uint64_t(1) << 22);
            ensure_u32(&w.dR, &w.capR, 1u << 15);
            ensure_u32(&w.dS, &w.capS, 1u << 15);
            dpairs_reserve(&w.res, uint64_t(1) << 22);
            check(cudaStreamCreateWithFlags(&w.stream, cudaStreamNonBlocking), "cudaStreamCreateWithFlags");
        }
        for (auto &w : s->workers) {
            Worker *wp = &w;
            Server *sp = s.get();
            w.th = std::thread([sp, wp] { sp->loop(wp); });
        }
    } catch (...) {
        server_destroy(s.release());
        throw;
    }
    return s.release();
}

uint64_t server_submit(Server *s, const uint32_t *R, uint32_t nR, const uint32_t *S, uint32_t nS, uint32_t theta,
                       uint64_t k) {
    auto q = std::make_shared<Request>();
    q->R.assign(R, R + nR);
    q->S.assign(S, S + nS);
    q->theta = theta;
    q->k = k;
    const uint32_t T = s->tile_width;
    q->units = std::min<uint32_t>(s->max_blocks, std::max<uint32_t>(2, (nR + T - 1) / T));
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) fail(RN_ECANCELLED, "the server is stopping");
        q->ticket = s->next_ticket++;
        q->t_submit = Clock::now();
        if (!s->have_first) {
            s->first_submit = q->t_submit;
            s->have_first = true;
        }
        s->submitted++;
        s->reqs[q->ticket] = q;
        s->pending.push_back(q);
    }
    s->cv_work.notify_all();
    return q->ticket;
}

void server_wait(Server *s, uint64_t ticket, uint32_t timeout_ms, rn_pairs *out) {
    std::shared_ptr<Request> q;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        auto it = s->reqs.find(ticket);
        if (it == s->reqs.end()) fail(RN_EINVAL, "unknown ticket (never issued, or already collected)");
        q = it->second;
        auto ready = [&] { return q->done; };
        if (timeout_ms == 0xFFFFFFFFu) s->cv_done.wait(lk, ready);
        else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready))
            fail(RN_ETIMEOUT, "request " + std::to_string(ticket) + " not done within " + std::to_string(timeout_ms) +
                                  " ms");
        s->reqs.erase(ticket);
    }
    if (q->status != RN_OK) fail(q->status, q->err);
    *out = q->out;
    q->out = rn_pairs{};
}

// Cancel a queued request: it leaves the queue and its wait returns RN_ECANCELLED.  A
// request already on the device runs to the end (no kernel is interrupted): RN_EBUSY.
void server_cancel(Server *s, uint64_t ticket) {
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->reqs.find(ticket);
        if (it == s->reqs.end()) fail(RN_EINVAL, "unknown ticket (never issued, or already collected)");
        std::shared_ptr<Request> q = it->second;
        if (q->done) fail(RN_EBUSY, "request " + std::to_string(ticket) + " has already finished");
        auto pos = std::find(s->pending.begin(), s->pending.end(), q);
        if (pos == s->pending.end()) fail(RN_EBUSY, "request " + std::to_string(ticket) + " is running");
        s->pending.erase(pos);
        q->status = RN_ECANCELLED;
        q->err = "request " + std::to_string(ticket) + " was cancelled";
        q->done = true;
        s->cancelled++;
    }
    s->cv_done.notify_all();
    s->cv_work.notify_all();  // the next request may fit now
}

void server_stats(Server *s, rn_serve_stats *out) {
    std::lock_guard<std::mutex> lk(s->mu);
    rn_serve_stats r{};
    r.submitted = s->submitted;
    r.completed = s->completed;
    r.failed = s->failed;
    r.cancelled = s->cancelled;
    r.groups = s->groups;
    r.grouped = s->grouped;
    r.pending = s->pending.size();
    r.running = s->running;
    r.pairs = s->pairs;
    const uint64_t region = slab_region_bytes();
    r.slab_bytes = uint64_t(s->units_total) * region;
    r.slab_bytes_in_use = uint64_t(s->units_in_use) * region;
    r.slab_bytes_peak = uint64_t(s->units_peak) * region;
    r.workers = uint32_t(s->workers.size());
    r.max_running = s->max_running;
    if (!s->latency_ms.empty()) {
        std::vector<double> l = s->latency_ms;
        std::sort(l.begin(), l.end());
        auto pct = [&](double p) { return l[std::min<size_t>(l.size() - 1, size_t(p * double(l.size() - 1) + 0.5))]; };
        r.p50_ms = pct(0.50);
        r.p99_ms = pct(0.99);
        r.max_ms = l.back();
        double sum = 0;
        for (double x : l) sum += x;
        r.mean_ms = sum / double(l.size());
        r.mean_queue_ms = s->queue_ms / double(l.size());
    }
    r.busy_s = s->busy_s;
    if (s->running) r.busy_s += ms_between(s->busy_since, Clock::now()) / 1e3;
    if (s->have_first && s->completed + s->failed) r.span_s = ms_between(s->first_submit, s->last_done) / 1e3;
    *out = r;
}

void server_reset_stats(Server *s) {
    std::lock_guard<std::mutex> lk(s->mu);
    s->submitted = s->pending.size() + s->running;
    s->completed = s->failed = s->cancelled = s->pairs = 0;
    s->groups = s->grouped = 0;
    s->max_running = s->running;
    s->units_peak = s->units_in_use;
    s->latency_ms.clear();
    s->queue_ms = 0;
    s->busy_s = 0;
    if (s->running) s->busy_since = Clock::now();
    s->have_first = false;
}

void server_destroy(Server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->pending.clear();
    }
    s->cv_work.notify_all();
    for (auto &w : s->workers)
        if (w.th.joinable()) w.th.join();
    for (auto &kv : s->reqs) rn_pairs_free(&kv.second->out);
    s->reqs.clear();
    for (auto &w : s->workers) {
        if (w.stream) cudaStreamSynchronize(w.stream);
        workspace_destroy(w.ws);
        device_free(w.dR);
        device_free(w.dS);
        dpairs_release(&w.res);
        if (w.stream) cudaStreamDestroy(w.stream);
    }
    device_free(s->arena);
    delete s;
}

}  // namespace rn
