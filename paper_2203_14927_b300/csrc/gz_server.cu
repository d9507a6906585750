// gz_server.cu -- serving many independent graphs on one GPU (host code only;
// the device work is the library's ingestion and query kernels).
//
// State: every graph has a FIFO of requests and is WAITING (no device memory
// yet), RESIDENT (a gz_handle holds its sketches), EVICTED (its sketches wait
// in pinned host memory as a checkpoint) or RELEASED.  `slots` worker
// threads, each with its own CUDA stream, loop:
//   - serve a resident idle graph with pending requests (oldest request
//     first): finishing resident graphs is what frees memory;
//   - else admit the waiting or evicted graph with the oldest request that
//     fits in the remaining budget (create, or restore its checkpoint);
//   - else, when such a graph has waited kEvictAfterMs, evict the least
//     recently used idle resident graph (checkpoint to pinned host memory,
//     free its device memory) to make room;
// taking up to max_batch requests of a graph, serving them in order on the
// worker's stream, reporting the completions, and releasing the graph's
// memory once it is closed and drained.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/gz.h"
#include "gz_handle.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t id;
    uint32_t kind;  // 0 update, 1 query
    std::vector<uint32_t> u, v;            // owned copy, or empty when borrowed
    const uint32_t *bu = nullptr, *bv = nullptr;  // the caller's arrays (GZ_SUBMIT_NOCOPY)
    size_t n = 0;
    uint32_t* labels = nullptr;
    double submit_ms = 0;
};

enum GraphState { WAITING = 0, RESIDENT = 1, RELEASED = 2, EVICTED = 3 };

// a graph that cannot be admitted for this long evicts an idle resident one
constexpr double kEvictAfterMs = 20.0;
constexpr size_t kPinChunk = size_t(256) << 20;

struct Graph {
    uint32_t V = 0;
    uint64_t seed = 0;
    gz_config cfg{};
    bool has_cfg = false;
    uint64_t bytes = 0;
    GraphState state = WAITING;
    bool busy = false, closed = false;
    gz_handle* h = nullptr;
    std::deque<Request> queue;
    double last_used_ms = 0;         // end of its last service
    std::vector<void*> chunks;       // an evicted graph's sketches, in pinned host chunks
    uint64_t evictions = 0;
};

}  // namespace

struct gz_server {
    gz_server_config cfg{};
    int device = 0;
    Clock::time_point t0;
    std::mutex mu;
    std::condition_variable work_cv, done_cv;
    std::vector<std::unique_ptr<Graph>> graphs;
    std::deque<gz_completion> completions;
    std::vector<std::thread> workers;
    std::vector<cudaStream_t> streams;
    uint64_t next_req = 1;
    uint64_t resident_bytes = 0, peak_bytes = 0, completed = 0, evictions = 0;
    uint64_t evicting_bytes = 0;  // resident bytes of graphs being checkpointed out
    double evict_ms = 0, restore_ms = 0;
    // pinned host memory for evicted sketches, in chunks of kPinChunk bytes
    // shared by every graph and kept until the server is destroyed (pinning
    // host memory costs far more than the copy into it)
    std::vector<void*> pin_free, pin_all;
    uint64_t outstanding = 0;  // submitted, not completed
    uint32_t busy_workers = 0;
    bool stop = false;
    std::string last_err;

    double now_ms() const {
        return std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
    }
};

namespace {

uint64_t graph_bytes(uint32_t V, const gz_config* cfg) {
    size_t b = 0;
    gz_memory_bytes(V, cfg, &b);
    // query scratch (labels, parents, members, ... and the merge accumulators)
    // and the host-input staging buffers
    uint32_t K = 0, R = 0;
    gz_geometry(V, &K, &R);
    const uint32_t cl = cfg && cfg->chunk_log2 ? cfg->chunk_log2 : 24;
    return b + (uint64_t)V * 96 + (uint64_t)gz::query_slots(V) * 84ull * R + (4ull << cl) * 4;
}

enum Task { NONE = 0, SERVE = 1, EVICT = 2 };

// Pick work under the lock (see the top of the file for the order).
Task pick(gz_server* s, uint32_t* gid) {
    const double now = s->now_ms();
    int best = -1, adm = -1, starving = -1, lru = -1;
    for (size_t i = 0; i < s->graphs.size(); ++i) {
        Graph* g = s->graphs[i].get();
        if (g->busy || g->state == RELEASED) continue;
        if (g->queue.empty()) {
            if (g->state == RESIDENT && !g->closed && g->h && !g->h->tiered &&
                (lru < 0 || g->last_used_ms < s->graphs[lru]->last_used_ms))
                lru = (int)i;
            continue;
        }
        const double t = g->queue.front().submit_ms;
        if (g->state == RESIDENT) {
            if (best < 0 || t < s->graphs[best]->queue.front().submit_ms) best = (int)i;
        } else if (s->resident_bytes + g->bytes <= s->cfg.hbm_budget) {
            if (adm < 0 || t < s->graphs[adm]->queue.front().submit_ms) adm = (int)i;
        } else if (now - t >= kEvictAfterMs) {
            if (starving < 0 || t < s->graphs[starving]->queue.front().submit_ms) starving = (int)i;
        }
    }
    // resident graphs first, unless an admissible graph has waited
    // kEvictAfterMs longer than the oldest resident request (no starvation)
    if (adm >= 0 && (best < 0 || s->graphs[adm]->queue.front().submit_ms + kEvictAfterMs <
                                     s->graphs[best]->queue.front().submit_ms)) {
        *gid = (uint32_t)adm;
        return SERVE;
    }
    if (best >= 0) {
        *gid = (uint32_t)best;
        return SERVE;
    }
    // evict only what the oldest starving graph still lacks once the
    // evictions under way have finished
    if (starving >= 0 && lru >= 0 &&
        s->resident_bytes - s->evicting_bytes + s->graphs[starving]->bytes > s->cfg.hbm_budget) {
        *gid = (uint32_t)lru;
        return EVICT;
    }
    return NONE;
}

// n pinned chunks: spare ones first, new ones for the rest
bool take_chunks(gz_server* s, size_t n, std::vector<void*>& out) {
    {
        std::lock_guard<std::mutex> lk(s->mu);
        while (out.size() < n && !s->pin_free.empty()) {
            out.push_back(s->pin_free.back());
            s->pin_free.pop_back();
        }
    }
    while (out.size() < n) {
        void* p = nullptr;
        if (cudaMallocHost(&p, kPinChunk) != cudaSuccess) return false;
        std::lock_guard<std::mutex> lk(s->mu);
        s->pin_all.push_back(p);
        out.push_back(p);
    }
    return true;
}

void give_chunks(gz_server* s, std::vector<void*>& chunks) {
    std::lock_guard<std::mutex> lk(s->mu);
    for (void* p : chunks) s->pin_free.push_back(p);
    chunks.clear();
}

// Copy an idle resident graph's sketches into pinned host chunks and free its
// device memory (outside the lock; the graph is marked busy).  The graph's
// stream is idle and its last request's status already reported.
gz_status evict_graph(gz_server* s, Graph* g) {
    gz_handle* h = g->h;
    gz_status st = gz_sync(h);
    if (st != GZ_OK) return st;
    const size_t bytes = (size_t)h->V * h->node_bytes;
    std::vector<void*> ch;
    if (!take_chunks(s, (bytes + kPinChunk - 1) / kPinChunk, ch)) {
        give_chunks(s, ch);
        return GZ_ENOMEM;
    }
    cudaError_t e = cudaSuccess;
    for (size_t i = 0; i < ch.size() && e == cudaSuccess; ++i)
        e = cudaMemcpyAsync(ch[i], h->d_sketch + i * kPinChunk, std::min(kPinChunk, bytes - i * kPinChunk),
                            cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        give_chunks(s, ch);
        return GZ_ECUDA;
    }
    g->chunks = std::move(ch);
    gz_destroy(h);
    g->h = nullptr;
    return GZ_OK;
}

// A fresh handle with the evicted graph's sketches (same V, seed and
// configuration, so the same hash keys); the chunks go back to the pool.
gz_status restore_graph(gz_server* s, Graph* g, cudaStream_t stream) {
    gz_status st = gz_create(g->V, g->seed, g->has_cfg ? &g->cfg : nullptr, stream, &g->h);
    if (st != GZ_OK) {
        g->h = nullptr;
        return st;
    }
    gz_handle* h = g->h;
    const size_t bytes = (size_t)h->V * h->node_bytes;
    cudaError_t e = cudaSuccess;
    for (size_t i = 0; i < g->chunks.size() && e == cudaSuccess; ++i)
        e = cudaMemcpyAsync(h->d_sketch + i * kPinChunk, g->chunks[i], std::min(kPinChunk, bytes - i * kPinChunk),
                            cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        gz_destroy(h);
        g->h = nullptr;
        return GZ_ECUDA;
    }
    give_chunks(s, g->chunks);
    return GZ_OK;
}

void worker_main(gz_server* s, int slot) {
    cudaSetDevice(s->device);
    cudaStream_t stream = s->streams[slot];
    for (;;) {
        uint32_t gid = 0;
        Graph* g = nullptr;
        std::vector<Request> batch;
        bool admit = false, restore = false;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            Task task = NONE;
            for (;;) {
                task = pick(s, &gid);
                if (task != NONE || s->stop) break;
                // an admission that waits for memory is re-examined after
                // kEvictAfterMs even when nothing else happens
                s->work_cv.wait_for(lk, std::chrono::milliseconds((int)kEvictAfterMs));
            }
            if (task == NONE) return;  // stopping and nothing left to do
            g = s->graphs[gid].get();
            g->busy = true;
            ++s->busy_workers;
            if (task == EVICT) {
                s->evicting_bytes += g->bytes;
                lk.unlock();
                gz_set_stream(g->h, stream);
                const double te = s->now_ms();
                const gz_status est = evict_graph(s, g);
                lk.lock();
                s->evict_ms += s->now_ms() - te;
                g->busy = false;
                --s->busy_workers;
                s->evicting_bytes -= g->bytes;
                if (est == GZ_OK) {
                    g->state = EVICTED;
                    s->resident_bytes -= g->bytes;
                    ++g->evictions;
                    ++s->evictions;
                    if (g->closed && g->queue.empty()) {  // closed while it was copied out
                        g->state = RELEASED;
                        for (void* p : g->chunks) s->pin_free.push_back(p);
                        g->chunks.clear();
                    }
                } else {
                    s->last_err = "eviction of graph " + std::to_string(gid) + " failed";
                }
                lk.unlock();
                s->work_cv.notify_all();
                s->done_cv.notify_all();
                continue;
            }
            if (g->state == WAITING || g->state == EVICTED) {
                admit = g->state == WAITING;
                restore = g->state == EVICTED;
                g->state = RESIDENT;  // memory is reserved now, taken below
                s->resident_bytes += g->bytes;
                s->peak_bytes = std::max(s->peak_bytes, s->resident_bytes);
            }
            const uint32_t take = std::min<size_t>(g->queue.size(), s->cfg.max_batch);
            for (uint32_t i = 0; i < take; ++i) {
                batch.push_back(std::move(g->queue.front()));
                g->queue.pop_front();
            }
        }
        gz_status create_st = GZ_OK;
        if (admit) {
            create_st = gz_create(g->V, g->seed, g->has_cfg ? &g->cfg : nullptr, stream, &g->h);
            if (create_st != GZ_OK) g->h = nullptr;
        } else if (restore) {
            const double tr = s->now_ms();
            create_st = restore_graph(s, g, stream);
            std::lock_guard<std::mutex> lk(s->mu);
            s->restore_ms += s->now_ms() - tr;
        } else if (g->h) {
            gz_set_stream(g->h, stream);  // the previous worker synchronised before releasing it
        }
        std::vector<gz_completion> done;
        done.reserve(batch.size());
        std::string err;
        // updates are queued back to back; the completion time of a run of
        // updates is taken when the stream next synchronises (a query, or
        // the end of the batch)
        size_t unsynced = 0;
        auto settle = [&](gz_status st) {
            const double t = s->now_ms();
            for (size_t i = done.size() - unsynced; i < done.size(); ++i) {
                done[i].done_ms = t;
                if (done[i].status == GZ_OK) done[i].status = st;
            }
            unsynced = 0;
        };
        for (Request& r : batch) {
            gz_completion c{};
            c.req_id = r.id;
            c.graph = gid;
            c.kind = r.kind;
            c.submit_ms = r.submit_ms;
            c.start_ms = s->now_ms();
            gz_status st = create_st;
            if (st == GZ_OK && !g->h) st = GZ_ENOMEM;
            if (st == GZ_OK && r.kind == 0) {
                st = gz_edge_update(g->h, r.bu, r.bv, r.n, 0);
                c.n_updates = r.n;
                c.status = st;
                done.push_back(c);
                ++unsynced;
            } else {
                if (st == GZ_OK) {
                    settle(gz_sync(g->h));
                    uint32_t ncc = 0;
                    st = gz_connected_components(g->h, r.labels, &ncc, nullptr);
                    c.n_components = ncc;
                }
                c.status = st;
                c.done_ms = s->now_ms();
                done.push_back(c);
            }
            if (st != GZ_OK && st != GZ_ESKETCH_FAIL && err.empty())
                err = "graph " + std::to_string(gid) + ": " + (g->h ? gz_last_error(g->h) : "no handle");
            std::vector<uint32_t>().swap(r.u);
            std::vector<uint32_t>().swap(r.v);
        }
        if (g->h) settle(gz_sync(g->h));
        else settle(GZ_OK);
        gz_handle* to_free = nullptr;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            for (const gz_completion& c : done) s->completions.push_back(c);
            if (!err.empty()) s->last_err = err;
            s->completed += done.size();
            s->outstanding -= done.size();
            g->busy = false;
            g->last_used_ms = s->now_ms();
            --s->busy_workers;
            if (create_st != GZ_OK) {
                // the graph cannot be admitted: its queued requests fail too
                for (Request& r : g->queue) {
                    gz_completion c{};
                    c.req_id = r.id;
                    c.graph = gid;
                    c.kind = r.kind;
                    c.status = create_st;
                    c.submit_ms = r.submit_ms;
                    c.start_ms = c.done_ms = s->now_ms();
                    s->completions.push_back(c);
                    ++s->completed;
                    --s->outstanding;
                }
                g->queue.clear();
            }
            if ((g->closed && g->queue.empty()) || create_st != GZ_OK) {
                if (g->state == RESIDENT) s->resident_bytes -= g->bytes;
                g->state = RELEASED;
                to_free = g->h;
                g->h = nullptr;
                for (void* p : g->chunks) s->pin_free.push_back(p);
                g->chunks.clear();
            }
        }
        if (to_free) gz_destroy(to_free);
        s->work_cv.notify_all();
        s->done_cv.notify_all();
    }
}

}  // namespace

extern "C" {

gz_status gz_server_create(const gz_server_config* cfg, gz_server** out) {
    if (!out) return GZ_EINVAL;
    *out = nullptr;
    gz_server* s = new (std::nothrow) gz_server();
    if (!s) return GZ_ENOMEM;
    if (cfg) s->cfg = *cfg;
    if (s->cfg.slots == 0) s->cfg.slots = 4;
    if (s->cfg.max_batch == 0) s->cfg.max_batch = 64;
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        return GZ_ECUDA;
    }
    if (s->cfg.hbm_budget == 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            delete s;
            return GZ_ECUDA;
        }
        s->cfg.hbm_budget = (uint64_t)(0.8 * fr);
    }
    // Graphs are admitted and released all the time; keep up to the budget of
    // freed memory in the device's stream-ordered pool instead of returning it
    // to the driver at every synchronisation (the pool's default), so an
    // admission reuses memory a released graph left.  This is a property of
    // the device's default pool, shared with the rest of the process.
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, s->device) == cudaSuccess) {
        uint64_t keep = s->cfg.hbm_budget;
        uint64_t cur = 0;
        if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &cur) == cudaSuccess && cur < keep)
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    // pinned chunks for evictions, pinned now rather than under load
    for (uint64_t b = 0; b < (uint64_t)s->cfg.host_pool_mb << 20; b += kPinChunk) {
        void* p = nullptr;
        if (cudaMallocHost(&p, kPinChunk) != cudaSuccess) {
            for (void* q : s->pin_all) cudaFreeHost(q);
            delete s;
            return GZ_ENOMEM;
        }
        s->pin_all.push_back(p);
        s->pin_free.push_back(p);
    }
    s->t0 = Clock::now();
    for (uint32_t i = 0; i < s->cfg.slots; ++i) {
        cudaStream_t st;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
            delete s;
            return GZ_ECUDA;
        }
        s->streams.push_back(st);
    }
    for (uint32_t i = 0; i < s->cfg.slots; ++i) s->workers.emplace_back(worker_main, s, (int)i);
    *out = s;
    return GZ_OK;
}

gz_status gz_server_destroy(gz_server* s) {
    if (!s) return GZ_EINVAL;
    gz_server_drain(s);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->work_cv.notify_all();
    for (std::thread& t : s->workers) t.join();
    for (auto& g : s->graphs)
        if (g->h) gz_destroy(g->h);
    for (void* p : s->pin_all) cudaFreeHost(p);
    for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
    delete s;
    return GZ_OK;
}

gz_status gz_server_add_graph(gz_server* s, uint32_t V, uint64_t seed, const gz_config* cfg, uint32_t* graph) {
    if (!s || !graph) return GZ_EINVAL;
    uint32_t K, R;
    if (gz_geometry(V, &K, &R) != GZ_OK) return GZ_EINVAL;
    std::unique_ptr<Graph> g(new (std::nothrow) Graph());
    if (!g) return GZ_ENOMEM;
    g->V = V;
    g->seed = seed;
    if (cfg) g->cfg = *cfg;
    // serving requests are small batches: partition buffers for 2^20 updates
    // unless the caller chose otherwise (larger batches are split by the call)
    if (g->cfg.chunk_log2 == 0) g->cfg.chunk_log2 = 20;
    // the server overlaps graphs on its worker streams; a graph's own
    // partition/update pipeline would only add a stream and buffers per graph
    g->cfg.no_pipeline = 1;
    g->has_cfg = true;
    g->bytes = graph_bytes(V, &g->cfg);
    std::lock_guard<std::mutex> lk(s->mu);
    if (g->bytes > s->cfg.hbm_budget) return GZ_ENOMEM;
    *graph = (uint32_t)s->graphs.size();
    s->graphs.push_back(std::move(g));
    return GZ_OK;
}

static gz_status submit(gz_server* s, uint32_t graph, Request&& r, uint64_t* req_id) {
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (graph >= s->graphs.size()) return GZ_EINVAL;
        Graph* g = s->graphs[graph].get();
        if (g->closed || g->state == RELEASED) return GZ_EINVAL;
        r.id = s->next_req++;
        r.submit_ms = s->now_ms();
        if (req_id) *req_id = r.id;
        g->queue.push_back(std::move(r));
        ++s->outstanding;
    }
    s->work_cv.notify_all();
    return GZ_OK;
}

gz_status gz_server_submit_update(gz_server* s, uint32_t graph, const uint32_t* u, const uint32_t* v, size_t n,
                                  uint32_t flags, uint64_t* req_id) {
    if (!s || (n && (!u || !v))) return GZ_EINVAL;
    Request r;
    r.kind = 0;
    r.n = n;
    if (flags & GZ_SUBMIT_NOCOPY) {
        r.bu = u;
        r.bv = v;
    } else {
        try {
            r.u.assign(u, u + n);
            r.v.assign(v, v + n);
        } catch (...) {
            return GZ_ENOMEM;
        }
        r.bu = r.u.data();
        r.bv = r.v.data();
    }
    return submit(s, graph, std::move(r), req_id);
}

gz_status gz_server_submit_query(gz_server* s, uint32_t graph, uint32_t* labels, uint64_t* req_id) {
    if (!s) return GZ_EINVAL;
    Request r;
    r.kind = 1;
    r.labels = labels;
    return submit(s, graph, std::move(r), req_id);
}

gz_status gz_server_close_graph(gz_server* s, uint32_t graph) {
    if (!s) return GZ_EINVAL;
    gz_handle* to_free = nullptr;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (graph >= s->graphs.size()) return GZ_EINVAL;
        Graph* g = s->graphs[graph].get();
        g->closed = true;
        if (!g->busy && g->queue.empty() && g->state != RELEASED) {
            if (g->state == RESIDENT) s->resident_bytes -= g->bytes;
            g->state = RELEASED;
            to_free = g->h;
            g->h = nullptr;
            for (void* p : g->chunks) s->pin_free.push_back(p);
            g->chunks.clear();
        }
    }
    if (to_free) gz_destroy(to_free);
    s->work_cv.notify_all();
    return GZ_OK;
}

gz_status gz_server_poll(gz_server* s, gz_completion* out, size_t max, size_t* n, int wait_ms) {
    if (!s || !n || (max && !out)) return GZ_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->completions.empty() && wait_ms > 0)
        s->done_cv.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return !s->completions.empty(); });
    size_t k = 0;
    while (k < max && !s->completions.empty()) {
        out[k++] = s->completions.front();
        s->completions.pop_front();
    }
    *n = k;
    return GZ_OK;
}

gz_status gz_server_drain(gz_server* s) {
    if (!s) return GZ_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    s->done_cv.wait(lk, [&] { return s->outstanding == 0; });
    return GZ_OK;
}

const char* gz_server_last_error(gz_server* s) {
    if (!s) return "null server";
    std::lock_guard<std::mutex> lk(s->mu);
    thread_local std::string copy;
    copy = s->last_err;
    return copy.c_str();
}

gz_status gz_server_set_budget(gz_server* s, uint64_t hbm_budget) {
    if (!s || !hbm_budget) return GZ_EINVAL;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->cfg.hbm_budget = hbm_budget;
    }
    cudaMemPool_t pool;
    uint64_t cur = 0;
    if (cudaDeviceGetDefaultMemPool(&pool, s->device) == cudaSuccess &&
        cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &cur) == cudaSuccess && cur < hbm_budget)
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &hbm_budget);
    s->work_cv.notify_all();
    return GZ_OK;
}

gz_status gz_server_stats_read(gz_server* s, gz_server_stats* out) {
    if (!s || !out) return GZ_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    std::memset(out, 0, sizeof(*out));
    out->resident_bytes = s->resident_bytes;
    out->peak_resident_bytes = s->peak_bytes;
    out->budget_bytes = s->cfg.hbm_budget;
    out->graphs = (uint32_t)s->graphs.size();
    for (auto& g : s->graphs) {
        out->resident_graphs += g->state == RESIDENT;
        out->waiting_graphs += g->state == WAITING && !g->queue.empty();
        out->evicted_graphs += g->state == EVICTED;
        out->pending_requests += (uint32_t)g->queue.size();
    }
    out->completed_requests = s->completed;
    out->evictions = s->evictions;
    out->evict_ms = s->evict_ms;
    out->pinned_chunks = (uint32_t)s->pin_all.size();
    out->restore_ms = s->restore_ms;
    return GZ_OK;
}

}  // extern "C"
