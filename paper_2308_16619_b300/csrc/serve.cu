// serve.cu -- csgv_serve_*: a decode server with a device-resident cache of
// decoded bricks (Sec. 4.1 of the paper: bricks are requested at a level of
// detail, decoded in parallel on the GPU into a cache, and evicted when not
// needed).
//
// A client submits a list of (brick, LOD) requests and gets a ticket.  A
// worker thread
//   * dedupes each request against the cache: a ready entry is a hit, an
//     entry still being decoded is shared, anything else is a miss;
//   * admits misses only while cache space can be found: a free slot of the
//     request's size (one free stack per LOD, as in the Shading Atlas
//     Streaming design the paper adapts), fresh space from the pool's top,
//     or the least recently used unpinned entry of the same LOD; if nothing
//     is pinned and space is still missing the cache is rebuilt (cleared);
//     otherwise the request waits until releases free space;
//   * launches admitted misses as batched decodes (one persistent launch per
//     batch) round-robin over several CUDA streams, so batches submitted
//     while others run overlap on the device (continuous batching);
//   * notices finished batches through CUDA events and completes tickets.
// Results are device pointers into the cache, valid until the ticket is
// released.  Latency per ticket = submit to completion, as seen by the worker.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "csgv_internal.cuh"
#include "../../include/csgv.h"

namespace csgv {
void set_last_error(const char *msg);  // api.cu
}

namespace {

using Clock = std::chrono::steady_clock;

struct Entry {
    uint32_t brick;
    uint8_t lod;
    bool ready = false;
    int32_t status = 0;
    uint64_t off = 0;  // in labels from the pool start
    uint32_t pins = 0;
    bool in_lru = false;
    bool transient = false;  // out-of-range request: owned by its ticket, never cached
    std::list<Entry *>::iterator lru_it;
};

struct Ticket {
    uint64_t id;
    std::vector<uint32_t> bricks;
    std::vector<uint8_t> lods;
    std::vector<Entry *> entries;  // filled as requests are admitted
    size_t admitted = 0;
    Clock::time_point t_submit, t_done;
    bool done = false;
};

struct Batch {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    bool busy = false;
    uint32_t cap = 0;
    uint32_t *ids_d = nullptr;
    uint8_t *lods_d = nullptr;
    uint64_t *offs_d = nullptr;
    int32_t *status_d = nullptr;
    uint32_t *ids_h = nullptr;  // pinned staging
    uint8_t *lods_h = nullptr;
    uint64_t *offs_h = nullptr;
    int32_t *status_h = nullptr;
    std::vector<Entry *> entries;
};

int set_err(int code, const char *msg) {
    csgv::set_last_error(msg);
    return code;
}

}  // namespace

struct csgv_server {
    const csgv_volume *vol = nullptr;
    int device = 0;
    uint32_t N = 0, b = 0;
    uint32_t *pool = nullptr;
    uint64_t pool_labels = 0, top = 0;
    std::vector<uint64_t> free_slots[csgv::kMaxN + 1];
    std::list<Entry *> lru[csgv::kMaxN + 1];
    std::unordered_map<uint64_t, Entry *> map;
    std::deque<Ticket *> waiting;
    std::unordered_map<uint64_t, Ticket *> tickets;
    std::vector<Entry *> to_launch;
    std::vector<Batch> batches;
    uint32_t max_batch = 0, next_batch = 0;
    uint64_t next_ticket = 1;
    csgv_serve_stats stats{};
    std::vector<double> latencies_ms;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread worker;
    bool stop = false;
    int fatal = 0;

    uint64_t slot_labels(uint32_t lod) const {
        const uint64_t s = (uint64_t)(b >> lod) * (b >> lod) * (b >> lod);
        return (s + 3) & ~3ull;  // 16-byte slots
    }
    static uint64_t key(uint32_t brick, uint32_t lod) { return ((uint64_t)brick << 8) | lod; }

    void lru_remove(Entry *e) {
        if (e->in_lru) {
            lru[e->lod].erase(e->lru_it);
            e->in_lru = false;
        }
    }
    void pin(Entry *e) {
        lru_remove(e);
        e->pins++;
    }
    void unpin(Entry *e) {
        if (e->pins && --e->pins == 0 && e->ready) {
            lru[e->lod].push_back(e);
            e->lru_it = std::prev(lru[e->lod].end());
            e->in_lru = true;
        }
    }
    // cache space for one block of `lod`; false if none can be found now
    bool alloc(uint32_t lod, uint64_t &off) {
        if (!free_slots[lod].empty()) {
            off = free_slots[lod].back();
            free_slots[lod].pop_back();
            return true;
        }
        const uint64_t s = slot_labels(lod);
        if (top + s <= pool_labels) {
            off = top;
            top += s;
            return true;
        }
        if (!lru[lod].empty()) {
            Entry *v = lru[lod].front();
            lru[lod].pop_front();
            v->in_lru = false;
            map.erase(key(v->brick, v->lod));
            off = v->off;
            delete v;
            stats.evictions++;
            return true;
        }
        // rebuild: nothing pinned and nothing decoding -> drop every entry, reset the pool
        bool busy = false;
        for (auto &kv : map)
            if (kv.second->pins || !kv.second->ready) busy = true;
        if (!busy && !map.empty()) {
            for (auto &kv : map) delete kv.second;
            map.clear();
            for (auto &l : lru) l.clear();
            for (auto &f : free_slots) f.clear();
            top = 0;
            stats.rebuilds++;
            if (top + s <= pool_labels) {
                off = top;
                top += s;
                return true;
            }
        }
        return false;
    }

    void admit() {
        while (!waiting.empty()) {
            Ticket *t = waiting.front();
            while (t->admitted < t->bricks.size()) {
                const uint32_t br = t->bricks[t->admitted], lod = t->lods[t->admitted];
                auto it = map.find(key(br, lod));
                if (it != map.end()) {
                    pin(it->second);
                    t->entries.push_back(it->second);
                    if (it->second->ready) stats.hits++;
                    else stats.shared++;
                } else {
                    uint64_t off;
                    if (br >= n_bricks || lod > N) {
                        // out of range: an entry that is ready with an error, no cache space
                        Entry *e = new Entry();
                        e->brick = br;
                        e->lod = (uint8_t)lod;
                        e->ready = true;
                        e->status = CSGV_ERR_RANGE;
                        e->transient = true;
                        t->entries.push_back(e);
                        t->admitted++;
                        admitted_any = true;
                        continue;
                    }
                    if (!alloc(lod, off)) return;  // wait for space: admission by free memory
                    Entry *e = new Entry();
                    e->brick = br;
                    e->lod = (uint8_t)lod;
                    e->off = off;
                    e->pins = 1;
                    map[key(br, lod)] = e;
                    t->entries.push_back(e);
                    to_launch.push_back(e);
                    stats.misses++;
                }
                t->admitted++;
            }
            waiting.pop_front();
            admitted_any = true;
        }
    }
    uint64_t n_bricks = 0;
    bool admitted_any = false;

    void launch() {
        while (!to_launch.empty()) {
            Batch *B = nullptr;
            for (size_t k = 0; k < batches.size(); k++) {
                Batch &c = batches[(next_batch + k) % batches.size()];
                if (!c.busy) {
                    B = &c;
                    next_batch = (uint32_t)((next_batch + k + 1) % batches.size());
                    break;
                }
            }
            if (!B) return;  // every stream busy: the rest joins later batches
            const uint32_t n = (uint32_t)std::min<size_t>(to_launch.size(), B->cap);
            B->entries.assign(to_launch.begin(), to_launch.begin() + n);
            to_launch.erase(to_launch.begin(), to_launch.begin() + n);
            for (uint32_t i = 0; i < n; i++) {
                B->ids_h[i] = B->entries[i]->brick;
                B->lods_h[i] = B->entries[i]->lod;
                B->offs_h[i] = B->entries[i]->off;
            }
            cudaError_t e = cudaMemcpyAsync(B->ids_d, B->ids_h, 4ull * n, cudaMemcpyHostToDevice, B->st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(B->lods_d, B->lods_h, n, cudaMemcpyHostToDevice, B->st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(B->offs_d, B->offs_h, 8ull * n, cudaMemcpyHostToDevice, B->st);
            int rc = e == cudaSuccess ? csgv_decode_bricks(vol, B->ids_d, B->lods_d, n, pool, B->offs_d, B->status_d, B->st)
                                      : CSGV_ERR_CUDA;
            if (rc == CSGV_OK) e = cudaMemcpyAsync(B->status_h, B->status_d, 4ull * n, cudaMemcpyDeviceToHost, B->st);
            if (rc == CSGV_OK && e == cudaSuccess) e = cudaEventRecord(B->ev, B->st);
            if (rc != CSGV_OK || e != cudaSuccess) {
                fatal = CSGV_ERR_CUDA;
                return;
            }
            B->busy = true;
            stats.batches++;
        }
    }

    bool complete() {
        bool any = false;
        for (Batch &B : batches) {
            if (!B.busy) continue;
            const cudaError_t q = cudaEventQuery(B.ev);
            if (q == cudaErrorNotReady) continue;
            if (q != cudaSuccess) {
                fatal = CSGV_ERR_CUDA;
                continue;
            }
            for (size_t i = 0; i < B.entries.size(); i++) {
                Entry *e = B.entries[i];
                e->status = B.status_h[i];
                e->ready = true;
                stats.decoded_labels += (uint64_t)(b >> e->lod) * (b >> e->lod) * (b >> e->lod);
            }
            B.entries.clear();
            B.busy = false;
            any = true;
        }
        if (any || admitted_any) {
            admitted_any = false;
            const auto now = Clock::now();
            for (auto &kv : tickets) {
                Ticket *t = kv.second;
                if (t->done || t->admitted < t->bricks.size()) continue;
                bool all = true;
                for (Entry *e : t->entries) all = all && e->ready;
                if (all) {
                    t->done = true;
                    t->t_done = now;
                    latencies_ms.push_back(std::chrono::duration<double, std::milli>(now - t->t_submit).count());
                    any = true;
                }
            }
        }
        return any;
    }

    void run() {
        cudaSetDevice(device);
        std::unique_lock<std::mutex> lk(mu);
        while (!stop) {
            admit();
            launch();
            const bool progressed = complete();
            if (progressed) cv_done.notify_all();
            bool in_flight = false;
            for (Batch &B : batches) in_flight = in_flight || B.busy;
            if (fatal) cv_done.notify_all();
            // short sleeps while batches run; wait for new work otherwise
            if (in_flight) cv_work.wait_for(lk, std::chrono::microseconds(20));
            else if (!progressed) cv_work.wait_for(lk, std::chrono::milliseconds(5));
        }
    }
};

extern "C" {

int csgv_serve_create(const csgv_volume *vol, const csgv_serve_config *cfg, csgv_server **out) {
    if (!vol || !out) return set_err(CSGV_ERR_INVALID_ARG, "NULL argument");
    csgv_volume_info inf;
    int rc = csgv_volume_info_get(vol, &inf);
    if (rc) return rc;
    const uint64_t cache_bytes = cfg && cfg->cache_bytes ? cfg->cache_bytes : (8ull << 30);
    const uint32_t max_batch = cfg && cfg->max_batch ? cfg->max_batch : 16384;
    const uint32_t n_streams = cfg && cfg->n_streams ? std::min<uint32_t>(cfg->n_streams, 16) : 3;
    csgv_server *s = new csgv_server();
    s->vol = vol;
    s->N = inf.N;
    s->b = 1u << inf.N;
    s->n_bricks = inf.n_bricks;
    cudaGetDevice(&s->device);
    s->pool_labels = cache_bytes / 4;
    s->max_batch = max_batch;
    if (cudaMalloc(&s->pool, s->pool_labels * 4) != cudaSuccess) {
        delete s;
        return set_err(CSGV_ERR_OOM, "cannot allocate the decoded-brick cache");
    }
    s->batches.resize(n_streams);
    for (Batch &B : s->batches) {
        B.cap = max_batch;
        cudaError_t e = cudaStreamCreateWithFlags(&B.st, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B.ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMalloc(&B.ids_d, 4ull * max_batch);
        if (e == cudaSuccess) e = cudaMalloc(&B.lods_d, (size_t)max_batch);
        if (e == cudaSuccess) e = cudaMalloc(&B.offs_d, 8ull * max_batch);
        if (e == cudaSuccess) e = cudaMalloc(&B.status_d, 4ull * max_batch);
        if (e == cudaSuccess) e = cudaMallocHost(&B.ids_h, 4ull * max_batch);
        if (e == cudaSuccess) e = cudaMallocHost(&B.lods_h, (size_t)max_batch);
        if (e == cudaSuccess) e = cudaMallocHost(&B.offs_h, 8ull * max_batch);
        if (e == cudaSuccess) e = cudaMallocHost(&B.status_h, 4ull * max_batch);
        if (e != cudaSuccess) {
            csgv_serve_destroy(s);
            return set_err(CSGV_ERR_OOM, "cannot allocate serve batch buffers");
        }
    }
    s->worker = std::thread([s] { s->run(); });
    *out = s;
    return CSGV_OK;
}

int csgv_serve_submit(csgv_server *s, const uint32_t *bricks_host, const uint8_t *lods_host, uint32_t n,
                      uint64_t *ticket) {
    if (!s || !ticket || (n && (!bricks_host || !lods_host))) return set_err(CSGV_ERR_INVALID_ARG, "NULL argument");
    Ticket *t = new Ticket();
    t->bricks.assign(bricks_host, bricks_host + n);
    t->lods.assign(lods_host, lods_host + n);
    t->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->fatal) {
            delete t;
            return set_err(s->fatal, "server stopped after a CUDA error");
        }
        t->id = s->next_ticket++;
        s->tickets[t->id] = t;
        s->waiting.push_back(t);
        s->stats.submitted++;
    }
    s->cv_work.notify_one();
    *ticket = t->id;
    return CSGV_OK;
}

int csgv_serve_poll(csgv_server *s, uint64_t ticket, uint32_t timeout_us, csgv_result *results) {
    if (!s) return set_err(CSGV_ERR_INVALID_ARG, "NULL server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return set_err(CSGV_ERR_INVALID_ARG, "unknown ticket");
    Ticket *t = it->second;
    const auto deadline = Clock::now() + std::chrono::microseconds(timeout_us);
    while (!t->done && !s->fatal) {
        if (timeout_us == 0) return CSGV_PENDING;
        if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && !t->done)
            return t->done ? CSGV_OK : CSGV_ERR_TIMEOUT;
    }
    if (!t->done) return set_err(s->fatal ? s->fatal : CSGV_ERR_CUDA, "server stopped after a CUDA error");
    if (results)
        for (size_t i = 0; i < t->entries.size(); i++) {
            Entry *e = t->entries[i];
            results[i].labels_dev = e->status == CSGV_OK ? s->pool + e->off : nullptr;
            results[i].status = e->status;
            results[i].lod = e->lod;
            results[i].brick = e->brick;
        }
    return CSGV_OK;
}

int csgv_serve_release(csgv_server *s, uint64_t ticket) {
    if (!s) return set_err(CSGV_ERR_INVALID_ARG, "NULL server");
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->tickets.find(ticket);
        if (it == s->tickets.end()) return set_err(CSGV_ERR_INVALID_ARG, "unknown ticket");
        Ticket *t = it->second;
        if (!t->done) return set_err(CSGV_ERR_INVALID_ARG, "ticket not finished: poll it until CSGV_OK first");
        for (Entry *e : t->entries) {
            if (e->transient) delete e;
            else s->unpin(e);
        }
        s->tickets.erase(it);
        delete t;
    }
    s->cv_work.notify_one();  // released space may admit waiting requests
    return CSGV_OK;
}

int csgv_serve_stats_get(csgv_server *s, csgv_serve_stats *out, double *latency_ms_host, uint32_t max_latencies,
                         uint32_t *n_latencies) {
    if (!s || !out) return set_err(CSGV_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->stats;
    out->cache_labels_used = s->top;
    out->cache_entries = s->map.size();
    uint32_t k = 0;
    if (latency_ms_host)
        for (; k < max_latencies && k < s->latencies_ms.size(); k++) latency_ms_host[k] = s->latencies_ms[k];
    if (n_latencies) *n_latencies = (uint32_t)s->latencies_ms.size();
    return CSGV_OK;
}

void csgv_serve_destroy(csgv_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    cudaSetDevice(s->device);
    for (Batch &B : s->batches) {
        if (B.st) cudaStreamSynchronize(B.st);
        if (B.ev) cudaEventDestroy(B.ev);
        if (B.st) cudaStreamDestroy(B.st);
        cudaFree(B.ids_d); cudaFree(B.lods_d); cudaFree(B.offs_d); cudaFree(B.status_d);
        cudaFreeHost(B.ids_h); cudaFreeHost(B.lods_h); cudaFreeHost(B.offs_h); cudaFreeHost(B.status_h);
    }
    for (auto &kv : s->map) delete kv.second;
    for (auto &kv : s->tickets) {
        for (Entry *e : kv.second->entries)
            if (e->transient) delete e;
        delete kv.second;
    }
    cudaFree(s->pool);
    delete s;
}

}  // extern "C"
