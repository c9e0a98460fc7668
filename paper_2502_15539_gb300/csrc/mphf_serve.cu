// Serving loop: continuous batching of query requests over resident MPHFs.
//
// Memory.  The HBM budget is one device arena, allocated once; a structure's
// pilots and remap table occupy one range of it while the structure is
// resident.  Structures are registered as serialized bytes kept in
// page-locked host memory.  Admitting one takes a free range (first fit)
// and queues its copy on a dedicated copy stream; evicting one returns its
// range.  Nothing on the serving path allocates or frees device memory, so
// nothing synchronizes the device.
//
// Admission is first come, first served: the oldest queued request whose
// structure is absent decides what is loaded next.  If its structure does not
// fit, resident structures are chosen least-recently-used and marked
// draining: their requests that arrived before the blocked one still run,
// later ones wait, and as soon as a draining structure is idle its range is
// freed.  So a large structure cannot starve behind busy small ones.
//
// Batching.  A dispatcher thread fills free slots; each slot owns a stream
// and a persistent batch executor.  A slot takes queued requests of loaded
// or loading structures in arrival order, up to a request and key budget,
// waits on the GPU for the copies of any structure still loading, and
// launches one batch.  Requests that arrive while batches run join the next
// free slot, so several batches overlap on the device.  Completion is
// observed through events; latency runs from a request's arrival time to
// that observation.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "mphf_internal.cuh"

using Clock = std::chrono::steady_clock;

namespace ptrhash {
int serialized_device_bytes(const void *blob, size_t len, uint64_t *bytes, uint64_t *n);
int handle_in_arena(const void *blob, size_t len, uint8_t *dev, cudaStream_t s, mphf_t **out);
}  // namespace ptrhash

namespace {

enum State { kAbsent, kLoading, kResident };

struct Entry {
    uint8_t *blob = nullptr;     // page-locked host copy (serialized)
    size_t len = 0;
    uint64_t dev_bytes = 0;      // arena bytes while resident
    State state = kAbsent;
    mphf_t *m = nullptr;         // handle into the arena
    uint64_t offset = 0;         // arena offset
    cudaEvent_t ready = nullptr; // end of the copy into the arena
    uint64_t last_use = 0;
    uint32_t queued = 0, inflight = 0;
    bool removed = false, draining = false;
};

struct Req {
    uint64_t ticket;
    uint32_t sid;
    const void *keys;
    const uint64_t *offsets;
    uint64_t count;
    uint32_t *out;
    Clock::time_point arrival;
};

struct Slot {
    cudaStream_t stream = nullptr;
    mphf_batch_t *batch = nullptr;
    cudaEvent_t done = nullptr;
    std::vector<Req> reqs;
    bool busy = false;
};

// First-fit range allocator over [0, cap).
struct Arena {
    uint8_t *base = nullptr;
    uint64_t cap = 0;
    std::map<uint64_t, uint64_t> free;   // offset -> size
    bool take(uint64_t bytes, uint64_t *off) {
        for (auto it = free.begin(); it != free.end(); ++it) {
            if (it->second < bytes) continue;
            *off = it->first;
            const uint64_t rest = it->second - bytes, at = it->first + bytes;
            free.erase(it);
            if (rest) free[at] = rest;
            return true;
        }
        return false;
    }
    void give(uint64_t off, uint64_t bytes) {
        auto it = free.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free.erase(nx);
        }
        if (it != free.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free.erase(it);
            }
        }
    }
};

}  // namespace

struct mphf_server {
    mphf_server_config cfg;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::vector<Entry> entries;
    std::deque<Req> queue;
    std::vector<Slot> slots;
    Arena arena;
    cudaStream_t copy_stream = nullptr;
    std::unordered_map<uint64_t, int> finished;   // ticket -> status
    std::vector<double> lat_us;
    uint64_t next_ticket = 1, use_clock = 0, resident_bytes = 0;
    uint64_t done_queries = 0, done_requests = 0, batches = 0, batch_requests = 0, evictions = 0, admissions = 0;
    uint64_t block_ticket = 0;                    // oldest request waiting for its structure (0: none)
    Clock::time_point t_first{}, t_last{};
    bool have_first = false;
    int error = MPHF_OK;
    bool stop = false;
    std::atomic<uint64_t> nudges{0};              // bumped with every cv_work notification
    std::thread dispatcher;
};

static void evict_locked(mphf_server *s, Entry &v) {
    mphf_free(v.m);   // non-owning handle: releases only the host object
    v.m = nullptr;
    s->arena.give(v.offset, v.dev_bytes);
    s->resident_bytes -= v.dev_bytes;
    v.state = kAbsent;
    v.draining = false;
    s->evictions++;
}

static bool has_old_request(const mphf_server *s, uint32_t sid, uint64_t ticket) {
    for (const Req &r : s->queue) {
        if (r.ticket > ticket) break;
        if (r.sid == sid) return true;
    }
    return false;
}

// First come, first served admission (see the file comment).
static void admit_locked(mphf_server *s) {
    for (;;) {
        const Req *oldest = nullptr;
        for (const Req &r : s->queue)
            if (s->entries[r.sid].state == kAbsent) { oldest = &r; break; }
        if (!oldest) { s->block_ticket = 0; return; }
        const uint32_t sid = oldest->sid;
        const uint64_t ticket = oldest->ticket;
        Entry &e = s->entries[sid];
        uint64_t off = 0;
        bool fits = s->arena.take(e.dev_bytes, &off);
        if (!fits) {
            // Mark least-recently-used residents as draining until they would
            // make room, then evict the ones that are already idle.
            uint64_t room = s->arena.cap - s->resident_bytes;
            std::vector<uint32_t> order;
            for (uint32_t j = 0; j < s->entries.size(); j++)
                if (s->entries[j].state != kAbsent) order.push_back(j);
            std::sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) {
                return s->entries[a].last_use < s->entries[b].last_use;
            });
            for (uint32_t j : order) {
                if (room >= e.dev_bytes) break;
                s->entries[j].draining = true;
                room += s->entries[j].dev_bytes;
            }
            for (uint32_t j : order) {
                Entry &v = s->entries[j];
                if (v.draining && v.inflight == 0 && !has_old_request(s, j, ticket)) evict_locked(s, v);
            }
            fits = s->arena.take(e.dev_bytes, &off);
            if (!fits) {
                // Fragmentation: free every idle resident, oldest use first.
                for (uint32_t j : order) {
                    Entry &v = s->entries[j];
                    if (v.state != kAbsent && v.inflight == 0 && !has_old_request(s, j, ticket)) {
                        evict_locked(s, v);
                        if ((fits = s->arena.take(e.dev_bytes, &off))) break;
                    }
                }
            }
        }
        if (!fits) { s->block_ticket = ticket; return; }   // wait for draining structures
        mphf_t *m = nullptr;
        int rc = ptrhash::handle_in_arena(e.blob, e.len, s->arena.base + off, s->copy_stream, &m);
        if (rc == MPHF_OK && cudaEventRecord(e.ready, s->copy_stream) != cudaSuccess) rc = MPHF_ERR_CUDA;
        if (rc) {
            s->arena.give(off, e.dev_bytes);
            s->error = rc;
            // Fail every queued request of this structure rather than spin.
            for (auto it = s->queue.begin(); it != s->queue.end();) {
                if (it->sid == sid) {
                    s->finished[it->ticket] = rc;
                    e.queued--;
                    it = s->queue.erase(it);
                } else {
                    ++it;
                }
            }
            s->cv_done.notify_all();
            continue;
        }
        e.m = m;
        e.offset = off;
        e.state = kLoading;
        s->resident_bytes += e.dev_bytes;
        s->admissions++;
        for (Entry &x : s->entries) x.draining = false;
        s->block_ticket = 0;
    }
}

// Returns whether a batch finished.
static bool complete_locked(mphf_server *s) {
    bool any = false;
    for (Entry &e : s->entries)
        if (e.state == kLoading && cudaEventQuery(e.ready) == cudaSuccess) e.state = kResident;
    for (Slot &sl : s->slots) {
        if (!sl.busy) continue;
        cudaError_t q = cudaEventQuery(sl.done);
        if (q == cudaErrorNotReady) continue;
        const int status = q == cudaSuccess ? MPHF_OK : MPHF_ERR_CUDA;
        if (q != cudaSuccess) s->error = MPHF_ERR_CUDA;
        const Clock::time_point now = Clock::now();
        for (const Req &r : sl.reqs) {
            s->finished[r.ticket] = status;
            s->lat_us.push_back(std::chrono::duration<double, std::micro>(now - r.arrival).count());
            s->done_queries += r.count;
            s->done_requests++;
            s->entries[r.sid].inflight--;
            if (!s->have_first || r.arrival < s->t_first) { s->t_first = r.arrival; s->have_first = true; }
        }
        s->t_last = now;
        sl.reqs.clear();
        sl.busy = false;
        any = true;
        s->cv_done.notify_all();
    }
    return any;
}

static bool dispatchable(const mphf_server *s, const Req &r) {
    const Entry &e = s->entries[r.sid];
    if (e.state == kAbsent) return false;
    if (e.draining && s->block_ticket && r.ticket > s->block_ticket) return false;
    return true;
}

// How long the dispatcher keeps polling after its last activity before it
// blocks on the condition variable.  Polling costs one host core while the
// server is busy; blocking adds a thread wake-up to the next request.
constexpr std::chrono::microseconds kPollWindow(200);

static void dispatcher_main(mphf_server *s) {
    cudaSetDevice(s->device);
    std::vector<mphf_request> creq;
    std::vector<uint32_t> waits;
    std::vector<cudaEvent_t> pending;
    // Activity: a batch launched or finished, or a request arrived.  Queued
    // requests alone are not activity: one that cannot be dispatched (its
    // structure waits for room) must not keep the dispatcher polling.
    Clock::time_point last_activity = Clock::now();
    uint64_t nudges_seen = s->nudges.load(std::memory_order_acquire);
    std::unique_lock<std::mutex> lock(s->mu);
    for (;;) {
        const bool any_busy = std::any_of(s->slots.begin(), s->slots.end(), [](const Slot &x) { return x.busy; });
        if (s->stop && s->queue.empty() && !any_busy) break;
        if (complete_locked(s)) last_activity = Clock::now();
        admit_locked(s);
        bool launched = false;
        for (Slot &sl : s->slots) {
            if (sl.busy || s->queue.empty()) continue;
            uint64_t keys = 0;
            for (auto it = s->queue.begin(); it != s->queue.end() && sl.reqs.size() < s->cfg.max_batch_requests;) {
                if (!dispatchable(s, *it) || (keys && keys + it->count > s->cfg.max_batch_keys)) { ++it; continue; }
                Entry &e = s->entries[it->sid];
                keys += it->count;
                e.queued--;
                e.inflight++;
                e.last_use = ++s->use_clock;
                sl.reqs.push_back(*it);
                it = s->queue.erase(it);
            }
            if (sl.reqs.empty()) break;
            creq.resize(sl.reqs.size());
            waits.clear();
            for (size_t i = 0; i < sl.reqs.size(); i++) {
                const Req &r = sl.reqs[i];
                const Entry &e = s->entries[r.sid];
                creq[i] = mphf_request{e.m, r.keys, r.offsets, r.count, r.out};
                if (e.state == kLoading && std::find(waits.begin(), waits.end(), r.sid) == waits.end()) waits.push_back(r.sid);
            }
            int rc = MPHF_OK;
            for (uint32_t sid : waits)
                if (cudaStreamWaitEvent(sl.stream, s->entries[sid].ready, 0) != cudaSuccess) rc = MPHF_ERR_CUDA;
            if (rc == MPHF_OK) rc = mphf_batch_run(sl.batch, creq.data(), (uint32_t)creq.size(), sl.stream);
            if (rc == MPHF_OK && cudaEventRecord(sl.done, sl.stream) != cudaSuccess) rc = MPHF_ERR_CUDA;
            if (rc) {
                s->error = rc;
                for (const Req &r : sl.reqs) {
                    s->finished[r.ticket] = rc;
                    s->entries[r.sid].inflight--;
                }
                sl.reqs.clear();
                s->cv_done.notify_all();
                continue;
            }
            sl.busy = true;
            s->batches++;
            s->batch_requests += creq.size();
            launched = true;
        }
        if (launched) {
            last_activity = Clock::now();
            continue;
        }
        // Nothing more can start now.  Poll for a finished batch or a new
        // request without holding the lock (holding it between polls starves
        // the threads that submit), then take it again to act on either.
        pending.clear();
        for (const Slot &sl : s->slots)
            if (sl.busy) pending.push_back(sl.done);
        Clock::time_point now = Clock::now();
        const uint64_t seen = s->nudges.load(std::memory_order_acquire);
        if (!pending.empty() || seen != nudges_seen) last_activity = now;   // batches in flight, or a new request
        nudges_seen = seen;
        if (now - last_activity < kPollWindow) {
            // With every slot busy a new request cannot start anyway; waking
            // for each one would only contend with a burst of submitters.
            const bool slot_free = pending.size() < s->slots.size();
            lock.unlock();
            for (;;) {
                bool finished = false;
                for (cudaEvent_t ev : pending)
                    if (cudaEventQuery(ev) != cudaErrorNotReady) { finished = true; break; }
                if (finished || (slot_free && s->nudges.load(std::memory_order_acquire) != seen)) break;
                if (pending.empty() && Clock::now() - last_activity >= kPollWindow) break;
                std::this_thread::yield();
            }
            lock.lock();
        } else if (!s->stop) {
            s->cv_work.wait_for(lock, std::chrono::milliseconds(2));   // a queued request restarts the polling
        }
    }
}

static void destroy_server(mphf_server *s) {
    for (Slot &sl : s->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        mphf_batch_free(sl.batch);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.stream) cudaStreamDestroy(sl.stream);
    }
    if (s->copy_stream) {
        cudaStreamSynchronize(s->copy_stream);
        cudaStreamDestroy(s->copy_stream);
    }
    for (Entry &e : s->entries) {
        mphf_free(e.m);
        if (e.ready) cudaEventDestroy(e.ready);
        cudaFreeHost(e.blob);
    }
    cudaFree(s->arena.base);
    delete s;
}

extern "C" {

int mphf_server_default_config(mphf_server_config *c) {
    if (!c) { ptrhash::set_error("NULL config"); return MPHF_ERR_ARG; }
    c->hbm_budget_bytes = 4ull << 30;
    c->max_batch_requests = 1024;
    c->max_batch_keys = 1ull << 24;
    c->slots = 4;
    return MPHF_OK;
}

int mphf_server_create(const mphf_server_config *cfg, mphf_server_t **out) {
    if (!out || !cfg) { ptrhash::set_error("NULL argument"); return MPHF_ERR_ARG; }
    *out = nullptr;
    if (cfg->slots < 1 || cfg->slots > 16 || cfg->max_batch_requests < 1 || cfg->max_batch_requests > 4096 ||
        cfg->max_batch_keys < 1 || cfg->hbm_budget_bytes < 256) {
        ptrhash::set_error("slots in [1,16], max_batch_requests in [1,4096], max_batch_keys >= 1, budget >= 256");
        return MPHF_ERR_ARG;
    }
    mphf_server *s = new (std::nothrow) mphf_server();
    if (!s) { ptrhash::set_error("host allocation"); return MPHF_ERR_OOM; }
    s->cfg = *cfg;
    cudaGetDevice(&s->device);
    s->arena.cap = cfg->hbm_budget_bytes & ~255ull;
    cudaError_t e = cudaMalloc(&s->arena.base, s->arena.cap);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        int rc = ptrhash::cuda_fail(e, "server arena");
        destroy_server(s);
        return rc;
    }
    s->arena.free[0] = s->arena.cap;
    s->slots.resize(cfg->slots);
    for (Slot &sl : s->slots) {
        e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
        int rc = e == cudaSuccess ? mphf_batch_create(cfg->max_batch_requests, &sl.batch) : ptrhash::cuda_fail(e, "server slot");
        if (rc) {
            destroy_server(s);
            return rc;
        }
    }
    s->dispatcher = std::thread(dispatcher_main, s);
    *out = s;
    return MPHF_OK;
}

void mphf_server_free(mphf_server_t *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
    }
    s->nudges.fetch_add(1, std::memory_order_release);
    s->cv_work.notify_all();
    if (s->dispatcher.joinable()) s->dispatcher.join();
    destroy_server(s);
}

int mphf_server_add(mphf_server_t *s, const void *serialized, size_t len, uint32_t *id) {
    if (!s || !serialized || !id) { ptrhash::set_error("NULL argument"); return MPHF_ERR_ARG; }
    Entry e;
    uint64_t n = 0;
    int rc = ptrhash::serialized_device_bytes(serialized, len, &e.dev_bytes, &n);
    if (rc) return rc;
    if (ptrhash::wide_values(n) || ((const uint8_t *)serialized)[28] & 1u) {
        ptrhash::set_error("n > 2^32 or a 128-bit string hash: not served (32-bit batched queries)");
        return MPHF_ERR_ARG;
    }
    if (e.dev_bytes > s->arena.cap) {
        ptrhash::set_error("structure of %llu bytes exceeds the HBM budget", (unsigned long long)e.dev_bytes);
        return MPHF_ERR_CAPACITY;
    }
    cudaError_t ce = cudaHostAlloc(&e.blob, len, cudaHostAllocDefault);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&e.ready, cudaEventDisableTiming);
    if (ce != cudaSuccess) {
        cudaFreeHost(e.blob);
        return ptrhash::cuda_fail(ce, "server add");
    }
    memcpy(e.blob, serialized, len);
    e.len = len;
    std::lock_guard<std::mutex> lock(s->mu);
    *id = (uint32_t)s->entries.size();
    s->entries.push_back(e);
    return MPHF_OK;
}

int mphf_server_remove(mphf_server_t *s, uint32_t id) {
    if (!s) { ptrhash::set_error("NULL server"); return MPHF_ERR_ARG; }
    std::unique_lock<std::mutex> lock(s->mu);
    if (id >= s->entries.size() || s->entries[id].removed) { ptrhash::set_error("unknown structure id"); return MPHF_ERR_ARG; }
    s->entries[id].removed = true;
    s->nudges.fetch_add(1, std::memory_order_release);
    s->cv_work.notify_all();
    s->cv_done.wait(lock, [&] { return s->entries[id].queued == 0 && s->entries[id].inflight == 0; });
    Entry &e = s->entries[id];
    if (e.state != kAbsent) {
        cudaEventSynchronize(e.ready);
        evict_locked(s, e);
        s->evictions--;   // a removal is not an eviction
    }
    return MPHF_OK;
}

static int submit_locked(mphf_server *s, const mphf_server_req &r, Clock::time_point arrival, uint64_t *ticket) {
    if (r.structure >= s->entries.size() || s->entries[r.structure].removed) {
        ptrhash::set_error("unknown structure id %u", r.structure);
        return MPHF_ERR_ARG;
    }
    if (r.count && (!r.keys_dev || !r.out_dev)) { ptrhash::set_error("NULL keys or out"); return MPHF_ERR_ARG; }
    Entry &e = s->entries[r.structure];
    Req q{s->next_ticket++, r.structure, r.keys_dev, r.offsets_dev, r.count, r.out_dev, arrival};
    e.queued++;
    s->queue.push_back(q);
    *ticket = q.ticket;
    s->nudges.fetch_add(1, std::memory_order_release);
    return MPHF_OK;
}

int mphf_server_submit(mphf_server_t *s, const mphf_server_req *r, uint64_t *ticket) {
    if (!s || !r || !ticket) { ptrhash::set_error("NULL argument"); return MPHF_ERR_ARG; }
    int rc;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        rc = submit_locked(s, *r, Clock::now(), ticket);
    }
    s->cv_work.notify_one();
    return rc;
}

int mphf_server_replay(mphf_server_t *s, const mphf_server_req *reqs, const double *arrival_us, uint32_t n,
                       uint64_t *tickets) {
    if (!s || (n && (!reqs || !arrival_us || !tickets))) { ptrhash::set_error("NULL argument"); return MPHF_ERR_ARG; }
    const Clock::time_point t0 = Clock::now();
    for (uint32_t i = 0; i < n; i++) {
        const Clock::time_point due = t0 + std::chrono::nanoseconds((int64_t)(arrival_us[i] * 1000.0));
        while (Clock::now() < due) {}
        int rc;
        {
            std::lock_guard<std::mutex> lock(s->mu);
            rc = submit_locked(s, reqs[i], due, &tickets[i]);
        }
        s->cv_work.notify_one();
        if (rc) return rc;
    }
    return MPHF_OK;
}

int mphf_server_wait(mphf_server_t *s, uint64_t ticket, uint64_t timeout_us, int *status) {
    if (!s) { ptrhash::set_error("NULL server"); return MPHF_ERR_ARG; }
    std::unique_lock<std::mutex> lock(s->mu);
    const bool ok = s->cv_done.wait_for(lock, std::chrono::microseconds(timeout_us),
                                        [&] { return s->finished.count(ticket) != 0; });
    if (!ok) {
        ptrhash::set_error("ticket %llu not done after %llu us", (unsigned long long)ticket, (unsigned long long)timeout_us);
        return MPHF_ERR_TIMEOUT;
    }
    if (status) *status = s->finished[ticket];
    return MPHF_OK;
}

int mphf_server_drain(mphf_server_t *s, uint64_t timeout_us) {
    if (!s) { ptrhash::set_error("NULL server"); return MPHF_ERR_ARG; }
    std::unique_lock<std::mutex> lock(s->mu);
    const bool ok = s->cv_done.wait_for(lock, std::chrono::microseconds(timeout_us), [&] {
        return s->queue.empty() && std::none_of(s->slots.begin(), s->slots.end(), [](const Slot &x) { return x.busy; });
    });
    if (!ok) {
        ptrhash::set_error("requests still pending after %llu us", (unsigned long long)timeout_us);
        return MPHF_ERR_TIMEOUT;
    }
    return s->error;
}

int mphf_server_stats(mphf_server_t *s, int reset, mphf_server_stats_t *out) {
    if (!s || !out) { ptrhash::set_error("NULL argument"); return MPHF_ERR_ARG; }
    std::lock_guard<std::mutex> lock(s->mu);
    memset(out, 0, sizeof(*out));
    std::vector<double> v = s->lat_us;
    if (!v.empty()) {
        std::sort(v.begin(), v.end());
        auto pct = [&](double p) { return v[std::min(v.size() - 1, (size_t)(p * (v.size() - 1) + 0.5))]; };
        out->p50_us = pct(0.50);
        out->p99_us = pct(0.99);
        out->max_us = v.back();
        double sum = 0;
        for (double x : v) sum += x;
        out->mean_us = sum / v.size();
    }
    out->requests = s->done_requests;
    out->queries = s->done_queries;
    out->batches = s->batches;
    out->mean_requests_per_batch = s->batches ? (double)s->batch_requests / s->batches : 0.0;
    out->admissions = s->admissions;
    out->evictions = s->evictions;
    out->resident_bytes = s->resident_bytes;
    const double span = s->have_first ? std::chrono::duration<double>(s->t_last - s->t_first).count() : 0.0;
    out->queries_per_s = span > 0 ? s->done_queries / span : 0.0;
    if (reset) {
        s->lat_us.clear();
        s->done_queries = s->done_requests = s->batches = s->batch_requests = 0;
        s->admissions = s->evictions = 0;
        s->have_first = false;
        s->finished.clear();
    }
    return MPHF_OK;
}

}  // extern "C"
