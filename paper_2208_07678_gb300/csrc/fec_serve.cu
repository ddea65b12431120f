// fec_serve.cu -- request loop with continuous batching.
//
// Requests (clouds of any size, each with its own d and size bounds) are
// copied into pinned staging at submit time and queued.  A fixed set of
// worker slots, each with its own CUDA stream and device workspace, takes
// requests as they arrive: a request is admitted when a slot is free and the
// sum of the workspace estimates of running requests stays within the memory
// budget, so requests that arrive while others run start as soon as slots and
// memory free up, and their work overlaps on the device.  Each request runs
// the same one-cloud pipeline as fec_cluster on its slot's stream, so its
// labels equal fec_cluster on that request alone (the result is unique).
//
// Latency of a request = submit -> completion (labels and count in host
// memory); poll only observes it.
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "fec_internal.cuh"
#include "fec_serve.h"

namespace fec {

namespace {

constexpr int kSlots = 4;
constexpr size_t kDefaultBudget = (size_t)40 << 30;  // 40 GiB when the context has none

struct Request {
    uint64_t ticket = 0;
    float *xyz = nullptr;   // pinned copy of the input (from the engine's pool)
    size_t xyz_cap = 0;
    int64_t n = 0;
    float d = 0;
    int64_t min_size = 0, max_size = 0;
    int32_t *labels_out = nullptr;
    size_t est = 0;         // workspace estimate (bytes)
    fec_status status = FEC_ERR_NOT_READY;
    int32_t k = 0;
    bool done = false;
};

}  // namespace

// Pinned host buffers reused across requests: allocating and freeing pinned
// memory per request would serialise the device (freeing pinned memory
// synchronises it).  Buffers come in power-of-two size classes.
struct PinnedPool {
    std::vector<std::pair<size_t, void *>> free_list;  // (capacity, pointer)
    size_t held = 0;

    void *get(size_t bytes, size_t &cap)
    {
        size_t c = 4096;
        while (c < bytes) c <<= 1;
        for (size_t i = 0; i < free_list.size(); ++i)
            if (free_list[i].first == c) {
                void *p = free_list[i].second;
                free_list.erase(free_list.begin() + i);
                cap = c;
                return p;
            }
        void *p = nullptr;
        if (cudaMallocHost(&p, c) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        held += c;
        cap = c;
        return p;
    }
    void put(void *p, size_t cap) { free_list.emplace_back(cap, p); }
    void release_all()
    {
        for (auto &e : free_list) cudaFreeHost(e.second);
        free_list.clear();
    }
};

struct ServeEngine {
    fec_ctx *owner = nullptr;
    PinnedPool pool;
    int device = 0;
    size_t budget = 0;
    size_t in_flight = 0;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> queue;
    std::unordered_map<uint64_t, Request *> all;
    std::vector<std::thread> workers;
    std::vector<fec_ctx *> slots;
    bool started = false;

    void start();
    void worker(int slot);
};

void ServeEngine::start()
{
    // called with mu held
    if (started) return;
    started = true;
    for (int i = 0; i < kSlots; ++i) {
        fec_options o{};
        o.device = device;
        o.mem_budget_bytes = 0;
        fec_ctx *c = nullptr;
        if (fec_create(&o, &c) != FEC_OK) break;
        slots.push_back(c);
    }
    for (size_t i = 0; i < slots.size(); ++i) workers.emplace_back(&ServeEngine::worker, this, (int)i);
}

void ServeEngine::worker(int slot)
{
    cudaSetDevice(device);
    fec_ctx *ctx = slots[slot];
    for (;;) {
        Request *r = nullptr;
        {
            std::unique_lock<std::mutex> lk(mu);
            cv_work.wait(lk, [&] {
                if (stop) return true;
                // admit the oldest request that fits the memory budget
                for (Request *q : queue)
                    if (in_flight + q->est <= budget) return true;
                return false;
            });
            if (stop && queue.empty()) return;
            for (auto it = queue.begin(); it != queue.end(); ++it)
                if (in_flight + (*it)->est <= budget) {
                    r = *it;
                    queue.erase(it);
                    break;
                }
            if (!r) continue;
            in_flight += r->est;
        }
        int32_t k = 0;
        fec_status s = fec_cluster(ctx, r->xyz, r->n, r->d, r->min_size, r->max_size,
                                   r->labels_out, &k);
        {
            std::lock_guard<std::mutex> lk(mu);
            in_flight -= r->est;
            r->status = s;
            r->k = k;
            r->done = true;
            if (r->xyz) pool.put(r->xyz, r->xyz_cap);
            r->xyz = nullptr;
        }
        cv_done.notify_all();
        cv_work.notify_all();
    }
}

ServeEngine *serve_create(fec_ctx *owner, const char *)
{
    ServeEngine *e = new ServeEngine();
    e->owner = owner;
    cudaGetDevice(&e->device);
    return e;
}

void serve_destroy(ServeEngine *e)
{
    if (!e) return;
    {
        std::lock_guard<std::mutex> lk(e->mu);
        e->stop = true;
    }
    e->cv_work.notify_all();
    for (auto &t : e->workers) t.join();
    for (auto &kv : e->all) {
        if (kv.second->xyz) e->pool.put(kv.second->xyz, kv.second->xyz_cap);
        delete kv.second;
    }
    for (fec_ctx *c : e->slots) fec_destroy(c);
    e->pool.release_all();
    delete e;
}

}  // namespace fec

using namespace fec;

// The owning context's budget and serving engine are reached through these
// accessors (fec_ctx is defined in fec_api.cu).
namespace fec {
size_t ctx_budget(const fec_ctx *ctx);
ServeEngine *ctx_serve(fec_ctx *ctx);
}  // namespace fec

extern "C" {

fec_status fec_serve_submit(fec_ctx *ctx, const float *xyz, int64_t n, float d, int64_t min_size,
                            int64_t max_size, int32_t *labels_out, uint64_t *ticket)
{
    if (!ctx || !ticket) return FEC_ERR_INVALID_ARG;
    if (n < 0 || n > FEC_MAX_POINTS || !(d > 0.0f) || !std::isfinite(d) || min_size < 0 ||
        max_size < min_size)
        return FEC_ERR_INVALID_ARG;
    if (n > 0 && (!xyz || !labels_out)) return FEC_ERR_INVALID_ARG;
    ServeEngine *e = ctx_serve(ctx);
    if (!e) return FEC_ERR_INVALID_ARG;
    Request *r = new Request();
    r->n = n;
    r->d = d;
    r->min_size = min_size;
    r->max_size = max_size;
    r->labels_out = labels_out;
    r->est = (size_t)fec_workspace_bytes(n, d);
    {
        std::lock_guard<std::mutex> lk(e->mu);
        if (!e->budget) {
            const size_t b = ctx_budget(ctx);
            e->budget = b ? b : kDefaultBudget;
        }
    }
    if (r->est > e->budget) {
        delete r;
        return FEC_ERR_BUSY;
    }
    if (n > 0) {
        {
            std::lock_guard<std::mutex> lk(e->mu);
            r->xyz = (float *)e->pool.get((size_t)n * 12, r->xyz_cap);
        }
        if (!r->xyz) {
            delete r;
            return FEC_ERR_OOM;
        }
        std::memcpy(r->xyz, xyz, (size_t)n * 12);
    }
    {
        std::lock_guard<std::mutex> lk(e->mu);
        e->start();
        r->ticket = e->next_ticket++;
        e->all[r->ticket] = r;
        e->queue.push_back(r);
        *ticket = r->ticket;
    }
    e->cv_work.notify_one();
    return FEC_OK;
}

fec_status fec_serve_poll(fec_ctx *ctx, uint64_t ticket, int32_t *num_clusters, int timeout_ms)
{
    if (!ctx) return FEC_ERR_INVALID_ARG;
    ServeEngine *e = ctx_serve(ctx);
    if (!e) return FEC_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(e->mu);
    auto it = e->all.find(ticket);
    if (it == e->all.end()) return FEC_ERR_INVALID_ARG;
    Request *r = it->second;
    if (!r->done) {
        if (timeout_ms == 0) return FEC_ERR_NOT_READY;
        if (timeout_ms < 0) {
            e->cv_done.wait(lk, [&] { return r->done; });
        } else if (!e->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms),
                                        [&] { return r->done; })) {
            return FEC_ERR_TIMEOUT;
        }
    }
    const fec_status s = r->status;
    if (num_clusters) *num_clusters = r->k;
    e->all.erase(it);
    delete r;
    return s;
}

}  // extern "C"
