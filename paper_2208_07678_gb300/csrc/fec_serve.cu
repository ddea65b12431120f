// fec_serve.cu -- request loop with continuous batching.
//
// Requests (clouds of any size, each with its own d and size bounds) are
// copied to device memory at submit time, on the engine's copy stream, into
// a region of the engine's input arena (one device allocation made when the
// engine starts; regions are handed out first-fit on the host, so no submit
// allocates device memory), and queued.  A fixed set of worker slots, each
// with its own CUDA stream and device workspace, takes requests as they
// arrive: a request is admitted when a slot is free and the memory budget
// allows (below), so requests that arrive while others run start as soon as
// slots and memory free up, and their work overlaps on the device.  Each
// request runs the same one-cloud pipeline as fec_cluster on its slot's
// stream, so its labels equal fec_cluster on that request alone (the result
// is unique).
//
// Memory: the arena takes a quarter of the budget (at most 2 GiB); the slots'
// workspaces share the rest.  A slot keeps its workspace between requests
// (grown as larger requests reach it), and a request is admitted on a free
// slot only when the workspaces of all slots, with that slot's grown to what
// the request needs, stay within the share; an idle slot whose workspace
// keeps a queued request from fitting releases it.  So the engine never holds
// more device memory than the budget.  A request whose workspace estimate
// exceeds the slots' share, or whose input does not fit the arena's free
// space, or that finds the queue full, is refused at submit with
// FEC_ERR_BUSY.  A request submitted with a deadline that has not started by
// then completes with FEC_ERR_TIMEOUT without running.
//
// Latency of a request = submit -> completion (labels and count in host
// memory); poll only observes it.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <ctime>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "fec_internal.cuh"
#include "fec_serve.h"

namespace fec {

// fec_api.cu
cudaStream_t ctx_stream(const fec_ctx *ctx);
int ctx_sms(const fec_ctx *ctx);
size_t ctx_ws_bytes(const fec_ctx *ctx);
size_t ctx_projected_bytes(const fec_ctx *ctx, size_t n, float d, size_t budget);
void ctx_set_budget(fec_ctx *ctx, size_t budget);
void ctx_release_workspace(fec_ctx *ctx);
fec_status ctx_grow(fec_ctx *ctx, size_t n, float d);

namespace {

constexpr int kSlots = 4;
constexpr size_t kDefaultBudget = (size_t)40 << 30;  // 40 GiB when the context has none
constexpr size_t kMaxQueued = 4096;                   // requests waiting for a slot
constexpr size_t kArenaMax = (size_t)2 << 30;
constexpr size_t kGranule = 256;                      // arena regions start 256-byte aligned

int64_t now_ns()
{
    timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (int64_t)ts.tv_sec * 1000000000LL + ts.tv_nsec;
}

// First-fit allocator of regions of one device buffer (host-side bookkeeping).
struct Arena {
    char *base = nullptr;
    size_t size = 0;
    std::map<size_t, size_t> free_;  // offset -> bytes, coalesced

    void reset(void *b, size_t s)
    {
        base = (char *)b;
        size = s;
        free_.clear();
        if (s) free_[0] = s;
    }
    static size_t round(size_t bytes) { return (bytes + kGranule - 1) / kGranule * kGranule; }
    bool alloc(size_t bytes, size_t &off)
    {
        bytes = round(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            off = it->first;
            const size_t rest = it->second - bytes;
            free_.erase(it);
            if (rest) free_[off + bytes] = rest;
            return true;
        }
        return false;
    }
    void release(size_t off, size_t bytes)
    {
        bytes = round(bytes);
        auto next = free_.lower_bound(off);
        if (next != free_.end() && off + bytes == next->first) {  // merge with the next region
            bytes += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {  // and with the previous one
                prev->second += bytes;
                return;
            }
        }
        free_[off] = bytes;
    }
};

struct Request {
    uint64_t ticket = 0;
    size_t arena_off = 0, arena_bytes = 0;  // the input's region of the arena (bytes 0: none)
    cudaEvent_t ready = nullptr;  // the copy has landed
    int64_t n = 0;
    float d = 0;
    int64_t min_size = 0, max_size = 0;
    int32_t *labels_out = nullptr;
    size_t est = 0;         // workspace estimate (bytes)
    int64_t submit_ns = 0, deadline_ns = 0;  // deadline 0: none
    fec_status status = FEC_ERR_NOT_READY;
    int32_t k = 0;
    bool done = false;
    int64_t done_ns = 0;    // CLOCK_MONOTONIC at completion
};

}  // namespace

struct ServeEngine {
    fec_ctx *owner = nullptr;
    cudaStream_t copy = nullptr;  // host -> device copies of submitted inputs
    int device = 0;
    size_t budget = 0;            // the whole engine's device memory
    size_t slot_budget = 0;       // what the slots' workspaces may hold together
    size_t held_total = 0;        // what they hold (sum of held[])
    std::vector<size_t> held;     // per slot: its workspace bytes, or what it may grow to while running
    size_t big_n = 0;             // largest request seen (points), and the smallest radius
    float small_d = 0;
    uint64_t next_ticket = 1;
    bool stop = false;
    bool started = false;
    void *arena_mem = nullptr;
    Arena arena;
    std::vector<cudaEvent_t> event_pool;
    fec_serve_stats stats{};
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> queue;
    std::unordered_map<uint64_t, Request *> all;
    std::vector<std::thread> workers;
    std::vector<fec_ctx *> slots;

    fec_status start();
    void worker(int slot);
    void finish(Request *r, fec_status s, int32_t k);  // with mu held
};

fec_status ServeEngine::start()
{
    // called with mu held
    if (started) return FEC_OK;
    const size_t arena_bytes = std::max<size_t>(std::min(budget / 4, kArenaMax), kGranule);
    if (cudaMalloc(&arena_mem, arena_bytes) != cudaSuccess) {
        cudaGetLastError();
        arena_mem = nullptr;
        return FEC_ERR_OOM;
    }
    arena.reset(arena_mem, arena_bytes);
    slot_budget = budget > arena_bytes ? budget - arena_bytes : 0;
    started = true;
    for (int i = 0; i < kSlots; ++i) {
        fec_options o{};
        o.device = device;
        o.mem_budget_bytes = 0;
        fec_ctx *c = nullptr;
        if (fec_create(&o, &c) != FEC_OK) break;
        slots.push_back(c);
    }
    held.assign(slots.size(), 0);
    for (size_t i = 0; i < slots.size(); ++i) workers.emplace_back(&ServeEngine::worker, this, (int)i);
    return FEC_OK;
}

void ServeEngine::finish(Request *r, fec_status s, int32_t k)
{
    if (r->arena_bytes) arena.release(r->arena_off, r->arena_bytes);
    r->arena_bytes = 0;
    if (r->ready) event_pool.push_back(r->ready);
    r->ready = nullptr;
    r->status = s;
    r->k = k;
    r->done_ns = now_ns();
    r->done = true;
}

void ServeEngine::worker(int slot)
{
    cudaSetDevice(device);
    fec_ctx *ctx = slots[slot];
    std::unique_lock<std::mutex> lk(mu);
    // the memory slot `slot` may hold while running q: the slots' share less
    // what the other slots hold
    auto allowed = [&]() -> size_t {
        const size_t others = held_total - held[slot];
        return others < slot_budget ? slot_budget - others : 0;
    };
    auto fits = [&](const Request *q, size_t *proj) {
        const size_t a = allowed();
        *proj = ctx_projected_bytes(ctx, (size_t)q->n, q->d, a);
        return *proj <= a;
    };
    for (;;) {
        size_t proj = 0;
        cv_work.wait(lk, [&] {
            if (stop) return true;
            if (queue.empty()) return false;
            for (Request *q : queue)
                if (fits(q, &proj)) return true;
            // nothing fits: release this idle slot's workspace if it has one
            return held[slot] > 0;
        });
        if (stop && queue.empty()) return;
        // drop requests whose deadline passed, then admit the oldest that fits
        const int64_t t = now_ns();
        bool expired = false;
        for (auto it = queue.begin(); it != queue.end();) {
            Request *q = *it;
            if (q->deadline_ns && t > q->deadline_ns) {
                it = queue.erase(it);
                finish(q, FEC_ERR_TIMEOUT, 0);
                stats.expired += 1;
                expired = true;
            } else {
                ++it;
            }
        }
        if (expired) cv_done.notify_all();
        Request *r = nullptr;
        for (auto it = queue.begin(); it != queue.end(); ++it)
            if (fits(*it, &proj)) {
                r = *it;
                queue.erase(it);
                break;
            }
        if (!r) {
            if (held[slot] > 0 && !queue.empty()) {
                // its workspace keeps the queue from fitting: give it back
                lk.unlock();
                ctx_release_workspace(ctx);
                lk.lock();
                held_total -= held[slot];
                held[slot] = 0;
                cv_work.notify_all();
            }
            continue;
        }
        // a slot grows once to the largest request (and smallest radius) seen
        // so far, when that fits, instead of again at every larger request
        const size_t gn = std::max(big_n, (size_t)r->n);
        const float gd = std::min(small_d, r->d);
        size_t pre = ctx_projected_bytes(ctx, gn, gd, allowed());
        const bool pregrow = pre <= allowed() && pre > proj;
        if (pregrow) proj = pre;
        // this slot may grow to proj bytes while it runs r
        const size_t grant = std::max(proj, held[slot]);
        held_total += grant - held[slot];
        held[slot] = grant;
        ctx_set_budget(ctx, allowed());
        const int64_t wait = t - r->submit_ns;
        stats.queue_wait_ns_sum += wait;
        stats.queue_wait_ns_max = std::max<int64_t>(stats.queue_wait_ns_max, wait);
        lk.unlock();
        int32_t k = 0;
        const cudaStream_t st = ctx_stream(ctx);
        const int64_t t_run = now_ns();
        if (pregrow) ctx_grow(ctx, gn, gd);
        if (r->ready) cudaStreamWaitEvent(st, r->ready, 0);
        const fec_status s = fec_cluster(ctx, r->n ? (const float *)(arena.base + r->arena_off) : nullptr,
                                         r->n, r->d, r->min_size, r->max_size, r->labels_out, &k);
        lk.lock();
        // what the workspace holds now (a retry with longer lists may have grown it)
        const size_t now_held = ctx_ws_bytes(ctx);
        held_total = held_total - held[slot] + now_held;
        held[slot] = now_held;
        finish(r, s, k);
        const int64_t run = r->done_ns - t_run;
        stats.completed += 1;
        stats.run_ns_sum += run;
        stats.run_ns_max = std::max<int64_t>(stats.run_ns_max, run);
        cv_done.notify_all();
        cv_work.notify_all();
    }
}

ServeEngine *serve_create(fec_ctx *owner, const char *)
{
    ServeEngine *e = new ServeEngine();
    e->owner = owner;
    cudaGetDevice(&e->device);
    if (cudaStreamCreateWithFlags(&e->copy, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        e->copy = nullptr;
    }
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
    if (e->copy) cudaStreamSynchronize(e->copy);
    for (auto &kv : e->all) {
        if (kv.second->ready) cudaEventDestroy(kv.second->ready);
        delete kv.second;
    }
    for (cudaEvent_t ev : e->event_pool) cudaEventDestroy(ev);
    for (fec_ctx *c : e->slots) fec_destroy(c);
    if (e->arena_mem) cudaFree(e->arena_mem);
    if (e->copy) cudaStreamDestroy(e->copy);
    delete e;
}

}  // namespace fec

using namespace fec;

// The owning context's budget and serving engine are reached through these
// accessors (fec_ctx is defined in fec_api.cu).
namespace fec {
size_t ctx_budget(const fec_ctx *ctx);
cudaStream_t ctx_stream(const fec_ctx *ctx);
ServeEngine *ctx_serve(fec_ctx *ctx);
size_t workspace_estimate(int sms, int64_t n, float d);  // fec_api.cu
}  // namespace fec

extern "C" {

fec_status fec_serve_submit_deadline(fec_ctx *ctx, const float *xyz, int64_t n, float d,
                                     int64_t min_size, int64_t max_size, int32_t *labels_out,
                                     int64_t deadline_us, uint64_t *ticket)
{
    if (!ctx || !ticket) return FEC_ERR_INVALID_ARG;
    if (n < 0 || n > FEC_MAX_POINTS || !(d > 0.0f) || !std::isfinite(d) || min_size < 0 ||
        max_size < min_size)
        return FEC_ERR_INVALID_ARG;
    if (n > 0 && (!xyz || !labels_out)) return FEC_ERR_INVALID_ARG;
    ServeEngine *e = ctx_serve(ctx);
    if (!e) return FEC_ERR_INVALID_ARG;
    const int64_t t_submit = now_ns();
    Request *r = new Request();
    r->n = n;
    r->d = d;
    r->min_size = min_size;
    r->max_size = max_size;
    r->labels_out = labels_out;
    r->est = workspace_estimate(ctx_sms(ctx), n, d);
    r->submit_ns = t_submit;
    r->deadline_ns = deadline_us > 0 ? t_submit + deadline_us * 1000 : 0;
    {
        std::unique_lock<std::mutex> lk(e->mu);
        if (!e->budget) {
            const size_t b = ctx_budget(ctx);
            e->budget = b ? b : kDefaultBudget;
        }
        fec_status st = e->start();
        if (st != FEC_OK) {
            delete r;
            return st;
        }
        // refused: can never fit the slots' memory, the queue is full, or the
        // arena has no room for the input now
        bool busy = r->est > e->slot_budget || e->queue.size() >= kMaxQueued;
        if (!busy && n > 0) {
            r->arena_bytes = (size_t)n * 12;
            if (!e->arena.alloc(r->arena_bytes, r->arena_off)) {
                r->arena_bytes = 0;
                busy = true;
            }
        }
        if (busy) {
            e->stats.rejected += 1;
            delete r;
            return FEC_ERR_BUSY;
        }
        if (n > 0 && !e->event_pool.empty()) {
            r->ready = e->event_pool.back();
            e->event_pool.pop_back();
        }
    }
    if (n > 0) {
        // Copy the input to its arena region now; the request's slot waits
        // for the event.  One copy stream, so copies land in submit order.
        // From pageable memory the call returns once the driver has staged
        // the input (the caller may reuse its buffer); from pinned host or
        // device memory the copy runs asynchronously (the buffer must stay
        // unchanged until the request completes).
        cudaError_t ce = cudaSuccess;
        if (!r->ready) ce = cudaEventCreateWithFlags(&r->ready, cudaEventDisableTiming);
        if (ce == cudaSuccess)
            ce = cudaMemcpyAsync(e->arena.base + r->arena_off, xyz, (size_t)n * 12, cudaMemcpyDefault,
                                 e->copy);
        if (ce == cudaSuccess) ce = cudaEventRecord(r->ready, e->copy);
        if (ce != cudaSuccess) {
            cudaGetLastError();
            std::lock_guard<std::mutex> lk(e->mu);
            e->arena.release(r->arena_off, r->arena_bytes);
            if (r->ready) e->event_pool.push_back(r->ready);
            delete r;
            return FEC_ERR_CUDA;
        }
    }
    {
        std::lock_guard<std::mutex> lk(e->mu);
        if ((size_t)n > e->big_n) e->big_n = (size_t)n;
        if (e->small_d == 0 || d < e->small_d) e->small_d = d;
        r->ticket = e->next_ticket++;
        e->all[r->ticket] = r;
        e->queue.push_back(r);
        e->stats.submitted += 1;
        e->stats.queue_max = std::max<int64_t>(e->stats.queue_max, (int64_t)e->queue.size());
        *ticket = r->ticket;
    }
    e->cv_work.notify_one();
    return FEC_OK;
}

fec_status fec_serve_submit(fec_ctx *ctx, const float *xyz, int64_t n, float d, int64_t min_size,
                            int64_t max_size, int32_t *labels_out, uint64_t *ticket)
{
    return fec_serve_submit_deadline(ctx, xyz, n, d, min_size, max_size, labels_out, 0, ticket);
}

fec_status fec_serve_poll(fec_ctx *ctx, uint64_t ticket, int32_t *num_clusters, int timeout_ms)
{
    return fec_serve_poll_timed(ctx, ticket, num_clusters, timeout_ms, nullptr);
}

fec_status fec_serve_poll_timed(fec_ctx *ctx, uint64_t ticket, int32_t *num_clusters,
                                int timeout_ms, int64_t *done_ns)
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
            return FEC_ERR_NOT_READY;
        }
    }
    const fec_status s = r->status;
    if (num_clusters) *num_clusters = r->k;
    if (done_ns) *done_ns = r->done_ns;
    e->all.erase(it);
    delete r;
    return s;
}

fec_status fec_serve_get_stats(fec_ctx *ctx, fec_serve_stats *out)
{
    if (!ctx || !out) return FEC_ERR_INVALID_ARG;
    ServeEngine *e = ctx_serve(ctx);
    if (!e) return FEC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(e->mu);
    *out = e->stats;
    out->queued = (int64_t)e->queue.size();
    out->arena_bytes = (int64_t)e->arena.size;
    return FEC_OK;
}

}  // extern "C"
