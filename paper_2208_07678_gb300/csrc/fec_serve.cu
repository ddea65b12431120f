// fec_serve.cu -- request loop with continuous batching.
//
// Requests (clouds of any size, each with its own d and size bounds) are
// copied to device memory at submit time, on the engine's copy stream, and
// queued.  A fixed set of
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
#include <ctime>
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

cudaStream_t ctx_stream(const fec_ctx *ctx);  // fec_api.cu
fec_status ctx_reserve(fec_ctx *ctx, size_t n, uint32_t slab_cap, size_t max_bytes);  // fec_api.cu

namespace {

constexpr int kSlots = 4;
constexpr size_t kDefaultBudget = (size_t)40 << 30;  // 40 GiB when the context has none

struct Request {
    uint64_t ticket = 0;
    float *xyz = nullptr;   // device copy of the input (stream-ordered allocation)
    cudaEvent_t ready = nullptr;  // the copy has landed
    int64_t n = 0;
    float d = 0;
    int64_t min_size = 0, max_size = 0;
    int32_t *labels_out = nullptr;
    size_t est = 0;         // workspace estimate (bytes)
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
    size_t budget = 0;
    size_t in_flight = 0;
    size_t hw_n = 0;         // largest request (points) and slab index seen so far
    uint32_t hw_slab = 0;
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
        // grow this slot's workspace to the largest request seen so far (while
        // that fits its share of the budget), so that slots do not each
        // re-allocate as ever larger requests reach them
        size_t hn = 0;
        uint32_t hs = 0;
        {
            std::lock_guard<std::mutex> lk(mu);
            hn = hw_n;
            hs = hw_slab;
        }
        ctx_reserve(ctx, hn, hs, budget / kSlots);
        int32_t k = 0;
        const cudaStream_t st = ctx_stream(ctx);
        if (r->ready) cudaStreamWaitEvent(st, r->ready, 0);
        fec_status s = fec_cluster(ctx, r->xyz, r->n, r->d, r->min_size, r->max_size,
                                   r->labels_out, &k);
        timespec ts;
        clock_gettime(CLOCK_MONOTONIC, &ts);
        if (r->xyz) cudaFreeAsync(r->xyz, st);
        r->xyz = nullptr;
        {
            std::lock_guard<std::mutex> lk(mu);
            in_flight -= r->est;
            r->status = s;
            r->k = k;
            r->done_ns = (int64_t)ts.tv_sec * 1000000000LL + ts.tv_nsec;
            r->done = true;
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
        if (kv.second->xyz) cudaFree(kv.second->xyz);
        if (kv.second->ready) cudaEventDestroy(kv.second->ready);
        delete kv.second;
    }
    for (fec_ctx *c : e->slots) fec_destroy(c);
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
        // Copy the input to the device now (the caller may reuse its buffer
        // once submit returns: a copy from pageable memory returns after the
        // driver has staged it); the request's slot waits for the event.
        if (!e->copy || cudaMallocAsync(&r->xyz, (size_t)n * 12, e->copy) != cudaSuccess) {
            cudaGetLastError();
            delete r;
            return FEC_ERR_OOM;
        }
        if (cudaMemcpyAsync(r->xyz, xyz, (size_t)n * 12, cudaMemcpyDefault, e->copy) != cudaSuccess ||
            cudaEventCreateWithFlags(&r->ready, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventRecord(r->ready, e->copy) != cudaSuccess) {
            cudaGetLastError();
            cudaFreeAsync(r->xyz, e->copy);
            delete r;
            return FEC_ERR_CUDA;
        }
    }
    {
        std::lock_guard<std::mutex> lk(e->mu);
        e->start();
        if ((size_t)n > e->hw_n) e->hw_n = (size_t)n;
        const uint32_t sc = make_params((uint32_t)n, d).slab_cap;
        if (sc > e->hw_slab) e->hw_slab = sc;
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
            return FEC_ERR_TIMEOUT;
        }
    }
    const fec_status s = r->status;
    if (num_clusters) *num_clusters = r->k;
    if (done_ns) *done_ns = r->done_ns;
    e->all.erase(it);
    if (r->ready) cudaEventDestroy(r->ready);
    delete r;
    return s;
}

}  // extern "C"
