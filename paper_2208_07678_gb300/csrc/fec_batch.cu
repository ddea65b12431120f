// fec_batch.cu -- many independent frames in one launch: the frames of a batch
// are spread over L concurrent lanes (a CUDA stream and a workspace each;
// largest frame first onto the least-loaded lane), and the whole fork/join
// launch sequence is captured once into a CUDA graph and replayed for every
// batch of the same shape.  Each frame runs exactly the one-cloud pipeline,
// so its labels equal fec_cluster on the frame alone.
//
// Autotuner: the first time a batch shape is seen, each lane count in
// {1, 2, 4, 8} (at most the number of frames) is captured and timed with
// CUDA events, and the fastest is kept (in memory, and in the context's
// tuning file when one was given: one "key lanes" line per shape).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "fec.h"
#include "fec_batch.h"
#include "fec_internal.cuh"

namespace fec {

fec_status status_from_bits(uint32_t s);  // fec_api.cu

namespace {

constexpr int kMaxLanes = 8;

struct Lane {
    cudaStream_t st = nullptr;
    cudaEvent_t done = nullptr;
    Workspace ws;
};

// Per-frame result, copied from the frame's plan when it finishes.
struct FrameResult {
    uint32_t status, k;
};

__global__ void k_frame_result(const Plan *plan, FrameResult *out)
{
    if (threadIdx.x == 0) {
        out->status = plan->status;
        out->k = plan->kept.n;
    }
}

struct GraphEntry {
    cudaGraphExec_t exec = nullptr;
};

bool on_device(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

struct BatchEngine {
    int device = 0;
    int sms = 1;
    std::string tune_path;
    Lane lanes[kMaxLanes];
    int nlanes = 0;
    size_t lane_cap = 0;        // points each lane workspace holds
    uint32_t lane_slab = 0;
    uint32_t list_scale = 1;
    size_t bytes = 0;           // device bytes held
    cudaEvent_t fork = nullptr, t0 = nullptr, t1 = nullptr;
    cudaStream_t cap = nullptr;  // capture stream (graphs are launched on the caller's stream)
    FrameResult *res_dev = nullptr, *res_host = nullptr;
    size_t res_cap = 0;
    float *xyz_stage = nullptr;  // device staging of host input
    int32_t *lab_stage = nullptr;
    size_t stage_cap = 0;
    std::map<std::string, GraphEntry> graphs;
    std::map<std::string, int> tuned;
    bool tune_loaded = false;

    void free_graphs()
    {
        for (auto &g : graphs)
            if (g.second.exec) cudaGraphExecDestroy(g.second.exec);
        graphs.clear();
    }
};

BatchEngine *batch_create(int device, int sms, const char *tune_path)
{
    BatchEngine *e = new BatchEngine();
    e->device = device;
    e->sms = sms;
    if (tune_path) e->tune_path = tune_path;
    return e;
}

void batch_destroy(BatchEngine *e)
{
    if (!e) return;
    cudaSetDevice(e->device);
    for (int i = 0; i < e->nlanes; ++i) cudaStreamSynchronize(e->lanes[i].st);
    e->free_graphs();
    for (int i = 0; i < kMaxLanes; ++i) {
        Lane &l = e->lanes[i];
        if (l.ws.base) cudaFree(l.ws.base);
        if (l.done) cudaEventDestroy(l.done);
        if (l.st) cudaStreamDestroy(l.st);
    }
    if (e->fork) cudaEventDestroy(e->fork);
    if (e->cap) cudaStreamDestroy(e->cap);
    if (e->t0) cudaEventDestroy(e->t0);
    if (e->t1) cudaEventDestroy(e->t1);
    if (e->res_dev) cudaFree(e->res_dev);
    if (e->res_host) cudaFreeHost(e->res_host);
    if (e->xyz_stage) cudaFree(e->xyz_stage);
    if (e->lab_stage) cudaFree(e->lab_stage);
    delete e;
}

namespace {

// Make kMaxLanes lanes that each hold `cap` points (only the lanes a run uses
// are allocated).
fec_status ensure_lanes(BatchEngine &e, int lanes, size_t cap, uint32_t slab, size_t budget)
{
    if (!e.fork) {
        if (cudaEventCreateWithFlags(&e.fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreate(&e.t0) != cudaSuccess || cudaEventCreate(&e.t1) != cudaSuccess ||
            cudaStreamCreateWithFlags(&e.cap, cudaStreamNonBlocking) != cudaSuccess)
            return FEC_ERR_CUDA;
    }
    if (cap < 4096) cap = 4096;
    const bool grow = cap > e.lane_cap || slab > e.lane_slab;
    if (grow) {
        for (int i = 0; i < e.nlanes; ++i) cudaStreamSynchronize(e.lanes[i].st);
        e.free_graphs();
        for (int i = 0; i < kMaxLanes; ++i)
            if (e.lanes[i].ws.base) {
                cudaFree(e.lanes[i].ws.base);
                e.lanes[i].ws.base = nullptr;
            }
        e.bytes = 0;
        e.lane_cap = std::max(cap, e.lane_cap);
        e.lane_slab = std::max(slab, e.lane_slab);
    }
    for (int i = 0; i < lanes; ++i) {
        Lane &l = e.lanes[i];
        if (!l.st && cudaStreamCreateWithFlags(&l.st, cudaStreamNonBlocking) != cudaSuccess)
            return FEC_ERR_CUDA;
        if (!l.done && cudaEventCreateWithFlags(&l.done, cudaEventDisableTiming) != cudaSuccess)
            return FEC_ERR_CUDA;
        if (l.ws.base) continue;
        Workspace probe;
        probe.sms = e.sms;
        probe.list_scale = e.list_scale;
        const size_t b = workspace_layout(probe, nullptr, e.lane_cap, e.lane_slab);
        if (budget && e.bytes + b > budget) return FEC_ERR_OOM;
        void *base = nullptr;
        if (cudaMalloc(&base, b) != cudaSuccess) {
            cudaGetLastError();
            return FEC_ERR_OOM;
        }
        l.ws.sms = e.sms;
        l.ws.device = e.device;
        l.ws.list_scale = e.list_scale;
        workspace_layout(l.ws, base, e.lane_cap, e.lane_slab);
        e.bytes += b;
    }
    e.nlanes = std::max(e.nlanes, lanes);
    return FEC_OK;
}

fec_status ensure_results(BatchEngine &e, size_t nb)
{
    if (nb <= e.res_cap) return FEC_OK;
    if (e.res_dev) cudaFree(e.res_dev);
    if (e.res_host) cudaFreeHost(e.res_host);
    e.res_dev = nullptr;
    e.res_host = nullptr;
    if (cudaMalloc(&e.res_dev, nb * sizeof(FrameResult)) != cudaSuccess ||
        cudaMallocHost(&e.res_host, nb * sizeof(FrameResult)) != cudaSuccess) {
        cudaGetLastError();
        e.res_cap = 0;
        return FEC_ERR_OOM;
    }
    e.res_cap = nb;
    e.free_graphs();  // graphs hold the old result pointers
    return FEC_OK;
}

std::string shape_key(const int64_t *offsets, int32_t nb, const float *d, const int64_t *mn,
                      const int64_t *mx, const float *xyz, const int32_t *labels, int lanes)
{
    // FNV-1a over everything the captured launch sequence depends on
    unsigned long long h = 1469598103934665603ull;
    auto mix = [&](const void *p, size_t n) {
        const unsigned char *b = (const unsigned char *)p;
        for (size_t i = 0; i < n; ++i) {
            h ^= b[i];
            h *= 1099511628211ull;
        }
    };
    mix(offsets, sizeof(int64_t) * (nb + 1));
    mix(d, sizeof(float) * nb);
    mix(mn, sizeof(int64_t) * nb);
    mix(mx, sizeof(int64_t) * nb);
    mix(&xyz, sizeof(xyz));
    mix(&labels, sizeof(labels));
    char buf[64];
    std::snprintf(buf, sizeof(buf), "%016llx/%d/%d", h, nb, lanes);
    return buf;
}

std::string tune_key(const int64_t *offsets, int32_t nb)
{
    int64_t mx = 0;
    for (int32_t f = 0; f < nb; ++f) mx = std::max(mx, offsets[f + 1] - offsets[f]);
    // shape bucket: frame count and total / largest size to 2 significant bits
    auto bucket = [](int64_t v) {
        int b = 0;
        while ((v >> b) > 3) ++b;
        return (int)((v >> b) << 8 | b);
    };
    char buf[64];
    std::snprintf(buf, sizeof(buf), "nb%d_tot%d_max%d", nb, bucket(offsets[nb]), bucket(mx));
    return buf;
}

void load_tuning(BatchEngine &e)
{
    if (e.tune_loaded) return;
    e.tune_loaded = true;
    if (e.tune_path.empty()) return;
    FILE *f = std::fopen(e.tune_path.c_str(), "r");
    if (!f) return;
    char key[128];
    int lanes = 0;
    while (std::fscanf(f, "%127s %d", key, &lanes) == 2)
        if (lanes >= 1 && lanes <= kMaxLanes) e.tuned[key] = lanes;
    std::fclose(f);
}

void save_tuning(const BatchEngine &e)
{
    if (e.tune_path.empty()) return;
    FILE *f = std::fopen(e.tune_path.c_str(), "w");
    if (!f) return;
    for (const auto &kv : e.tuned) std::fprintf(f, "%s %d\n", kv.first.c_str(), kv.second);
    std::fclose(f);
}

// Capture the batch into a graph on `main` with `lanes` lanes.
fec_status capture(BatchEngine &e, int lanes, const float *xyz,
                   const int64_t *offsets, int32_t nb, const float *d, const int64_t *mn,
                   const int64_t *mx, int32_t *labels, cudaGraphExec_t *out)
{
    // largest frame first onto the least-loaded lane
    std::vector<int32_t> order(nb);
    for (int32_t f = 0; f < nb; ++f) order[f] = f;
    std::sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
        return offsets[a + 1] - offsets[a] > offsets[b + 1] - offsets[b];
    });
    std::vector<std::vector<int32_t>> plan(lanes);
    std::vector<int64_t> load(lanes, 0);
    for (int32_t f : order) {
        const int64_t n = offsets[f + 1] - offsets[f];
        const int l = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        plan[l].push_back(f);
        load[l] += n + 4096;  // a small per-frame cost for launch overhead
    }
    cudaGraph_t graph = nullptr;
    cudaStream_t main = e.cap;
    if (cudaStreamBeginCapture(main, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return FEC_ERR_CUDA;
    cudaError_t err = cudaEventRecord(e.fork, main);
    for (int l = 0; l < lanes && err == cudaSuccess; ++l) {
        Lane &ln = e.lanes[l];
        err = cudaStreamWaitEvent(ln.st, e.fork, 0);
        for (int32_t f : plan[l]) {
            if (err != cudaSuccess) break;
            const int64_t n = offsets[f + 1] - offsets[f];
            if (n == 0) {
                err = cudaMemsetAsync(e.res_dev + f, 0, sizeof(FrameResult), ln.st);
                continue;
            }
            err = enqueue_cluster(ln.ws, xyz + 3 * offsets[f], make_params((uint32_t)n, d[f]),
                                  mn[f], mx[f], labels + offsets[f], ln.st);
            if (err == cudaSuccess) {
                k_frame_result<<<1, 32, 0, ln.st>>>(ln.ws.plan, e.res_dev + f);
                err = cudaGetLastError();
            }
        }
        if (err == cudaSuccess) err = cudaEventRecord(ln.done, ln.st);
        if (err == cudaSuccess) err = cudaStreamWaitEvent(main, ln.done, 0);
    }
    const cudaError_t end = cudaStreamEndCapture(main, &graph);
    if (err != cudaSuccess || end != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return FEC_ERR_CUDA;
    }
    const cudaError_t inst = cudaGraphInstantiate(out, graph, 0);
    cudaGraphDestroy(graph);
    if (inst != cudaSuccess) {
        cudaGetLastError();
        return FEC_ERR_CUDA;
    }
    return FEC_OK;
}

fec_status get_graph(BatchEngine &e, cudaStream_t main, int lanes, const float *xyz,
                     const int64_t *offsets, int32_t nb, const float *d, const int64_t *mn,
                     const int64_t *mx, int32_t *labels, cudaGraphExec_t *exec)
{
    const std::string key = shape_key(offsets, nb, d, mn, mx, xyz, labels, lanes);
    auto it = e.graphs.find(key);
    if (it != e.graphs.end()) {
        *exec = it->second.exec;
        return FEC_OK;
    }
    if (e.graphs.size() > 64) e.free_graphs();
    GraphEntry g;
    const fec_status s = capture(e, lanes, xyz, offsets, nb, d, mn, mx, labels, &g.exec);
    if (s != FEC_OK) return s;
    e.graphs[key] = g;
    *exec = g.exec;
    return FEC_OK;
}

}  // namespace

fec_status batch_run(BatchEngine *e, cudaStream_t main, size_t budget, const float *xyz,
                     const int64_t *offsets, int32_t nb, const float *d, const int64_t *mn,
                     const int64_t *mx, int32_t *labels, int32_t *num_clusters)
{
    const int64_t total = offsets[nb];
    int64_t nmax = 0;
    uint32_t slab = 0;
    for (int32_t f = 0; f < nb; ++f) {
        nmax = std::max(nmax, offsets[f + 1] - offsets[f]);
        slab = std::max(slab, make_params(1, d[f]).slab_cap);
    }
    // inputs and outputs in device memory (host buffers are staged)
    const bool dev_in = on_device(xyz), dev_out = on_device(labels);
    if ((!dev_in || !dev_out) && (size_t)total > e->stage_cap) {
        if (e->xyz_stage) cudaFree(e->xyz_stage);
        if (e->lab_stage) cudaFree(e->lab_stage);
        e->xyz_stage = nullptr;
        e->lab_stage = nullptr;
        e->stage_cap = 0;
        e->free_graphs();
        if (cudaMalloc(&e->xyz_stage, (size_t)total * 12) != cudaSuccess ||
            cudaMalloc(&e->lab_stage, (size_t)total * 4) != cudaSuccess) {
            cudaGetLastError();
            return FEC_ERR_OOM;
        }
        e->stage_cap = (size_t)total;
    }
    const float *xin = dev_in ? xyz : e->xyz_stage;
    int32_t *lout = dev_out ? labels : e->lab_stage;
    fec_status s = ensure_results(*e, (size_t)nb);
    if (s != FEC_OK) return s;
    if (!dev_in &&
        cudaMemcpyAsync(e->xyz_stage, xyz, (size_t)total * 12, cudaMemcpyHostToDevice, main) !=
            cudaSuccess)
        return FEC_ERR_CUDA;

    load_tuning(*e);
    const std::string tk = tune_key(offsets, nb);
    int lanes = 0;
    auto tit = e->tuned.find(tk);
    if (tit != e->tuned.end()) lanes = std::min<int>(tit->second, std::max<int32_t>(nb, 1));
    for (int attempt = 0;; ++attempt) {
        if (lanes == 0) {
            // autotune the lane count on this batch
            float best = 1e30f;
            int best_l = 1;
            for (int l = 1; l <= kMaxLanes && l <= std::max<int32_t>(nb, 1); l *= 2) {
                s = ensure_lanes(*e, l, (size_t)nmax, slab, budget);
                if (s != FEC_OK) break;
                cudaGraphExec_t ex = nullptr;
                s = get_graph(*e, main, l, xin, offsets, nb, d, mn, mx, lout, &ex);
                if (s != FEC_OK) return s;
                cudaGraphLaunch(ex, main);  // warm-up
                cudaEventRecord(e->t0, main);
                for (int r = 0; r < 2; ++r) cudaGraphLaunch(ex, main);
                cudaEventRecord(e->t1, main);
                if (cudaEventSynchronize(e->t1) != cudaSuccess) return FEC_ERR_CUDA;
                float ms = 0;
                cudaEventElapsedTime(&ms, e->t0, e->t1);
                if (ms < best) {
                    best = ms;
                    best_l = l;
                }
            }
            lanes = best_l;
            e->tuned[tk] = lanes;
            save_tuning(*e);
        }
        s = ensure_lanes(*e, lanes, (size_t)nmax, slab, budget);
        if (s != FEC_OK) return s;
        cudaGraphExec_t ex = nullptr;
        s = get_graph(*e, main, lanes, xin, offsets, nb, d, mn, mx, lout, &ex);
        if (s != FEC_OK) return s;
        if (cudaGraphLaunch(ex, main) != cudaSuccess ||
            cudaMemcpyAsync(e->res_host, e->res_dev, nb * sizeof(FrameResult),
                            cudaMemcpyDeviceToHost, main) != cudaSuccess ||
            cudaStreamSynchronize(main) != cudaSuccess) {
            cudaGetLastError();
            return FEC_ERR_CUDA;
        }
        uint32_t bits = 0;
        for (int32_t f = 0; f < nb; ++f) bits |= e->res_host[f].status;
        if ((bits & ST_QUEUE_OVERFLOW) && attempt < 3) {
            // boundary lists too small for some frame: larger lists, re-capture
            e->list_scale *= 4;
            for (int i = 0; i < e->nlanes; ++i) cudaStreamSynchronize(e->lanes[i].st);
            e->free_graphs();
            for (int i = 0; i < kMaxLanes; ++i)
                if (e->lanes[i].ws.base) {
                    cudaFree(e->lanes[i].ws.base);
                    e->lanes[i].ws.base = nullptr;
                }
            e->bytes = 0;
            continue;
        }
        // frames are independent: report the first error, numbers for all
        fec_status worst = FEC_OK;
        for (int32_t f = 0; f < nb; ++f) {
            const fec_status fs = status_from_bits(e->res_host[f].status);
            num_clusters[f] = fs == FEC_OK ? (int32_t)e->res_host[f].k : 0;
            if (fs != FEC_OK && worst == FEC_OK) worst = fs;
        }
        if (!dev_out &&
            (cudaMemcpyAsync(labels, e->lab_stage, (size_t)total * 4, cudaMemcpyDeviceToHost,
                             main) != cudaSuccess ||
             cudaStreamSynchronize(main) != cudaSuccess))
            return FEC_ERR_CUDA;
        return worst;
    }
}

size_t batch_bytes(const BatchEngine *e) { return e ? e->bytes : 0; }

}  // namespace fec
