// fec_batch.cu -- many independent frames in one device pass.
//
// The frames of a batch are grouped by their radius d (exact float value; the
// grid geometry depends on it), and every group runs as ONE call of the
// pipeline over all of its frames: the frame table (see Frame) makes the sort
// segmented by frame, the cell table start a new cell at every frame, the
// size bounds and the numbering per frame, so a group of a hundred frames
// takes the same ~20 launches as one cloud, with every kernel persistent over
// all the group's points.  Groups run concurrently on up to 8 lanes (a CUDA
// stream and a workspace each), and the whole fork/join sequence -- the
// labels' -1 fill, the frame tables' uploads, every group's pipeline and the
// per-frame results -- is captured once into a CUDA graph and replayed for
// every batch of the same shape.  Each frame's labels equal fec_cluster on
// the frame alone (the result is unique).
//
// Autotuner: the first time a batch shape is seen, the launch configuration
// is tuned on it by coordinate descent, each candidate captured and timed with
// CUDA events: the number of lanes (how many groups run at once), the largest
// region of the neighbour step (cells per block, 256 / 512 / 1024), the
// schedule of that step (its last grid-full of regions cut 1, 2 or 4 times
// smaller, so that the blocks finish together) and the sub-cell size above
// which a warp instead of a thread reduces a sub-cell (points per warp, 32 /
// 64 / 128).  The winner is kept in memory and in the context's tuning file
// when one was given (one "key lanes region big tail" line per shape).
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

// Per-frame result, written on the device when the frame's group finishes.
struct FrameResult {
    uint32_t status, k;
    uint32_t slab_need;  // slab-index entries the frame's group needs
    uint32_t pad;
};

// Results of one group: its status bits and each frame's kept clusters.
__global__ void k_group_result(const Plan *plan, const Frame *fr, uint32_t nf,
                               const int32_t *__restrict__ batch_index, FrameResult *out)
{
    grid_enter();
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nf; i += gridDim.x * blockDim.x) {
        FrameResult r;
        r.status = plan->status;
        r.k = nf == 1 ? plan->kept_n : fr[i].kept;
        r.slab_need = plan->slab_need;
        r.pad = 0;
        out[batch_index[i]] = r;
    }
}

// The launch configuration the tuner picks.
struct Config {
    int lanes = 1;
    uint32_t region = kRegionCellsPerBlock;
    uint32_t big = kBigSubcell;
    uint32_t tail = kRegionTailDiv;
};

// Frames of one radius, run as one pipeline call.
struct Group {
    float d = 0;
    std::vector<int32_t> frames;  // batch frame indices, in input order, none empty
    uint32_t n = 0;               // points
    int lane = 0;
};

struct GraphEntry {
    cudaGraphExec_t exec = nullptr;
    Frame *tables = nullptr;       // pinned: every group's frame table (uploaded by the graph)
    int32_t *index_host = nullptr; // pinned: batch index of every group frame
    int32_t *index_dev = nullptr;
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

void free_entry(GraphEntry &g)
{
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.tables) cudaFreeHost(g.tables);
    if (g.index_host) cudaFreeHost(g.index_host);
    if (g.index_dev) cudaFree(g.index_dev);
    g = GraphEntry();
}

}  // namespace

struct BatchEngine {
    int device = 0;
    int sms = 1;
    std::string tune_path;
    Lane lanes[kMaxLanes];
    size_t lane_cap[kMaxLanes] = {};  // points each lane workspace holds
    uint32_t lane_nf[kMaxLanes] = {};  // frames it holds
    uint32_t slab_cap = 0;             // slab-index entries of every lane workspace
    uint32_t list_scale = 1;
    size_t bytes = 0;                  // device bytes held by lane workspaces
    cudaEvent_t fork = nullptr, t0 = nullptr, t1 = nullptr;
    cudaStream_t cap = nullptr;        // capture stream (graphs are launched on the caller's stream)
    FrameResult *res_dev = nullptr, *res_host = nullptr;
    size_t res_cap = 0;
    float *xyz_stage = nullptr;        // device staging of host input
    int32_t *lab_stage = nullptr;
    size_t stage_cap = 0;
    std::map<std::string, GraphEntry> graphs;
    std::map<std::string, Config> tuned;
    bool tune_loaded = false;

    void free_graphs()
    {
        for (auto &g : graphs) free_entry(g.second);
        graphs.clear();
    }
    void free_lanes()
    {
        for (int i = 0; i < kMaxLanes; ++i)
            if (lanes[i].st) cudaStreamSynchronize(lanes[i].st);
        free_graphs();
        for (int i = 0; i < kMaxLanes; ++i) {
            if (lanes[i].ws.base) cudaFree(lanes[i].ws.base);
            lanes[i].ws = Workspace();
            lane_cap[i] = 0;
            lane_nf[i] = 0;
        }
        bytes = 0;
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
    e->free_lanes();
    for (int i = 0; i < kMaxLanes; ++i) {
        Lane &l = e->lanes[i];
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

// Groups of the batch by radius (frames in input order, empty ones left
// out), split so that no group has more than kMaxFramesPerCall frames, and
// spread over `lanes` lanes: largest group first onto the least-loaded lane.
std::vector<Group> make_groups(const int64_t *offsets, int32_t nb, const float *d, int lanes)
{
    std::vector<Group> groups;
    std::map<uint32_t, size_t> open;  // radius bits -> group being filled
    for (int32_t f = 0; f < nb; ++f) {
        const int64_t n = offsets[f + 1] - offsets[f];
        if (n == 0) continue;
        uint32_t bits;
        std::memcpy(&bits, &d[f], 4);
        auto it = open.find(bits);
        if (it == open.end() || groups[it->second].frames.size() >= kMaxFramesPerCall) {
            groups.push_back(Group());
            groups.back().d = d[f];
            open[bits] = groups.size() - 1;
            it = open.find(bits);
        }
        Group &g = groups[it->second];
        g.frames.push_back(f);
        g.n += (uint32_t)n;
    }
    std::vector<size_t> order(groups.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = i;
    std::sort(order.begin(), order.end(), [&](size_t a, size_t b) { return groups[a].n > groups[b].n; });
    std::vector<uint64_t> load(std::max(lanes, 1), 0);
    for (size_t i : order) {
        const int l = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        groups[i].lane = l;
        load[l] += groups[i].n + 65536;  // a fixed cost per group for its launches
    }
    return groups;
}

// Slab-index entries a group of n points starts with (a LiDAR frame of
// 160 m needs about 640 at d = 0.25 m); a group that needs more grows them
// and runs again.
uint32_t slab_guess(uint64_t n) { return (uint32_t)std::max<uint64_t>(1u << 16, n / 8); }

// Lane workspaces large enough for their groups.
fec_status ensure_lanes(BatchEngine &e, const std::vector<Group> &groups, int lanes, size_t budget)
{
    if (!e.fork) {
        if (cudaEventCreateWithFlags(&e.fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreate(&e.t0) != cudaSuccess || cudaEventCreate(&e.t1) != cudaSuccess ||
            cudaStreamCreateWithFlags(&e.cap, cudaStreamNonBlocking) != cudaSuccess)
            return FEC_ERR_CUDA;
    }
    size_t need_n[kMaxLanes] = {};
    uint32_t need_nf[kMaxLanes] = {};
    uint32_t slab = e.slab_cap;
    for (const Group &g : groups) {
        need_n[g.lane] = std::max<size_t>(need_n[g.lane], g.n);
        need_nf[g.lane] = std::max<uint32_t>(need_nf[g.lane], (uint32_t)g.frames.size());
        slab = std::max(slab, slab_guess(g.n));
    }
    if (slab > e.slab_cap) {  // every lane's slab index grows: start over
        e.free_lanes();
        e.slab_cap = slab;
    }
    for (int i = 0; i < lanes; ++i) {
        Lane &l = e.lanes[i];
        if (!l.st && cudaStreamCreateWithFlags(&l.st, cudaStreamNonBlocking) != cudaSuccess)
            return FEC_ERR_CUDA;
        if (!l.done && cudaEventCreateWithFlags(&l.done, cudaEventDisableTiming) != cudaSuccess)
            return FEC_ERR_CUDA;
        const size_t cap = std::max<size_t>(need_n[i], 4096);
        const uint32_t nf = std::max<uint32_t>(need_nf[i], 1);
        if (l.ws.base && cap <= e.lane_cap[i] && nf <= e.lane_nf[i]) continue;
        if (l.ws.base) {  // too small: graphs hold its pointers
            cudaStreamSynchronize(l.st);
            e.free_graphs();
            cudaFree(l.ws.base);
            e.bytes -= l.ws.bytes;
            l.ws = Workspace();
        }
        const size_t cap2 = std::max(cap, e.lane_cap[i]);
        const uint32_t nf2 = std::max(nf, e.lane_nf[i]);
        Workspace probe;
        probe.sms = e.sms;
        probe.list_scale = e.list_scale;
        const size_t b = workspace_layout(probe, nullptr, cap2, e.slab_cap, nf2);
        if (budget && e.bytes + b > budget) return FEC_ERR_OOM;
        void *base = nullptr;
        if (cudaMalloc(&base, b) != cudaSuccess) {
            cudaGetLastError();
            return FEC_ERR_OOM;
        }
        l.ws.sms = e.sms;
        l.ws.device = e.device;
        l.ws.list_scale = e.list_scale;
        workspace_layout(l.ws, base, cap2, e.slab_cap, nf2);
        e.lane_cap[i] = cap2;
        e.lane_nf[i] = nf2;
        e.bytes += b;
    }
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
                      const int64_t *mx, const float *xyz, const int32_t *labels, const Config &c)
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
    char buf[96];
    std::snprintf(buf, sizeof(buf), "%016llx/%d/%d/%u/%u/%u", h, nb, c.lanes, c.region, c.big, c.tail);
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
    char line[256], key[128];
    while (std::fgets(line, sizeof(line), f)) {
        // "key lanes region big [tail]" (files without the tail use the default)
        Config c;
        unsigned region = 0, big = 0, tail = kRegionTailDiv;
        const int got = std::sscanf(line, "%127s %d %u %u %u", key, &c.lanes, &region, &big, &tail);
        if (got < 4 || c.lanes < 1 || c.lanes > kMaxLanes || region < kRegionMinCells ||
            region > kRegionCellsPerBlock || big < 1 || big > (unsigned)kHugeSubcell || tail < 1 ||
            tail > 8)
            continue;
        c.region = region;
        c.big = big;
        c.tail = tail;
        e.tuned[key] = c;
    }
    std::fclose(f);
}

void save_tuning(const BatchEngine &e)
{
    if (e.tune_path.empty()) return;
    FILE *f = std::fopen(e.tune_path.c_str(), "w");
    if (!f) return;
    for (const auto &kv : e.tuned)
        std::fprintf(f, "%s %d %u %u %u\n", kv.first.c_str(), kv.second.lanes, kv.second.region,
                     kv.second.big, kv.second.tail);
    std::fclose(f);
}

// Capture the batch into a graph with configuration c.
fec_status capture(BatchEngine &e, const Config &c, const std::vector<Group> &groups,
                   const float *xyz, const int64_t *offsets, int32_t nb, const int64_t *mn,
                   const int64_t *mx, int32_t *labels, GraphEntry &g)
{
    // frame tables and batch indices of every group, in pinned memory that
    // the graph's uploads read from
    size_t total = 0;
    for (const Group &gr : groups) total += gr.frames.size();
    if (total) {
        if (cudaMallocHost(&g.tables, total * sizeof(Frame)) != cudaSuccess ||
            cudaMallocHost(&g.index_host, total * sizeof(int32_t)) != cudaSuccess ||
            cudaMalloc(&g.index_dev, total * sizeof(int32_t)) != cudaSuccess) {
            cudaGetLastError();
            free_entry(g);
            return FEC_ERR_OOM;
        }
    }
    std::vector<size_t> first(groups.size());
    size_t at = 0;
    for (size_t gi = 0; gi < groups.size(); ++gi) {
        first[gi] = at;
        uint32_t pos = 0, tile = 0;
        for (int32_t f : groups[gi].frames) {
            Frame fr{};
            fr.in_off = (uint32_t)offsets[f];
            fr.pos_off = pos;
            fr.n = (uint32_t)(offsets[f + 1] - offsets[f]);
            fr.tile0 = tile;
            fr.min_size = mn[f];
            fr.max_size = mx[f];
            pos += fr.n;
            tile += frame_tiles(fr.n);
            g.tables[at] = fr;
            g.index_host[at] = f;
            ++at;
        }
    }
    const uint32_t rows = (uint32_t)offsets[nb];
    cudaGraph_t graph = nullptr;
    cudaStream_t main = e.cap;
    if (cudaStreamBeginCapture(main, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        free_entry(g);
        return FEC_ERR_CUDA;
    }
    // every label starts at -1 (empty frames and dropped points keep it);
    // the groups write their frames' kept points only
    cudaError_t err = cudaMemsetAsync(labels, 0xff, (size_t)rows * 4, main);
    if (err == cudaSuccess && total)
        err = cudaMemcpyAsync(g.index_dev, g.index_host, total * sizeof(int32_t),
                              cudaMemcpyHostToDevice, main);
    // frames without points: no clusters
    for (int32_t f = 0; f < nb && err == cudaSuccess; ++f)
        if (offsets[f + 1] == offsets[f]) err = cudaMemsetAsync(e.res_dev + f, 0, sizeof(FrameResult), main);
    if (err == cudaSuccess) err = cudaEventRecord(e.fork, main);
    for (int l = 0; l < c.lanes && err == cudaSuccess; ++l) {
        Lane &ln = e.lanes[l];
        err = cudaStreamWaitEvent(ln.st, e.fork, 0);
        for (size_t gi = 0; gi < groups.size() && err == cudaSuccess; ++gi) {
            const Group &gr = groups[gi];
            if (gr.lane != l) continue;
            const uint32_t nf = (uint32_t)gr.frames.size();
            err = cudaMemcpyAsync(ln.ws.frames, g.tables + first[gi], nf * sizeof(Frame),
                                  cudaMemcpyHostToDevice, ln.st);
            if (err != cudaSuccess) break;
            Params prm = make_params(gr.n, gr.d);
            prm.nf = nf;
            prm.ntiles = 0;
            for (int32_t f : gr.frames) prm.ntiles += frame_tiles((uint64_t)(offsets[f + 1] - offsets[f]));
            prm.rows = rows;
            prm.slab_cap = e.slab_cap;
            prm.region_cells = c.region;
            prm.big_subcell = c.big;
            prm.region_tail = c.tail;
            FrontArgs fa;
            fa.single = false;
            err = enqueue_cluster(ln.ws, xyz, prm, fa, labels, false, ln.st);
            if (err == cudaSuccess) {
                launch(k_group_result, (nf + 255) / 256, 256, 0, ln.st, ln.ws.plan, ln.ws.frames, nf,
                                                                     g.index_dev + first[gi], e.res_dev);
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
        free_entry(g);
        return FEC_ERR_CUDA;
    }
    const cudaError_t inst = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (inst != cudaSuccess) {
        cudaGetLastError();
        free_entry(g);
        return FEC_ERR_CUDA;
    }
    return FEC_OK;
}

fec_status get_graph(BatchEngine &e, const Config &c, const std::vector<Group> &groups,
                     size_t budget, const float *xyz, const int64_t *offsets, int32_t nb,
                     const float *d, const int64_t *mn, const int64_t *mx, int32_t *labels,
                     cudaGraphExec_t *exec)
{
    fec_status s = ensure_lanes(e, groups, c.lanes, budget);
    if (s != FEC_OK) return s;
    const std::string key = shape_key(offsets, nb, d, mn, mx, xyz, labels, c);
    auto it = e.graphs.find(key);
    if (it != e.graphs.end()) {
        *exec = it->second.exec;
        return FEC_OK;
    }
    if (e.graphs.size() > 64) e.free_graphs();
    GraphEntry g;
    s = capture(e, c, groups, xyz, offsets, nb, mn, mx, labels, g);
    if (s != FEC_OK) return s;
    e.graphs[key] = g;
    *exec = g.exec;
    return FEC_OK;
}

// Milliseconds per replay of configuration c (one warm-up, two timed).
fec_status time_config(BatchEngine &e, cudaStream_t main, const Config &c, size_t budget,
                       const float *xyz, const int64_t *offsets, int32_t nb, const float *d,
                       const int64_t *mn, const int64_t *mx, int32_t *labels, float *ms)
{
    const std::vector<Group> groups = make_groups(offsets, nb, d, c.lanes);
    cudaGraphExec_t ex = nullptr;
    const fec_status s = get_graph(e, c, groups, budget, xyz, offsets, nb, d, mn, mx, labels, &ex);
    if (s != FEC_OK) return s;
    cudaGraphLaunch(ex, main);
    cudaEventRecord(e.t0, main);
    for (int r = 0; r < 2; ++r) cudaGraphLaunch(ex, main);
    cudaEventRecord(e.t1, main);
    if (cudaEventSynchronize(e.t1) != cudaSuccess) return FEC_ERR_CUDA;
    cudaEventElapsedTime(ms, e.t0, e.t1);
    return FEC_OK;
}

// Coordinate descent over lanes, then region size, then the region schedule,
// then the warp threshold.
fec_status autotune(BatchEngine &e, cudaStream_t main, size_t budget, const float *xyz,
                    const int64_t *offsets, int32_t nb, const float *d, const int64_t *mn,
                    const int64_t *mx, int32_t *labels, Config *out)
{
    const int ngroups = (int)make_groups(offsets, nb, d, 1).size();
    Config best;
    float best_ms = 1e30f;
    auto consider = [&](const Config &c) -> fec_status {
        float ms = 0;
        const fec_status s = time_config(e, main, c, budget, xyz, offsets, nb, d, mn, mx, labels, &ms);
        if (s == FEC_ERR_OOM) return FEC_OK;  // too large for the budget: not a candidate
        if (s != FEC_OK) return s;
        if (ms < best_ms) {
            best_ms = ms;
            best = c;
        }
        return FEC_OK;
    };
    for (int l = 1; l <= kMaxLanes && l <= std::max(ngroups, 1); l *= 2) {
        Config c;
        c.lanes = l;
        const fec_status s = consider(c);
        if (s != FEC_OK) return s;
    }
    if (best_ms >= 1e30f) return FEC_ERR_OOM;
    const Config base_r = best;
    for (uint32_t r : {256u, 512u, 1024u}) {
        if (r == base_r.region) continue;
        Config c = base_r;
        c.region = r;
        const fec_status s = consider(c);
        if (s != FEC_OK) return s;
    }
    const Config base_t = best;
    for (uint32_t t : {1u, 2u, 4u}) {
        if (t == base_t.tail) continue;
        Config c = base_t;
        c.tail = t;
        const fec_status s = consider(c);
        if (s != FEC_OK) return s;
    }
    const Config base_b = best;
    for (uint32_t b : {32u, 64u, 128u}) {
        if (b == base_b.big) continue;
        Config c = base_b;
        c.big = b;
        const fec_status s = consider(c);
        if (s != FEC_OK) return s;
    }
    *out = best;
    return FEC_OK;
}

}  // namespace

fec_status batch_run(BatchEngine *e, cudaStream_t main, size_t budget, const float *xyz,
                     const int64_t *offsets, int32_t nb, const float *d, const int64_t *mn,
                     const int64_t *mx, int32_t *labels, int32_t *num_clusters)
{
    const int64_t total = offsets[nb];
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
    for (int attempt = 0;; ++attempt) {
        auto tit = e->tuned.find(tk);
        Config cfg;
        if (tit != e->tuned.end()) {
            cfg = tit->second;
        } else {
            s = autotune(*e, main, budget, xin, offsets, nb, d, mn, mx, lout, &cfg);
            if (s != FEC_OK) return s;
            e->tuned[tk] = cfg;
            save_tuning(*e);
        }
        const std::vector<Group> groups = make_groups(offsets, nb, d, cfg.lanes);
        cudaGraphExec_t ex = nullptr;
        s = get_graph(*e, cfg, groups, budget, xin, offsets, nb, d, mn, mx, lout, &ex);
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
        if ((bits & (ST_QUEUE_OVERFLOW | ST_SIZE_OVERFLOW)) && attempt < 3) {
            // boundary lists or a slab index too small for some group: grow
            // them (every lane), capture again
            if (bits & ST_QUEUE_OVERFLOW) e->list_scale *= 4;
            uint32_t need = e->slab_cap;
            for (int32_t f = 0; f < nb; ++f) need = std::max(need, e->res_host[f].slab_need);
            const uint32_t old = e->slab_cap;
            e->free_lanes();
            e->slab_cap = std::max(need, old);
            if (!(bits & ST_QUEUE_OVERFLOW) && e->slab_cap == old) break;  // nothing to grow
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
    // growing did not help: report the statuses as they are
    fec_status worst = FEC_OK;
    for (int32_t f = 0; f < nb; ++f) {
        const fec_status fs = status_from_bits(e->res_host[f].status);
        num_clusters[f] = fs == FEC_OK ? (int32_t)e->res_host[f].k : 0;
        if (fs != FEC_OK && worst == FEC_OK) worst = fs;
    }
    return worst;
}

size_t batch_bytes(const BatchEngine *e) { return e ? e->bytes : 0; }

}  // namespace fec
