// fec_api.cu -- contexts, workspace, the one-cloud pipeline on a stream, and
// the C ABI declared in include/fec.h.
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include <cuda.h>

#include "fec.h"
#include "fec_batch.h"
#include "fec_internal.cuh"
#include "fec_serve.h"

// Single calls of at least this many points read the plan's outcome back
// after the bounding-box kernel (one 16-byte copy and a stream
// synchronisation) and launch only the sort passes of the key width it chose;
// smaller calls skip that round trip and launch the passes of both widths,
// of which those of the other width return at once (120k frame: 0.195 ->
// 0.188 ms).
#ifndef FEC_READBACK_MIN_POINTS
#define FEC_READBACK_MIN_POINTS 1000000
#endif

namespace fec {

// ---------------------------------------------------------------------------
// Parameters
// ---------------------------------------------------------------------------

Params make_params(uint32_t n, float d)
{
    Params p{};
    p.n = n;
    // T2 = floor((d*1024)^2); any two valid points are closer than
    // sqrt(3) * 2^24 units, so clamping T2 at 3 * 2^48 changes no decision.
    const double s = (double)d * 1024.0;
    double t = std::floor(s * s);
    const double cap = 3.0 * 281474976710656.0;
    if (t > cap) t = cap;
    p.T2 = (int64_t)t;
    int64_t R = (int64_t)std::sqrt((double)p.T2);
    while (R * R > p.T2) --R;
    while ((R + 1) * (R + 1) <= p.T2) ++R;
    p.R = (int32_t)R;
    int64_t h = (R + 1) / 2;
    if (h < 1) h = 1;
    if (h > (1 << 24)) h = 1 << 24;
    p.h = (int32_t)h;
    p.S = (int32_t)(2 * h);
    p.slab_cap = (uint32_t)(((1u << 24) - 1) / (uint32_t)p.S + 2);
    p.packed = p.S <= 1024 ? 1u : 0u;
    // floor(rel / S) for rel < 2^24 as (rel * m) >> s: with s = 24 + ceil(log2 S)
    // and m = ceil(2^s / S) the product overshoots rel / S by less than 1/S.
    uint32_t lg = 0;
    while (((int64_t)1 << lg) < (int64_t)p.S) ++lg;
    p.div_s = 24 + lg;
    p.div_m = (uint32_t)((((uint64_t)1 << p.div_s) + (uint64_t)p.S - 1) / (uint64_t)p.S);
    // one frame (a single cloud) unless the caller lays out several
    p.nf = 1;
    p.ntiles = frame_tiles(n);
    p.rows = n;
    return p;
}

static int bitlen_host(uint64_t v)
{
    int b = 0;
    while (v) {
        ++b;
        v >>= 1;
    }
    return b;
}

int max_sort_passes(const Params &prm)
{
    const int b = bitlen_host(((1u << 24) - 1) / (uint32_t)prm.S);
    int bits = 3 * b + 3;
    if (bits > 64) bits = 64;
    return (bits + kRadixBits - 1) / kRadixBits;
}


// ---------------------------------------------------------------------------
// Workspace
// ---------------------------------------------------------------------------

size_t workspace_layout(Workspace &ws, void *base, size_t cap_n, uint32_t slab_cap, uint32_t nf_cap)
{
    size_t off = 0;
    auto take = [&](size_t bytes) -> void * {
        off = (off + 255) & ~(size_t)255;
        void *p = base ? (void *)((char *)base + off) : nullptr;
        off += bytes;
        return p;
    };
    const size_t n = cap_n;
    if (nf_cap < 1) nf_cap = 1;
    ws.plan = (Plan *)take(sizeof(Plan));
    ws.frames = (Frame *)take(sizeof(Frame) * nf_cap);
    ws.fhist = (uint32_t *)take(4 * (size_t)nf_cap * kMaxPasses * kRadixBins);
    ws.xyz = (float *)take(12 * n);
    ws.labels = (int32_t *)take(4 * n);
    ws.keys_a = take(8 * n);
    ws.keys_b = take(8 * n);
    ws.vals_a = take(8 * n);
    ws.vals_b = take(8 * n);
    ws.sort_status = (uint32_t *)take(4 * sort_status_words(max_tiles(n, nf_cap)));
    ws.scan_status = (unsigned long long *)take(8 * (n / kScanTile + 2));
    ws.rec = (Rec *)take(sizeof(Rec) * n);
    ws.sc_of = (uint32_t *)take(4 * n);
    ws.sc_start = (uint32_t *)take(4 * (n + 2));
    ws.scode = (uint8_t *)take(n);
    ws.cocc = (uint8_t *)take(n);
    ws.box = (SubBox *)take(sizeof(SubBox) * n);
    ws.sminidx = (uint32_t *)take(4 * n);
    ws.parent = (uint32_t *)take(4 * n);
    ws.csize = (uint32_t *)take(4 * n);
    ws.cmin = (uint32_t *)take(4 * n);
    ws.crank = (int32_t *)take(4 * n);
    ws.big = (uint32_t *)take(4 * n);
    ws.cell_key = (unsigned long long *)take(8 * n);
    ws.cell_sc = (uint32_t *)take(4 * (n + 2));
    ws.cframe = (uint32_t *)take(4 * n);
    ws.slab_lo = (uint32_t *)take(4 * (size_t)slab_cap);
    ws.slab_hi = (uint32_t *)take(4 * (size_t)slab_cap);
    const size_t lists = 2 * n * (size_t)(ws.list_scale ? ws.list_scale : 1);
    ws.pairq_cap = lists;
    ws.pairq = (uint2 *)take(sizeof(uint2) * lists);
    ws.reps = (uint32_t *)take(4 * n);
    // dense column index: 2^col_bits entries, about 4 per point (64 Ki..64 Mi)
    uint32_t cb = 16;
    while (cb < 26 && ((size_t)1 << cb) < 4 * n) ++cb;
    ws.col_bits = cb;
    ws.col_lo = (uint32_t *)take(4 * ((size_t)1 << cb));
    ws.col_hi = (uint32_t *)take(4 * ((size_t)1 << cb));
    ws.edges_cap = lists;
    ws.edges = (uint2 *)take(sizeof(uint2) * lists);
    size_t es = 1024;
    while (es < n / 8) es <<= 1;
    ws.edge_set_size = es;
    ws.edge_set = (unsigned long long *)take(sizeof(unsigned long long) * es);
    const size_t words = n / 32 + 1;
    ws.rank_bits = (uint32_t *)take(4 * words);
    ws.rank_prefix = (uint32_t *)take(4 * words);
    ws.rank_status = (unsigned long long *)take(8 * (words / 2048 + 2));
    ws.nb_first = (uint32_t *)take(4 * 13 * n);
    ws.nb_cnt = (uint8_t *)take(32 * n);
    ws.scratch_words = (size_t)region_grid(ws, n) * region_scratch(ws, n);
    ws.scratch = (uint32_t *)take(4 * ws.scratch_words);
    off = (off + 255) & ~(size_t)255;
    if (base) {
        ws.base = base;
        ws.bytes = off;
        ws.cap_n = cap_n;
        ws.slab_cap = slab_cap;
        ws.nf_cap = nf_cap;
    }
    return off;
}

// ---------------------------------------------------------------------------
// Pipeline
// ---------------------------------------------------------------------------

cudaError_t enqueue_cluster(Workspace &ws, const float *xyz, const Params &prm_in,
                            const FrontArgs &fa, int32_t *labels, bool fill_labels, cudaStream_t st)
{
    Params prm = prm_in;
    prm.col_bits = ws.col_bits;
    cudaError_t e = enqueue_front(ws, xyz, prm, fa, st);
    if (e != cudaSuccess) return e;
    return enqueue_back(ws, xyz, prm, labels, fill_labels, st);
}

cudaError_t enqueue_back(Workspace &ws, const float *xyz, const Params &prm_in, int32_t *labels,
                         bool fill_labels, cudaStream_t st, const KeyLayout *known)
{
    Params prm = prm_in;
    prm.col_bits = ws.col_bits;
    const int sort_grid = ws.sms;  // per SM; the sort multiplies by its occupancy
    cudaError_t e = cudaSuccess;
    // a2: the passes of the width the plan selected, when the host knows it;
    // else both key widths (the kernels of the other width return at once)
    const bool pk = prm.packed != 0;
    const bool run32 = !known || !known->key64, run64 = !known || known->key64;
    const int p64 = known ? known->passes : max_sort_passes(prm);
    if (run32) {
        e = launch_sort(ws, "onesweep_u32", &ws.plan->sort, ws.keys_a, ws.vals_a, ws.keys_b,
                        ws.vals_b, false, pk, !pk, ws.sort_status, prm.ntiles,
                        known ? known->passes : 4, sort_grid, st, &ws.plan->status,
                        main_sort_source(ws, xyz, prm));
        if (e != cudaSuccess) return e;
    }
    if (run64 && p64 > 4) {
        e = launch_sort(ws, "onesweep_u64", &ws.plan->sort, ws.keys_a, ws.vals_a, ws.keys_b,
                        ws.vals_b, true, pk, !pk, ws.sort_status, prm.ntiles, p64, sort_grid, st,
                        &ws.plan->status, main_sort_source(ws, xyz, prm));
        if (e != cudaSuccess) return e;
    }
    e = enqueue_cells(ws, xyz, prm, st);
    if (e != cudaSuccess) return e;
    e = enqueue_union(ws, prm, st);
    if (e != cudaSuccess) return e;
    return enqueue_labels(ws, prm, labels, fill_labels, st);
}

// The summary of a finished call: the head of its plan (status, counts,
// counters; everything before the sort control block), copied to pinned
// host memory.
constexpr size_t kSummaryBytes = offsetof(Plan, sort);
using Summary = Plan;

fec_status status_from_bits(uint32_t s)
{
    if (s & ST_DEBUG_BOUNDS) return FEC_ERR_INTERNAL;
    if (s & ST_NONFINITE) return FEC_ERR_NONFINITE;
    if (s & (ST_OUT_OF_RANGE | ST_KEY_OVERFLOW)) return FEC_ERR_OUT_OF_RANGE;
    if (s & (ST_WAIT_TIMEOUT | ST_UNION_CAP)) return FEC_ERR_NOT_CONVERGED;
    if (s & ST_SIZE_OVERFLOW) return FEC_ERR_OUT_OF_RANGE;
    if (s & ST_QUEUE_OVERFLOW) return FEC_ERR_OOM;
    return FEC_OK;
}

// ---------------------------------------------------------------------------
// Tracing
// ---------------------------------------------------------------------------

struct Trace {
    cudaEvent_t start = nullptr;
    std::vector<cudaEvent_t> pool;
    std::vector<const char *> names;
    int used = 0;
    struct Acc {
        const char *name;
        int64_t launches;
        double ms;
    };
    std::vector<Acc> acc;

    bool init(int n)
    {
        if (start) return true;
        if (cudaEventCreate(&start) != cudaSuccess) return false;
        pool.resize(n);
        names.resize(n);
        for (auto &e : pool)
            if (cudaEventCreate(&e) != cudaSuccess) return false;
        return true;
    }
    void destroy()
    {
        if (start) cudaEventDestroy(start);
        for (auto &e : pool)
            if (e) cudaEventDestroy(e);
        start = nullptr;
        pool.clear();
    }
    void begin(cudaStream_t st)
    {
        used = 0;
        cudaEventRecord(start, st);
    }
    // after the stream has been synchronised
    void end()
    {
        cudaEvent_t prev = start;
        for (int i = 0; i < used; ++i) {
            float ms = 0;
            cudaEventElapsedTime(&ms, prev, pool[i]);
            prev = pool[i];
            bool hit = false;
            for (auto &a : acc)
                if (a.name == names[i] || std::strcmp(a.name, names[i]) == 0) {
                    a.launches += 1;
                    a.ms += ms;
                    hit = true;
                    break;
                }
            if (!hit) acc.push_back({names[i], 1, (double)ms});
        }
        used = 0;
    }
};

void trace_mark(const Workspace &ws, const char *name, cudaStream_t st)
{
    Trace *t = ws.trace;
    if (!t || t->used >= (int)t->pool.size()) return;
    cudaEventRecord(t->pool[t->used], st);
    t->names[t->used] = name;
    ++t->used;
}

namespace {

// Driver entry points for the current context's ID, taken through the
// runtime once (no link against the driver library is needed).
using PfnCtxGetCurrent = CUresult (*)(CUcontext *);
using PfnCtxGetId = CUresult (*)(CUcontext, unsigned long long *);
std::once_flag g_pfn_once;
PfnCtxGetCurrent g_ctx_get_current = nullptr;
PfnCtxGetId g_ctx_get_id = nullptr;

}  // namespace

unsigned long long current_ctx_id()
{
    std::call_once(g_pfn_once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_get_current = (PfnCtxGetCurrent)f;
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_get_id = (PfnCtxGetId)f;
        cudaGetLastError();
    });
    if (!g_ctx_get_current || !g_ctx_get_id) return 0;
    CUcontext c = nullptr;
    if (g_ctx_get_current(&c) != CUDA_SUCCESS || !c) return 0;
    unsigned long long id = 0;
    if (g_ctx_get_id(c, &id) != CUDA_SUCCESS) return 0;
    return id;
}

bool ctx_setup_needed(std::atomic<unsigned long long> &done_in)
{
    const unsigned long long id = current_ctx_id();
    if (id != 0 && done_in.load(std::memory_order_acquire) == id) return false;
    return true;
}

void ctx_setup_done(std::atomic<unsigned long long> &done_in)
{
    done_in.store(current_ctx_id(), std::memory_order_release);
}

int sm_count()
{
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 1;
}

}  // namespace fec

using namespace fec;

struct fec_ctx {
    int device = 0;
    size_t budget = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    Workspace ws;
    Summary *summary_host = nullptr;  // pinned; its first kSummaryBytes are valid
    fec_stats last{};
    std::mutex mu;
    ServeEngine *serve = nullptr;
    BatchEngine *batch = nullptr;
    Trace trace;
    bool tracing = false;
    uint32_t wait_cap = kWaitCap;    // iteration caps of the device loops (fec_set_iteration_caps)
    uint32_t union_cap = kUnionCap;
    char *pinned = nullptr;          // pinned staging of pageable inputs and outputs
    size_t pinned_bytes = 0;
};

namespace {

// Where a caller's buffer lives: device (or managed), pinned host, or
// pageable host memory.
enum class Mem { Device, Pinned, Pageable };
Mem mem_kind(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return Mem::Pageable;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return Mem::Device;
    return a.type == cudaMemoryTypeHost ? Mem::Pinned : Mem::Pageable;
}

// Pinned staging of at least `bytes` (grown with a quarter of headroom).  A
// pageable input goes through it: a CPU copy plus an asynchronous DMA
// instead of the driver's pageable copy path.
char *pinned_stage(fec_ctx *ctx, size_t bytes)
{
    if (bytes <= ctx->pinned_bytes) return ctx->pinned;
    if (ctx->pinned) {
        cudaStreamSynchronize(ctx->stream);
        cudaFreeHost(ctx->pinned);
    }
    ctx->pinned = nullptr;
    ctx->pinned_bytes = 0;
    const size_t want = bytes + bytes / 4;
    if (cudaMallocHost((void **)&ctx->pinned, want) != cudaSuccess) {
        cudaGetLastError();
        ctx->pinned = nullptr;
        return nullptr;
    }
    ctx->pinned_bytes = want;
    return ctx->pinned;
}

fec_status check_args(int64_t n, float d, int64_t min_size, int64_t max_size)
{
    if (n < 0 || n > FEC_MAX_POINTS) return FEC_ERR_INVALID_ARG;
    if (!std::isfinite(d) || !(d > 0.0f)) return FEC_ERR_INVALID_ARG;
    if (min_size < 0 || max_size < min_size) return FEC_ERR_INVALID_ARG;
    return FEC_OK;
}

// Grow the workspace to hold n points at slab capacity slab_cap.
// The size a workspace grows to for n points at slab capacity slab_cap: a
// quarter more points than it holds now (so that slowly growing clouds do
// not re-allocate every call), or exactly n when that would exceed budget.
struct Growth {
    size_t cap, bytes;
    uint32_t slab;
};
Growth growth_for(const Workspace &ws, size_t n, uint32_t slab_cap, size_t budget)
{
    Growth g;
    g.cap = n;
    if (ws.base && g.cap < ws.cap_n + ws.cap_n / 4) g.cap = ws.cap_n + ws.cap_n / 4;
    if (g.cap < 4096) g.cap = 4096;
    g.slab = slab_cap > ws.slab_cap ? slab_cap : ws.slab_cap;
    Workspace probe;
    probe.sms = ws.sms;
    probe.list_scale = ws.list_scale;
    g.bytes = workspace_layout(probe, nullptr, g.cap, g.slab);
    if (budget && g.bytes > budget) {
        g.cap = n < 4096 ? 4096 : n;  // without headroom
        g.bytes = workspace_layout(probe, nullptr, g.cap, g.slab);
    }
    return g;
}

fec_status ensure_workspace(fec_ctx *ctx, size_t n, uint32_t slab_cap, bool force = false)
{
    Workspace &ws = ctx->ws;
    if (!force && ws.base && n <= ws.cap_n && slab_cap <= ws.slab_cap) return FEC_OK;
    const Growth g = growth_for(ws, n, slab_cap, ctx->budget);
    if (ctx->budget && g.bytes > ctx->budget) return FEC_ERR_OOM;
    const size_t cap = g.cap, bytes = g.bytes;
    const uint32_t sc = g.slab;
    // Stream-ordered: the old workspace is released and the new one taken on
    // the context's stream, so growing it stalls no other stream (a plain
    // free would synchronise the whole device).
    if (ws.base) {
        cudaFreeAsync(ws.base, ctx->stream);
        ws.base = nullptr;
        ws.cap_n = 0;
    }
    void *base = nullptr;
    if (cudaMallocAsync(&base, bytes, ctx->stream) != cudaSuccess) {
        cudaGetLastError();
        return FEC_ERR_OOM;
    }
    workspace_layout(ws, base, cap, sc);
    return FEC_OK;
}

fec_status finish(fec_ctx *ctx, int64_t n, const Params &prm, int32_t *num_clusters)
{
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return FEC_ERR_CUDA;
    const Summary &s = *ctx->summary_host;
    fec_stats &st = ctx->last;
    st.n = n;
    st.cells = s.M_c;
    st.subcells = s.M_s;
    st.num_clusters = s.kept_n;
    st.key_bits = s.key_bits;
    st.workspace_bytes = (int64_t)ctx->ws.bytes;
    st.R = prm.R;
    st.h = prm.h;
    st.T2 = prm.T2;
    st.pair_checks = (int64_t)s.ctr[CTR_PAIRS];
    st.pair_box_joins = (int64_t)s.ctr[CTR_BOX_JOINS];
    st.pair_point_tests = (int64_t)s.ctr[CTR_POINT_TESTS];
    st.pair_same_root = (int64_t)s.ctr[CTR_SAME_ROOT];
    st.point_evals = (int64_t)s.ctr[CTR_POINT_EVALS];
    st.pairs_queued = (int64_t)s.ctr[CTR_QUEUED];
    st.boundary_edges = (int64_t)s.ctr[CTR_EDGES];
    const fec_status f = status_from_bits(s.status);
    if (f == FEC_OK && num_clusters) *num_clusters = (int32_t)s.kept_n;
    return f;
}

}  // namespace

namespace fec {

fec_status cluster_once(fec_ctx *ctx, const float *xyz, int64_t n, int64_t min_size,
                        int64_t max_size, int32_t *labels, int32_t *num_clusters,
                        const Params &prm);

// One cloud on the context's stream; device or host pointers.  Caller holds ctx->mu.
fec_status cluster_locked(fec_ctx *ctx, const float *xyz, int64_t n, float d, int64_t min_size,
                          int64_t max_size, int32_t *labels, int32_t *num_clusters)
{
    Params prm = make_params((uint32_t)n, d);
    prm.wait_cap = ctx->wait_cap;
    prm.union_cap = ctx->union_cap;
    fec_status s = ensure_workspace(ctx, (size_t)n, prm.slab_cap);
    if (s != FEC_OK) return s;
    // The boundary-edge and pair lists hold 2 entries per point; a cloud that
    // needs more (it is reported by the device) is re-run with larger lists.
    for (int attempt = 0;; ++attempt) {
        s = cluster_once(ctx, xyz, n, min_size, max_size, labels, num_clusters, prm);
        if (!(ctx->summary_host->status & ST_QUEUE_OVERFLOW) || attempt == 3) return s;
        ctx->ws.list_scale *= 4;
        s = ensure_workspace(ctx, (size_t)n, prm.slab_cap, true);
        if (s != FEC_OK) return s;
    }
}

fec_status cluster_once(fec_ctx *ctx, const float *xyz, int64_t n, int64_t min_size,
                        int64_t max_size, int32_t *labels, int32_t *num_clusters,
                        const Params &prm)
{
    Workspace &ws = ctx->ws;
    ws.trace = ctx->tracing ? &ctx->trace : nullptr;
    if (ws.trace) ws.trace->begin(ctx->stream);
    const float *xin = xyz;
    const Mem in_kind = mem_kind(xyz), out_kind = mem_kind(labels);
    // pinned staging of a pageable input (a pageable output is copied by the
    // driver: a CPU copy into freshly allocated caller memory would pay its
    // page faults on the critical path)
    char *stage = nullptr;
    if (in_kind == Mem::Pageable) {
        stage = pinned_stage(ctx, (size_t)n * 12);
        if (!stage) return FEC_ERR_OOM;
    }
    if (in_kind != Mem::Device) {
        const void *src = xyz;
        if (in_kind == Mem::Pageable) {
            std::memcpy(stage, xyz, (size_t)n * 12);
            src = stage;
        }
        if (cudaMemcpyAsync(ws.xyz, src, (size_t)n * 12, cudaMemcpyHostToDevice, ctx->stream) !=
            cudaSuccess)
            return FEC_ERR_CUDA;
        FEC_MARK(ws, "h2d_xyz", ctx->stream);
        xin = ws.xyz;
    }
    const bool dev_out = out_kind == Mem::Device;
    int32_t *lout = dev_out ? labels : ws.labels;
    FrontArgs fa;
    fa.single = true;
    fa.min_size = min_size;
    fa.max_size = max_size;
    Params pc = prm;
    pc.col_bits = ws.col_bits;
    if (enqueue_front(ws, xin, pc, fa, ctx->stream) != cudaSuccess) return FEC_ERR_CUDA;
#if FEC_READBACK_MIN_POINTS > 0
    if ((uint64_t)n < (uint64_t)FEC_READBACK_MIN_POINTS) {  // small cloud: no read-back
        if (enqueue_back(ws, xin, pc, lout, true, ctx->stream, nullptr) != cudaSuccess) return FEC_ERR_CUDA;
        if (!dev_out && cudaMemcpyAsync(labels, ws.labels, (size_t)n * 4, cudaMemcpyDeviceToHost,
                                        ctx->stream) != cudaSuccess)
            return FEC_ERR_CUDA;
        if (cudaMemcpyAsync(ctx->summary_host, ws.plan, kSummaryBytes, cudaMemcpyDeviceToHost,
                            ctx->stream) != cudaSuccess)
            return FEC_ERR_CUDA;
        const fec_status st0 = finish(ctx, n, prm, num_clusters);
        if (ws.trace) ws.trace->end();
        ws.trace = nullptr;
        return st0;
    }
#endif
    // The plan's outcome back on the host (16 bytes): a data error ends the
    // call here, and the sort launches exactly the passes of the key width
    // the plan selected (no launches that would only return).
    uint32_t *front = ctx->summary_host->front;
    if (cudaMemcpyAsync(front, ws.plan->front, sizeof(uint32_t) * 4, cudaMemcpyDeviceToHost,
                        ctx->stream) != cudaSuccess ||
        cudaStreamSynchronize(ctx->stream) != cudaSuccess)
        return FEC_ERR_CUDA;
    if (front[0] & (ST_NONFINITE | ST_OUT_OF_RANGE | ST_KEY_OVERFLOW | ST_SIZE_OVERFLOW)) {
        if (ws.trace) ws.trace->end();
        ws.trace = nullptr;
        ctx->summary_host->status = front[0];
        ctx->last = fec_stats{};
        ctx->last.n = n;
        return status_from_bits(front[0]);
    }
    KeyLayout kl;
    kl.key64 = front[1] != 0;
    kl.passes = (int)front[2];
    if (enqueue_back(ws, xin, pc, lout, true, ctx->stream, &kl) != cudaSuccess) return FEC_ERR_CUDA;
    if (!dev_out) {
        if (cudaMemcpyAsync(labels, ws.labels, (size_t)n * 4, cudaMemcpyDeviceToHost,
                            ctx->stream) != cudaSuccess)
            return FEC_ERR_CUDA;
        FEC_MARK(ws, "d2h_labels", ctx->stream);
    }
    if (cudaMemcpyAsync(ctx->summary_host, ws.plan, kSummaryBytes,
                        cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess)
        return FEC_ERR_CUDA;
    FEC_MARK(ws, "summary", ctx->stream);
    const fec_status st = finish(ctx, n, prm, num_clusters);
    if (ws.trace) ws.trace->end();
    ws.trace = nullptr;
    return st;
}

size_t ctx_budget(const fec_ctx *ctx) { return ctx->budget; }
cudaStream_t ctx_stream(const fec_ctx *ctx) { return ctx->stream; }
ServeEngine *ctx_serve(fec_ctx *ctx) { return ctx->serve; }
int ctx_sms(const fec_ctx *ctx) { return ctx->ws.sms; }
// Device bytes ctx's workspace holds now.
size_t ctx_ws_bytes(const fec_ctx *ctx) { return ctx->ws.base ? ctx->ws.bytes : 0; }
// Bytes it will hold while clustering n points at radius d within budget
// (its present size when that already fits).
size_t ctx_projected_bytes(const fec_ctx *ctx, size_t n, float d, size_t budget)
{
    const Workspace &ws = ctx->ws;
    const uint32_t slab = make_params((uint32_t)n, d).slab_cap;
    if (ws.base && n <= ws.cap_n && slab <= ws.slab_cap) return ws.bytes;
    return growth_for(ws, n, slab, budget).bytes;
}
// Grow ctx's workspace for n points at radius d, within its budget.
fec_status ctx_grow(fec_ctx *ctx, size_t n, float d)
{
    std::lock_guard<std::mutex> lock(ctx->mu);
    cudaSetDevice(ctx->device);
    return ensure_workspace(ctx, n, make_params((uint32_t)n, d).slab_cap);
}
void ctx_set_budget(fec_ctx *ctx, size_t budget)
{
    std::lock_guard<std::mutex> lock(ctx->mu);
    ctx->budget = budget;
}
// Release ctx's workspace (after its stream's work); the next call allocates anew.
void ctx_release_workspace(fec_ctx *ctx)
{
    std::lock_guard<std::mutex> lock(ctx->mu);
    Workspace &ws = ctx->ws;
    if (!ws.base) return;
    cudaSetDevice(ctx->device);
    cudaFreeAsync(ws.base, ctx->stream);
    cudaStreamSynchronize(ctx->stream);
    ws.base = nullptr;
    ws.cap_n = 0;
    ws.bytes = 0;
    ws.slab_cap = 0;
}

// Device workspace bytes fec_cluster takes for n points at radius d on a
// device of `sms` SMs (the region step's scratch scales with the SM count).
size_t workspace_estimate(int sms, int64_t n, float d)
{
    const Params prm = make_params((uint32_t)n, d);
    Workspace probe;
    probe.sms = sms > 0 ? sms : 1;
    return workspace_layout(probe, nullptr, (size_t)(n < 4096 ? 4096 : n), prm.slab_cap);
}

}  // namespace fec

extern "C" {

const char *fec_status_string(fec_status s)
{
    switch (s) {
    case FEC_OK: return "FEC_OK";
    case FEC_ERR_INVALID_ARG: return "FEC_ERR_INVALID_ARG";
    case FEC_ERR_NONFINITE: return "FEC_ERR_NONFINITE";
    case FEC_ERR_OUT_OF_RANGE: return "FEC_ERR_OUT_OF_RANGE";
    case FEC_ERR_OOM: return "FEC_ERR_OOM";
    case FEC_ERR_CUDA: return "FEC_ERR_CUDA";
    case FEC_ERR_NOT_CONVERGED: return "FEC_ERR_NOT_CONVERGED";
    case FEC_ERR_NOT_READY: return "FEC_ERR_NOT_READY";
    case FEC_ERR_BUSY: return "FEC_ERR_BUSY";
    case FEC_ERR_TIMEOUT: return "FEC_ERR_TIMEOUT";
    case FEC_ERR_INTERNAL: return "FEC_ERR_INTERNAL";
    }
    return "FEC_ERR_UNKNOWN";
}

int64_t fec_workspace_bytes(int64_t n, float d)
{
    if (n < 0 || n > FEC_MAX_POINTS || !std::isfinite(d) || !(d > 0.0f)) return -1;
    // the current device's SM count; 160 when no device can be queried
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
        cudaGetLastError();
        sms = 160;
    }
    return (int64_t)workspace_estimate(sms, n, d);
}

fec_status fec_create(const fec_options *opt, fec_ctx **out)
{
    if (!out) return FEC_ERR_INVALID_ARG;
    *out = nullptr;
    fec_ctx *ctx = new (std::nothrow) fec_ctx();
    if (!ctx) return FEC_ERR_OOM;
    ctx->device = opt ? opt->device : 0;
    ctx->budget = opt ? opt->mem_budget_bytes : 0;
    if (cudaSetDevice(ctx->device) != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return FEC_ERR_CUDA;
    }
    if (opt && opt->cuda_stream) {
        ctx->stream = (cudaStream_t)opt->cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete ctx;
            return FEC_ERR_CUDA;
        }
        ctx->own_stream = true;
    }
    ctx->ws.device = ctx->device;
    ctx->ws.sms = sm_count();
    {
        // keep freed workspaces in the device's stream-ordered pool for reuse
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, ctx->device) == cudaSuccess) {
            uint64_t keep = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
        cudaGetLastError();
    }
    if (cudaMallocHost(&ctx->summary_host, sizeof(Summary)) != cudaSuccess) {
        cudaGetLastError();
        fec_destroy(ctx);
        return FEC_ERR_OOM;
    }
    ctx->serve = serve_create(ctx, opt ? opt->autotune_cache : nullptr);
    ctx->batch = batch_create(ctx->device, ctx->ws.sms, opt ? opt->autotune_cache : nullptr);
    *out = ctx;
    return FEC_OK;
}

void fec_destroy(fec_ctx *ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->serve) serve_destroy(ctx->serve);
    if (ctx->batch) batch_destroy(ctx->batch);
    ctx->trace.destroy();
    if (ctx->ws.base && ctx->stream) cudaFreeAsync(ctx->ws.base, ctx->stream);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    if (ctx->summary_host) cudaFreeHost(ctx->summary_host);
    if (ctx->pinned) cudaFreeHost(ctx->pinned);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

fec_status fec_cluster(fec_ctx *ctx, const float *xyz, int64_t n, float d, int64_t min_size,
                       int64_t max_size, int32_t *labels, int32_t *num_clusters)
{
    if (!ctx || !num_clusters) return FEC_ERR_INVALID_ARG;
    fec_status s = check_args(n, d, min_size, max_size);
    if (s != FEC_OK) return s;
    if (n > 0 && (!xyz || !labels)) return FEC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(ctx->mu);
    if (cudaSetDevice(ctx->device) != cudaSuccess) return FEC_ERR_CUDA;
    if (n == 0) {
        *num_clusters = 0;
        ctx->last = fec_stats{};
        return FEC_OK;
    }
    return cluster_locked(ctx, xyz, n, d, min_size, max_size, labels, num_clusters);
}

fec_status fec_cluster_batch(fec_ctx *ctx, const float *xyz, const int64_t *offsets, int32_t nb,
                             const float *d, const int64_t *min_size, const int64_t *max_size,
                             int32_t *labels, int32_t *num_clusters)
{
    if (!ctx || nb < 0 || (nb > 0 && (!offsets || !d || !min_size || !max_size || !num_clusters)))
        return FEC_ERR_INVALID_ARG;
    if (nb == 0) return FEC_OK;
    if (offsets[0] != 0) return FEC_ERR_INVALID_ARG;
    for (int32_t f = 0; f < nb; ++f) {
        if (offsets[f + 1] < offsets[f]) return FEC_ERR_INVALID_ARG;
        const fec_status s = check_args(offsets[f + 1] - offsets[f], d[f], min_size[f], max_size[f]);
        if (s != FEC_OK) return s;
    }
    if (offsets[nb] > 0 && (!xyz || !labels)) return FEC_ERR_INVALID_ARG;
    if (offsets[nb] > FEC_MAX_POINTS) return FEC_ERR_INVALID_ARG;  // rows must fit 32 bits
    std::lock_guard<std::mutex> lock(ctx->mu);
    if (cudaSetDevice(ctx->device) != cudaSuccess) return FEC_ERR_CUDA;
    if (offsets[nb] == 0) {
        for (int32_t f = 0; f < nb; ++f) num_clusters[f] = 0;
        return FEC_OK;
    }
    const fec_status s = batch_run(ctx->batch, ctx->stream, ctx->budget, xyz, offsets, nb, d,
                                   min_size, max_size, labels, num_clusters);
    ctx->last = fec_stats{};
    ctx->last.n = offsets[nb];
    ctx->last.workspace_bytes = (int64_t)(ctx->ws.bytes + batch_bytes(ctx->batch));
    return s;
}

fec_status fec_set_iteration_caps(fec_ctx *ctx, uint32_t wait_cap, uint32_t union_cap)
{
    if (!ctx) return FEC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(ctx->mu);
    ctx->wait_cap = wait_cap;
    ctx->union_cap = union_cap;
    return FEC_OK;
}

fec_status fec_trace_enable(fec_ctx *ctx, int enable)
{
    if (!ctx) return FEC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(ctx->mu);
    if (cudaSetDevice(ctx->device) != cudaSuccess) return FEC_ERR_CUDA;
    ctx->trace.acc.clear();
    if (enable && !ctx->trace.init(512)) return FEC_ERR_CUDA;
    ctx->tracing = enable != 0;
    return FEC_OK;
}

int fec_trace_read(const fec_ctx *ctx, fec_trace_entry *out, int cap)
{
    if (!ctx || cap < 0) return -1;
    const auto &acc = ctx->trace.acc;
    if (out)
        for (int i = 0; i < cap && i < (int)acc.size(); ++i) {
            out[i].name = acc[i].name;
            out[i].launches = acc[i].launches;
            out[i].total_ms = acc[i].ms;
        }
    return (int)acc.size();
}

fec_status fec_get_stats(const fec_ctx *ctx, fec_stats *out)
{
    if (!ctx || !out) return FEC_ERR_INVALID_ARG;
    *out = ctx->last;
    return FEC_OK;
}

}  // extern "C"
