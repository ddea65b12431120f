// fec_noalloc.cu -- fec_cluster_noalloc: the one-cloud pipeline with its
// workspace in a fixed, statically allocated device array, for callers that
// must not allocate device memory (see include/fec.h).
//
// The array below is part of the library's device image: every GPU that loads
// the library holds it until the process exits.  Host code cannot use the
// symbol as a device address, so the address is looked up with
// cudaGetSymbolAddress (with the device current) and passed to the kernels.
// The lookup is a set-up step done on the first call on each device, and
// again whenever the CUDA context current on that device is not the one the
// cached address was taken in (a caller's own context, or a new primary
// context after cudaDeviceReset): an address is valid only in the context
// whose module it came from.  Contexts are told apart by the driver's
// context ID (current_ctx_id), which is never reused within a process.  Every call shares the
// array and leaves the last call's contents in it; the pipeline clears what
// must start at zero at the start of each call.  Calls are serialised by a
// host mutex and each returns only after its GPU work has finished, because
// two calls whose work overlapped on the GPU would race on the shared array.
#include <cmath>
#include <cstring>
#include <mutex>

#include "fec.h"
#include "fec_internal.cuh"

namespace fec {

fec_status status_from_bits(uint32_t s);  // fec_api.cu

namespace {

constexpr int64_t kMaxPoints = FEC_NOALLOC_MAX_POINTS;
constexpr uint32_t kSlabCap = 65536;                 // slab entries (brick rows of 16 major-axis cells)
constexpr size_t kScratchBytes = (size_t)16 << 20;   // 16 MiB per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// The array's device address in one context of one device.
struct DeviceSlot {
    unsigned long long ctx_id = 0;  // driver context ID the address belongs to (0: none)
    void *base = nullptr;
    int sms = 0;
};

std::mutex g_mu;
DeviceSlot g_slot[kMaxDevices];

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
}  // namespace fec

using namespace fec;

extern "C" fec_status fec_cluster_noalloc(const float *xyz, int64_t n, float d, int64_t min_size,
                                          int64_t max_size, int32_t *labels,
                                          int32_t *num_clusters, void *cuda_stream)
{
    if (!num_clusters || n < 0 || n > kMaxPoints) return FEC_ERR_INVALID_ARG;
    if (!std::isfinite(d) || !(d > 0.0f)) return FEC_ERR_INVALID_ARG;
    if (min_size < 0 || max_size < min_size) return FEC_ERR_INVALID_ARG;
    if (n > 0 && (!xyz || !labels)) return FEC_ERR_INVALID_ARG;
    *num_clusters = 0;
    if (n == 0) return FEC_OK;

    std::lock_guard<std::mutex> lock(g_mu);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return FEC_ERR_CUDA;
    DeviceSlot &slot = g_slot[dev];
    // Set-up: the device address of the array in the current context (first
    // call on this device, or the context changed since).
    const unsigned long long ctx_id = current_ctx_id();
    if (!slot.base || ctx_id == 0 || ctx_id != slot.ctx_id) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
            cudaGetLastError();
            slot = DeviceSlot();
            return FEC_ERR_CUDA;
        }
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            sms < 1) {
            slot = DeviceSlot();
            return FEC_ERR_CUDA;
        }
        slot.base = ptr;
        slot.sms = sms;
        slot.ctx_id = current_ctx_id();  // the lookup made a context current if none was
    }
    Workspace ws;
    ws.device = dev;
    ws.sms = slot.sms;
    {
        Workspace probe;
        probe.sms = ws.sms;
        if (workspace_layout(probe, nullptr, (size_t)kMaxPoints, kSlabCap) > kScratchBytes)
            return FEC_ERR_OOM;  // cannot happen with the constants above; checked anyway
    }
    workspace_layout(ws, slot.base, (size_t)kMaxPoints, kSlabCap);
    cudaStream_t st = (cudaStream_t)cuda_stream;

    Params prm = make_params((uint32_t)n, d);
    if (prm.slab_cap > kSlabCap) prm.slab_cap = kSlabCap;  // wider clouds are rejected on device

    const float *xin = xyz;
    if (!on_device(xyz)) {
        if (cudaMemcpyAsync(ws.xyz, xyz, (size_t)n * 12, cudaMemcpyHostToDevice, st) != cudaSuccess)
            return FEC_ERR_CUDA;
        xin = ws.xyz;
    }
    const bool dev_out = on_device(labels);
    int32_t *lout = dev_out ? labels : ws.labels;

    // The same stages as fec_cluster, on the static workspace.
    FrontArgs fa;
    fa.single = true;
    fa.min_size = min_size;
    fa.max_size = max_size;
    cudaError_t e = enqueue_cluster(ws, xin, prm, fa, lout, true, st);
    if (e == cudaSuccess && !dev_out)
        e = cudaMemcpyAsync(labels, ws.labels, (size_t)n * 4, cudaMemcpyDeviceToHost, st);
    uint32_t status_bits = 0, k = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&status_bits, &ws.plan->status, sizeof(uint32_t),
                            cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&k, &ws.plan->kept_n, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return FEC_ERR_CUDA;
    }
    const fec_status s = status_from_bits(status_bits);
    if (s == FEC_OK) *num_clusters = (int32_t)k;
    return s;
}
