/*
 * fec.h -- C ABI of the GB300 exact Euclidean clustering library (FEC,
 * "Fast Euclidean Clustering for Point Cloud Segmentation", arxiv 2208.07678).
 *
 * The library labels every point of an unorganised 3-D cloud with the
 * connected component of the graph that joins two points when their
 * Euclidean distance is at most d (Eq. 1, Section 2.2), drops components
 * whose size lies outside [min_size, max_size] (the size bounds shared with
 * PCL's Euclidean cluster extraction, Section 3.1; Algorithm 1's Th_max is
 * read as max_size), and numbers the kept components 0..k-1 in increasing
 * order of their smallest point index.  Dropped points get label -1.
 *
 * Exactness.  Coordinates are quantised to integer units of 1/1024 m,
 * q = rint(x * 1024) (round half to even), and two points join iff
 * dx^2 + dy^2 + dz^2 <= T2 with T2 = floor((d * 1024)^2) computed in double.
 * The result is unique, so labels are bit-identical run to run and to any
 * correct implementation of the same definition.
 *
 * Limits.  0 <= n <= FEC_MAX_POINTS.  |q| < 2^23 on every axis (|x| < 8192 m).
 * d finite and > 0.  0 <= min_size <= max_size (INT64_MAX = unbounded).  The
 * uniform grid with cell side about d over the cloud's bounding box must be
 * addressable with a 61-bit cell key (always true for d >= 1 cm over an
 * 8 km cube); otherwise FEC_ERR_OUT_OF_RANGE.
 *
 * Memory.  Every buffer passed in is owned by the caller.  A context owns its
 * device workspace and grows it on demand within mem_budget_bytes.  Pointers
 * may be host or device memory (detected per call with
 * cudaPointerGetAttributes); host buffers are staged through the context.
 *
 * Errors.  No call throws or aborts.  On an error the outputs are unspecified
 * and nothing leaks.  A CUDA error leaves the context usable only if the
 * device context itself survived.
 */
#ifndef FEC_H
#define FEC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FEC_MAX_POINTS ((int64_t)1 << 30)

typedef enum {
    FEC_OK = 0,
    FEC_ERR_INVALID_ARG = 1,    /* bad pointer, n, d, or size bounds */
    FEC_ERR_NONFINITE = 2,      /* a coordinate is NaN or +-Inf */
    FEC_ERR_OUT_OF_RANGE = 3,   /* |rint(x*1024)| >= 2^23, or grid key > 61 bits */
    FEC_ERR_OOM = 4,            /* workspace above mem_budget_bytes, or cudaMalloc failed */
    FEC_ERR_CUDA = 5,           /* a CUDA runtime call failed */
    FEC_ERR_NOT_CONVERGED = 6,  /* a bounded device loop hit its iteration cap */
    FEC_ERR_NOT_READY = 7,      /* fec_serve_poll: request still queued or running */
    FEC_ERR_BUSY = 8,           /* fec_serve_submit: request can never fit the budget / queue full */
    FEC_ERR_TIMEOUT = 9,        /* serving: the request's deadline passed before it started */
    FEC_ERR_INTERNAL = 10       /* debug builds (FEC_DEBUG) only: a device bounds check failed */
} fec_status;

typedef struct fec_ctx fec_ctx;

typedef struct {
    int device;               /* CUDA device ordinal */
    size_t mem_budget_bytes;  /* cap on device workspace; 0 = no cap */
    void *cuda_stream;        /* cudaStream_t to run on; NULL = a stream owned by the context */
    const char *autotune_cache; /* path of the batch tuner's cache file; NULL = in memory only */
} fec_options;

/* Per-call counters of the last fec_cluster / fec_cluster_batch call. */
typedef struct {
    int64_t n;                /* points */
    int64_t cells;            /* occupied grid cells (side S = 2h units) */
    int64_t subcells;         /* occupied sub-cells (side h units; each is a clique) */
    int64_t num_clusters;     /* kept clusters */
    int64_t key_bits;         /* bits of the sort key actually used */
    int64_t workspace_bytes;  /* device workspace held by the context */
    int32_t R;                /* floor(sqrt(T2)): largest joined offset per axis, units */
    int32_t h;                /* sub-cell side, units */
    int64_t T2;               /* squared join radius, units^2 */
    int64_t pair_checks;      /* sub-cell pairs examined by the neighbour step */
    int64_t pair_box_joins;   /* ... joined from their bounding boxes alone */
    int64_t pair_point_tests; /* ... that needed point-level tests */
    int64_t pair_same_root;   /* ... of those, skipped as already joined */
    int64_t point_evals;      /* point-level distance evaluations */
    int64_t pairs_queued;     /* pairs deferred to the warp-per-pair pass */
    int64_t boundary_edges;   /* edges between regions, joined after the region pass */
} fec_stats;

/* Create a context on options->device (options may be NULL: device 0, no
 * budget, own stream).  *out receives the context.  Thread-compatible: one
 * thread at a time per context for fec_cluster / fec_cluster_batch. */
fec_status fec_create(const fec_options *options, fec_ctx **out);

/* Destroy a context; waits for its serving requests and frees everything.
 * NULL is a no-op. */
void fec_destroy(fec_ctx *ctx);

/* Cluster one cloud (Eq. 1; Algorithm 1's input and output).
 *   xyz          float32 [n][3], x y z interleaved, host or device memory.
 *   n            number of points, 0 <= n <= FEC_MAX_POINTS.
 *   d            join radius in metres (distance <= d joins), finite, > 0.
 *   min_size, max_size  inclusive size bounds of kept clusters.
 *   labels       int32 [n], host or device memory, written in input order:
 *                0..k-1 by smallest point index, -1 for dropped points.
 *                After any status other than FEC_OK its contents are
 *                unspecified.
 *   num_clusters host int32: k, the number of kept clusters.
 * Synchronous: returns after labels and num_clusters are written.
 * Precedence of data errors: NONFINITE before OUT_OF_RANGE. */
fec_status fec_cluster(fec_ctx *ctx, const float *xyz, int64_t n, float d, int64_t min_size,
                       int64_t max_size, int32_t *labels, int32_t *num_clusters);

/* Cluster nb independent frames in one device pass (frames of uneven size,
 * per-frame d and size bounds).  Frame f holds points offsets[f] ..
 * offsets[f+1]-1 of the concatenated xyz.  Labels are frame-local (each frame
 * numbered 0..k_f-1 exactly as fec_cluster would number it alone).  Frames
 * that share a radius run together as one pass of the pipeline (a sort
 * segmented by frame, a cell table and size filter per frame), radius groups
 * run concurrently, and the whole batch is captured into a CUDA graph that is
 * replayed for later batches of the same shape (offsets, radii, bounds and
 * buffers); the launch configuration is tuned on the first batch of a shape
 * (see fec_options.autotune_cache).
 *   xyz          float32 [offsets[nb]][3], host or device.
 *   offsets      host int64 [nb+1], offsets[0] = 0, non-decreasing,
 *                offsets[nb] <= FEC_MAX_POINTS.
 *   d, min_size, max_size  host arrays [nb].
 *   labels       int32 [offsets[nb]], host or device.
 *   num_clusters host int32 [nb].
 * Same exactness and error rules as fec_cluster; a data error in any frame
 * fails the whole call. */
fec_status fec_cluster_batch(fec_ctx *ctx, const float *xyz, const int64_t *offsets, int32_t nb,
                             const float *d, const int64_t *min_size, const int64_t *max_size,
                             int32_t *labels, int32_t *num_clusters);

/* Serving: submit one request.  The input is copied into the engine's device
 * input arena (no device allocation per request): from pageable host memory
 * the call returns once the copy has been staged, so the caller may reuse
 * its buffer; from pinned host or device memory the copy runs asynchronously
 * and the buffer must stay unchanged until fec_serve_poll returns a final
 * status for the ticket.  labels_out (host memory, int32 [n]) must stay
 * valid until then too.  Requests
 * run concurrently on the context's device as workspace slots and the memory
 * budget allow (continuous batching); each result equals fec_cluster on that
 * request alone.  Memory: the engine's whole device footprint stays within
 * the context's budget (40 GiB when it has none): a quarter of it, at most
 * 2 GiB, is the input arena, the rest the slots' workspaces.
 * FEC_ERR_BUSY, and no ticket, when the request can never fit the slots'
 * memory, when 4,096 requests are already waiting, or when the arena has no
 * room for its input right now (submit again once earlier requests finish).
 * Thread-safe. */
fec_status fec_serve_submit(fec_ctx *ctx, const float *xyz, int64_t n, float d, int64_t min_size,
                            int64_t max_size, int32_t *labels_out, uint64_t *ticket);

/* Serving: fec_serve_submit with a deadline.  deadline_us > 0: if the
 * request has not started deadline_us microseconds after submit, it is
 * dropped without running and completes with FEC_ERR_TIMEOUT (labels_out
 * untouched); <= 0: no deadline.  Thread-safe. */
fec_status fec_serve_submit_deadline(fec_ctx *ctx, const float *xyz, int64_t n, float d,
                                     int64_t min_size, int64_t max_size, int32_t *labels_out,
                                     int64_t deadline_us, uint64_t *ticket);

/* Serving: wait up to timeout_ms (0 = just check, <0 = forever) for a ticket.
 * FEC_OK: labels_out and *num_clusters are final and the ticket is released.
 * FEC_ERR_NOT_READY: still queued or running when the wait ended; the ticket
 * stays valid.  FEC_ERR_INVALID_ARG: unknown ticket.  Any other status
 * (FEC_ERR_TIMEOUT for a request whose deadline passed, or a clustering
 * error) is the request's final status and releases the ticket.
 * Thread-safe. */
fec_status fec_serve_poll(fec_ctx *ctx, uint64_t ticket, int32_t *num_clusters, int timeout_ms);

/* Serving: fec_serve_poll that also reports when the request completed:
 * *done_ns (if not NULL) is the CLOCK_MONOTONIC time, in nanoseconds, at
 * which its labels and cluster count were final in host memory (set with
 * FEC_OK and with a final error).  Lets a caller measure submit-to-completion
 * latency independently of how often it polls.  Thread-safe. */
fec_status fec_serve_poll_timed(fec_ctx *ctx, uint64_t ticket, int32_t *num_clusters,
                                int timeout_ms, int64_t *done_ns);

/* Serving counters since the engine started (times in nanoseconds). */
typedef struct {
    int64_t submitted;         /* requests accepted by submit */
    int64_t completed;         /* requests that ran (any final status but FEC_ERR_TIMEOUT) */
    int64_t rejected;          /* submits refused with FEC_ERR_BUSY */
    int64_t expired;           /* requests dropped at their deadline (FEC_ERR_TIMEOUT) */
    int64_t queued;            /* requests waiting for a slot now */
    int64_t queue_max;         /* most requests ever waiting at once */
    int64_t queue_wait_ns_sum; /* submit -> start, summed over started requests */
    int64_t queue_wait_ns_max;
    int64_t run_ns_sum;        /* start -> completion, summed */
    int64_t run_ns_max;
    int64_t arena_bytes;       /* size of the device input arena */
} fec_serve_stats;

fec_status fec_serve_get_stats(fec_ctx *ctx, fec_serve_stats *out);

/* Counters of the last fec_cluster / fec_cluster_batch call on ctx. */
fec_status fec_get_stats(const fec_ctx *ctx, fec_stats *out);

/* Tracing: per-kernel device time, measured with CUDA events recorded on
 * the context's stream after every launch of fec_cluster /
 * fec_cluster_batch while enabled.  The time charged to a launch is the
 * interval since the previous event on the stream (the launch itself plus any
 * idle gap before it).  Enabling clears the accumulators. */
typedef struct {
    const char *name;    /* kernel or copy name (static string) */
    int64_t launches;    /* launches recorded */
    double total_ms;     /* summed device time */
} fec_trace_entry;

fec_status fec_trace_enable(fec_ctx *ctx, int enable);

/* Copy up to cap accumulated entries into out (out may be NULL to count);
 * returns the number of distinct names, or -1 on a bad argument. */
int fec_trace_read(const fec_ctx *ctx, fec_trace_entry *out, int cap);

/* Failure-path control.  Every loop on the device that waits on other
 * blocks (the decoupled look-back of the radix sort and of the cell-table
 * scan) or walks the global union-find (finds, unions and the flatten) is
 * bounded: after wait_cap spin iterations, or union_cap steps, it gives up,
 * the call's remaining kernels return at once, and the call returns
 * FEC_ERR_NOT_CONVERGED with its labels unspecified (never FEC_OK with wrong
 * labels).  The caps of the Section 2.2 pipeline are FEC_DEFAULT_WAIT_CAP
 * and FEC_DEFAULT_UNION_CAP, far above what any correct run needs; this call
 * sets them for later fec_cluster calls on ctx (not the batch or serving
 * paths), so that tests can make a wait or a union run out on purpose
 * (wait_cap 0: any wait gives up at once; union_cap 0: any find that has to
 * walk, or any union, gives up).  The device and the context stay usable:
 * set the defaults back and the next call is exact again.  Thread-compatible
 * like fec_cluster. */
#define FEC_DEFAULT_WAIT_CAP ((uint32_t)1 << 22)
#define FEC_DEFAULT_UNION_CAP ((uint32_t)1 << 20)
fec_status fec_set_iteration_caps(fec_ctx *ctx, uint32_t wait_cap, uint32_t union_cap);

/* Device workspace bytes fec_cluster needs for n points at radius d. */
int64_t fec_workspace_bytes(int64_t n, float d);

/* Largest cloud fec_cluster_noalloc accepts. */
#define FEC_NOALLOC_MAX_POINTS ((int64_t)32768)

/* Cluster one cloud without allocating any memory.  The paper has no
 * counterpart: this entry point exists for callers that cannot call
 * cudaMalloc or any allocator -- code running inside a host application
 * that owns all device memory through its own pool, real-time loops where an
 * allocation (and its implicit device synchronisation) is not allowed, or
 * plug-ins loaded by a framework that forbids allocating outside its
 * allocator.  It computes exactly what fec_cluster computes, with the same
 * argument rules, but its workspace is a 16 MiB array that is part of the
 * library's device image (every GPU that loads the library holds it until
 * the process exits), so it needs no context and allocates nothing.
 *   xyz, labels  caller-owned, host or device memory, as for fec_cluster.
 *   n            at most FEC_NOALLOC_MAX_POINTS; larger n gives
 *                FEC_ERR_INVALID_ARG.  A cloud longer than 1,048,576 grid
 *                cells (of side about d) along its longest axis gives
 *                FEC_ERR_OUT_OF_RANGE, and one that needs more boundary
 *                lists than the array holds gives FEC_ERR_OOM.
 *   cuda_stream  cudaStream_t to run on (NULL = the default stream).
 * The first call on each device does a set-up step: it looks up the array's
 * device address (cudaGetSymbolAddress, with that device current), which is
 * then reused; make that first call before any stream capture begins.  The
 * address belongs to the CUDA context it was taken in, so the set-up is
 * repeated when a later call finds a different context current on the device
 * (the caller's own context, or a new one after cudaDeviceReset).  All calls
 * share the one array, which keeps the last call's contents: each call clears
 * what must start at zero, and calls are serialised inside the library and
 * return only when their GPU work is done (the call synchronises
 * cuda_stream), because calls whose GPU work overlapped would race on the
 * array. */
fec_status fec_cluster_noalloc(const float *xyz, int64_t n, float d, int64_t min_size,
                               int64_t max_size, int32_t *labels, int32_t *num_clusters,
                               void *cuda_stream);

/* Static string naming a status. */
const char *fec_status_string(fec_status status);

#ifdef __cplusplus
}
#endif

#endif /* FEC_H */
