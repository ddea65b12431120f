// fec_internal.cuh -- device-side plan, workspace layout and helpers shared by
// the CUDA translation units of the library (not part of the public ABI).
//
// The pipeline for one cloud (Eq. 1 as connected components; Algorithm 1's
// input/output) runs without host round trips until the final read-back:
//
//   a1  quantise + bounding box + validation, plan      k_bbox (its last block: plan_body)
//   a1  grid keys (cell of side S=2h, sub-cell bits)    k_keys (+ radix digit histograms)
//   a2  LSD radix sort of (key, index), onesweep        k_onesweep (per 8-bit digit)
//   a3  cell table: sub-cell/cell heads, scan, gather   k_cells, k_subcell_stats (+ slab index)
//   a4  neighbour lists, neighbour test + union         k_nbrs, k_region, k_edges, k_pairs
//       (27-cell stencil, region-local union-find)
//   a5  flatten + component statistics                  k_flatten_stats
//   a6  size filter, order by smallest index, labels    k_kept, sort, k_rank, k_labels
//
// Sizes that only the device knows (key bits, cells, sub-cells, kept count)
// live in Plan / SortCtl in device memory; kernels read them and grid-stride.
#pragma once

#include <atomic>
#include <cstddef>
#include <cstdint>
#include <type_traits>
#include <utility>

#include <cuda_runtime.h>

#include "fec.h"

namespace fec {

// Status bits set by kernels (Plan::status).
enum : uint32_t {
    ST_NONFINITE = 1u << 0,
    ST_OUT_OF_RANGE = 1u << 1,
    ST_KEY_OVERFLOW = 1u << 2,     // cell key would need > 61 bits
    ST_WAIT_TIMEOUT = 1u << 3,     // a look-back wait hit its cap
    ST_UNION_CAP = 1u << 4,        // a union/find loop hit its cap
    ST_SIZE_OVERFLOW = 1u << 5,    // a device count exceeded its buffer
    ST_QUEUE_OVERFLOW = 1u << 6,   // more boundary edges / pairs than the lists hold
    ST_DEBUG_BOUNDS = 1u << 7,     // FEC_DEBUG builds: a device bounds check failed
};
// Status bits after which a call's remaining kernels return at once: a wait
// or union loop gave up, or a device count went out of range, so later
// stages would index through wrong offsets.
constexpr uint32_t kAbortBits = ST_WAIT_TIMEOUT | ST_UNION_CAP | ST_SIZE_OVERFLOW | ST_DEBUG_BOUNDS;

// Work counters of the union step (Plan::ctr).
enum {
    CTR_PAIRS = 0,        // sub-cell pairs examined
    CTR_BOX_JOINS = 1,    // pairs joined by the box-diameter test alone
    CTR_POINT_TESTS = 2,  // pairs that needed point-level tests
    CTR_SAME_ROOT = 3,    // ... of which skipped because already joined
    CTR_POINT_EVALS = 4,  // point-level distance evaluations
    CTR_QUEUED = 5,       // pairs queued for the warp-per-pair kernel
    CTR_EDGES = 6,        // edges between regions joined after the region step
};

// Kernels are launched with programmatic stream serialisation (grid_enter(),
// launch()); 0 gives plain stream order.
#ifndef FEC_PDL
#define FEC_PDL 1
#endif

constexpr int kRadixBits = 8;
constexpr int kRadixBins = 1 << kRadixBits;
constexpr int kMaxPasses = 8;            // 64-bit keys
#ifndef FEC_SORT_THREADS
#define FEC_SORT_THREADS 256
#endif
#ifndef FEC_SORT_IPT
#define FEC_SORT_IPT 10
#endif
#ifndef FEC_SORT_MINB
#define FEC_SORT_MINB 4
#endif
constexpr int kSortThreads = FEC_SORT_THREADS;
constexpr int kSortIPT = FEC_SORT_IPT;   // items per thread
constexpr int kSortMinBlocks = FEC_SORT_MINB;
constexpr int kSortTile = kSortThreads * kSortIPT;   // 2560 keys per tile
constexpr int kScanThreads = 256;
constexpr int kScanIPT = 8;
constexpr int kScanTile = kScanThreads * kScanIPT;   // 2048 positions per tile
constexpr int kBigSubcell = 64;          // sub-cells above this size are reduced by a warp,
constexpr int kHugeSubcell = 2048;       //   above this size by a block
constexpr uint32_t kMaxFramesPerCall = 4096;  // frames of one call (one radius group)
constexpr uint32_t kRegionScratch = 32768;  // undecided in-region pairs kept per block
#ifndef FEC_REGION_CELLS
#define FEC_REGION_CELLS 1024
#endif
#ifndef FEC_REGION_THREADS
#define FEC_REGION_THREADS 512
#endif
#ifndef FEC_REGION_BLOCKS
#define FEC_REGION_BLOCKS 2
#endif
constexpr uint32_t kRegionCellsPerBlock = FEC_REGION_CELLS;
#ifndef FEC_REGION_TAIL_DIV
#define FEC_REGION_TAIL_DIV 2
#endif
constexpr uint32_t kRegionTailDiv = FEC_REGION_TAIL_DIV;  // default split of the last regions
constexpr int kRegionThreads = FEC_REGION_THREADS;
constexpr int kRegionBlocksPerSM = FEC_REGION_BLOCKS;
constexpr uint32_t kWaitCap = 1u << 22;  // default: spin iterations before a wait gives up
constexpr uint32_t kUnionCap = 1u << 20; // default: steps of one union or find before it gives up
static_assert(kWaitCap == FEC_DEFAULT_WAIT_CAP && kUnionCap == FEC_DEFAULT_UNION_CAP,
              "the header's default caps");

// Control block of one radix sort (device memory).
struct SortCtl {
    uint32_t n;         // number of keys
    uint32_t npasses;   // 8-bit digit passes to run
    uint32_t key64;     // 1: 64-bit keys, 0: 32-bit keys
    uint32_t parity;    // pass p uses look-back array (p + parity) & 1, which starts clear
    uint32_t wait_cap;  // spin iterations of a look-back wait before it gives up
    uint32_t hist[kMaxPasses][kRadixBins];   // digit counts of every pass (unsegmented sorts)
    uint32_t tile_counter[kMaxPasses];       // dynamic tile ids of every pass
};

// One frame of a call.  A call clusters nf independent clouds ("frames")
// that share the radius d in one pass of the pipeline: frame f's points are
// rows in_off .. in_off+n-1 of the call's input (and of its labels) and
// positions pos_off .. pos_off+n-1 of the sorted arrays; keys are
// frame-local, the sort is segmented by frame (its tiles never straddle
// two frames), cells and sub-cells of different frames never meet, and the
// kept components of each frame are numbered from 0.  A single cloud is the
// frame table {0, 0, n}.  Static fields are written by the host (or by
// k_init for a single cloud); the rest on the device.
struct __align__(16) Frame {
    uint32_t in_off;     // first input row
    uint32_t pos_off;    // first sorted position
    uint32_t n;          // points (> 0)
    uint32_t tile0;      // first tile of the frame in the sort (kSortTile points each)
    long long min_size, max_size;  // inclusive size bounds of kept clusters
    int32_t lo[3];       // bounding box of q per original axis (device)
    uint32_t kept;       // kept clusters (device)
    int32_t hi[3];
    uint32_t nslab;      // slab-index entries: brick rows of the frame's major cell coordinate (device)
    uint32_t slab_base;  // first slab-index entry of the frame (device)
    uint32_t pad[3];
};

// Frame of a sorted position, of an input row, of a sort tile: the last
// frame whose first one is at or before it (frames are in input order and
// none is empty, so these offsets increase strictly).
__device__ __forceinline__ uint32_t frame_search(const Frame *__restrict__ fr, uint32_t nf,
                                                 uint32_t v, int field)
{
    uint32_t lo = 0, hi = nf;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        const uint32_t at = field == 0 ? fr[mid].pos_off : (field == 1 ? fr[mid].in_off : fr[mid].tile0);
        if (at <= v) lo = mid;
        else hi = mid;
    }
    return lo;
}
__device__ __forceinline__ uint32_t frame_of_pos(const Frame *fr, uint32_t nf, uint32_t p)
{
    return nf > 1 ? frame_search(fr, nf, p, 0) : 0u;
}
__device__ __forceinline__ uint32_t frame_of_row(const Frame *fr, uint32_t nf, uint32_t i)
{
    return nf > 1 ? frame_search(fr, nf, i, 1) : 0u;
}
__device__ __forceinline__ uint32_t frame_of_tile(const Frame *fr, uint32_t nf, uint32_t t)
{
    return nf > 1 ? frame_search(fr, nf, t, 2) : 0u;
}

// Per-call plan (device memory), written by plan_body / k_cells / kernels.
struct Plan {
    // written by plan_body for the host: status, key64, passes of the main
    // sort, key bits (one 16-byte read-back decides which sort passes to
    // launch)
    uint32_t front[4];
    int32_t perm[3];           // permuted axis p -> original axis (p0 major .. p2 minor)
    uint32_t bits[3];          // bits of the cell coordinate per permuted axis
    uint32_t key_bits;         // total sort-key bits (cell key bits + 3)
    uint32_t status;           // ST_* bits
    uint32_t M_s, M_c;         // occupied sub-cells and cells
    uint32_t n_big;            // sub-cells with more than kBigSubcell points (up to kHugeSubcell)
    uint32_t n_huge;           // sub-cells with more than kHugeSubcell points
    uint32_t scan_tile_counter;
    uint32_t pairq_n;           // pairs queued for point-level tests
    uint32_t use_cols;          // 1: the dense column index covers the grid
    uint32_t edges_n;           // boundary edges emitted by the neighbour step
    uint32_t region_counter;    // dynamic regions of the neighbour step
    uint32_t slab_need;         // slab-index entries the frames need (all frames)
    uint32_t rank_tile_counter; // dynamic tiles of the kept-component ranking scan
    uint32_t bbox_done;         // blocks of k_bbox finished (the last one lays out the plan)
    uint32_t kept_n;            // kept components
    unsigned long long ctr[8];  // work counters of the union step (CTR_*)
    // Everything above is the call's summary, read back by the host in one
    // copy of offsetof(Plan, sort) bytes after the call's last kernel.
    SortCtl sort;              // main (key, index) sort
};

// Host-side constants of one call, passed by value.
struct Params {
    uint32_t n;
    int64_t T2;          // squared join radius in units^2
    int32_t R;           // floor(sqrt(T2))
    int32_t h;           // sub-cell side (units); cells have side S = 2h
    int32_t S;
    uint32_t slab_cap;   // entries of the slab index (>= max major cell coordinate + 1)
    uint32_t col_bits;   // log2 of the dense column index capacity
    uint32_t packed;     // 1: sort values carry the in-cell offsets (S <= 1024)
    // floor(rel / S) == (rel * div_m) >> div_s for every rel < 2^24
    uint32_t div_m, div_s;
    uint32_t wait_cap = kWaitCap;    // iterations of a look-back wait before it gives up
    uint32_t union_cap = kUnionCap;  // steps of a union or find before it gives up
    // frames of the call (see Frame): nf, their sort tiles, and the length
    // of the call's input / label arrays (rows)
    uint32_t nf = 1;
    uint32_t ntiles = 0;
    uint32_t rows = 0;
    // tunables: largest region of the neighbour step (cells, 32..1024), how
    // many times smaller its last grid-full of regions is cut (its schedule),
    // and the sub-cell size above which a warp, not a thread, reduces a
    // sub-cell
    uint32_t region_cells = kRegionCellsPerBlock;
    uint32_t region_tail = kRegionTailDiv;
    uint32_t big_subcell = kBigSubcell;
};

// Quantised point record in cell order: coordinates and the original index.
struct __align__(16) Rec {
    int32_t x, y, z;
    uint32_t idx;
};

// Per sub-cell: bounding box, first record, record count, smallest index.
struct __align__(16) SubBox {
    int32_t lx, ly, lz;
    uint32_t start;
    int32_t hx, hy, hz;
    uint32_t count;
};

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------

// q = rint(x * 1024) (round half to even).  x * 1024 is exact in float.
// Returns 0 if valid, 1 if non-finite, 2 if |q| >= 2^23.
__device__ __forceinline__ int quantize1(float x, int32_t &q)
{
    if (!isfinite(x)) {
        q = 0;
        return 1;
    }
    float r = rintf(x * 1024.0f);
    if (fabsf(r) >= 8388608.0f) {
        q = 0;
        return 2;
    }
    q = __float2int_rn(r);
    return 0;
}

// Layout of a cell key (the sort key without its 3 sub-cell bits).  With
// b0, b1, b2 bits of cell coordinate along the permuted axes p0 (major), p1,
// p2 (minor), the columns (c0, c1) are grouped in bricks of 2^B0 x 2^B1
// columns (B = FEC_KEY_BRICK, less on an axis with fewer bits):
//   [ c0 >> B0 | c1 >> B1 | c0 mod 2^B0 | c1 mod 2^B1 | c2 ]
// so that a run of consecutive cells (a region of the neighbour step) is a
// compact block of columns instead of a one-cell-thick slice along p0: fewer
// neighbour pairs cross regions.  (Host and device: a CPU test checks the
// layout's round trips, tests/key_layout_main.cu.)  A column's cells stay consecutive (c2 is
// the lowest field), and the "slab" of c0 is the key range of its brick row,
// c0 >> B0.
#ifndef FEC_KEY_BRICK
#define FEC_KEY_BRICK 4
#endif
struct CellKeyLayout {
    uint32_t b0, b1, b2, B0, B1;
    __host__ __device__ __forceinline__ void load(const Plan *plan)
    {
        b0 = plan->bits[0];
        b1 = plan->bits[1];
        b2 = plan->bits[2];
        B0 = b0 < (uint32_t)FEC_KEY_BRICK ? b0 : (uint32_t)FEC_KEY_BRICK;
        B1 = b1 < (uint32_t)FEC_KEY_BRICK ? b1 : (uint32_t)FEC_KEY_BRICK;
    }
    // cell key of column (c0, c1) at c2 = 0
    __host__ __device__ __forceinline__ unsigned long long column(unsigned long long c0, unsigned long long c1) const
    {
        const unsigned long long m0 = (1ull << B0) - 1, m1 = (1ull << B1) - 1;
        return ((c0 >> B0) << (b2 + b1 + B0)) | ((c1 >> B1) << (b2 + B1 + B0)) | ((c0 & m0) << (b2 + B1)) |
               ((c1 & m1) << b2);
    }
    __host__ __device__ __forceinline__ void decode(unsigned long long ck, unsigned long long &c0,
                                           unsigned long long &c1, unsigned long long &c2) const
    {
        const unsigned long long m0 = (1ull << B0) - 1, m1 = (1ull << B1) - 1;
        c2 = ck & ((1ull << b2) - 1);
        c1 = (((ck >> (b2 + B1 + B0)) & ((1ull << (b1 - B1)) - 1)) << B1) | ((ck >> b2) & m1);
        c0 = ((ck >> (b2 + b1 + B0)) << B0) | ((ck >> (b2 + B1)) & m0);
    }
    // slab (brick row) of a major coordinate
    __host__ __device__ __forceinline__ unsigned long long slab_of(unsigned long long c0) const { return c0 >> B0; }
};

// Grid coordinates of a quantised point under the plan.  The sort key is
// the cell key (CellKeyLayout) above [s_p0 s_p1 s_p2] (s = which half of the
// cell along each permuted axis), so every original axis a has fixed places
// in it: the low lw[a] bits of its cell coordinate at bit lsh[a], the other
// hw[a] bits at bit hsh[a], and its half at bit kbit[a].  These are resolved
// once in load(), so a point's key is a few shifts with no per-point axis
// selection.
struct GridMap {
    int32_t lo[3];
    uint32_t lsh[3], hsh[3], lw[3], hw[3], kbit[3];
    int32_t S, h;
    uint32_t div_m, div_s;  // floor(rel / S) == (rel * div_m) >> div_s for rel < 2^24

    __host__ __device__ __forceinline__ void load(const Plan *plan, const Params &prm, const Frame &fr)
    {
        CellKeyLayout L;
        L.load(plan);
#pragma unroll
        for (int a = 0; a < 3; ++a) {  // constant indices only (no local memory)
            lo[a] = fr.lo[a];
            const int p = plan->perm[0] == a ? 0 : (plan->perm[1] == a ? 1 : 2);
            // p0: low B0 bits at b2 + B1, the rest at b2 + b1 + B0; p1: low B1
            // bits at b2, the rest at b2 + B1 + B0; p2: all b2 bits at 0
            lw[a] = p == 0 ? L.B0 : (p == 1 ? L.B1 : L.b2);
            hw[a] = p == 0 ? L.b0 - L.B0 : (p == 1 ? L.b1 - L.B1 : 0u);
            lsh[a] = 3u + (p == 0 ? L.b2 + L.B1 : (p == 1 ? L.b2 : 0u));
            hsh[a] = 3u + (p == 0 ? L.b2 + L.b1 + L.B0 : (p == 1 ? L.b2 + L.B1 + L.B0 : 0u));
            // an empty field holds zeros: shift by 0, never by the key's width
            if (lw[a] == 0) lsh[a] = 0;
            if (hw[a] == 0) hsh[a] = 0;
            kbit[a] = 2u - (uint32_t)p;
        }
        S = prm.S;
        h = prm.h;
        div_m = prm.div_m;
        div_s = prm.div_s;
    }
    // Another frame of the same call: only the grid origin changes.
    __host__ __device__ __forceinline__ void set_frame(const Frame &fr)
    {
#pragma unroll
        for (int a = 0; a < 3; ++a) lo[a] = fr.lo[a];
    }
    // Cell coordinate and offset inside the cell, per original axis.
    __host__ __device__ __forceinline__ void cell_of(const int32_t q[3], uint32_t c[3], uint32_t off[3]) const
    {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const uint32_t rel = (uint32_t)(q[a] - lo[a]);
            c[a] = (uint32_t)(((unsigned long long)rel * div_m) >> div_s);
            off[a] = rel - c[a] * (uint32_t)S;
        }
    }
    // Sort key of a point (KeyT: uint32 when the key has at most 32 bits).
    template <typename KeyT>
    __host__ __device__ __forceinline__ KeyT key_of(const uint32_t c[3], const uint32_t off[3]) const
    {
        KeyT k = 0;
#pragma unroll
        for (int a = 0; a < 3; ++a)
            k |= ((KeyT)(c[a] & ((1u << lw[a]) - 1u)) << lsh[a]) | ((KeyT)(c[a] >> lw[a]) << hsh[a]) |
                 ((KeyT)(off[a] >= (uint32_t)h ? 1u : 0u) << kbit[a]);
        return k;
    }
    // Sort payload of the packed layout: the original index in the low 32
    // bits and the point's offsets inside its cell (original axes x, y, z,
    // 10 bits each, S <= 1024) above it.
    __host__ __device__ __forceinline__ unsigned long long payload_of(const uint32_t off[3], uint32_t idx) const
    {
        return (unsigned long long)idx | ((unsigned long long)off[0] << 32) |
               ((unsigned long long)off[1] << 42) | ((unsigned long long)off[2] << 52);
    }
    // Inverse of key_of() + payload_of(): the quantised coordinates of a point.
    template <typename KeyT>
    __host__ __device__ __forceinline__ void unpack(KeyT key, unsigned long long v, int32_t q[3]) const
    {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const uint32_t c = (uint32_t)((key >> lsh[a]) & (((KeyT)1 << lw[a]) - 1)) |
                               ((uint32_t)((key >> hsh[a]) & (((KeyT)1 << hw[a]) - 1)) << lw[a]);
            q[a] = lo[a] + (int32_t)(c * (uint32_t)S) + (int32_t)((v >> (32 + 10 * a)) & 1023u);
        }
    }
};

// A sub-cell's representative point, stored as its offset from the low corner
// of the sub-cell's box, 10 bits per axis (4 bytes instead of a 16-byte
// record); kNoRep when an offset does not fit (boxes over 1,022 units wide,
// possible only for d above 1 m), which leaves the pair to the point tests.
constexpr uint32_t kNoRep = 0xffffffffu;
__device__ __forceinline__ uint32_t pack_rep(const Rec &r, int32_t lx, int32_t ly, int32_t lz)
{
    const uint32_t ox = (uint32_t)(r.x - lx), oy = (uint32_t)(r.y - ly), oz = (uint32_t)(r.z - lz);
    return (ox < 1023u && oy < 1023u && oz < 1023u) ? (ox | (oy << 10) | (oz << 20)) : kNoRep;
}

__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed(uint32_t *p, uint32_t v)
{
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_relaxed64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed64(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint32_t lanemask_lt()
{
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

// Backoff inside bounded spin loops.
__device__ __forceinline__ void spin_pause(uint32_t it)
{
    if (it > 16) __nanosleep(it > 1024 ? 256 : 32);
}

// Union-find over sub-cells.  Invariant: parent[x] <= x, roots satisfy
// parent[r] == r, so the root of a set is its smallest member.  Every loop
// takes at most `cap` steps; a walk cut short sets ok = false (the caller
// flags ST_UNION_CAP, which stops the rest of the call).
__device__ __forceinline__ uint32_t uf_find(uint32_t *parent, uint32_t x, uint32_t cap, bool &ok)
{
    uint32_t cur = ld_relaxed(parent + x);
    if (cur == x) return x;
    uint32_t prev = x;
    for (uint32_t it = 0; it < cap; ++it) {
        uint32_t next = ld_relaxed(parent + cur);
        if (next == cur) return cur;
        // path halving: prev skips to cur's parent (still an ancestor)
        st_relaxed(parent + prev, next);
        prev = cur;
        cur = next;
    }
    ok = false;
    return cur;
}

// Join the sets of a and b: hook the larger root under the smaller.
// Returns false if a loop hit its cap (the caller flags ST_UNION_CAP).
__device__ __forceinline__ bool uf_unite(uint32_t *parent, uint32_t a, uint32_t b, uint32_t cap)
{
    bool ok = true;
    for (uint32_t it = 0; it < cap; ++it) {
        a = uf_find(parent, a, cap, ok);
        b = uf_find(parent, b, cap, ok);
        if (!ok) return false;
        if (a == b) return true;
        if (a < b) {
            uint32_t t = a;
            a = b;
            b = t;
        }
        // a > b: make b the parent of root a, if a is still a root
        uint32_t old = atomicCAS(parent + a, a, b);
        if (old == a) return true;
        a = old;
    }
    return false;
}

// True when an earlier stage of this call gave up (kAbortBits): the kernel
// must return at once.  Read once at entry, so every block of a kernel that
// waits on its peers decides the same way (blocks that start late and see
// the bit take no tile, so no tile is left unpublished).
__device__ __forceinline__ bool call_aborted(const uint32_t *status)
{
    return (*(volatile const uint32_t *)status & kAbortBits) != 0;
}
// The same decision taken once per block (thread 0 reads, every thread gets
// its answer), for kernels with block barriers: a bit set by another block
// between two threads' reads cannot split the block.  Every thread of the
// block must call it.
__device__ __forceinline__ bool block_aborted(const uint32_t *status)
{
    return __syncthreads_or(threadIdx.x == 0 && call_aborted(status)) != 0;
}

// Debug builds (-DFEC_DEBUG=1, libfec_debug.so) check the indices of the
// gathers and scatters that depend on device-computed offsets.
// FEC_IN_BOUNDS(status, i, n) is true when i < n; otherwise it sets
// ST_DEBUG_BOUNDS in the call's status (the call ends with FEC_ERR_INTERNAL
// and its later kernels return at once) and the caller skips the access.
// Release builds compile it to `true` and evaluate neither i nor n.
#ifndef FEC_DEBUG
#define FEC_DEBUG 0
#endif
#if FEC_DEBUG
__device__ __forceinline__ bool debug_in_bounds(uint32_t *status, unsigned long long i,
                                                unsigned long long n)
{
    if (i < n) return true;
    atomicOr(status, ST_DEBUG_BOUNDS);
    return false;
}
#define FEC_IN_BOUNDS(status, i, n) \
    ::fec::debug_in_bounds((status), (unsigned long long)(i), (unsigned long long)(n))
#else
#define FEC_IN_BOUNDS(status, i, n) true
#endif

// Programmatic dependent launch.  Kernels are launched (launch() below) so
// that the launch of a kernel is prepared while the previous kernel of the
// stream is still running, and its blocks start as that kernel's blocks
// exit, without the gap of a plain stream dependency.  Every kernel calls
// grid_enter() before its first access to global memory: it waits until the
// previous kernel has finished and its writes are visible (so ordering stays
// transitive along the stream: each kernel finishes only after its
// predecessor has).  No kernel signals its dependents early: resident blocks
// of the next kernel waiting beside a running one measured slower (map, batch)
// than dependents released as blocks exit.  Outside such a launch the wait
// returns at once.
__device__ __forceinline__ void grid_enter()
{
#if FEC_PDL
    asm volatile("griddepcontrol.wait;" ::: "memory");
#endif
}

// ---------------------------------------------------------------------------
// Host launchers (one stream; all asynchronous)
// ---------------------------------------------------------------------------

// Device workspace of one context, carved from a single allocation.  All
// arrays are sized for cap_n points (every per-cell / per-sub-cell array is
// bounded by the number of points).
struct Trace;  // per-launch CUDA-event tracing (fec_api.cu)

struct Workspace {
    Trace *trace = nullptr;        // non-null while tracing is enabled
    int device = 0;
    int sms = 0;
    size_t cap_n = 0;
    uint32_t slab_cap = 0;
    uint32_t nf_cap = 1;           // frames the table holds
    Frame *frames = nullptr;       // frame table (nf_cap)
    uint32_t *fhist = nullptr;     // per frame: digit counts of every pass of the main sort
    void *base = nullptr;
    size_t bytes = 0;
    Plan *plan = nullptr;
    float *xyz = nullptr;          // staging of host input
    int32_t *labels = nullptr;     // staging of host output
    void *keys_a = nullptr;        // 8 * cap_n bytes each (32- or 64-bit keys)
    void *keys_b = nullptr;
    void *vals_a = nullptr;        // 8 * cap_n bytes each (32-bit index or 64-bit packed payload)
    void *vals_b = nullptr;
    uint32_t *sort_status = nullptr;
    unsigned long long *scan_status = nullptr;
    Rec *rec = nullptr;
    uint32_t *sc_of = nullptr;
    uint32_t *sc_start = nullptr;  // cap_n + 1
    uint8_t *scode = nullptr;      // per sub-cell: which half of its cell on each axis
    uint8_t *cocc = nullptr;       // per cell: bit s set when its sub-cell with code s exists
    SubBox *box = nullptr;
    uint32_t *sminidx = nullptr;
    uint32_t *parent = nullptr;
    uint32_t *csize = nullptr;
    uint32_t *cmin = nullptr;
    int32_t *crank = nullptr;
    uint32_t *big = nullptr;
    unsigned long long *cell_key = nullptr;
    uint32_t *cell_sc = nullptr;   // cap_n + 1
    uint32_t *cframe = nullptr;    // per cell: its frame
    uint32_t *slab_lo = nullptr;   // slab_cap
    uint32_t *slab_hi = nullptr;
    uint2 *pairq = nullptr;        // sub-cell pairs queued for point tests
    uint32_t *reps = nullptr;      // per sub-cell: its point nearest the box centre (pack_rep)
    uint32_t *col_lo = nullptr;    // dense column index: cells of column (c0, c1) are
    uint32_t *col_hi = nullptr;    //   [col_lo, col_hi) of the sorted cell array
    uint32_t col_bits = 0;         // log2 of its capacity
    uint2 *edges = nullptr;        // boundary edges of the neighbour step
    size_t edges_cap = 0;
    unsigned long long *edge_set = nullptr;  // hash set of joined root pairs (power of two)
    size_t edge_set_size = 0;
    uint32_t *nb_first = nullptr;  // per cell: first sub-cell of each neighbour cell (13)
    uint8_t *nb_cnt = nullptr;     // per cell, 32 bytes: neighbour occupancies and offsets
    uint32_t *rank_bits = nullptr;   // bitmap over positions: smallest rows of kept components
    uint32_t *rank_prefix = nullptr; // per bitmap word: set bits before it
    unsigned long long *rank_status = nullptr;  // look-back status of the ranking scan
    uint32_t *scratch = nullptr;   // per block of the neighbour step: undecided in-region pairs
    size_t scratch_words = 0;
    uint32_t list_scale = 1;       // boundary-edge and pair lists hold list_scale * 2 * cap_n
    size_t pairq_cap = 0;
    // The kept-component list reuses the key buffers once the cell table is built.
    uint32_t *kept_key_a() const { return (uint32_t *)keys_a; }
    uint32_t *kept_val_a() const { return (uint32_t *)keys_a + cap_n; }
};

// Record a trace mark named `name` after the launch just enqueued on st
// (no-op unless tracing is enabled).
void trace_mark(const Workspace &ws, const char *name, cudaStream_t st);
#define FEC_MARK(ws, name, st) trace_mark((ws), (name), (st))

// Enqueue kernel k on st with `grid` blocks of `block` threads and `smem`
// bytes of dynamic shared memory, allowed to be scheduled before the
// previous kernel of st has finished (the kernel's grid_enter() waits for
// it).  Launch errors are left for the caller's cudaGetLastError().
template <typename... P, typename... A>
inline void launch(void (*k)(P...), uint32_t grid, uint32_t block, size_t smem, cudaStream_t st,
                   A &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = FEC_PDL;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k, std::forward<A>(args)...);
}

// Blocks of a grid-stride kernel over `items` work items, `per_block` per
// block and step: as many as the items need, at most `per_sm` per SM.
inline int grid_for(const Workspace &ws, uint64_t items, uint64_t per_block, int per_sm)
{
    const uint64_t want = (items + per_block - 1) / per_block;
    const uint64_t cap = (uint64_t)ws.sms * (uint64_t)per_sm;
    return (int)(want < 1 ? 1 : (want < cap ? want : cap));
}

// Regions have kRegionCellsPerBlock cells, fewer (down to kRegionMinCells)
// when the cloud has too few cells to give every block of the grid two.
#ifndef FEC_REGION_MIN_CELLS
#define FEC_REGION_MIN_CELLS 32
#endif
constexpr uint32_t kRegionMinCells = FEC_REGION_MIN_CELLS;

// Blocks of the region kernel for n points (kRegionBlocksPerSM per SM, at most
// one per possible region of the smallest size).
inline uint32_t region_grid(const Workspace &ws, uint64_t n)
{
    const uint64_t regions = (n + kRegionMinCells - 1) / kRegionMinCells;
    const uint64_t g = (uint64_t)ws.sms * kRegionBlocksPerSM;
    return (uint32_t)(regions < g ? (regions ? regions : 1) : g);
}

// Scratch entries of each region block (undecided pairs inside its region):
// kRegionScratch for full-size regions, in proportion for the smaller regions
// a cloud of n points can get.
inline uint32_t region_scratch(const Workspace &ws, uint64_t n)
{
    const uint64_t g = region_grid(ws, n);
    uint64_t rc = n / (2 * g);
    if (rc < kRegionMinCells) rc = kRegionMinCells;
    if (rc > kRegionCellsPerBlock) rc = kRegionCellsPerBlock;
    return (uint32_t)(kRegionScratch * rc / kRegionCellsPerBlock);
}

// Bytes of a workspace for cap_n points, slab_cap slab entries and nf_cap
// frames; with a non-null base, also carves the arrays into ws.
size_t workspace_layout(Workspace &ws, void *base, size_t cap_n, uint32_t slab_cap,
                        uint32_t nf_cap = 1);
// Sort tiles of a frame of n points, and the tiles a workspace must hold.
inline uint32_t frame_tiles(uint64_t n) { return (uint32_t)((n + kSortTile - 1) / kSortTile); }
inline uint32_t max_tiles(size_t cap_n, uint32_t nf_cap)
{
    return (uint32_t)(cap_n / kSortTile) + nf_cap + 1;
}

// Host-side constants for n points at radius d.
Params make_params(uint32_t n, float d);
// Upper bound of 8-bit passes of the main sort over any cloud at this S.
int max_sort_passes(const Params &prm);

// How a call's frame table is set: by k_init for a single cloud (single =
// true, with its size bounds), else uploaded by the host before the call.
struct FrontArgs {
    bool single = true;
    long long min_size = 0, max_size = 0;
};
// a1 (init, bbox, plan, keys) for the call's prm.n points at xyz (device).
cudaError_t enqueue_front(Workspace &ws, const float *xyz, const Params &prm, const FrontArgs &fa,
                          cudaStream_t st);
// The main sort's key layout, when the host has read it back from the plan:
// only its passes of its width are launched (else both widths are launched
// and the kernels of the width the plan does not select return at once).
struct KeyLayout {
    bool key64 = false;
    int passes = 0;
};
// Everything after enqueue_front (a2 .. a6).
cudaError_t enqueue_back(Workspace &ws, const float *xyz, const Params &prm, int32_t *labels,
                         bool fill_labels, cudaStream_t st, const KeyLayout *known = nullptr);
// a3 (cell table, sub-cell stats, slab index).
cudaError_t enqueue_cells(Workspace &ws, const float *xyz, const Params &prm, cudaStream_t st);
// a4 + a5 + kept list of a6 (size bounds from the frame table).
cudaError_t enqueue_union(Workspace &ws, const Params &prm, cudaStream_t st);
// a6 rank + labels (labels: device pointer, prm.rows entries; fill: set
// every label to -1 first, else the caller has done so).
cudaError_t enqueue_labels(Workspace &ws, const Params &prm, int32_t *labels, bool fill,
                           cudaStream_t st);
// The whole pipeline for one call (device pointers), no host
// synchronisation: prm.nf frames of prm.n points in total that share the
// radius, rows prm.rows of xyz and labels.  prm comes from make_params(n, d)
// (one frame); callers may lower its slab capacity or iteration caps, or lay
// out several frames (the table then uploaded before the call, fa.single
// false).  fill_labels: set all prm.rows labels to -1 first (else the caller
// has done so).
cudaError_t enqueue_cluster(Workspace &ws, const float *xyz, const Params &prm,
                            const FrontArgs &fa, int32_t *labels, bool fill_labels,
                            cudaStream_t st);

// Onesweep radix sort of (key, value) over ctl->npasses 8-bit digits, with
// digit histograms already in ctl->hist.  Keys are 32- or 64-bit, values 32-
// or 64-bit; values may be the identity index 0..n-1 for the first pass.
// Kernels for a key width that ctl->key64 does not select return at once, so
// both widths can be enqueued blindly.  The result lands in keys_a/vals_a if
// npasses is even, else in keys_b/vals_b.
// Where the first pass of a sort gets its keys: from keys_a/vals_a (xyz
// null), or computed from the coordinates under the plan (packed payloads;
// the key kernel then only makes the histograms).
// The frames (non-null: a segmented sort, see k_onesweep) and their digit
// histograms.
struct SortSource {
    const float *xyz = nullptr;
    const Plan *plan = nullptr;
    Params prm{};
    const Frame *frames = nullptr;
    const uint32_t *fhist = nullptr;
};
// tiles: how many tiles the sort can have at most (sizes the grid).
cudaError_t launch_sort(const Workspace &ws, const char *name, SortCtl *ctl, void *keys_a,
                        void *vals_a, void *keys_b, void *vals_b, bool key64, bool val64,
                        bool identity_vals, uint32_t *tile_status, uint32_t tiles, int max_passes,
                        int grid, cudaStream_t st, uint32_t *status,
                        const SortSource &src = SortSource());
// The main sort's source, matching enqueue_front (which stores keys only
// when the payloads are not packed): segmented by the call's frames.
inline SortSource main_sort_source(const Workspace &ws, const float *xyz, const Params &prm)
{
    SortSource s;
    s.prm = prm;
    s.frames = ws.frames;
    s.fhist = ws.fhist;
    if (prm.packed) {
        s.xyz = xyz;
        s.plan = ws.plan;
    }
    return s;
}
// uint32 words between the two look-back arrays of a workspace's sorts.
inline size_t sort_tstride(const Workspace &ws)
{
    return ((size_t)max_tiles(ws.cap_n, ws.nf_cap) + 1) * kRadixBins;
}
// uint32 words of look-back status (two arrays) for a sort of `tiles` tiles.
inline size_t sort_status_words(uint32_t tiles)
{
    return 2 * ((size_t)tiles + 1) * kRadixBins;
}

int sm_count();

// ID of the CUDA context current on this thread (unique within the process,
// never reused), or 0 when it cannot be told.  Per-context set-up (function
// attributes, symbol addresses) is keyed on it: a device reset or a second
// device gives a new context, whose set-up must be done again.
unsigned long long current_ctx_id();
// True when the set-up recorded in done_in was not made in the current
// context (or the context cannot be told); ctx_setup_done records it.
bool ctx_setup_needed(std::atomic<unsigned long long> &done_in);
void ctx_setup_done(std::atomic<unsigned long long> &done_in);

}  // namespace fec
