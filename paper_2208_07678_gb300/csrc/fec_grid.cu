// fec_grid.cu -- voxel-grid construction: quantisation and bounding box,
// grid keys, and the cell table built from the sorted keys.
//
// The grid replaces Algorithm 1's kd-tree (Section 2.2) and its radius query
// FindNeighbor: with R = floor(sqrt(T2)) the largest per-axis offset of two
// joined points, cells of side S = 2h >= R (h = ceil(R/2)) guarantee that every
// joined pair lies in the same or an adjacent cell (27-cell stencil).  Each
// cell is split into 2x2x2 sub-cells of side h; since 3(h-1)^2 <= T2, all
// points of one sub-cell are pairwise within d, so a sub-cell is a clique and
// becomes one union-find node.
#include <algorithm>

#include "fec_internal.cuh"

namespace fec {

namespace {

__device__ __forceinline__ uint32_t bitlen(uint32_t v) { return v ? 32u - __clz(v) : 0u; }

template <typename T>
__device__ __forceinline__ T warp_min(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
template <typename T>
__device__ __forceinline__ T warp_max(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

}  // namespace

// Reset the plan and the frame table for a call of n points in nf frames
// (one block does the plan; every block clears its share of the frames'
// device fields and per-frame histograms).  A single cloud (single = 1)
// also gets its one frame's static fields here, so it needs no upload.
__global__ void k_init(Plan *plan, Frame *fr, uint32_t nf, uint32_t *fhist, uint32_t n,
                       uint32_t wait_cap, int single, long long min_size, long long max_size)
{
    grid_enter();
    const int t = threadIdx.x;
    if (blockIdx.x == 0) {
        if (t < 3) {
            plan->perm[t] = t;
            plan->bits[t] = 0;
        }
        if (t == 0) {
            plan->key_bits = 0;
            plan->status = 0;
            plan->M_s = 0;
            plan->M_c = 0;
            plan->n_big = 0;
            plan->n_huge = 0;
            plan->scan_tile_counter = 0;
            plan->pairq_n = 0;
            plan->use_cols = 0;
            plan->edges_n = 0;
            plan->region_counter = 0;
            plan->slab_need = 0;
            plan->rank_tile_counter = 0;
            plan->bbox_done = 0;
            plan->sort.n = n;
            plan->sort.npasses = 0;
            plan->sort.key64 = 0;
            plan->sort.parity = 0;
            plan->sort.wait_cap = wait_cap;
            plan->kept_n = 0;
        }
        if (t < 8) plan->ctr[t] = 0;
        if (t < kMaxPasses) plan->sort.tile_counter[t] = 0;
    }
    const uint32_t gt = blockIdx.x * blockDim.x + t, gs = gridDim.x * blockDim.x;
    for (uint32_t f = gt; f < nf; f += gs) {
        Frame &F = fr[f];
        if (single) {
            F.in_off = 0;
            F.pos_off = 0;
            F.n = n;
            F.tile0 = 0;
            F.min_size = min_size;
            F.max_size = max_size;
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            F.lo[a] = INT32_MAX;
            F.hi[a] = INT32_MIN;
        }
        F.kept = 0;
        F.nslab = 0;
        F.slab_base = 0;
    }
    const size_t hw = (size_t)nf * kMaxPasses * kRadixBins;
    for (size_t i = gt; i < hw; i += gs) fhist[i] = 0;
}

// Block-wide min / max of three values per thread into s (thread 0 reads).
__device__ __forceinline__ void block_box(int32_t lo[3], int32_t hi[3], int32_t (*s_lo)[8],
                                          int32_t (*s_hi)[8])
{
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int32_t vl = warp_min(lo[a]), vh = warp_max(hi[a]);
        if (l == 0) {
            s_lo[a][w] = vl;
            s_hi[a][w] = vh;
        }
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        const int a = threadIdx.x;
        int32_t vl = INT32_MAX, vh = INT32_MIN;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            vl = min(vl, s_lo[a][k]);
            vh = max(vh, s_hi[a][k]);
        }
        s_lo[a][0] = vl;
        s_hi[a][0] = vh;
    }
    __syncthreads();
}

// Work units of the bounding-box and key kernels: each sort tile (which never
// straddles two frames) split into kUnitsPerTile chunks of about 1,024 points.  Unit u covers
// frame-local indices [first, first + count) of frame f (count may be 0).
constexpr uint32_t kUnitsPerTile = kSortTile >= 2048 ? kSortTile / 1024 : 1;
constexpr uint32_t kUnit = kSortTile / kUnitsPerTile;  // about 1024 points
static_assert(kUnit * kUnitsPerTile == kSortTile, "units split a tile evenly");
struct TileSpan {
    uint32_t f, first, count;
};
__device__ __forceinline__ TileSpan unit_span(const Frame *__restrict__ fr, uint32_t nf, uint32_t u)
{
    const uint32_t t = u / kUnitsPerTile;
    TileSpan sp;
    sp.f = frame_of_tile(fr, nf, t);
    sp.first = (t - fr[sp.f].tile0) * (uint32_t)kSortTile + (u - t * kUnitsPerTile) * kUnit;
    const uint32_t n = fr[sp.f].n;
    sp.count = sp.first < n ? min(kUnit, n - sp.first) : 0u;
    return sp;
}
// The units block b takes: with several frames a contiguous share
// [lo, hi) of the call's units (so that its units mostly belong to one
// frame), with one frame every gridDim.x-th unit from blockIdx.x (the whole
// grid then sweeps the input in order).
struct UnitRange {
    uint32_t lo, hi, step;
};
__device__ __forceinline__ UnitRange block_units(uint32_t ntiles, uint32_t nf)
{
    const uint64_t U = (uint64_t)ntiles * kUnitsPerTile;
    if (nf == 1) return UnitRange{blockIdx.x, (uint32_t)U, gridDim.x};
    return UnitRange{(uint32_t)(U * blockIdx.x / gridDim.x), (uint32_t)(U * (blockIdx.x + 1) / gridDim.x), 1u};
}

// Twelve floats (four points) of rows [row, row + cnt) of xyz: three 16-byte
// loads when the rows are aligned and complete.
__device__ __forceinline__ void load_rows4(const float *__restrict__ xyz, uint32_t row, uint32_t cnt,
                                           bool vec, float f[12])
{
    if (vec && cnt == 4) {
        const float4 *src = reinterpret_cast<const float4 *>(xyz + 3 * (size_t)row);
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            const float4 v = __ldcs(src + t);
            f[4 * t + 0] = v.x;
            f[4 * t + 1] = v.y;
            f[4 * t + 2] = v.z;
            f[4 * t + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int t = 0; t < 12; ++t) f[t] = (uint32_t)t < 3 * cnt ? __ldcs(xyz + 3 * (size_t)row + t) : 0.0f;
    }
}

// a1: choose the axis order (largest cell extent major, smallest minor) and
// the key layout, the same for every frame of the call (from the largest
// extent per axis over the frames); lay out each frame's part of the slab
// index; disable the rest of the pipeline on a data error.  Run by one
// whole block (256 threads), the last of the bounding-box kernel, after
// every block's boxes are in memory: the boxes are read past the L1 cache,
// which may hold lines of the frame table from before.
__device__ __forceinline__ void plan_body(Plan *plan, Frame *__restrict__ fr, const Params &prm)
{
    __shared__ uint32_t s_cm[3];
    __shared__ uint32_t s_scan[256];
    __shared__ int s_perm0;
    __shared__ uint32_t s_stop;
    const int t = threadIdx.x;
    if (t < 3) s_cm[t] = 0;
    if (t == 0) s_stop = (*(volatile uint32_t *)&plan->status & (ST_NONFINITE | ST_OUT_OF_RANGE)) ? 1u : 0u;
    __syncthreads();
    // the host's 16-byte read-back of the outcome
    auto publish = [&]() {
        plan->front[0] = plan->status;
        plan->front[1] = plan->sort.key64;
        plan->front[2] = plan->sort.npasses;
        plan->front[3] = plan->key_bits;
    };
    if (s_stop) {
        if (t == 0) {
            plan->sort.n = 0;
            publish();
        }
        return;
    }
    for (uint32_t f = t; f < prm.nf; f += blockDim.x)
        for (int a = 0; a < 3; ++a)
            atomicMax(&s_cm[a], (uint32_t)(((int64_t)__ldcg(&fr[f].hi[a]) - __ldcg(&fr[f].lo[a])) / prm.S));
    __syncthreads();
    if (t == 0) {
        uint32_t cm[3] = {s_cm[0], s_cm[1], s_cm[2]};
        int perm[3] = {0, 1, 2};
        for (int i = 0; i < 3; ++i)
            for (int j = i + 1; j < 3; ++j)
                if (cm[perm[j]] > cm[perm[i]]) {
                    int tt = perm[i];
                    perm[i] = perm[j];
                    perm[j] = tt;
                }
        uint32_t total = 0;
        for (int p = 0; p < 3; ++p) {
            plan->perm[p] = perm[p];
            plan->bits[p] = bitlen(cm[perm[p]]);
            total += plan->bits[p];
        }
        s_perm0 = perm[0];
        if (total > 61) {
            plan->status |= ST_KEY_OVERFLOW;
            plan->sort.n = 0;
            s_stop = 1;
            publish();
        } else {
            plan->key_bits = total + 3;
            plan->use_cols =
                (prm.nf == 1 && plan->bits[0] + plan->bits[1] <= prm.col_bits) ? 1u : 0u;
            plan->sort.npasses = (total + 3 + kRadixBits - 1) / kRadixBits;
            plan->sort.key64 = (total + 3) > 32 ? 1u : 0u;
        }
    }
    __syncthreads();
    if (s_stop) return;
    // each frame's slab entries (the brick rows of its major cell
    // coordinates), laid out in frame order: an exclusive scan in chunks of
    // 256 frames
    const int p0 = s_perm0;
    CellKeyLayout L;
    L.load(plan);
    uint32_t carry = 0;
    for (uint32_t c0 = 0; c0 < prm.nf; c0 += blockDim.x) {
        const uint32_t f = c0 + t;
        uint32_t ns = 0;
        if (f < prm.nf)
            ns = (uint32_t)L.slab_of(
                     (unsigned long long)(((int64_t)__ldcg(&fr[f].hi[p0]) - __ldcg(&fr[f].lo[p0])) / prm.S)) + 1u;
        s_scan[t] = ns;
        __syncthreads();
        for (int o = 1; o < 256; o <<= 1) {
            const uint32_t v = t >= o ? s_scan[t - o] : 0u;
            __syncthreads();
            s_scan[t] += v;
            __syncthreads();
        }
        if (f < prm.nf) {
            fr[f].nslab = ns;
            fr[f].slab_base = carry + s_scan[t] - ns;
        }
        carry += s_scan[255];
        __syncthreads();
    }
    if (t == 0) {
        plan->slab_need = carry;
        if (carry > prm.slab_cap) {  // the host grows the slab index and runs the call again
            plan->status |= ST_SIZE_OVERFLOW;
            plan->sort.n = 0;
        }
        publish();
    }
}

// a1: validate and quantise every coordinate, reduce each frame's bounding
// box of q.  A block keeps its partial box until one of its units belongs
// to another frame (a single cloud: once, at the end).  The last block to
// finish then runs plan_body.
template <bool MULTI>
__global__ void __launch_bounds__(256) k_bbox(const float *__restrict__ xyz, Plan *plan,
                                              Frame *__restrict__ fr, Params prm)
{
    grid_enter();
    __shared__ int32_t s_lo[3][8], s_hi[3][8];
    __shared__ uint32_t s_st;
    int32_t lo[3] = {INT32_MAX, INT32_MAX, INT32_MAX};
    int32_t hi[3] = {INT32_MIN, INT32_MIN, INT32_MIN};
    uint32_t st = 0;
    if (threadIdx.x == 0) s_st = 0;
    uint32_t cur = 0xffffffffu;  // frame of the partial box (block-uniform)
    auto flush = [&]() {
        block_box(lo, hi, s_lo, s_hi);
        if (threadIdx.x < 3 && s_lo[threadIdx.x][0] != INT32_MAX) {
            atomicMin(&fr[cur].lo[threadIdx.x], s_lo[threadIdx.x][0]);
            atomicMax(&fr[cur].hi[threadIdx.x], s_hi[threadIdx.x][0]);
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            lo[a] = INT32_MAX;
            hi[a] = INT32_MIN;
        }
        __syncthreads();
    };
    // groups of four rows [row0 + 4 g0, row0 + count), every gstep-th
    auto rows = [&](uint32_t row0, uint32_t count, uint32_t g0, uint32_t gstep) {
        const bool vec = ((reinterpret_cast<uintptr_t>(xyz) & 15) == 0) && (row0 & 3u) == 0;
        for (uint32_t gi = g0; 4 * gi < count; gi += gstep) {
            const uint32_t cnt = min(4u, count - 4 * gi);
            float f[12];
            load_rows4(xyz, row0 + 4 * gi, cnt, vec, f);
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                if ((uint32_t)k >= 3 * cnt) break;
                const int a = k % 3;
                int32_t q;
                const int e = quantize1(f[k], q);
                if (e == 1) st |= ST_NONFINITE;
                else if (e == 2) st |= ST_OUT_OF_RANGE;
                else {
                    lo[a] = min(lo[a], q);
                    hi[a] = max(hi[a], q);
                }
            }
        }
    };
    if (!MULTI) {  // one frame: the whole grid sweeps its rows
        cur = 0;
        rows(fr[0].in_off, prm.n, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
    } else {
        const UnitRange ur = block_units(prm.ntiles, prm.nf);
        for (uint32_t u = ur.lo; u < ur.hi; u += ur.step) {
            const TileSpan sp = unit_span(fr, prm.nf, u);
            if (sp.f != cur) {
                if (cur != 0xffffffffu) flush();
                cur = sp.f;
            }
            rows(fr[sp.f].in_off + sp.first, sp.count, threadIdx.x, blockDim.x);
        }
    }
    if (cur != 0xffffffffu) flush();
    if (st) atomicOr(&s_st, st);
    __syncthreads();
    // the last block to finish lays out the plan (every block's boxes and
    // status bits are in memory before it counts itself done)
    __shared__ bool s_last;
    if (threadIdx.x == 0) {
        if (s_st) atomicOr(&plan->status, s_st);
        __threadfence();
        s_last = atomicAdd(&plan->bbox_done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        plan_body(plan, fr, prm);
    }
}

// Arrays zeroed by the key kernel for the later stages.
struct Clears {
    uint32_t *sort_status;          // look-back array 0 of the main sort
    size_t sort_words;
    unsigned long long *scan_status;  // cell-table look-back
    size_t scan_words;
    uint32_t *slab_lo, *slab_hi;    // slab index
    size_t slab_words;
    uint32_t *col_lo, *col_hi;      // dense column index (size from the plan)
    uint32_t *rank_bits;            // kept-component bitmap
    size_t rank_words;
    unsigned long long *rank_status;  // its scan's look-back
    size_t rank_status_words;
    size_t max_words;
};

// a1: grid keys of all points, plus each frame's digit histograms of every
// radix pass.  With STORE false only the histograms are made: the sort's
// first pass then computes the keys and payloads again from the coordinates
// it reads, which saves writing and re-reading them (packed layout only).
// A block's shared-memory histograms go to the frame's global ones when one
// of its units belongs to another frame.
template <typename KeyT, bool STORE, bool MULTI>
__device__ __forceinline__ void keys_body(const float *__restrict__ xyz, Plan *plan, const Params &prm,
                                          const Frame *__restrict__ fr, uint32_t *__restrict__ fhist,
                                          KeyT *__restrict__ keys, const Clears &clr,
                                          uint32_t (*h)[kRadixBins])
{
    SortCtl *ctl = &plan->sort;
    if (ctl->n == 0) return;
    // arrays the later stages need zeroed (in place of separate memsets)
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < clr.max_words;
         i += (size_t)gridDim.x * blockDim.x) {
        if (i < clr.sort_words) clr.sort_status[i] = 0;
        if (i < clr.scan_words) clr.scan_status[i] = 0;
        if (i < clr.slab_words) {
            clr.slab_lo[i] = 0;
            clr.slab_hi[i] = 0;
        }
        if (i < clr.rank_words) clr.rank_bits[i] = 0;
        if (i < clr.rank_status_words) clr.rank_status[i] = 0;
    }
    // the dense column index, when the plan uses it (its size is known now)
    if (plan->use_cols) {
        const size_t ncol = (size_t)1 << (plan->bits[0] + plan->bits[1]);
        for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < ncol;
             i += (size_t)gridDim.x * blockDim.x) {
            clr.col_lo[i] = 0;
            clr.col_hi[i] = 0;
        }
    }
    const int np = (int)ctl->npasses;
    for (int i = threadIdx.x; i < kMaxPasses * kRadixBins; i += blockDim.x) (&h[0][0])[i] = 0;
    GridMap g;
    g.load(plan, prm, fr[0]);
    __syncthreads();
    uint32_t cur = 0xffffffffu;  // frame whose counts are in h (block-uniform)
    auto flush = [&]() {
        __syncthreads();
        uint32_t *dst = fhist + (size_t)cur * kMaxPasses * kRadixBins;
        for (int i = threadIdx.x; i < np * kRadixBins; i += blockDim.x) {
            const uint32_t v = (&h[0][0])[i];
            if (v) atomicAdd(dst + i, v);
            (&h[0][0])[i] = 0;
        }
        __syncthreads();
    };
    // four consecutive points per thread and step: groups of four rows
    // [row0 + 4 g0, row0 + count), every gstep-th, at positions from pos0
    auto rows = [&](uint32_t row0, uint32_t pos0, uint32_t count, uint32_t g0, uint32_t gstep) {
        const bool vec = ((reinterpret_cast<uintptr_t>(xyz) & 15) == 0) && (row0 & 3u) == 0;
        const bool vst = (pos0 & 3u) == 0;
        for (uint32_t gi = g0; 4 * gi < count; gi += gstep) {
            const uint32_t cnt = min(4u, count - 4 * gi);
            float f[12];
            load_rows4(xyz, row0 + 4 * gi, cnt, vec, f);
            KeyT k[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                int32_t q[3];
#pragma unroll
                for (int a = 0; a < 3; ++a) quantize1(f[3 * u + a], q[a]);
                uint32_t c[3], off[3];
                g.cell_of(q, c, off);
                k[u] = g.key_of<KeyT>(c, off);
            }
            if (STORE) {
                const uint32_t p = pos0 + 4 * gi;
                if (cnt == 4 && vst) {
                    if (sizeof(KeyT) == 4) {
                        reinterpret_cast<uint4 *>(keys + p)[0] =
                            make_uint4((uint32_t)k[0], (uint32_t)k[1], (uint32_t)k[2], (uint32_t)k[3]);
                    } else {
                        reinterpret_cast<ulonglong2 *>(keys + p)[0] = make_ulonglong2(k[0], k[1]);
                        reinterpret_cast<ulonglong2 *>(keys + p)[1] = make_ulonglong2(k[2], k[3]);
                    }
                } else {
                    for (uint32_t u = 0; u < cnt; ++u) keys[p + u] = k[u];
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if ((uint32_t)u >= cnt) break;
                for (int p = 0; p < np; ++p)
                    atomicAdd(&h[p][(uint32_t)(k[u] >> (p * kRadixBits)) & 255u], 1u);
            }
        }
    };
    if (!MULTI) {  // one frame: the whole grid sweeps its rows
        cur = 0;
        rows(fr[0].in_off, 0u, ctl->n, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
    } else {
        const UnitRange ur = block_units(prm.ntiles, prm.nf);
        for (uint32_t u = ur.lo; u < ur.hi; u += ur.step) {
            const TileSpan sp = unit_span(fr, prm.nf, u);
            if (sp.f != cur) {
                if (cur != 0xffffffffu) flush();
                cur = sp.f;
                g.set_frame(fr[sp.f]);
            }
            rows(fr[sp.f].in_off + sp.first, fr[sp.f].pos_off + sp.first, sp.count, threadIdx.x,
                 blockDim.x);
        }
    }
    if (cur != 0xffffffffu) flush();
}

// The key kernel for either key width (the plan selects it on the device).
template <bool STORE, bool MULTI>
__global__ void __launch_bounds__(256)
    k_keys(const float *__restrict__ xyz, Plan *plan, Params prm, const Frame *__restrict__ fr,
           uint32_t *__restrict__ fhist, void *__restrict__ keys, Clears clr)
{
    grid_enter();
    __shared__ uint32_t h[kMaxPasses][kRadixBins];
    if (plan->sort.key64)
        keys_body<unsigned long long, STORE, MULTI>(xyz, plan, prm, fr, fhist, (unsigned long long *)keys,
                                                    clr, h);
    else
        keys_body<uint32_t, STORE, MULTI>(xyz, plan, prm, fr, fhist, (uint32_t *)keys, clr, h);
}

// a3: cell table from the sorted keys, in one pass with a decoupled look-back
// scan of two head flags (new sub-cell, new cell).  Also gathers the sorted
// point records (quantised coordinates + original index).
//   sc_of[p]      sub-cell of sorted position p
//   sc_start[a]   first sorted position of sub-cell a (sc_start[M_s] = n)
//   scode[a]      sub-cell code of a: which half of its cell on each axis
//   cell_key[c]   cell key of cell c; cell_sc[c] first sub-cell of cell c
//   cframe[c]     frame of cell c
// A frame's first position always starts a new cell and sub-cell (keys are
// frame-local, so two frames' cells never merge).
struct CellsSmem {
    uint32_t tile;
    unsigned long long warp[kScanThreads / 32];
    unsigned long long prefix;
    Rec rec[kScanTile];     // the tile's records, staged for coalesced stores
    uint32_t sc[kScanTile];
};

template <typename KeyT, typename ValT, bool MULTI>
__device__ __forceinline__ void cells_body(Plan *plan, const Params &prm, const KeyT *__restrict__ keys_a,
                                           const ValT *__restrict__ vals_a,
                                           const KeyT *__restrict__ keys_b,
                                           const ValT *__restrict__ vals_b,
                                           const float *__restrict__ xyz, Rec *__restrict__ rec,
                                           uint32_t *__restrict__ sc_of,
                                           uint32_t *__restrict__ sc_start, uint8_t *__restrict__ scode,
                                           unsigned long long *__restrict__ cell_key,
                                           uint32_t *__restrict__ cell_sc,
                                           uint32_t *__restrict__ cframe,
                                           const Frame *__restrict__ fr,
                                           unsigned long long *__restrict__ tstat, CellsSmem &C)
{
    const SortCtl *ctl = &plan->sort;
    const uint32_t n = ctl->n;
    if (n == 0 || block_aborted(&plan->status)) return;
    const uint32_t wait_cap = prm.wait_cap;
    const bool in_b = (ctl->npasses & 1u) != 0;
    const KeyT *__restrict__ keys = in_b ? keys_b : keys_a;
    const ValT *__restrict__ vals = in_b ? vals_b : vals_a;
    constexpr bool PACKED = sizeof(ValT) == 8;
    GridMap g;
    if (PACKED) g.load(plan, prm, fr[0]);
    uint32_t gframe = 0;  // frame whose origin g holds
    const uint32_t ntiles = (n + kScanTile - 1) / kScanTile;
    const uint32_t nf = prm.nf;

    constexpr unsigned long long kAgg = 1ull << 62, kIncl = 2ull << 62;
    constexpr unsigned long long kMask = (1ull << 62) - 1;
    uint32_t &s_tile = C.tile;
    unsigned long long *s_warp = C.warp;
    unsigned long long &s_prefix = C.prefix;
    Rec *s_rec = C.rec;
    uint32_t *s_sc = C.sc;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    for (;;) {
        if (tid == 0) s_tile = atomicAdd(&plan->scan_tile_counter, 1u);
        __syncthreads();
        const uint32_t tile = s_tile;
        if (tile >= ntiles) break;
        const uint32_t p0 = tile * kScanTile + tid * kScanIPT;

        KeyT k[kScanIPT];
        unsigned long long flag[kScanIPT];  // (cell head << 31) | sub-cell head
        KeyT prev = (p0 > 0 && p0 - 1 < n) ? keys[p0 - 1] : KeyT(0);
        // frame of the thread's first position, and which of its positions
        // start a frame (bit i: position p0 + i)
        const uint32_t f0 = (MULTI && p0 < n) ? frame_of_pos(fr, nf, p0) : 0u;
        uint32_t fstarts = p0 == 0 ? 1u : 0u;
        if (MULTI) {
            uint32_t wf = f0, wstart = fr[f0].pos_off;
            uint32_t wnext = wf + 1 < nf ? fr[wf + 1].pos_off : 0xffffffffu;
#pragma unroll
            for (int i = 0; i < kScanIPT; ++i) {
                const uint32_t p = p0 + i;
                while (p >= wnext) {
                    ++wf;
                    wstart = wnext;
                    wnext = wf + 1 < nf ? fr[wf + 1].pos_off : 0xffffffffu;
                }
                if (p == wstart) fstarts |= 1u << i;
            }
        }
        unsigned long long run = 0;
        const bool full = p0 + kScanIPT <= n;
        if (full) {  // the thread's keys in 16-byte loads
            constexpr int per = 16 / sizeof(KeyT);
#pragma unroll
            for (int v = 0; v < kScanIPT / per; ++v) {
                const uint4 w = __ldcs(reinterpret_cast<const uint4 *>(keys + p0) + v);
                const KeyT *e = reinterpret_cast<const KeyT *>(&w);
#pragma unroll
                for (int t = 0; t < per; ++t) k[v * per + t] = e[t];
            }
        }
        // the payloads too, so that their loads overlap the scan and look-back
        ValT vv[kScanIPT];
        if (full) {
            constexpr int per = 16 / sizeof(ValT);
#pragma unroll
            for (int v = 0; v < kScanIPT / per; ++v) {
                const uint4 w = __ldcs(reinterpret_cast<const uint4 *>(vals + p0) + v);
                const ValT *e = reinterpret_cast<const ValT *>(&w);
#pragma unroll
                for (int t = 0; t < per; ++t) vv[v * per + t] = e[t];
            }
        } else {
#pragma unroll
            for (int i = 0; i < kScanIPT; ++i) vv[i] = (p0 + i < n) ? vals[p0 + i] : (ValT)0;
        }
#pragma unroll
        for (int i = 0; i < kScanIPT; ++i) {
            const uint32_t p = p0 + i;
            unsigned long long f = 0;
            if (p < n) {
                if (!full) k[i] = keys[p];
                const bool fh = (fstarts >> i) & 1u;  // includes p == 0
                const bool sh = fh || k[i] != prev;
                const bool ch = fh || (k[i] >> 3) != (prev >> 3);
                f = ((unsigned long long)ch << 31) | (unsigned long long)sh;
                prev = k[i];
            } else {
                k[i] = KeyT(0);
            }
            run += f;
            flag[i] = run;  // inclusive within the thread
        }
        // block exclusive scan of the thread totals
        unsigned long long incl = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        if (lane == 31) s_warp[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            unsigned long long tot = 0;
            for (int w = 0; w < kScanThreads / 32; ++w) tot += s_warp[w];
            __syncwarp();
            if (lane == 0) {
                unsigned long long acc = 0;
                for (int w = 0; w < kScanThreads / 32; ++w) {
                    const unsigned long long v = s_warp[w];
                    s_warp[w] = acc;
                    acc += v;
                }
                st_relaxed64(tstat + tile, (tile == 0 ? kIncl : kAgg) | tot);
            }
            // look-back, 32 preceding tiles per step (one per lane)
            unsigned long long prefix = 0;
            if (tile > 0) {
                int64_t p = (int64_t)tile - 1;
                uint32_t it = 0;
                for (;;) {
                    const int64_t q = p - lane;
                    unsigned long long sv = q >= 0 ? ld_relaxed64(tstat + q) : kIncl;
                    // the nearest inclusive entry, and everything before it published
                    uint32_t incl_m = __ballot_sync(0xffffffffu, (sv & ~kMask) == kIncl);
                    const int stop = incl_m ? __ffs(incl_m) - 1 : 31;
                    bool ready = (sv & ~kMask) != 0 || lane > stop;
                    while (!__all_sync(0xffffffffu, ready)) {
                        if (++it > wait_cap) {
                            if (lane == 0) atomicOr(&plan->status, ST_WAIT_TIMEOUT);
                            break;
                        }
                        spin_pause(it);
                        if (!ready) {
                            sv = ld_relaxed64(tstat + q);
                            ready = (sv & ~kMask) != 0;
                        }
                        incl_m = __ballot_sync(0xffffffffu, (sv & ~kMask) == kIncl);
                    }
                    const int stop2 = incl_m ? __ffs(incl_m) - 1 : 31;
                    unsigned long long part = (lane <= stop2 && q >= 0) ? (sv & kMask) : 0ull;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
                    prefix += part;
                    if (incl_m || it > wait_cap) break;
                    p -= 32;
                }
                if (lane == 0) st_relaxed64(tstat + tile, kIncl | ((prefix + tot) & kMask));
            }
            if (lane == 0) s_prefix = prefix;
        }
        // The sorted records do not depend on the prefix: staged here, the
        // other warps build them while warp 0 looks back.
        {
            uint32_t fr_i = f0;
#pragma unroll
            for (int i = 0; i < kScanIPT; ++i) {
                const uint32_t p = p0 + i;
                if (p >= n) break;
                if (i > 0 && ((fstarts >> i) & 1u)) ++fr_i;
                if (MULTI && PACKED && fr_i != gframe) {  // the grid origin of the position's frame
                    g.set_frame(fr[fr_i]);
                    gframe = fr_i;
                }
                const uint32_t idx = (uint32_t)vv[i];
                Rec r;
                if (PACKED) {
                    int32_t q[3];
                    g.unpack<KeyT>(k[i], (unsigned long long)vv[i], q);
                    r.x = q[0];
                    r.y = q[1];
                    r.z = q[2];
                } else if (idx < prm.rows) {  // gather from the input (cells wider than 1024 units)
                    quantize1(xyz[3 * (size_t)idx + 0], r.x);
                    quantize1(xyz[3 * (size_t)idx + 1], r.y);
                    quantize1(xyz[3 * (size_t)idx + 2], r.z);
                } else {  // only after a look-back timeout (reported below)
                    r.x = r.y = r.z = 0;
                }
                r.idx = idx;
                s_rec[tid * kScanIPT + i] = r;
            }
        }
        __syncthreads();
        const unsigned long long base = s_prefix + s_warp[warp] + (incl - run);

        unsigned long long before = base;
        uint32_t fcur = f0;
#pragma unroll
        for (int i = 0; i < kScanIPT; ++i) {
            const uint32_t p = p0 + i;
            if (p >= n) break;
            if (i > 0 && ((fstarts >> i) & 1u)) ++fcur;
            const unsigned long long cur = base + flag[i];
            const uint32_t sc = (uint32_t)(cur & 0x7fffffffull) - 1u;
            const uint32_t c = (uint32_t)(cur >> 31) - 1u;
            const bool sh = (cur & 0x7fffffffull) != (before & 0x7fffffffull);
            const bool ch = (cur >> 31) != (before >> 31);
            before = cur;
            const uint32_t idx = (uint32_t)vv[i];
            if (sc >= n || c >= n || idx >= prm.rows) {  // only after a look-back timeout
                atomicOr(&plan->status, ST_SIZE_OVERFLOW);
                continue;
            }
            s_sc[tid * kScanIPT + i] = sc;
            if (sh) {
                sc_start[sc] = p;
                scode[sc] = (uint8_t)(k[i] & 7u);
            }
            if (ch) {
                cell_key[c] = (unsigned long long)(k[i] >> 3);
                cell_sc[c] = sc;
                if (MULTI) cframe[c] = fcur;
            }
            if (p == n - 1) {
                plan->M_s = sc + 1;
                plan->M_c = c + 1;
                sc_start[sc + 1] = n;
                cell_sc[c + 1] = sc + 1;
            }
        }
        __syncthreads();
        // the tile's records and sub-cell indices, written out coalesced
        const uint32_t tile_n = min((uint32_t)kScanTile, n - tile * (uint32_t)kScanTile);
        for (uint32_t j = tid; j < tile_n; j += kScanThreads) {
            __stcs(reinterpret_cast<int4 *>(rec) + (size_t)tile * kScanTile + j,
                   reinterpret_cast<const int4 *>(s_rec)[j]);
            __stcs(sc_of + (size_t)tile * kScanTile + j, s_sc[j]);
        }
        __syncthreads();
    }
}

// The cell-table kernel for either key width (the plan selects it on the
// device); the payload width is known on the host.
template <typename ValT, bool MULTI>
__global__ void __launch_bounds__(kScanThreads, MULTI ? 3 : 4)  // the frame walk needs registers
    k_cells(Plan *plan, Params prm, const void *__restrict__ keys_a, const ValT *__restrict__ vals_a,
            const void *__restrict__ keys_b, const ValT *__restrict__ vals_b,
            const float *__restrict__ xyz, Rec *__restrict__ rec, uint32_t *__restrict__ sc_of,
            uint32_t *__restrict__ sc_start, uint8_t *__restrict__ scode,
            unsigned long long *__restrict__ cell_key, uint32_t *__restrict__ cell_sc,
            uint32_t *__restrict__ cframe, const Frame *__restrict__ fr,
            unsigned long long *__restrict__ tstat)
{
    grid_enter();
    __shared__ CellsSmem C;
    using u64 = unsigned long long;
    if (plan->sort.key64)
        cells_body<u64, ValT, MULTI>(plan, prm, (const u64 *)keys_a, vals_a, (const u64 *)keys_b, vals_b, xyz,
                              rec, sc_of, sc_start, scode, cell_key, cell_sc, cframe, fr, tstat, C);
    else
        cells_body<uint32_t, ValT, MULTI>(plan, prm, (const uint32_t *)keys_a, vals_a,
                                   (const uint32_t *)keys_b, vals_b, xyz, rec, sc_of, sc_start,
                                   scode, cell_key, cell_sc, cframe, fr, tstat, C);
}

// The nominal (grid) centre of the sub-cell containing q, as the cell origin
// org (in quantised coordinates) and twice the centre's offset from it,
// cen2 = 2*s*h + h - 1 per axis (s = which half of the cell).  A point p of
// the same sub-cell lies at 2*(p - org) - cen2 from the centre, in units of
// half a quantum; both terms stay well inside 32 bits.
__device__ __forceinline__ void subcell_centre(const int32_t q[3], const int32_t lo[3], int32_t S,
                                               int32_t h, int32_t org[3], int32_t cen2[3])
{
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const uint32_t rel = (uint32_t)(q[a] - lo[a]);
        const uint32_t c = rel / (uint32_t)S;
        const uint32_t off = rel - c * (uint32_t)S;
        org[a] = (int32_t)((uint32_t)lo[a] + c * (uint32_t)S);
        cen2[a] = (off >= (uint32_t)h ? 2 * h : 0) + h - 1;
    }
}

// Grid origin (bounding-box corner) of the frame holding sorted position p.
__device__ __forceinline__ void frame_origin(const Frame *__restrict__ fr, uint32_t nf, uint32_t p,
                                             int32_t lo[3])
{
    const Frame &F = fr[frame_of_pos(fr, nf, p)];
    lo[0] = F.lo[0];
    lo[1] = F.lo[1];
    lo[2] = F.lo[2];
}

__device__ __forceinline__ float centre_dist2(const Rec &r, const int32_t org[3],
                                              const int32_t cen2[3])
{
    const float dx = (float)(2 * (r.x - org[0]) - cen2[0]);
    const float dy = (float)(2 * (r.y - org[1]) - cen2[1]);
    const float dz = (float)(2 * (r.z - org[2]) - cen2[2]);
    return dx * dx + dy * dy + dz * dz;
}

// a3: slab index over the brick rows of the major cell coordinate (see
// CellKeyLayout): cells of slab x occupy [slab_lo[x], slab_hi[x]) of the
// sorted cell array (empty: lo == hi == 0); and, when it fits, the dense
// column index over (c_p0, c_p1) (the cell key above c_p2) the same way.
// One thread per cell; run by the sub-cell statistics kernel after its own
// loop (the two read only the cell table).
__device__ __forceinline__ void slab_index(const Plan *plan, const unsigned long long *__restrict__ cell_key,
                                           const uint32_t *__restrict__ cell_sc,
                                           const uint8_t *__restrict__ scode,
                                           uint32_t *__restrict__ slab_lo, uint32_t *__restrict__ slab_hi,
                                           uint32_t *__restrict__ col_lo, uint32_t *__restrict__ col_hi,
                                           uint8_t *__restrict__ cocc, const uint32_t *__restrict__ cframe,
                                           const Frame *__restrict__ fr, uint32_t nf)
{
    const uint32_t M = plan->M_c;
    CellKeyLayout L;
    L.load(plan);
    const uint32_t b2 = L.b2;
    const uint32_t sh = L.b2 + L.b1 + L.B0;  // key bits below the brick row
    const bool cols = plan->use_cols != 0;
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < M; c += gridDim.x * blockDim.x) {
        const unsigned long long k = cell_key[c];
        const unsigned long long x = k >> sh, col = k >> b2;
        const unsigned long long kp = c > 0 ? cell_key[c - 1] : ~0ull;
        const unsigned long long kn = c + 1 < M ? cell_key[c + 1] : ~0ull;
        // slab x of the cell's frame; a frame change also ends a slab
        const uint32_t f = nf > 1 ? cframe[c] : 0u;
        const bool fprev = nf > 1 && c > 0 && cframe[c - 1] != f;
        const bool fnext = nf > 1 && c + 1 < M && cframe[c + 1] != f;
        const uint32_t se = fr[f].slab_base + (uint32_t)x;
        if (c == 0 || fprev || (kp >> sh) != x) slab_lo[se] = c;
        if (c + 1 == M || fnext || (kn >> sh) != x) slab_hi[se] = c + 1;
        if (cols) {
            if (c == 0 || (kp >> b2) != col) col_lo[col] = c;
            if (c + 1 == M || (kn >> b2) != col) col_hi[col] = c + 1;
        }
        // occupancy of the cell: bit s set when sub-cell code s is present
        // (its sub-cells are stored in increasing code order)
        uint32_t occ = 0;
        const uint32_t e = min(cell_sc[c + 1], cell_sc[c] + 8u);
        for (uint32_t a = cell_sc[c]; a < e; ++a) occ |= 1u << (scode[a] & 7u);
        cocc[c] = (uint8_t)occ;
    }
}

// a3: per sub-cell box, count, smallest original index and representative
// (the point nearest the sub-cell's nominal centre), in one pass over its
// points; initialise the union-find and component arrays.  Sub-cells above
// prm.big_subcell points are queued for k_subcell_large.  Then the slab and
// column index and the cell occupancies (slab_index).
__global__ void __launch_bounds__(256)
    k_subcell_stats(Plan *plan, Params prm, const Rec *__restrict__ rec,
                    const uint32_t *__restrict__ sc_start, SubBox *__restrict__ box,
                    uint32_t *__restrict__ sminidx, uint32_t *__restrict__ parent,
                    uint32_t *__restrict__ csize, uint32_t *__restrict__ cmin,
                    int32_t *__restrict__ crank, uint32_t *__restrict__ big, uint32_t *__restrict__ reps,
                    const Frame *__restrict__ fr, const unsigned long long *__restrict__ cell_key,
                    const uint32_t *__restrict__ cell_sc, const uint8_t *__restrict__ scode,
                    uint32_t *__restrict__ slab_lo, uint32_t *__restrict__ slab_hi,
                    uint32_t *__restrict__ col_lo, uint32_t *__restrict__ col_hi,
                    uint8_t *__restrict__ cocc, const uint32_t *__restrict__ cframe)
{
    grid_enter();
    if (call_aborted(&plan->status)) return;
    const uint32_t M = plan->M_s;
    const int32_t lo0[3] = {fr[0].lo[0], fr[0].lo[1], fr[0].lo[2]};  // one frame: its origin
    for (uint32_t a = blockIdx.x * blockDim.x + threadIdx.x; a < M; a += gridDim.x * blockDim.x) {
        parent[a] = a;
        csize[a] = 0;
        cmin[a] = 0xffffffffu;
        crank[a] = -1;
        const uint32_t s = sc_start[a], e = sc_start[a + 1];
        if (s >= e || e > plan->sort.n) {  // only after a look-back timeout
            atomicOr(&plan->status, ST_SIZE_OVERFLOW);
            box[a] = SubBox{0, 0, 0, 0, 0, 0, 0, 0};
            sminidx[a] = 0;
            reps[a] = kNoRep;
            continue;
        }
        if (e - s > prm.big_subcell) {
            // medium sub-cells from the front of the list, huge ones from its middle
            // (at most n/65 and n/2049 of them)
            if (e - s > (uint32_t)kHugeSubcell) {
                const uint32_t j = atomicAdd(&plan->n_huge, 1u);
                if (FEC_IN_BOUNDS(&plan->status, j, plan->sort.n / (kHugeSubcell + 1) + 1))
                    big[plan->sort.n / 2 + j] = a;
            } else {
                const uint32_t j = atomicAdd(&plan->n_big, 1u);
                if (FEC_IN_BOUNDS(&plan->status, j, plan->sort.n / 2)) big[j] = a;
            }
            continue;
        }
        SubBox b;
        b.lx = b.ly = b.lz = INT32_MAX;
        b.hx = b.hy = b.hz = INT32_MIN;
        uint32_t mi = 0xffffffffu;
        const Rec r0 = rec[s];
        int32_t org[3], cen2[3];
        const int32_t q0[3] = {r0.x, r0.y, r0.z};
        int32_t lo[3] = {lo0[0], lo0[1], lo0[2]};
        if (prm.nf > 1) frame_origin(fr, prm.nf, s, lo);
        subcell_centre(q0, lo, prm.S, prm.h, org, cen2);
        float best = __int_as_float(0x7f800000);
        Rec rp = r0;
        for (uint32_t p = s; p < e; ++p) {
            const Rec r = rec[p];
            b.lx = min(b.lx, r.x); b.hx = max(b.hx, r.x);
            b.ly = min(b.ly, r.y); b.hy = max(b.hy, r.y);
            b.lz = min(b.lz, r.z); b.hz = max(b.hz, r.z);
            mi = min(mi, r.idx);
            const float dd = centre_dist2(r, org, cen2);
            if (dd < best) {
                best = dd;
                rp = r;
            }
        }
        b.start = s;
        b.count = e - s;
        box[a] = b;
        sminidx[a] = mi;
        reps[a] = pack_rep(rp, b.lx, b.ly, b.lz);
    }
    slab_index(plan, cell_key, cell_sc, scode, slab_lo, slab_hi, col_lo, col_hi, cocc, cframe, fr, prm.nf);
}

// a3: the same for the queued sub-cells of big_subcell..kHugeSubcell points,
// one warp per sub-cell (block `blk` of `nblk` blocks doing this part).
__device__ __forceinline__ void subcell_big(Plan *plan, const Params &prm, const Rec *__restrict__ rec,
                                            const uint32_t *__restrict__ sc_start,
                                            const uint32_t *__restrict__ big, SubBox *__restrict__ box,
                                            uint32_t *__restrict__ sminidx, uint32_t *__restrict__ reps,
                                            const Frame *__restrict__ fr, uint32_t blk, uint32_t nblk)
{
    if (call_aborted(&plan->status)) return;
    const uint32_t nb = plan->n_big;
    const int l = threadIdx.x & 31;
    const uint32_t nwarps = nblk * (blockDim.x >> 5);
    for (uint32_t j = blk * (blockDim.x >> 5) + (threadIdx.x >> 5); j < nb; j += nwarps) {
        const uint32_t a = big[j];
        const uint32_t s = sc_start[a], e = sc_start[a + 1];
        const Rec r0 = rec[s];
        int32_t org[3], cen2[3];
        const int32_t q0[3] = {r0.x, r0.y, r0.z};
        int32_t lo[3];
        frame_origin(fr, prm.nf, s, lo);
        subcell_centre(q0, lo, prm.S, prm.h, org, cen2);
        int32_t L[3] = {INT32_MAX, INT32_MAX, INT32_MAX}, H[3] = {INT32_MIN, INT32_MIN, INT32_MIN};
        uint32_t mi = 0xffffffffu;
        unsigned long long bk = ~0ull;
        for (uint32_t p = s + l; p < e; p += 32) {
            const Rec r = rec[p];
            L[0] = min(L[0], r.x); H[0] = max(H[0], r.x);
            L[1] = min(L[1], r.y); H[1] = max(H[1], r.y);
            L[2] = min(L[2], r.z); H[2] = max(H[2], r.z);
            mi = min(mi, r.idx);
            const unsigned long long k =
                ((unsigned long long)__float_as_uint(centre_dist2(r, org, cen2)) << 32) | (p - s);
            bk = k < bk ? k : bk;
        }
#pragma unroll
        for (int a3 = 0; a3 < 3; ++a3) {
            L[a3] = warp_min(L[a3]);
            H[a3] = warp_max(H[a3]);
        }
        mi = warp_min(mi);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long u = __shfl_xor_sync(0xffffffffu, bk, o);
            bk = u < bk ? u : bk;
        }
        if (l == 0) {
            SubBox b;
            b.lx = L[0]; b.ly = L[1]; b.lz = L[2];
            b.hx = H[0]; b.hy = H[1]; b.hz = H[2];
            b.start = s;
            b.count = e - s;
            box[a] = b;
            sminidx[a] = mi;
            reps[a] = pack_rep(rec[s + (uint32_t)bk], b.lx, b.ly, b.lz);
        }
    }
}

// a3: the same for the queued sub-cells above kHugeSubcell points, one block
// per sub-cell (block `blk` of `nblk` blocks doing this part).
__device__ __forceinline__ void subcell_huge(Plan *plan, const Params &prm, const Rec *__restrict__ rec,
                                             const uint32_t *__restrict__ sc_start,
                                             const uint32_t *__restrict__ big, SubBox *__restrict__ box,
                                             uint32_t *__restrict__ sminidx, uint32_t *__restrict__ reps,
                                             const Frame *__restrict__ fr, uint32_t blk, uint32_t nblk)
{
    __shared__ int32_t s_v[7][8];
    __shared__ unsigned long long s_k[8];
    if (block_aborted(&plan->status)) return;
    const uint32_t nb = plan->n_huge;
    big += plan->sort.n / 2;
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    for (uint32_t j = blk; j < nb; j += nblk) {
        const uint32_t a = big[j];
        const uint32_t s = sc_start[a], e = sc_start[a + 1];
        const Rec r0 = rec[s];
        int32_t org[3], cen2[3];
        const int32_t q0[3] = {r0.x, r0.y, r0.z};
        int32_t lo[3];
        frame_origin(fr, prm.nf, s, lo);
        subcell_centre(q0, lo, prm.S, prm.h, org, cen2);
        int32_t L[3] = {INT32_MAX, INT32_MAX, INT32_MAX}, H[3] = {INT32_MIN, INT32_MIN, INT32_MIN};
        uint32_t mi = 0xffffffffu;
        unsigned long long bk = ~0ull;
        for (uint32_t p = s + threadIdx.x; p < e; p += blockDim.x) {
            const Rec r = rec[p];
            L[0] = min(L[0], r.x); H[0] = max(H[0], r.x);
            L[1] = min(L[1], r.y); H[1] = max(H[1], r.y);
            L[2] = min(L[2], r.z); H[2] = max(H[2], r.z);
            mi = min(mi, r.idx);
            const unsigned long long k =
                ((unsigned long long)__float_as_uint(centre_dist2(r, org, cen2)) << 32) | (p - s);
            bk = k < bk ? k : bk;
        }
#pragma unroll
        for (int a3 = 0; a3 < 3; ++a3) {
            L[a3] = warp_min(L[a3]);
            H[a3] = warp_max(H[a3]);
        }
        mi = warp_min(mi);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long u = __shfl_xor_sync(0xffffffffu, bk, o);
            bk = u < bk ? u : bk;
        }
        if (l == 0) {
            for (int a3 = 0; a3 < 3; ++a3) {
                s_v[a3][w] = L[a3];
                s_v[3 + a3][w] = H[a3];
            }
            s_v[6][w] = (int32_t)mi;
            s_k[w] = bk;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            SubBox b;
            int32_t LL[3] = {INT32_MAX, INT32_MAX, INT32_MAX}, HH[3] = {INT32_MIN, INT32_MIN, INT32_MIN};
            uint32_t m = 0xffffffffu;
            unsigned long long kk = ~0ull;
            for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
                for (int a3 = 0; a3 < 3; ++a3) {
                    LL[a3] = min(LL[a3], s_v[a3][k]);
                    HH[a3] = max(HH[a3], s_v[3 + a3][k]);
                }
                m = min(m, (uint32_t)s_v[6][k]);
                kk = s_k[k] < kk ? s_k[k] : kk;
            }
            b.lx = LL[0]; b.ly = LL[1]; b.lz = LL[2];
            b.hx = HH[0]; b.hy = HH[1]; b.hz = HH[2];
            b.start = s;
            b.count = e - s;
            box[a] = b;
            sminidx[a] = m;
            reps[a] = pack_rep(rec[s + (uint32_t)kk], b.lx, b.ly, b.lz);
        }
        __syncthreads();
    }
}

// a3: the large sub-cells, in one launch: the first `huge_blocks` blocks take
// the huge ones (a block each), the rest the big ones (a warp each).
__global__ void __launch_bounds__(256)
    k_subcell_large(Plan *plan, Params prm, const Rec *__restrict__ rec,
                    const uint32_t *__restrict__ sc_start, const uint32_t *__restrict__ big,
                    SubBox *__restrict__ box, uint32_t *__restrict__ sminidx, uint32_t *__restrict__ reps,
                    const Frame *__restrict__ fr, uint32_t huge_blocks)
{
    grid_enter();
    if (blockIdx.x < huge_blocks)
        subcell_huge(plan, prm, rec, sc_start, big, box, sminidx, reps, fr, blockIdx.x, huge_blocks);
    else
        subcell_big(plan, prm, rec, sc_start, big, box, sminidx, reps, fr, blockIdx.x - huge_blocks,
                    gridDim.x - huge_blocks);
}

cudaError_t enqueue_front(Workspace &ws, const float *xyz, const Params &prm, const FrontArgs &fa,
                          cudaStream_t st)
{
    // one frame: four points per thread over the whole grid; several:
    // blocks take contiguous runs of 1024-point units (frame-aligned)
    const bool multi = prm.nf > 1;
    const int grid = multi ? (int)std::min<uint64_t>((uint64_t)prm.ntiles * kUnitsPerTile,
                                                     (uint64_t)ws.sms * 8)
                           : grid_for(ws, prm.n, 1024, 8);
    const uint64_t hist_words = (uint64_t)prm.nf * kMaxPasses * kRadixBins;
    const int igrid = (int)std::min<uint64_t>((hist_words + 2047) / 2048, (uint64_t)ws.sms * 4);
    launch(k_init, igrid < 1 ? 1 : igrid, 256, 0, st, ws.plan, ws.frames, prm.nf, ws.fhist, prm.n,
                                                  prm.wait_cap, fa.single ? 1 : 0, fa.min_size,
                                                  fa.max_size);
    FEC_MARK(ws, "k_init", st);
    if (multi) launch(k_bbox<true>, grid, 256, 0, st, xyz, ws.plan, ws.frames, prm);
    else launch(k_bbox<false>, grid, 256, 0, st, xyz, ws.plan, ws.frames, prm);
    FEC_MARK(ws, "k_bbox", st);
    Clears clr;
    clr.sort_status = ws.sort_status;
    clr.sort_words = ((size_t)prm.ntiles + 1) * kRadixBins;  // look-back array 0, this call's tiles
    clr.scan_status = ws.scan_status;
    clr.scan_words = (size_t)prm.n / kScanTile + 2;
    clr.slab_lo = ws.slab_lo;
    clr.slab_hi = ws.slab_hi;
    clr.slab_words = prm.slab_cap;
    clr.col_lo = ws.col_lo;
    clr.col_hi = ws.col_hi;
    clr.rank_bits = ws.rank_bits;
    clr.rank_words = ((size_t)prm.n + 31) / 32;
    clr.rank_status = ws.rank_status;
    clr.rank_status_words = clr.rank_words / 2048 + 2;
    clr.max_words = std::max({clr.sort_words, clr.scan_words, clr.slab_words, clr.rank_words});
    // packed layout: the sort's first pass computes the keys itself
    if (prm.packed && !multi)
        launch(k_keys<false, false>, grid, 256, 0, st, xyz, ws.plan, prm, ws.frames, ws.fhist, ws.keys_a, clr);
    else if (prm.packed)
        launch(k_keys<false, true>, grid, 256, 0, st, xyz, ws.plan, prm, ws.frames, ws.fhist, ws.keys_a, clr);
    else if (!multi)
        launch(k_keys<true, false>, grid, 256, 0, st, xyz, ws.plan, prm, ws.frames, ws.fhist, ws.keys_a, clr);
    else
        launch(k_keys<true, true>, grid, 256, 0, st, xyz, ws.plan, prm, ws.frames, ws.fhist, ws.keys_a, clr);
    FEC_MARK(ws, "k_keys", st);
    return cudaGetLastError();
}

cudaError_t enqueue_cells(Workspace &ws, const float *xyz, const Params &prm, cudaStream_t st)
{
    // the look-back status and the slab index were cleared by the key kernel
    const int grid = grid_for(ws, prm.n, kScanTile, 8);
    const int grid1 = grid_for(ws, prm.n, 256, 8);  // one item per thread
    using u32 = uint32_t;
    using u64 = unsigned long long;
    // one frame, or several (frame starts, frame origins, cell frames)
    const u64 *va64 = (const u64 *)ws.vals_a, *vb64 = (const u64 *)ws.vals_b;
    const u32 *va32 = (const u32 *)ws.vals_a, *vb32 = (const u32 *)ws.vals_b;
#define FEC_CELLS_ARGS(va, vb)                                                                   \
    ws.plan, prm, ws.keys_a, va, ws.keys_b, vb, xyz, ws.rec, ws.sc_of, ws.sc_start, ws.scode,     \
        ws.cell_key, ws.cell_sc, ws.cframe, ws.frames, ws.scan_status
    if (prm.packed && prm.nf == 1)
        launch(k_cells<u64, false>, grid, kScanThreads, 0, st, FEC_CELLS_ARGS(va64, vb64));
    else if (prm.packed)
        launch(k_cells<u64, true>, grid, kScanThreads, 0, st, FEC_CELLS_ARGS(va64, vb64));
    else if (prm.nf == 1)
        launch(k_cells<u32, false>, grid, kScanThreads, 0, st, FEC_CELLS_ARGS(va32, vb32));
    else
        launch(k_cells<u32, true>, grid, kScanThreads, 0, st, FEC_CELLS_ARGS(va32, vb32));
#undef FEC_CELLS_ARGS
    FEC_MARK(ws, "k_cells", st);
    launch(k_subcell_stats, grid1, 256, 0, st, ws.plan, prm, ws.rec, ws.sc_start, ws.box, ws.sminidx,
           ws.parent, ws.csize, ws.cmin, ws.crank, ws.big, ws.reps, ws.frames, ws.cell_key, ws.cell_sc,
           ws.scode, ws.slab_lo, ws.slab_hi, ws.col_lo, ws.col_hi, ws.cocc, ws.cframe);
    FEC_MARK(ws, "k_subcell_stats", st);
    const int huge_blocks = grid_for(ws, prm.n / (kHugeSubcell + 1), 1, 2);
    const int big_blocks = grid_for(ws, prm.n / (prm.big_subcell + 1), 8, 4);
    launch(k_subcell_large, huge_blocks + big_blocks, 256, 0, st, ws.plan, prm, ws.rec, ws.sc_start, ws.big,
                                                             ws.box, ws.sminidx, ws.reps, ws.frames,
                                                             (uint32_t)huge_blocks);
    FEC_MARK(ws, "k_subcell_large", st);
    return cudaGetLastError();
}

}  // namespace fec
