// fec_union.cu -- a4 neighbour test + union, a5 flatten, a6 size filter and
// canonical relabelling.
//
// a4 replaces Algorithm 1's main loop (FindNeighbor + the segment-merge loop
// that rewrites labels across the whole cloud): every cell is visited once
// by a warp, which finds its half-stencil neighbour cells (13 of the 26;
// the other half is covered by the neighbours' own visits) through the slab
// index, and decides every sub-cell pair (a in this cell, b in the cell or a
// neighbour):
//   - box gap above R: no edge;
//   - box diameter within R: edge (all cross pairs within d);
//   - otherwise the warp tests point pairs until the first hit.
// Edges join union-find sets (hook the larger root under the smaller with
// atomicCAS); pairs whose sub-cells already share a root are skipped.
//
// a6: components outside [min_size, max_size] are dropped; kept components
// are sorted by their smallest point index and numbered 0..k-1.
#include "fec_internal.cuh"

namespace fec {

namespace {

constexpr int kUnionThreads = 256;

// Squared distance of an offset, compared against T2.  Narrow form: each
// |component| is clamped to R+1 (anything above R already fails the test),
// so the sum of squares stays below 2^31 when R+1 <= 26754.
template <bool WIDE>
struct Metric {
    using T = typename std::conditional<WIDE, long long, int>::type;
    T T2;
    int R1;
    __device__ __forceinline__ T axis(int d) const
    {
        if (WIDE) return (T)d;
        return (T)min(abs(d), R1);
    }
    __device__ __forceinline__ bool within(int dx, int dy, int dz) const
    {
        const T x = axis(dx), y = axis(dy), z = axis(dz);
        return x * x + y * y + z * z <= T2;
    }
    // squared gap between a point and a box
    __device__ __forceinline__ bool point_box(const Rec &p, const SubBox &b) const
    {
        const int gx = max(0, max(b.lx - p.x, p.x - b.hx));
        const int gy = max(0, max(b.ly - p.y, p.y - b.hy));
        const int gz = max(0, max(b.lz - p.z, p.z - b.hz));
        return within(gx, gy, gz);
    }
    __device__ __forceinline__ bool box_gap(const SubBox &a, const SubBox &b) const
    {
        const int gx = max(0, max(b.lx - a.hx, a.lx - b.hx));
        const int gy = max(0, max(b.ly - a.hy, a.ly - b.hy));
        const int gz = max(0, max(b.lz - a.hz, a.lz - b.hz));
        return within(gx, gy, gz);
    }
    __device__ __forceinline__ bool box_diam(const SubBox &a, const SubBox &b) const
    {
        const int mx = max(a.hx - b.lx, b.hx - a.lx);
        const int my = max(a.hy - b.ly, b.hy - a.ly);
        const int mz = max(a.hz - b.lz, b.hz - a.lz);
        return within(mx, my, mz);
    }
};

// Squared distances in float, used only to order candidates (the decisions
// below are always taken with the exact integer Metric).
__device__ __forceinline__ float d2f(const Rec &p, const Rec &q)
{
    const float dx = (float)(p.x - q.x), dy = (float)(p.y - q.y), dz = (float)(p.z - q.z);
    return dx * dx + dy * dy + dz * dz;
}
__device__ __forceinline__ float d2boxf(const Rec &p, const SubBox &b)
{
    const float gx = (float)max(0, max(b.lx - p.x, p.x - b.hx));
    const float gy = (float)max(0, max(b.ly - p.y, p.y - b.hy));
    const float gz = (float)max(0, max(b.lz - p.z, p.z - b.hz));
    return gx * gx + gy * gy + gz * gz;
}

// Warp-wide argmin over records [start, start + count) of the float squared
// distance to a box (to_box) or to a point.  Non-negative floats order like
// their bit patterns, so (bits << 32 | index) reduces with an integer min.
__device__ __forceinline__ uint32_t warp_argmin(const Rec *__restrict__ rec, uint32_t start,
                                                uint32_t count, bool to_box, SubBox b, Rec q)
{
    const int lane = threadIdx.x & 31;
    float best = __int_as_float(0x7f800000);
    uint32_t bi = 0;
    for (uint32_t i = lane; i < count; i += 32) {
        const Rec p = rec[start + i];
        const float k = to_box ? d2boxf(p, b) : d2f(p, q);
        if (k < best) {
            best = k;
            bi = i;
        }
    }
    unsigned long long pk = ((unsigned long long)__float_as_uint(best) << 32) | bi;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long u = __shfl_xor_sync(0xffffffffu, pk, o);
        pk = u < pk ? u : pk;
    }
    return (uint32_t)pk;
}

// Whole-warp decision for sub-cells a and b whose boxes are neither
// separated nor within d: is some point pair within d?  Warp-uniform result;
// *evals counts point-level distance evaluations.
//   1. Exact pruning: if no point of A is within d of B's box (or vice
//      versa), there is no edge.
//   2. Witness search: alternate nearest-point queries A -> B -> A -> B
//      starting from A's point nearest to B's box; any pair found within d
//      is an edge.  In dense regions this finds a witness in O(|A| + |B|).
//   3. Otherwise every candidate pair is tested.
template <bool WIDE>
__device__ __forceinline__ bool warp_pair_test(uint32_t a, uint32_t b, const SubBox *__restrict__ box,
                                               const Rec *__restrict__ rec, const Metric<WIDE> &m,
                                               unsigned long long &evals)
{
    const int lane = threadIdx.x & 31;
    const SubBox A = box[a], B = box[b];
    evals += A.count + B.count;
    // 1. exact pruning by point-to-box distance
    bool anyA = false, anyB = false;
    for (uint32_t i = lane; i < A.count; i += 32) anyA |= m.point_box(rec[A.start + i], B);
    if (!__any_sync(0xffffffffu, anyA)) return false;
    for (uint32_t i = lane; i < B.count; i += 32) anyB |= m.point_box(rec[B.start + i], A);
    if (!__any_sync(0xffffffffu, anyB)) return false;
    // 2. witness search
    Rec pa = rec[A.start + warp_argmin(rec, A.start, A.count, true, B, Rec{})];
    for (int round = 0; round < 2; ++round) {
        const Rec pb = rec[B.start + warp_argmin(rec, B.start, B.count, false, A, pa)];
        evals += A.count + B.count;
        if (m.within(pa.x - pb.x, pa.y - pb.y, pa.z - pb.z)) return true;
        pa = rec[A.start + warp_argmin(rec, A.start, A.count, false, B, pb)];
        if (m.within(pa.x - pb.x, pa.y - pb.y, pa.z - pb.z)) return true;
    }
    // 3. exhaustive over candidates near the other box
    for (uint32_t ca = 0; ca < A.count; ca += 32) {
        const bool in = ca + lane < A.count;
        Rec p;
        p.x = p.y = p.z = 0;
        p.idx = 0;
        if (in) p = rec[A.start + ca + lane];
        const bool cand = in && m.point_box(p, B);
        if (!__any_sync(0xffffffffu, cand)) continue;
        for (uint32_t j = 0; j < B.count; ++j) {
            const Rec q = rec[B.start + j];
            if (!m.point_box(q, A)) continue;  // uniform across the warp
            ++evals;
            if (__any_sync(0xffffffffu, cand && m.within(p.x - q.x, p.y - q.y, p.z - q.z)))
                return true;
        }
    }
    return false;
}

// One thread decides a pair alone (used only when the pair queue is full).
template <bool WIDE>
__device__ __noinline__ bool thread_pair_test(uint32_t a, uint32_t b, const SubBox *__restrict__ box,
                                              const Rec *__restrict__ rec, const Metric<WIDE> &m)
{
    const SubBox A = box[a], B = box[b];
    for (uint32_t i = 0; i < A.count; ++i) {
        const Rec p = rec[A.start + i];
        if (!m.point_box(p, B)) continue;
        for (uint32_t j = 0; j < B.count; ++j) {
            const Rec q = rec[B.start + j];
            if (m.within(p.x - q.x, p.y - q.y, p.z - q.z)) return true;
        }
    }
    return false;
}

// Box-level decision for a sub-cell pair: 0 = no edge (boxes farther than
// d), 1 = edge (box diameter within d, or the two representatives within
// d), 2 = undecided (needs point tests).
template <bool WIDE>
__device__ __forceinline__ int box_decide(const SubBox &A, const SubBox &B, uint32_t ra,
                                          uint32_t rb, const Metric<WIDE> &m)
{
    if (!m.box_gap(A, B)) return 0;
    if (m.box_diam(A, B)) return 1;
    if (ra != kNoRep && rb != kNoRep &&  // the two representatives (packed, see pack_rep)
        m.within((A.lx + (int)(ra & 1023u)) - (B.lx + (int)(rb & 1023u)),
                 (A.ly + (int)((ra >> 10) & 1023u)) - (B.ly + (int)((rb >> 10) & 1023u)),
                 (A.lz + (int)(ra >> 20)) - (B.lz + (int)(rb >> 20))))
        return 1;
    return 2;
}

// Cells of column (n0, n1) with minor coordinate in [z_lo, z_hi] (at most
// 3): through the dense column index when the plan enables it, else by
// binary search in the slab (brick row) of n0.  Returns how many were
// written to out[].
__device__ __forceinline__ int column_cells(unsigned long long n0, unsigned long long n1,
                                            unsigned long long z_lo, unsigned long long z_hi,
                                            const CellKeyLayout &L, const Plan *plan,
                                            uint32_t slab_base, uint32_t nslab,
                                            const unsigned long long *__restrict__ cell_key,
                                            const uint32_t *__restrict__ slab_lo,
                                            const uint32_t *__restrict__ slab_hi,
                                            const uint32_t *__restrict__ col_lo,
                                            const uint32_t *__restrict__ col_hi, uint32_t out[3])
{
    uint32_t lo, end;
    const unsigned long long colkey = L.column(n0, n1);
    if (plan->use_cols) {
        const unsigned long long col = colkey >> L.b2;
        lo = col_lo[col];
        end = col_hi[col];
    } else {
        const unsigned long long x = L.slab_of(n0);
        if (x >= nslab) return 0;  // beyond the frame's slabs
        lo = slab_lo[slab_base + x];
        end = slab_hi[slab_base + x];
    }
    const unsigned long long tlo = colkey | z_lo, thi = colkey | z_hi;
    uint32_t hi = end;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (cell_key[mid] < tlo) lo = mid + 1;
        else hi = mid;
    }
    int k = 0;
    for (uint32_t q = lo; q < end && k < 3; ++q) {
        if (cell_key[q] > thi) break;
        out[k++] = q;
    }
    return k;
}

// The half-stencil neighbour cells of cell c (13 of the 26; the other half
// is covered by the neighbours' own visits), one column per lane: lanes
// 0..3 take columns (0,+1), (+1,-1), (+1,0), (+1,+1) over dz in {-1,0,+1},
// lane 4 takes (0,0,+1), the next cell of the same column (of the same
// frame).  Each lane returns its cells in f[0..2] and their count.
__device__ __forceinline__ int stencil_lane(int lane, uint32_t c, uint32_t M, unsigned long long ck,
                                            const CellKeyLayout &L, const Plan *plan,
                                            uint32_t slab_base, uint32_t nslab, bool next_same,
                                            const unsigned long long *__restrict__ cell_key,
                                            const uint32_t *__restrict__ slab_lo,
                                            const uint32_t *__restrict__ slab_hi,
                                            const uint32_t *__restrict__ col_lo,
                                            const uint32_t *__restrict__ col_hi, uint32_t f[3])
{
    const unsigned long long m1 = (1ull << L.b1) - 1, m2 = (1ull << L.b2) - 1;
    unsigned long long c0, c1, c2;
    L.decode(ck, c0, c1, c2);
    if (lane == 4) {
        if (c2 < m2 && c + 1 < M && next_same && cell_key[c + 1] == ck + 1) {
            f[0] = c + 1;
            return 1;
        }
        return 0;
    }
    if (lane > 3) return 0;
    const long long d0 = lane == 0 ? 0 : 1;
    const long long d1 = lane == 0 ? 1 : lane - 2;
    const long long n0 = (long long)c0 + d0, n1 = (long long)c1 + d1;
    const unsigned long long m0 = (1ull << L.b0) - 1;
    if (n1 < 0 || (unsigned long long)n1 > m1 || (unsigned long long)n0 > m0) return 0;
    return column_cells((unsigned long long)n0, (unsigned long long)n1, c2 > 0 ? c2 - 1 : 0,
                        c2 < m2 ? c2 + 1 : m2, L, plan, slab_base, nslab, cell_key, slab_lo,
                        slab_hi, col_lo, col_hi, f);
}

// Position of the r-th (from 0) set bit of the 8-bit mask m (r < popc(m)).
__device__ __forceinline__ uint32_t select8(uint32_t m, uint32_t r)
{
    uint32_t pos = 0;
    const uint32_t c4 = __popc(m & 15u);
    if (r >= c4) {
        r -= c4;
        pos = 4;
    }
    const uint32_t c2 = __popc((m >> pos) & 3u);
    if (r >= c2) {
        r -= c2;
        pos += 2;
    }
    if (r >= ((m >> pos) & 1u)) pos += 1;
    return pos;
}

// ceil(65536 / n) for n = 1..8: i / n == (i * kRecip[n]) >> 16 for i < 8192.
__constant__ uint32_t kRecip[9] = {0, 65536, 32768, 21846, 16384, 13108, 10923, 9363, 8192};

// a4: half-stencil neighbour lists, one thread per cell: for each of the
// cell's K <= 13 neighbour cells, its first sub-cell, its sub-cell occupancy
// (bit s set when its sub-cell with code s exists; sub-cells are stored in
// code order, so the r-th sub-cell has the r-th set bit's code) and its
// offset from the cell (per permuted axis, in sub-cell-code bit order:
// bit 2 = p0, bit 1 = p1, bit 0 = p2).  32 bytes per cell:
//   nb_first[c * 13 + k]
//   nb[c * 32 + k]      occupancy of neighbour k              (k < K)
//   nb[c * 32 + 13]     occupancy of the cell itself
//   nb[c * 32 + 15]     K
//   nb[c * 32 + 16 + k] axes at +1 | axes at -1 << 3          (k < K)
// (p0 is never at -1 in the half stencil, so two bits hold the -1 axes.)
__global__ void __launch_bounds__(256, 4)
    k_nbrs(Plan *plan, Params prm, const unsigned long long *__restrict__ cell_key,
           const uint32_t *__restrict__ cell_sc, const uint32_t *__restrict__ slab_lo,
           const uint32_t *__restrict__ slab_hi, const uint32_t *__restrict__ col_lo,
           const uint32_t *__restrict__ col_hi, const uint8_t *__restrict__ cocc,
           uint32_t *__restrict__ nb_first, uint8_t *__restrict__ nb_cnt,
           unsigned long long *__restrict__ edge_set, uint32_t edge_set_size,
           const uint32_t *__restrict__ cframe, const Frame *__restrict__ fr)
{
    grid_enter();
    if (call_aborted(&plan->status)) return;
    // the boundary-edge hash set of k_edges starts empty
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < edge_set_size;
         i += gridDim.x * blockDim.x)
        edge_set[i] = ~0ull;
    const uint32_t M = plan->M_c;
    CellKeyLayout L;
    L.load(plan);
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < M; c += gridDim.x * blockDim.x) {
        const unsigned long long ck = cell_key[c];
        unsigned long long e0, e1, e2;  // the cell's coordinates
        L.decode(ck, e0, e1, e2);
        uint32_t wv[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        int K = 0;
        // the cell's frame: its part of the slab index; the next cell must be of it too
        const uint32_t fc = prm.nf > 1 ? cframe[c] : 0u;
        const uint32_t sbase = fr[fc].slab_base, nslab = fr[fc].nslab;
        const bool next_same = prm.nf == 1 || (c + 1 < M && cframe[c + 1] == fc);
#pragma unroll
        for (int col = 0; col < 5; ++col) {
            uint32_t f[3];
            const int nf = stencil_lane(col == 0 ? 4 : col - 1, c, M, ck, L, plan, sbase, nslab,
                                        next_same, cell_key, slab_lo, slab_hi, col_lo, col_hi, f);
            for (int t = 0; t < nf; ++t) {
                if (!FEC_IN_BOUNDS(&plan->status, f[t], M) || !FEC_IN_BOUNDS(&plan->status, K, 13)) break;
                const uint32_t q = f[t], first = cell_sc[q];
                nb_first[(size_t)c * 13 + K] = first;
                unsigned long long n0, n1, n2;
                L.decode(cell_key[q], n0, n1, n2);
                const long long d0 = (long long)n0 - (long long)e0;
                const long long d1 = (long long)n1 - (long long)e1;
                const long long d2 = (long long)n2 - (long long)e2;
                const uint32_t plus = (d0 == 1 ? 4u : 0u) | (d1 == 1 ? 2u : 0u) | (d2 == 1 ? 1u : 0u);
                const uint32_t minus = (d1 == -1 ? 2u : 0u) | (d2 == -1 ? 1u : 0u);
                // K < 13, so the word indices below stay in range (unrolled: registers)
#pragma unroll
                for (int wi = 0; wi < 4; ++wi) {
                    if ((K >> 2) == wi) {
                        wv[wi] |= (uint32_t)cocc[q] << (8 * (K & 3));
                        wv[4 + wi] |= (plus | (minus << 3)) << (8 * (K & 3));
                    }
                }
                ++K;
            }
        }
        wv[3] |= ((uint32_t)cocc[c] << 8) | ((uint32_t)K << 24);
        reinterpret_cast<uint4 *>(nb_cnt)[2 * (size_t)c] = make_uint4(wv[0], wv[1], wv[2], wv[3]);
        reinterpret_cast<uint4 *>(nb_cnt)[2 * (size_t)c + 1] = make_uint4(wv[4], wv[5], wv[6], wv[7]);
    }
}

// ---------------------------------------------------------------------------
// a4: region-local connectivity.  A block takes a region of kRegionCells
// consecutive cells (fewer when the cloud is small, so that every block gets
// work; in key order, i.e. a compact piece of space) and keeps a
// union-find over the region's sub-cells in shared memory.  Its warps take
// the region's cells one at a time and decide sub-cell pairs 32 at a time:
// the cell's own pairs and its half-stencil neighbour pairs (13 of the 26
// neighbour cells; the other half is covered by the neighbours' own visits).
//   phase A: pairs already joined in the region are skipped; box gap above
//            d = no edge; box diameter or representatives within d = edge
//            (joined in shared memory, or emitted as a boundary edge when
//            the neighbour lies in another region);
//   phase B: the undecided pairs still apart: inside the region a warp tests
//            points (witness search) and joins on a hit; across regions
//            they are queued for k_pairs;
//   phase C: every sub-cell's global parent = its region-local root.
// Only boundary edges and cross-region pairs leave the block, through
// shared-memory buffers flushed in chunks.
// ---------------------------------------------------------------------------
#ifndef FEC_REGION_TAIL_ROUNDS
#define FEC_REGION_TAIL_ROUNDS 1
#endif
constexpr uint32_t kRegionTailRounds = FEC_REGION_TAIL_ROUNDS;
constexpr int kRegionCells = (int)kRegionCellsPerBlock;
constexpr int kRegionWarps = kRegionThreads / 32;
constexpr int kRegionSubs = 8 * kRegionCells;
static_assert(kRegionSubs <= 65536, "region-local sub-cell indices are 16-bit");
#ifndef FEC_REGION_BUF
#define FEC_REGION_BUF 1024
#endif
constexpr int kRegionBuf = FEC_REGION_BUF;

using RegionPar = uint16_t;
struct RegionSmem {
    RegionPar par[kRegionSubs];            // union-find parent, region-local (< 2^16)
    uint2 ebuf[kRegionBuf];   // boundary edges
    uint2 qbuf[kRegionBuf];   // cross-region undecided pairs
    uint32_t ecount, qcount, next, region, rend, pad[3];
    // per cell slot (two per warp, one per half-warp), per neighbour sub-cell
    // (in stencil order): its index, and its code (bits 0-2) with its cell's
    // axes at +1 (bits 3-5) and at -1 (bits 6-7); per own sub-cell: its code
    uint32_t nsub[2 * kRegionWarps][112];
    uint8_t ninfo[2 * kRegionWarps][112];
    uint8_t ocode[2 * kRegionWarps][8];
    uint32_t qa[kRegionWarps][64];         // queued pairs (a, b) of each warp
    uint32_t qb[kRegionWarps][64];
};

__device__ __forceinline__ uint32_t s_find(volatile RegionPar *par, uint32_t x)
{
    for (;;) {
        const uint32_t p = par[x];
        if (p == x) return x;
        const uint32_t g = par[p];
        if (g == p) return p;
        par[x] = g;  // path halving (g is an ancestor of x)
        x = g;
    }
}

__device__ __forceinline__ void s_unite(RegionPar *par, uint32_t a, uint32_t b)
{
    volatile RegionPar *vp = par;
    for (;;) {
        a = s_find(vp, a);
        b = s_find(vp, b);
        if (a == b) return;
        if (a < b) {
            const uint32_t t = a;
            a = b;
            b = t;
        }
        const uint32_t old = atomicCAS(reinterpret_cast<unsigned short *>(par + a), (unsigned short)a,
                                       (unsigned short)b);
        if (old == a) return;
        a = old;
    }
}

// Warp-aggregated append of the lanes in `mask` to a shared-memory buffer;
// when the buffer is full the entries go straight to the global list (or,
// if that is full too, are handled by `overflow`).  Unused buffer slots keep
// the sentinel written at block start.
template <typename F>
__device__ __forceinline__ void buf_append(uint32_t mask, bool mine, uint2 v, uint2 *sbuf,
                                           uint32_t *scount, uint2 *glist, uint32_t *gcount,
                                           uint32_t gcap, F overflow)
{
    if (!mask) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(mask) - 1;
    const uint32_t e = __popc(mask), rank = __popc(mask & lanemask_lt());
    uint32_t slot = 0;
    if (lane == leader) slot = atomicAdd(scount, e);
    slot = __shfl_sync(0xffffffffu, slot, leader);
    if (slot + e <= (uint32_t)kRegionBuf) {
        if (mine) sbuf[slot + rank] = v;
        return;
    }
    uint32_t g = 0;
    if (lane == leader) g = atomicAdd(gcount, e);
    g = __shfl_sync(0xffffffffu, g, leader);
    if (mine) {
        if (g + rank < gcap) glist[g + rank] = v;
        else overflow(v);
    }
}

template <bool WIDE>
__global__ void __launch_bounds__(kRegionThreads, kRegionBlocksPerSM)
    k_region(Plan *plan, Params prm, const unsigned long long *__restrict__ cell_key,
             const uint32_t *__restrict__ cell_sc, const SubBox *__restrict__ box,
             const uint32_t *__restrict__ reps, const Rec *__restrict__ rec, uint32_t *parent,
             const uint32_t *__restrict__ nb_first, const uint8_t *__restrict__ nb_cnt,
             uint2 *__restrict__ pairq, uint32_t qcap, uint2 *__restrict__ edges, uint32_t ecap,
             uint32_t *__restrict__ scratch, uint32_t scap)
{
    grid_enter();
    extern __shared__ __align__(16) unsigned char region_smem[];
    RegionSmem &S = *reinterpret_cast<RegionSmem *>(region_smem);
    if (block_aborted(&plan->status)) return;
    const uint32_t M = plan->M_c;
    const uint32_t Ms = plan->M_s;  // read in debug builds only

    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    uint32_t *status = &plan->status;
    Metric<WIDE> m;
    m.T2 = (typename Metric<WIDE>::T)prm.T2;
    m.R1 = prm.R + 1;
    uint32_t n_pairs = 0, n_yes = 0, n_und = 0, n_same = 0, n_queued = 0, n_edges = 0;
    unsigned long long n_evals = 0;
    volatile RegionPar *vpar = S.par;
    // this block's list of undecided in-region pairs (local indices a | b << 16
    // would not fit 8192 sub-cells twice, so two u16 halves of a u32: a, b < 8192)
    uint32_t *const my_scratch = scratch + (size_t)blockIdx.x * scap;
    const uint32_t wcap = scap / kRegionWarps;  // scratch entries per warp

    // Global lists full (more boundary pairs than points): report instead of
    // joining here, which would race with other blocks' phase C.
    auto edge_overflow = [&](uint2) { atomicOr(status, ST_QUEUE_OVERFLOW); };
    auto pair_overflow = [&](uint2) { atomicOr(status, ST_QUEUE_OVERFLOW); };

    for (;;) {
        if (tid == 0) {
            // region size: kRegionCells, or fewer cells when the cloud has too
            // few cells to give every block two regions.  The last
            // kRegionTailRounds * grid full regions' worth of cells is cut into
            // regions prm.region_tail times smaller, so that blocks finish together.
            const uint32_t rc =
                min(prm.region_cells, max(kRegionMinCells, M / (2u * gridDim.x)));
            const uint32_t rt = max(kRegionMinCells, rc / max(prm.region_tail, 1u));
            const uint64_t tail = (uint64_t)kRegionTailRounds * gridDim.x * rc;
            const uint64_t full = M > tail ? (M - tail) / rc : 0;  // full-size regions
            const uint32_t r = atomicAdd(&plan->region_counter, 1u);
            const uint64_t lo = r < full ? (uint64_t)r * rc : full * rc + (uint64_t)(r - full) * rt;
            const uint64_t hi = lo + (r < full ? rc : rt);
            S.region = lo < M ? (uint32_t)lo : M;
            S.rend = lo < M ? (uint32_t)(hi < M ? hi : M) : M;
        }
        __syncthreads();
        const uint32_t c_lo = S.region, c_hi = S.rend;
        if (c_lo >= M) break;
        const uint32_t s0 = cell_sc[c_lo], s1 = cell_sc[c_hi], ns = s1 - s0;
        if (!FEC_IN_BOUNDS(status, ns, kRegionSubs + 1)) break;  // block-uniform
        for (uint32_t i = tid; i < ns; i += blockDim.x) S.par[i] = (uint16_t)i;
        for (int i = tid; i < kRegionBuf; i += blockDim.x) {
            S.ebuf[i] = make_uint2(0xffffffffu, 0xffffffffu);
            S.qbuf[i] = make_uint2(0xffffffffu, 0xffffffffu);
        }
        if (tid == 0) {
            S.ecount = 0;
            S.qcount = 0;
            S.next = c_lo;
        }
        __syncthreads();

        uint32_t wcount = 0;  // entries this warp put in its scratch slice
        // phase A: the warp enumerates the pairs of its cells (one cell after
        // another), drops those that no point pair can join, and queues the
        // rest in shared memory; every 32 queued pairs are decided together.
        uint32_t qn = 0;                  // pairs in the warp's queue
        uint32_t qh = 0;                  // its first entry (a ring of 64)
        // Each half-warp (16 lanes) enumerates one cell, so that the two
        // cells' set-up loads are in flight together.
        const int hw = lane >> 4, hl = lane & 15;
        const int cs = 2 * w + hw;        // this half's cell slot in shared memory
        uint32_t a_lo = 0, na = 0, own = 0, P0 = 0, P = 0, rcp = 0, next_i = 0, Pmax = 0;
        bool cells_left = true;
        for (;;) {
            while (qn < 32 && cells_left) {
                if (next_i >= Pmax) {  // set up the warp's next two cells
                    uint32_t c0 = 0;
                    if (lane == 0) c0 = atomicAdd(&S.next, 2u);
                    c0 = __shfl_sync(0xffffffffu, c0, 0);
                    if (c0 >= c_hi) {
                        cells_left = false;
                        break;
                    }
                    const uint32_t c = c0 + hw;
                    const bool have = c < c_hi;
                    a_lo = have ? cell_sc[c] : 0u;
                    // neighbour record (32 bytes): occupancies, offsets, K
                    const uint32_t cw = (have && hl < 8) ? reinterpret_cast<const uint32_t *>(nb_cnt)[(size_t)c * 8 + hl] : 0u;
                    // loaded with the record, not after it (13 entries per cell below M)
                    const uint32_t first = (have && hl < 13) ? nb_first[(size_t)c * 13 + hl] : 0u;
                    const uint32_t w3 = __shfl_sync(0xffffffffu, cw, 3, 16);
                    const int K = (int)(w3 >> 24);
                    own = (w3 >> 8) & 255u;
                    na = __popc(own);
                    const uint32_t ow = __shfl_sync(0xffffffffu, cw, (hl >> 2) & 3, 16);
                    const uint32_t mw = __shfl_sync(0xffffffffu, cw, 4 + ((hl >> 2) & 3), 16);
                    const uint32_t occ = (ow >> (8 * (hl & 3))) & 255u;
                    const uint32_t cnt = hl < K ? (uint32_t)__popc(occ) : 0u;
                    uint32_t ci = cnt;
#pragma unroll
                    for (int o = 1; o < 16; o <<= 1) {
                        const uint32_t u = __shfl_up_sync(0xffffffffu, ci, o, 16);
                        if (hl >= o) ci += u;
                    }
                    const uint32_t T = __shfl_sync(0xffffffffu, ci, 15, 16);
                    if (hl < K) {
                        const uint32_t nm = ((mw >> (8 * (hl & 3))) & 31u) << 3;
                        uint32_t rest = occ;
                        for (uint32_t j = ci - cnt, b = first; j < ci; ++j, ++b) {
                            if (!FEC_IN_BOUNDS(status, j, 112)) break;
                            S.nsub[cs][j] = b;
                            S.ninfo[cs][j] = (uint8_t)(nm | (__ffs(rest) - 1));
                            rest &= rest - 1;
                        }
                    }
                    if ((uint32_t)hl < na) S.ocode[cs][hl] = (uint8_t)select8(own, hl);
                    __syncwarp();
                    P0 = na * (na - 1) / 2;
                    P = P0 + na * T;
                    rcp = kRecip[na];
                    next_i = 0;
                    Pmax = max(P, __shfl_xor_sync(0xffffffffu, P, 16));
                    continue;
                }
                const uint32_t i = next_i + hl;
                next_i += 16;
                bool possible = false;
                uint32_t a = 0, b = 0;
                if (i < P) {
                    if (i < P0) {
                        // own pair i = ib (ib - 1) / 2 + ia, ia < ib < na <= 8
                        const uint32_t ib = 1u + (i >= 1) + (i >= 3) + (i >= 6) + (i >= 10) +
                                            (i >= 15) + (i >= 21);
                        a = a_lo + (i - ib * (ib - 1) / 2);
                        b = a_lo + ib;
                        possible = true;
                    } else {
                        const uint32_t j = i - P0;
                        const uint32_t jb = (j * rcp) >> 16;
                        const uint32_t ia = j - jb * na;
                        b = S.nsub[cs][jb];
                        a = a_lo + ia;
                        // Sub-cells three sub-cell steps apart on an axis are
                        // more than 2h >= R apart: along an axis where the
                        // neighbour cell is at +1, a in the lower half and b
                        // in the upper half (at -1: the reverse) cannot join.
                        const uint32_t A = S.ocode[cs][ia];
                        const uint32_t info = S.ninfo[cs][jb];
                        const uint32_t B = info & 7u;
                        possible = ((((info >> 3) & 7u) & ~A & B) | ((info >> 6) & A & ~B)) == 0;
                    }
                }
                const uint32_t pm = __ballot_sync(0xffffffffu, possible);
                if (possible) {
                    const uint32_t slot = (qh + qn + __popc(pm & lanemask_lt())) & 63u;
                    S.qa[w][slot] = a;
                    S.qb[w][slot] = b;
                }
                qn += __popc(pm);
            }
            if (qn == 0) break;
            __syncwarp();
            // decide the first min(qn, 32) queued pairs, one per lane
            const uint32_t mq = qn < 32 ? qn : 32;
            uint32_t a = 0, b = 0;
            int dec = 0;
            bool local = true;
            uint32_t root_a = 0, root_b = 0;  // local pairs: their roots at the check
            const uint32_t qs = (qh + lane) & 63u;
            if ((uint32_t)lane < mq && FEC_IN_BOUNDS(status, S.qa[w][qs] - s0, ns) &&
                FEC_IN_BOUNDS(status, S.qb[w][qs], Ms)) {
                a = S.qa[w][qs];
                b = S.qb[w][qs];
                local = b - s0 < ns;
                const SubBox BA = box[a], BB = box[b];
                const uint32_t RA = reps[a], RB = reps[b];
                if (local) {
                    root_a = s_find(vpar, a - s0);
                    root_b = s_find(vpar, b - s0);
                }
                if (local && root_a == root_b) {
                    ++n_same;
                } else {
                    ++n_pairs;
                    dec = box_decide<WIDE>(BA, BB, RA, RB, m);
                }
            }
            qh = (qh + mq) & 63u;  // the queue is a ring: the rest stays in place
            qn -= mq;
            if (dec == 1 && local) {
                ++n_yes;
                s_unite(S.par, root_a, root_b);  // from the roots found at the check
            }
            const bool emit = dec == 1 && !local;
            n_edges += emit ? 1 : 0;
            buf_append(__ballot_sync(0xffffffffu, emit), emit, make_uint2(a, b), S.ebuf,
                       &S.ecount, edges, &plan->edges_n, ecap, edge_overflow);
            const bool und = dec == 2;
            n_und += und ? 1 : 0;
            const bool cross = und && !local;
            n_queued += cross ? 1 : 0;
            buf_append(__ballot_sync(0xffffffffu, cross), cross, make_uint2(a, b), S.qbuf,
                       &S.qcount, pairq, &plan->pairq_n, qcap, pair_overflow);
            // undecided pairs inside the region: the block's scratch list
            // (or, when it is full, the global queue)
            const bool keep = und && local;
            const uint32_t kmask = __ballot_sync(0xffffffffu, keep);
            bool spill = false;
            if (kmask) {
                // this warp's own slice of the block's scratch list
                const uint32_t slot = wcount + __popc(kmask & lanemask_lt());
                wcount += __popc(kmask);
                if (keep) {
                    if (slot < wcap) my_scratch[w * wcap + slot] = (a - s0) | ((b - s0) << 16);
                    else spill = true;
                }
            }
            // scratch full: test those pairs right here
            uint32_t smask = __ballot_sync(0xffffffffu, spill);
            while (smask) {
                const int src = __ffs(smask) - 1;
                smask &= smask - 1;
                const uint32_t pa = __shfl_sync(0xffffffffu, a, src) - s0;
                const uint32_t pb = __shfl_sync(0xffffffffu, b, src) - s0;
                const uint32_t fa = s_find(vpar, pa), fb = s_find(vpar, pb);
                if (fa == fb) continue;  // warp-uniform
                if (warp_pair_test<WIDE>(s0 + pa, s0 + pb, box, rec, m, n_evals) && lane == 0)
                    s_unite(S.par, fa, fb);
                __syncwarp();
            }
            __syncwarp();
        }
        __syncthreads();
        // phase B: the region's undecided pairs still apart, warp witness tests
        // (each warp takes its own slice, which it filled in phase A)
        {
            const uint32_t nsc = min(wcount, wcap);
            for (uint32_t base = 0; base < nsc; base += 32) {
                const uint32_t i = base + lane;
                uint32_t la = 0, lb = 0;
                bool live = false;
                if (i < nsc) {
                    const uint32_t v = my_scratch[w * wcap + i];
                    la = v & 0xffffu;
                    lb = v >> 16;
                    live = FEC_IN_BOUNDS(status, la, ns) && FEC_IN_BOUNDS(status, lb, ns) &&
                           s_find(vpar, la) != s_find(vpar, lb);
                }
                uint32_t lmask = __ballot_sync(0xffffffffu, live);
                while (lmask) {
                    const int src = __ffs(lmask) - 1;
                    lmask &= lmask - 1;
                    const uint32_t pa = __shfl_sync(0xffffffffu, la, src);
                    const uint32_t pb = __shfl_sync(0xffffffffu, lb, src);
                    // warp-uniform: every lane reads the same shared words
                    const uint32_t fa = s_find(vpar, pa), fb = s_find(vpar, pb);
                    if (fa == fb) continue;
                    if (warp_pair_test<WIDE>(s0 + pa, s0 + pb, box, rec, m, n_evals) && lane == 0)
                        s_unite(S.par, fa, fb);
                    __syncwarp();
                }
            }
        }
        __syncthreads();
        // phase C: local roots become global parents; flush the buffers
        for (uint32_t i = tid; i < ns; i += blockDim.x) parent[s0 + i] = s0 + s_find(vpar, i);
        const uint32_t ne = min(S.ecount, (uint32_t)kRegionBuf);
        const uint32_t nq = min(S.qcount, (uint32_t)kRegionBuf);
        __shared__ uint32_t s_g[2];
        if (tid == 0) {
            s_g[0] = ne ? atomicAdd(&plan->edges_n, ne) : 0;
            s_g[1] = nq ? atomicAdd(&plan->pairq_n, nq) : 0;
        }
        __syncthreads();
        for (uint32_t i = tid; i < ne; i += blockDim.x) {
            const uint2 v = S.ebuf[i];
            const uint32_t g = s_g[0] + i;
            if (g < ecap) edges[g] = v;
            else if (v.x != 0xffffffffu) edge_overflow(v);
        }
        for (uint32_t i = tid; i < nq; i += blockDim.x) {
            const uint2 v = S.qbuf[i];
            const uint32_t g = s_g[1] + i;
            if (g < qcap) pairq[g] = v;
            else if (v.x != 0xffffffffu) pair_overflow(v);
        }
        __syncthreads();
    }
    n_pairs = __reduce_add_sync(0xffffffffu, n_pairs);
    n_yes = __reduce_add_sync(0xffffffffu, n_yes);
    n_und = __reduce_add_sync(0xffffffffu, n_und);
    n_same = __reduce_add_sync(0xffffffffu, n_same);
    n_queued = __reduce_add_sync(0xffffffffu, n_queued);
    n_edges = __reduce_add_sync(0xffffffffu, n_edges);
    if (lane == 0) {
        atomicAdd(&plan->ctr[CTR_PAIRS], (unsigned long long)n_pairs);
        atomicAdd(&plan->ctr[CTR_BOX_JOINS], (unsigned long long)(n_yes + n_edges));
        atomicAdd(&plan->ctr[CTR_EDGES], (unsigned long long)n_edges);
        atomicAdd(&plan->ctr[CTR_POINT_TESTS], (unsigned long long)n_und);
        atomicAdd(&plan->ctr[CTR_SAME_ROOT], (unsigned long long)n_same);
        atomicAdd(&plan->ctr[CTR_QUEUED], (unsigned long long)n_queued);
        atomicAdd(&plan->ctr[CTR_POINT_EVALS], n_evals);
    }
}

// a4: the boundary edges found by k_region, one union per distinct pair of
// region-local roots.  After k_region every sub-cell points at its region
// root, so many boundary edges name the same pair of roots; a hash set keeps
// the first of each, and only that one joins (the rest would only add load on
// the giant component's root).  A full probe window falls back to joining.
__global__ void __launch_bounds__(256)
    k_edges(Plan *plan, const uint2 *__restrict__ edges, uint32_t ecap, uint32_t *parent,
            unsigned long long *__restrict__ set, uint32_t set_mask, uint32_t union_cap)
{
    grid_enter();
    if (call_aborted(&plan->status)) return;
    const uint32_t ne = min(plan->edges_n, ecap);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < ne; i += gridDim.x * blockDim.x) {
        const uint2 e = edges[i];
        if (e.x == 0xffffffffu) continue;  // unused buffer slot
        if (!FEC_IN_BOUNDS(&plan->status, e.x, plan->M_s) || !FEC_IN_BOUNDS(&plan->status, e.y, plan->M_s))
            continue;
        uint32_t ra = parent[e.x], rb = parent[e.y];
        if (ra == rb) continue;
        if (ra > rb) {
            const uint32_t t = ra;
            ra = rb;
            rb = t;
        }
        const unsigned long long key = ((unsigned long long)ra << 32) | rb;
        uint32_t h = (uint32_t)((key * 0x9E3779B97F4A7C15ull) >> 32) & set_mask;
        bool first = true;
        for (int probe = 0; probe < 32; ++probe) {
            const unsigned long long old = atomicCAS(set + h, ~0ull, key);
            if (old == ~0ull) break;          // inserted: this edge is the first
            if (old == key) {                 // already seen
                first = false;
                break;
            }
            h = (h + 1) & set_mask;
        }
        if (first && !uf_unite(parent, ra, rb, union_cap)) atomicOr(&plan->status, ST_UNION_CAP);
    }
}

// a4, last part: the queued pairs, one warp per pair after a parallel root
// check of 32 pairs at a time (most were joined meanwhile).
template <bool WIDE>
__global__ void __launch_bounds__(kUnionThreads, 2)
    k_pairs(Plan *plan, Params prm, const SubBox *__restrict__ box, const Rec *__restrict__ rec,
            uint32_t *parent, const uint2 *__restrict__ pairq, uint32_t qcap)
{
    grid_enter();
    if (block_aborted(&plan->status)) return;
    const uint32_t nq = min(plan->pairq_n, qcap);
    const int lane = threadIdx.x & 31;
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    uint32_t *status = &plan->status;
    Metric<WIDE> m;
    m.T2 = (typename Metric<WIDE>::T)prm.T2;
    m.R1 = prm.R + 1;
    unsigned long long n_same = 0, n_evals = 0;
    const uint32_t cap = prm.union_cap;
    for (uint32_t base = gw * 32; base < nq; base += nw * 32) {
        const uint32_t i = base + lane;
        uint2 pr = make_uint2(0, 0);
        bool live = false;
        if (i < nq) {
            pr = pairq[i];
            bool ok = true;
            live = pr.x != 0xffffffffu && FEC_IN_BOUNDS(status, pr.x, plan->M_s) &&
                   FEC_IN_BOUNDS(status, pr.y, plan->M_s) && uf_find(parent, pr.x, cap, ok) != uf_find(parent, pr.y, cap, ok);
            if (!ok) atomicOr(status, ST_UNION_CAP);
            if (!live) ++n_same;
        }
        uint32_t mask = __ballot_sync(0xffffffffu, live);
        while (mask) {
            const int src = __ffs(mask) - 1;
            mask &= mask - 1;
            const uint32_t pa = __shfl_sync(0xffffffffu, pr.x, src);
            const uint32_t pb = __shfl_sync(0xffffffffu, pr.y, src);
            if (warp_pair_test<WIDE>(pa, pb, box, rec, m, n_evals) && lane == 0 &&
                !uf_unite(parent, pa, pb, cap))
                atomicOr(status, ST_UNION_CAP);
        }
    }
    n_same = __reduce_add_sync(0xffffffffu, (uint32_t)n_same);
    if (lane == 0) {
        atomicAdd(&plan->ctr[CTR_SAME_ROOT], n_same);
        atomicAdd(&plan->ctr[CTR_POINT_EVALS], n_evals);
    }
}

// a5: every sub-cell points at its root; component sizes and smallest
// original index, aggregated per warp before the atomics.
constexpr int kFlatSlots = 512;  // per-block table of component sums

__global__ void __launch_bounds__(256, 4)
    k_flatten_stats(Plan *plan, const uint32_t *__restrict__ sc_start, const uint32_t *__restrict__ sminidx,
                    uint32_t *parent, uint32_t *__restrict__ csize, uint32_t *__restrict__ cmin,
                    uint32_t union_cap)
{
    grid_enter();
    if (block_aborted(&plan->status)) return;
    // Each block takes one contiguous range of sub-cells (a compact piece of
    // space, so few distinct components) and sums sizes and smallest indices
    // per root in a shared-memory table; roots that find no free slot go
    // straight to the global arrays.
    __shared__ uint32_t t_root[kFlatSlots], t_size[kFlatSlots], t_min[kFlatSlots];
    for (int i = threadIdx.x; i < kFlatSlots; i += blockDim.x) {
        t_root[i] = 0xffffffffu;
        t_size[i] = 0;
        t_min[i] = 0xffffffffu;
    }
    __syncthreads();
    const uint32_t M = plan->M_s;
    const int lane = threadIdx.x & 31;
    const uint32_t per = (M + gridDim.x - 1) / gridDim.x;
    const uint32_t lo = blockIdx.x * per, hi = min(M, lo + per);
    for (uint32_t base = lo + (threadIdx.x & ~31u); base < hi; base += blockDim.x) {
        const uint32_t a = base + lane;
        const bool valid = a < hi;
        uint32_t r = 0xffffffffu, cnt = 0, mi = 0xffffffffu;
        if (valid) {
            // read-only walk: unions are finished, pointers only get shorter
            r = a;
            bool found = false;
            for (uint32_t it = 0; it <= union_cap; ++it) {
                const uint32_t p = ld_relaxed(parent + r);
                if (p == r) {
                    found = true;
                    break;
                }
                if (!FEC_IN_BOUNDS(&plan->status, p, M)) break;
                r = p;
            }
            if (!found) atomicOr(&plan->status, ST_UNION_CAP);
            cnt = sc_start[a + 1] - sc_start[a];  // the sub-cell's points (not its 32-byte box)
            mi = sminidx[a];
            st_relaxed(parent + a, r);
        }
        uint32_t active = __ballot_sync(0xffffffffu, valid);
        while (active) {
            const int leader = __ffs(active) - 1;
            const uint32_t r0 = __shfl_sync(0xffffffffu, r, leader);
            const bool in = valid && r == r0;
            const uint32_t sm = __reduce_add_sync(0xffffffffu, in ? cnt : 0u);
            const uint32_t mn = __reduce_min_sync(0xffffffffu, in ? mi : 0xffffffffu);
            if (lane == leader) {
                uint32_t slot = (r0 * 2654435761u) >> (32 - 9);
                bool placed = false;
                for (int probe = 0; probe < 8; ++probe) {
                    const uint32_t cur = atomicCAS(&t_root[slot], 0xffffffffu, r0);
                    if (cur == 0xffffffffu || cur == r0) {
                        atomicAdd(&t_size[slot], sm);
                        atomicMin(&t_min[slot], mn);
                        placed = true;
                        break;
                    }
                    slot = (slot + 1) & (kFlatSlots - 1);
                }
                if (!placed) {
                    atomicAdd(csize + r0, sm);
                    atomicMin(cmin + r0, mn);
                }
            }
            active &= ~__ballot_sync(0xffffffffu, in);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kFlatSlots; i += blockDim.x) {
        const uint32_t r0 = t_root[i];
        if (r0 == 0xffffffffu) continue;
        atomicAdd(csize + r0, t_size[i]);
        atomicMin(cmin + r0, t_min[i]);
    }
}

// a6: numbering of the kept components by their smallest point index,
// without sorting them: each kept component sets one bit at the sorted
// position of its smallest input row (position order is row order within a
// frame, and frames are in row order), a scan counts the set bits before
// every bitmap word, and a component's number is the count of set bits
// before its own (minus those before its frame's first position).
//
// k_kept: list the kept components (position of the smallest row, root),
// set their bits, count them (per frame too).
__global__ void __launch_bounds__(256)
    k_kept(Plan *plan, const uint32_t *__restrict__ parent, const uint32_t *__restrict__ csize,
           const uint32_t *__restrict__ cmin, Frame *__restrict__ fr, uint32_t nf,
           uint32_t *__restrict__ kept_key, uint32_t *__restrict__ kept_val,
           uint32_t *__restrict__ rank_bits)
{
    grid_enter();
    if (block_aborted(&plan->status)) return;
    const uint32_t M = plan->M_s;
    const int lane = threadIdx.x & 31;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t base = (blockIdx.x * blockDim.x + threadIdx.x) & ~31u; base < M; base += stride) {
        const uint32_t a = base + lane;
        bool keep = false;
        uint32_t pos = 0;
        if (a < M && parent[a] == a) {
            // the bounds of the component's frame (the frame of its smallest row)
            const uint32_t row = cmin[a];
            const uint32_t f = frame_of_row(fr, nf, row);
            const long long s = (long long)csize[a];
            keep = s >= fr[f].min_size && s <= fr[f].max_size &&
                   FEC_IN_BOUNDS(&plan->status, row - fr[f].in_off, fr[f].n);
            pos = fr[f].pos_off + (row - fr[f].in_off);
            if (keep) {
                atomicOr(rank_bits + (pos >> 5), 1u << (pos & 31u));
                if (nf > 1) atomicAdd(&fr[f].kept, 1u);
            }
        }
        const uint32_t mask = __ballot_sync(0xffffffffu, keep);
        if (!mask) continue;
        const int leader = __ffs(mask) - 1;
        uint32_t slot = 0;
        if (lane == leader) slot = atomicAdd(&plan->kept_n, (uint32_t)__popc(mask));
        slot = __shfl_sync(0xffffffffu, slot, leader) + __popc(mask & lanemask_lt());
        if (keep && FEC_IN_BOUNDS(&plan->status, slot, M)) {
            kept_key[slot] = pos;
            kept_val[slot] = a;
        }
    }
}

// k_rankscan: rank_prefix[w] = set bits in words 0..w-1 of the bitmap (one
// pass, decoupled look-back over tiles of kRankTileWords words; waits
// bounded by prm.wait_cap like the sort's).
constexpr int kRankThreads = 256;
constexpr int kRankWordsPerThread = 8;
constexpr uint32_t kRankTileWords = kRankThreads * kRankWordsPerThread;
__global__ void __launch_bounds__(kRankThreads)
    k_rankscan(Plan *plan, Params prm, const uint32_t *__restrict__ rank_bits,
               uint32_t *__restrict__ rank_prefix, unsigned long long *__restrict__ tstat)
{
    grid_enter();
    __shared__ uint32_t s_tile, s_warp[kRankThreads / 32];
    __shared__ unsigned long long s_prefix;
    if (block_aborted(&plan->status)) return;
    constexpr unsigned long long kAgg = 1ull << 62, kIncl = 2ull << 62, kMask = (1ull << 62) - 1;
    const uint32_t nwords = (plan->sort.n + 31) / 32;
    const uint32_t ntiles = (nwords + kRankTileWords - 1) / kRankTileWords;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (;;) {
        if (tid == 0) s_tile = atomicAdd(&plan->rank_tile_counter, 1u);
        __syncthreads();
        const uint32_t tile = s_tile;
        if (tile >= ntiles) break;
        const uint32_t w0 = tile * kRankTileWords + tid * kRankWordsPerThread;
        uint32_t c[kRankWordsPerThread], run = 0;
#pragma unroll
        for (int i = 0; i < kRankWordsPerThread; ++i) {
            c[i] = w0 + i < nwords ? (uint32_t)__popc(rank_bits[w0 + i]) : 0u;
            run += c[i];
        }
        uint32_t incl = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        if (lane == 31) s_warp[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            uint32_t tot = 0;
            for (int w = 0; w < kRankThreads / 32; ++w) tot += s_warp[w];
            __syncwarp();
            if (lane == 0) {
                uint32_t acc = 0;
                for (int w = 0; w < kRankThreads / 32; ++w) {
                    const uint32_t v = s_warp[w];
                    s_warp[w] = acc;
                    acc += v;
                }
                st_relaxed64(tstat + tile, (tile == 0 ? kIncl : kAgg) | tot);
            }
            unsigned long long prefix = 0;
            if (tile > 0) {  // look-back, one preceding tile per lane per step
                int64_t p = (int64_t)tile - 1;
                uint32_t it = 0;
                for (;;) {
                    const int64_t q = p - lane;
                    unsigned long long sv = q >= 0 ? ld_relaxed64(tstat + q) : kIncl;
                    while (!__all_sync(0xffffffffu, (sv & ~kMask) != 0)) {
                        if (++it > prm.wait_cap) {
                            if (lane == 0) atomicOr(&plan->status, ST_WAIT_TIMEOUT);
                            break;
                        }
                        spin_pause(it);
                        if ((sv & ~kMask) == 0) sv = ld_relaxed64(tstat + q);
                    }
                    const uint32_t incl_m = __ballot_sync(0xffffffffu, (sv & ~kMask) == kIncl);
                    const int stop = incl_m ? __ffs(incl_m) - 1 : 31;
                    unsigned long long part = (lane <= stop && q >= 0) ? (sv & kMask) : 0ull;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
                    prefix += part;
                    if (incl_m || it > prm.wait_cap) break;
                    p -= 32;
                }
                if (lane == 0) st_relaxed64(tstat + tile, kIncl | ((prefix + tot) & kMask));
            }
            if (lane == 0) s_prefix = prefix;
        }
        __syncthreads();
        uint32_t before = (uint32_t)s_prefix + s_warp[warp] + (incl - run);
#pragma unroll
        for (int i = 0; i < kRankWordsPerThread; ++i) {
            if (w0 + i < nwords) rank_prefix[w0 + i] = before;
            before += c[i];
        }
        __syncthreads();
    }
}

// Set bits of the bitmap before position p.
__device__ __forceinline__ uint32_t bits_before(const uint32_t *__restrict__ bits,
                                                const uint32_t *__restrict__ prefix, uint32_t p)
{
    const uint32_t w = p >> 5, b = p & 31u;
    return prefix[w] + (uint32_t)__popc(bits[w] & ((1u << b) - 1u));
}

// k_rank: every kept root's number within its frame.
__global__ void __launch_bounds__(256)
    k_rank(Plan *plan, const uint32_t *__restrict__ kept_key, const uint32_t *__restrict__ kept_val,
           const uint32_t *__restrict__ rank_bits, const uint32_t *__restrict__ rank_prefix,
           const Frame *__restrict__ fr, uint32_t nf, int32_t *__restrict__ crank)
{
    grid_enter();
    if (call_aborted(&plan->status)) return;
    const uint32_t k = plan->kept_n;
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < k; t += gridDim.x * blockDim.x) {
        const uint32_t pos = kept_key[t];
        if (!FEC_IN_BOUNDS(&plan->status, pos, plan->sort.n) ||
            !FEC_IN_BOUNDS(&plan->status, kept_val[t], plan->M_s))
            continue;
        uint32_t r = bits_before(rank_bits, rank_prefix, pos);
        if (nf > 1) r -= bits_before(rank_bits, rank_prefix, fr[frame_of_pos(fr, nf, pos)].pos_off);
        crank[kept_val[t]] = (int32_t)r;
    }
}

// a6: the label of every sub-cell (its root's rank, or -1), written over the
// component-size array, which is not needed after k_kept; and every label of
// the output set to -1 (coalesced), so that k_labels writes kept points only.
__global__ void __launch_bounds__(256)
    k_sclabel(Plan *plan, const uint32_t *__restrict__ parent, const int32_t *__restrict__ crank,
              int32_t *__restrict__ sclab, int32_t *__restrict__ labels, uint32_t n)
{
    grid_enter();
    if (call_aborted(&plan->status)) return;
    const uint32_t M = plan->M_s;
    for (uint32_t a = blockIdx.x * blockDim.x + threadIdx.x; a < M; a += gridDim.x * blockDim.x)
        if (FEC_IN_BOUNDS(&plan->status, parent[a], M)) sclab[a] = crank[parent[a]];
    // 16-byte stores when the output is 16-byte aligned (a batch frame's
    // labels start anywhere), else 4-byte stores
    const uint32_t n4 = (reinterpret_cast<uintptr_t>(labels) & 15) ? 0u : n / 4;  // n: labels to fill
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < n4; q += gridDim.x * blockDim.x)
        __stcs(reinterpret_cast<int4 *>(labels) + q, make_int4(-1, -1, -1, -1));
    for (uint32_t i = 4 * n4 + blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        labels[i] = -1;
}

// a6: labels of the kept points in input order (the others are already -1),
// eight sorted positions per thread and step; a step whose eight points all
// belong to dropped components reads no indices.
__global__ void __launch_bounds__(256)
    k_labels(Plan *plan, const uint32_t *__restrict__ idx_a, const uint32_t *__restrict__ idx_b,
             uint32_t idx_stride, const uint32_t *__restrict__ sc_of,
             const int32_t *__restrict__ sclab, int32_t *__restrict__ labels, uint32_t rows)
{
    grid_enter();
    if (call_aborted(&plan->status)) return;
    const uint32_t n = plan->sort.n;
    const uint32_t *__restrict__ idx = (plan->sort.npasses & 1u) ? idx_b : idx_a;
    const uint32_t n8 = n / 8;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < n8; q += gridDim.x * blockDim.x) {
        uint32_t i[8], sc[8];
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const uint4 v = __ldcs(reinterpret_cast<const uint4 *>(sc_of) + 2 * (size_t)q + t);
            sc[4 * t] = v.x;
            sc[4 * t + 1] = v.y;
            sc[4 * t + 2] = v.z;
            sc[4 * t + 3] = v.w;
        }
        int32_t l[8];
        bool any = false;
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            l[t] = FEC_IN_BOUNDS(&plan->status, sc[t], plan->M_s) ? sclab[sc[t]] : -1;
            any |= l[t] >= 0;
        }
        if (!any) continue;
        if (idx_stride == 2) {
            const uint4 *src = reinterpret_cast<const uint4 *>(idx) + 4 * (size_t)q;
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const uint4 v = __ldcs(src + t);
                i[2 * t] = v.x;
                i[2 * t + 1] = v.z;
            }
        } else {
            const uint4 *src = reinterpret_cast<const uint4 *>(idx) + 2 * (size_t)q;
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                const uint4 v = __ldcs(src + t);
                i[4 * t] = v.x;
                i[4 * t + 1] = v.y;
                i[4 * t + 2] = v.z;
                i[4 * t + 3] = v.w;
            }
        }
#pragma unroll
        for (int t = 0; t < 8; ++t)
            if (l[t] >= 0 && i[t] < rows) labels[i[t]] = l[t];
    }
    for (uint32_t p = n8 * 8 + blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += gridDim.x * blockDim.x) {
        const int32_t l = FEC_IN_BOUNDS(&plan->status, sc_of[p], plan->M_s) ? sclab[sc_of[p]] : -1;
        const uint32_t i = idx[(size_t)p * idx_stride];
        if (l >= 0 && i < rows) labels[i] = l;
    }
}

}  // namespace

cudaError_t enqueue_union(Workspace &ws, const Params &prm, cudaStream_t st)
{
    const uint32_t qcap = (uint32_t)ws.pairq_cap;
    const uint32_t ecap = (uint32_t)ws.edges_cap;
    const bool wide = prm.R + 1 > 26754;
    const size_t smem = sizeof(RegionSmem);
    static std::atomic<unsigned long long> attr_ctx{0};  // context the attributes were set in
    if (ctx_setup_needed(attr_ctx)) {
        cudaFuncSetAttribute(k_region<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(k_region<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        ctx_setup_done(attr_ctx);
    }
    const int grid1 = grid_for(ws, prm.n, 256, 8);  // one item (cell, sub-cell, edge) per thread
    launch(k_nbrs, grid1, 256, 0, st, ws.plan, prm, ws.cell_key, ws.cell_sc, ws.slab_lo, ws.slab_hi,
                                        ws.col_lo, ws.col_hi, ws.cocc, ws.nb_first, ws.nb_cnt,
                                        ws.edge_set, (uint32_t)ws.edge_set_size, ws.cframe, ws.frames);
    FEC_MARK(ws, "k_nbrs", st);
    const uint32_t rgrid = region_grid(ws, prm.n);
    const uint32_t scap = region_scratch(ws, ws.cap_n);
    if (!wide)
        launch(k_region<false>, rgrid, kRegionThreads, smem, st,
            ws.plan, prm, ws.cell_key, ws.cell_sc, ws.box, ws.reps, ws.rec, ws.parent, ws.nb_first,
            ws.nb_cnt, ws.pairq, qcap, ws.edges, ecap, ws.scratch, scap);
    else
        launch(k_region<true>, rgrid, kRegionThreads, smem, st,
            ws.plan, prm, ws.cell_key, ws.cell_sc, ws.box, ws.reps, ws.rec, ws.parent, ws.nb_first,
            ws.nb_cnt, ws.pairq, qcap, ws.edges, ecap, ws.scratch, scap);
    FEC_MARK(ws, "k_region", st);
    launch(k_edges, grid1, 256, 0, st, ws.plan, ws.edges, ecap, ws.parent, ws.edge_set,
                                        (uint32_t)(ws.edge_set_size - 1), prm.union_cap);
    FEC_MARK(ws, "k_edges", st);
    if (!wide)
        launch(k_pairs<false>, grid_for(ws, prm.n, 64, 2), kUnionThreads, 0, st, ws.plan, prm, ws.box, ws.rec, ws.parent,
                                                             ws.pairq, qcap);
    else
        launch(k_pairs<true>, grid_for(ws, prm.n, 64, 2), kUnionThreads, 0, st, ws.plan, prm, ws.box, ws.rec, ws.parent,
                                                            ws.pairq, qcap);
    FEC_MARK(ws, "k_pairs", st);
    launch(k_flatten_stats, grid1, 256, 0, st, ws.plan, ws.sc_start, ws.sminidx, ws.parent, ws.csize,
                                                 ws.cmin, prm.union_cap);
    FEC_MARK(ws, "k_flatten_stats", st);
    launch(k_kept, grid1, 256, 0, st, ws.plan, ws.parent, ws.csize, ws.cmin, ws.frames, prm.nf,
                                  ws.kept_key_a(), ws.kept_val_a(), ws.rank_bits);
    FEC_MARK(ws, "k_kept", st);
    return cudaGetLastError();
}

cudaError_t enqueue_labels(Workspace &ws, const Params &prm, int32_t *labels, bool fill,
                           cudaStream_t st)
{
    const int grid1 = grid_for(ws, prm.n, 256, 8);
    const uint64_t words = ((uint64_t)prm.n + 31) / 32;
    launch(k_rankscan, grid_for(ws, words, kRankTileWords, 4), kRankThreads, 0, st,
        ws.plan, prm, ws.rank_bits, ws.rank_prefix, ws.rank_status);
    FEC_MARK(ws, "k_rankscan", st);
    launch(k_rank, grid_for(ws, prm.n, 256, 4), 256, 0, st, ws.plan, ws.kept_key_a(), ws.kept_val_a(),
                                                        ws.rank_bits, ws.rank_prefix, ws.frames,
                                                        prm.nf, ws.crank);
    FEC_MARK(ws, "k_rank", st);
    // sorted original indices: the 32-bit values, or the low half of the packed payloads
    int32_t *sclab = (int32_t *)ws.csize;  // component sizes are no longer needed
    launch(k_sclabel, grid1, 256, 0, st, ws.plan, ws.parent, ws.crank, sclab, labels, fill ? prm.rows : 0u);
    FEC_MARK(ws, "k_sclabel", st);
    launch(k_labels, grid_for(ws, prm.n, 2048, 8), 256, 0, st, ws.plan, (const uint32_t *)ws.vals_a,
                                         (const uint32_t *)ws.vals_b, prm.packed ? 2u : 1u, ws.sc_of,
                                         sclab, labels, prm.rows);
    FEC_MARK(ws, "k_labels", st);
    return cudaGetLastError();
}

}  // namespace fec
