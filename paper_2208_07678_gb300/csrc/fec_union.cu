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
constexpr int kUnionWarps = kUnionThreads / 32;
constexpr int kUnionChunk = 4;

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
__device__ __forceinline__ int box_decide(const SubBox &A, const SubBox &B, const Rec &ra,
                                          const Rec &rb, const Metric<WIDE> &m)
{
    if (!m.box_gap(A, B)) return 0;
    if (m.box_diam(A, B) || m.within(ra.x - rb.x, ra.y - rb.y, ra.z - rb.z)) return 1;
    return 2;
}

// Pairs (ia < ib) of the up to 8 sub-cells of one cell.
__constant__ uint8_t kPairA[28] = {0, 0, 0, 0, 0, 0, 0, 1, 1, 1, 1, 1, 1, 2,
                                   2, 2, 2, 2, 3, 3, 3, 3, 4, 4, 4, 5, 5, 6};
__constant__ uint8_t kPairB[28] = {1, 2, 3, 4, 5, 6, 7, 2, 3, 4, 5, 6, 7, 3,
                                   4, 5, 6, 7, 4, 5, 6, 7, 5, 6, 7, 6, 7, 7};

// Hand out cells in chunks (dynamic schedule: work per cell varies by
// orders of magnitude between sparse and dense regions).
struct CellSchedule {
    uint32_t base = 0, left = 0;
    __device__ __forceinline__ bool next(uint32_t *counter, uint32_t M, uint32_t &c)
    {
        for (;;) {
            if (left == 0) {
                uint32_t got = 0;
                if ((threadIdx.x & 31) == 0) got = atomicAdd(counter, (uint32_t)kUnionChunk);
                base = __shfl_sync(0xffffffffu, got, 0);
                left = kUnionChunk;
                if (base >= M) return false;
            }
            c = base++;
            --left;
            if (c < M) return true;
            left = 0;
        }
    }
};

// a4, first half: components inside each cell.  A warp takes a cell, decides
// its <= 28 sub-cell pairs (boxes, representatives, then point tests) with a
// warp-local union-find, and writes lroot = parent = the smallest sub-cell of
// each in-cell component.  No global atomics on the union-find.
template <bool WIDE>
__global__ void __launch_bounds__(kUnionThreads, 4)
    k_local(Plan *plan, Params prm, const uint32_t *__restrict__ cell_sc,
            const SubBox *__restrict__ box, const Rec *__restrict__ reps,
            const Rec *__restrict__ rec, uint32_t *__restrict__ parent,
            uint32_t *__restrict__ lroot)
{
    __shared__ SubBox s_box[kUnionWarps][8];
    __shared__ Rec s_rep[kUnionWarps][8];
    __shared__ uint8_t s_lp[kUnionWarps][8];
    const uint32_t M = plan->M_c;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    Metric<WIDE> m;
    m.T2 = (typename Metric<WIDE>::T)prm.T2;
    m.R1 = prm.R + 1;
    unsigned long long n_pairs = 0, n_yes = 0, n_tests = 0, n_evals = 0;
    CellSchedule sched;
    uint32_t c;
    while (sched.next(&plan->local_counter, M, c)) {
        const uint32_t a_lo = cell_sc[c], na = cell_sc[c + 1] - a_lo;
        if (na == 1) {
            if (lane == 0) lroot[a_lo] = a_lo;
            continue;
        }
        if (lane < (int)na) {
            s_box[w][lane] = box[a_lo + lane];
            s_rep[w][lane] = reps[a_lo + lane];
            s_lp[w][lane] = (uint8_t)lane;
        }
        __syncwarp();
        int dec = 0;
        const int ia = lane < 28 ? kPairA[lane] : 0, ib = lane < 28 ? kPairB[lane] : 0;
        if (lane < 28 && ib < (int)na)
            dec = box_decide<WIDE>(s_box[w][ia], s_box[w][ib], s_rep[w][ia], s_rep[w][ib], m);
        const uint32_t yes = __ballot_sync(0xffffffffu, dec == 1);
        uint32_t und = __ballot_sync(0xffffffffu, dec == 2);
        n_pairs += na * (na - 1) / 2;
        n_yes += __popc(yes);
        n_tests += __popc(und);
        // local union-find over <= 8 entries, kept by lane 0 (root = smallest)
        if (lane == 0) {
            for (uint32_t y = yes; y; y &= y - 1) {
                const int p = __ffs(y) - 1;
                int x = kPairA[p], z = kPairB[p];
                while (s_lp[w][x] != x) x = s_lp[w][x];
                while (s_lp[w][z] != z) z = s_lp[w][z];
                if (x != z) s_lp[w][max(x, z)] = (uint8_t)min(x, z);
            }
        }
        __syncwarp();
        while (und) {
            const int p = __ffs(und) - 1;
            und &= und - 1;
            int x = kPairA[p], z = kPairB[p];
            while (s_lp[w][x] != x) x = s_lp[w][x];
            while (s_lp[w][z] != z) z = s_lp[w][z];
            if (x == z) continue;  // warp-uniform: s_lp is read by every lane
            if (warp_pair_test<WIDE>(a_lo + kPairA[p], a_lo + kPairB[p], box, rec, m, n_evals)) {
                if (lane == 0) s_lp[w][max(x, z)] = (uint8_t)min(x, z);
            }
            __syncwarp();
        }
        if (lane < (int)na) {
            int x = lane;
            while (s_lp[w][x] != x) x = s_lp[w][x];
            lroot[a_lo + lane] = a_lo + x;
            parent[a_lo + lane] = a_lo + x;
        }
        __syncwarp();
    }
    n_yes = __reduce_add_sync(0xffffffffu, (uint32_t)(lane == 0 ? n_yes : 0));
    if (lane == 0) {
        atomicAdd(&plan->ctr[CTR_PAIRS], n_pairs);
        atomicAdd(&plan->ctr[CTR_BOX_JOINS], n_yes);
        atomicAdd(&plan->ctr[CTR_POINT_TESTS], n_tests);
        atomicAdd(&plan->ctr[CTR_POINT_EVALS], n_evals);
    }
}

// a4, second half: pairs across neighbouring cells.  A warp takes a cell,
// finds its half-stencil neighbour cells (13 of the 26; the other half is
// covered by the neighbours' own visits) through the slab index, and decides
// every sub-cell pair (a in the cell, b in a neighbour) from boxes and
// representatives.  Pairs are grouped by in-cell component pair
// (lroot[a], lroot[b]): a group with any decided edge joins the two
// components once; a group with only undecided pairs checks the global roots
// once and, if they differ, queues its pairs for k_pairs.
template <bool WIDE>
__global__ void __launch_bounds__(kUnionThreads, 4)
    k_global(Plan *plan, Params prm, const unsigned long long *__restrict__ cell_key,
             const uint32_t *__restrict__ cell_sc, const SubBox *__restrict__ box,
             const Rec *__restrict__ reps, const Rec *__restrict__ rec,
             const uint32_t *__restrict__ lroot, uint32_t *parent,
             const uint32_t *__restrict__ slab_lo, const uint32_t *__restrict__ slab_hi,
             uint2 *__restrict__ pairq, uint32_t qcap)
{
    __shared__ uint32_t s_nb[kUnionWarps][16];
    __shared__ uint32_t s_pre[kUnionWarps][17];
    __shared__ SubBox s_box[kUnionWarps][8];
    __shared__ Rec s_rep[kUnionWarps][8];
    __shared__ uint32_t s_lr[kUnionWarps][8];

    const uint32_t M = plan->M_c;
    const uint32_t b1 = plan->bits[1], b2 = plan->bits[2];
    const unsigned long long m1 = (1ull << b1) - 1, m2 = (1ull << b2) - 1;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t *status = &plan->status;
    Metric<WIDE> m;
    m.T2 = (typename Metric<WIDE>::T)prm.T2;
    m.R1 = prm.R + 1;

    unsigned long long n_pairs = 0, n_yes = 0, n_tests = 0, n_same = 0, n_queued = 0;
    CellSchedule sched;
    uint32_t c;
    while (sched.next(&plan->union_counter, M, c)) {
        const unsigned long long ck = cell_key[c];
        const unsigned long long c0 = ck >> (b1 + b2);
        const unsigned long long c1 = (ck >> b2) & m1, c2 = ck & m2;
        const uint32_t a_lo = cell_sc[c], na = cell_sc[c + 1] - a_lo;
        if (lane < (int)na) {
            s_box[w][lane] = box[a_lo + lane];
            s_rep[w][lane] = reps[a_lo + lane];
            s_lr[w][lane] = lroot[a_lo + lane];
        }

        // Neighbour cells of the half stencil.  Lanes 0..3 search columns
        // (0,+1), (+1,-1), (+1,0), (+1,+1) over dz in {-1,0,+1}; lane 4
        // checks (0,0,+1), the next cell of the same column.
        uint32_t f0 = 0, f1 = 0, f2 = 0;  // found neighbour cells (registers)
        int nf = 0;
        if (lane < 4) {
            const long long d0 = lane == 0 ? 0 : 1;
            const long long d1 = lane == 0 ? 1 : lane - 2;
            const long long n0 = (long long)c0 + d0, n1 = (long long)c1 + d1;
            if (n1 >= 0 && (unsigned long long)n1 <= m1 && (unsigned long long)n0 < prm.slab_cap) {
                uint32_t lo = slab_lo[n0];
                const uint32_t end = slab_hi[n0];
                uint32_t hi = end;
                const unsigned long long col = ((unsigned long long)n0 << (b1 + b2)) |
                                               ((unsigned long long)n1 << b2);
                const unsigned long long tlo = col | (c2 > 0 ? c2 - 1 : 0);
                const unsigned long long thi = col | (c2 < m2 ? c2 + 1 : m2);
                while (lo < hi) {
                    const uint32_t mid = (lo + hi) >> 1;
                    if (cell_key[mid] < tlo) lo = mid + 1;
                    else hi = mid;
                }
                for (uint32_t q = lo; q < end && nf < 3; ++q) {
                    if (cell_key[q] > thi) break;
                    if (nf == 0) f0 = q;
                    else if (nf == 1) f1 = q;
                    else f2 = q;
                    ++nf;
                }
            }
        } else if (lane == 4) {
            if (c2 < m2 && c + 1 < M && cell_key[c + 1] == ck + 1) {
                f0 = c + 1;
                nf = 1;
            }
        }
        int incl = nf;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        const int K = __shfl_sync(0xffffffffu, incl, 31);
        if (nf > 0) s_nb[w][incl - nf] = f0;
        if (nf > 1) s_nb[w][incl - nf + 1] = f1;
        if (nf > 2) s_nb[w][incl - nf + 2] = f2;
        __syncwarp();
        uint32_t cnt = 0;
        if (lane < K) {
            const uint32_t q = s_nb[w][lane];
            cnt = cell_sc[q + 1] - cell_sc[q];
        }
        uint32_t ci = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, ci, o);
            if (lane >= o) ci += u;
        }
        if (lane <= K) s_pre[w][lane] = ci - cnt;  // lane K holds the total
        __syncwarp();
        const uint32_t T = s_pre[w][K];
        const uint32_t P = na * T;
        n_pairs += P;

        for (uint32_t base = 0; base < P; base += 32) {
            const uint32_t i = base + lane;
            int dec = 0;
            uint32_t a = 0, b = 0;
            unsigned long long key = 0;
            if (i < P) {
                const uint32_t ia = i % na, jb = i / na;
                int k = 0;
                while (k + 1 < K && s_pre[w][k + 1] <= jb) ++k;
                const uint32_t q = s_nb[w][k];
                b = cell_sc[q] + (jb - s_pre[w][k]);
                a = a_lo + ia;
                dec = box_decide<WIDE>(s_box[w][ia], box[b], s_rep[w][ia], reps[b], m);
                if (dec) key = ((unsigned long long)s_lr[w][ia] << 32) | lroot[b];
            }
            const uint32_t active = __ballot_sync(0xffffffffu, dec != 0);
            const uint32_t yes_m = __ballot_sync(0xffffffffu, dec == 1);
            n_yes += __popc(yes_m);
            n_tests += __popc(active & ~yes_m);
            bool enq = false;
            if (dec) {
                const uint32_t peers = __match_any_sync(active, key);
                const int leader = __ffs(peers) - 1;
                const uint32_t ra = (uint32_t)(key >> 32), rb = (uint32_t)key;
                if (peers & yes_m) {
                    if (lane == leader && !uf_unite(parent, ra, rb)) atomicOr(status, ST_UNION_CAP);
                } else {
                    int same = 0;
                    if (lane == leader) same = uf_find(parent, ra) == uf_find(parent, rb);
                    same = __shfl_sync(peers, same, leader);
                    if (same) {
                        if (lane == leader) n_same += __popc(peers);
                    } else {
                        enq = true;
                    }
                }
            }
            const uint32_t qmask = __ballot_sync(0xffffffffu, enq);
            if (qmask) {
                n_queued += __popc(qmask);
                const int leader = __ffs(qmask) - 1;
                uint32_t slot = 0;
                if (lane == leader) slot = atomicAdd(&plan->pairq_n, (uint32_t)__popc(qmask));
                slot = __shfl_sync(0xffffffffu, slot, leader) + __popc(qmask & lanemask_lt());
                if (enq) {
                    if (slot < qcap) {
                        pairq[slot] = make_uint2(a, b);
                    } else if (thread_pair_test<WIDE>(a, b, box, rec, m)) {
                        // queue full: decide this pair alone (slow, but exact)
                        if (!uf_unite(parent, a, b)) atomicOr(status, ST_UNION_CAP);
                    }
                }
            }
        }
        __syncwarp();
    }
    n_same = __reduce_add_sync(0xffffffffu, (uint32_t)n_same);
    if (lane == 0) {
        atomicAdd(&plan->ctr[CTR_PAIRS], n_pairs);
        atomicAdd(&plan->ctr[CTR_BOX_JOINS], n_yes);
        atomicAdd(&plan->ctr[CTR_POINT_TESTS], n_tests);
        atomicAdd(&plan->ctr[CTR_SAME_ROOT], n_same);
        atomicAdd(&plan->ctr[CTR_QUEUED], n_queued);
    }
}

// a4, last part: the queued pairs, one warp per pair after a parallel root
// check of 32 pairs at a time (most were joined meanwhile).
template <bool WIDE>
__global__ void __launch_bounds__(kUnionThreads, 2)
    k_pairs(Plan *plan, Params prm, const SubBox *__restrict__ box, const Rec *__restrict__ rec,
            uint32_t *parent, const uint2 *__restrict__ pairq, uint32_t qcap)
{
    const uint32_t nq = min(plan->pairq_n, qcap);
    const int lane = threadIdx.x & 31;
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    uint32_t *status = &plan->status;
    Metric<WIDE> m;
    m.T2 = (typename Metric<WIDE>::T)prm.T2;
    m.R1 = prm.R + 1;
    unsigned long long n_same = 0, n_evals = 0;
    for (uint32_t base = gw * 32; base < nq; base += nw * 32) {
        const uint32_t i = base + lane;
        uint2 pr = make_uint2(0, 0);
        bool live = false;
        if (i < nq) {
            pr = pairq[i];
            live = uf_find(parent, pr.x) != uf_find(parent, pr.y);
            if (!live) ++n_same;
        }
        uint32_t mask = __ballot_sync(0xffffffffu, live);
        while (mask) {
            const int src = __ffs(mask) - 1;
            mask &= mask - 1;
            const uint32_t pa = __shfl_sync(0xffffffffu, pr.x, src);
            const uint32_t pb = __shfl_sync(0xffffffffu, pr.y, src);
            if (warp_pair_test<WIDE>(pa, pb, box, rec, m, n_evals) && lane == 0 &&
                !uf_unite(parent, pa, pb))
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
__global__ void __launch_bounds__(256)
    k_flatten_stats(Plan *plan, const SubBox *__restrict__ box, const uint32_t *__restrict__ sminidx,
                    uint32_t *parent, uint32_t *__restrict__ csize, uint32_t *__restrict__ cmin)
{
    const uint32_t M = plan->M_s;
    const int lane = threadIdx.x & 31;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t base = (blockIdx.x * blockDim.x + threadIdx.x) & ~31u; base < M; base += stride) {
        const uint32_t a = base + lane;
        const bool valid = a < M;
        uint32_t r = 0xffffffffu, cnt = 0, mi = 0xffffffffu;
        if (valid) {
            // read-only walk: unions are finished, pointers only get shorter
            r = a;
            for (uint32_t it = 0; it < kUnionCap; ++it) {
                const uint32_t p = ld_relaxed(parent + r);
                if (p == r) break;
                r = p;
            }
            cnt = box[a].count;
            mi = sminidx[a];
        }
        uint32_t active = __ballot_sync(0xffffffffu, valid);
        if (valid) st_relaxed(parent + a, r);
        while (active) {
            const int leader = __ffs(active) - 1;
            const uint32_t r0 = __shfl_sync(0xffffffffu, r, leader);
            const bool in = valid && r == r0;
            const uint32_t s = __reduce_add_sync(0xffffffffu, in ? cnt : 0u);
            const uint32_t mn = __reduce_min_sync(0xffffffffu, in ? mi : 0xffffffffu);
            if (lane == leader) {
                atomicAdd(csize + r0, s);
                atomicMin(cmin + r0, mn);
            }
            active &= ~__ballot_sync(0xffffffffu, in);
        }
    }
}

// a6: list the kept components (root, smallest index) for the ordering sort.
__global__ void __launch_bounds__(256)
    k_kept(Plan *plan, const uint32_t *__restrict__ parent, const uint32_t *__restrict__ csize,
           const uint32_t *__restrict__ cmin, long long min_size, long long max_size,
           uint32_t *__restrict__ kept_key, uint32_t *__restrict__ kept_val)
{
    const uint32_t M = plan->M_s;
    const int lane = threadIdx.x & 31;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t base = (blockIdx.x * blockDim.x + threadIdx.x) & ~31u; base < M; base += stride) {
        const uint32_t a = base + lane;
        bool keep = false;
        if (a < M && parent[a] == a) {
            const long long s = (long long)csize[a];
            keep = s >= min_size && s <= max_size;
        }
        const uint32_t mask = __ballot_sync(0xffffffffu, keep);
        if (!mask) continue;
        const int leader = __ffs(mask) - 1;
        uint32_t slot = 0;
        if (lane == leader) slot = atomicAdd(&plan->kept.n, (uint32_t)__popc(mask));
        slot = __shfl_sync(0xffffffffu, slot, leader) + __popc(mask & lanemask_lt());
        if (keep) {
            kept_key[slot] = cmin[a];
            kept_val[slot] = a;
        }
    }
}

// a6: rank of each kept root in smallest-index order.
__global__ void __launch_bounds__(256)
    k_rank(Plan *plan, const uint32_t *__restrict__ va, const uint32_t *__restrict__ vb,
           int32_t *__restrict__ crank)
{
    const uint32_t k = plan->kept.n;
    const uint32_t *__restrict__ v = (plan->kept.npasses & 1u) ? vb : va;
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < k; t += gridDim.x * blockDim.x)
        crank[v[t]] = (int32_t)t;
}

// a6: labels in input order.
__global__ void __launch_bounds__(256)
    k_labels(Plan *plan, const uint32_t *__restrict__ idx_a, const uint32_t *__restrict__ idx_b,
             const uint32_t *__restrict__ sc_of, const uint32_t *__restrict__ parent,
             const int32_t *__restrict__ crank, int32_t *__restrict__ labels)
{
    const uint32_t n = plan->sort.n;
    const uint32_t *__restrict__ idx = (plan->sort.npasses & 1u) ? idx_b : idx_a;
    for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const uint32_t i = idx[p];
        if (i < n) labels[i] = crank[parent[sc_of[p]]];
    }
}

}  // namespace

cudaError_t enqueue_union(Workspace &ws, const Params &prm, long long min_size,
                          long long max_size, cudaStream_t st)
{
    const uint32_t qcap = (uint32_t)ws.pairq_cap;
    const bool wide = prm.R + 1 > 26754;
    if (!wide)
        k_local<false><<<ws.sms * 4, kUnionThreads, 0, st>>>(ws.plan, prm, ws.cell_sc, ws.box,
                                                             ws.reps, ws.rec, ws.parent, ws.lroot);
    else
        k_local<true><<<ws.sms * 4, kUnionThreads, 0, st>>>(ws.plan, prm, ws.cell_sc, ws.box,
                                                            ws.reps, ws.rec, ws.parent, ws.lroot);
    FEC_MARK(ws, "k_local", st);
    if (!wide)
        k_global<false><<<ws.sms * 4, kUnionThreads, 0, st>>>(
            ws.plan, prm, ws.cell_key, ws.cell_sc, ws.box, ws.reps, ws.rec, ws.lroot, ws.parent,
            ws.slab_lo, ws.slab_hi, ws.pairq, qcap);
    else
        k_global<true><<<ws.sms * 4, kUnionThreads, 0, st>>>(
            ws.plan, prm, ws.cell_key, ws.cell_sc, ws.box, ws.reps, ws.rec, ws.lroot, ws.parent,
            ws.slab_lo, ws.slab_hi, ws.pairq, qcap);
    FEC_MARK(ws, "k_global", st);
    if (!wide)
        k_pairs<false><<<ws.sms * 2, kUnionThreads, 0, st>>>(ws.plan, prm, ws.box, ws.rec, ws.parent,
                                                             ws.pairq, qcap);
    else
        k_pairs<true><<<ws.sms * 2, kUnionThreads, 0, st>>>(ws.plan, prm, ws.box, ws.rec, ws.parent,
                                                            ws.pairq, qcap);
    FEC_MARK(ws, "k_pairs", st);
    k_flatten_stats<<<ws.sms * 8, 256, 0, st>>>(ws.plan, ws.box, ws.sminidx, ws.parent, ws.csize,
                                                 ws.cmin);
    FEC_MARK(ws, "k_flatten_stats", st);
    k_kept<<<ws.sms * 8, 256, 0, st>>>(ws.plan, ws.parent, ws.csize, ws.cmin, min_size, max_size,
                                        ws.kept_key_a(), ws.kept_val_a());
    FEC_MARK(ws, "k_kept", st);
    return cudaGetLastError();
}

cudaError_t enqueue_labels(Workspace &ws, int32_t *labels, cudaStream_t st)
{
    k_rank<<<ws.sms * 4, 256, 0, st>>>(ws.plan, ws.kept_val_a(), ws.kept_val_b(), ws.crank);
    FEC_MARK(ws, "k_rank", st);
    k_labels<<<ws.sms * 8, 256, 0, st>>>(ws.plan, ws.vals_a, ws.vals_b, ws.sc_of, ws.parent,
                                         ws.crank, labels);
    FEC_MARK(ws, "k_labels", st);
    return cudaGetLastError();
}

}  // namespace fec
