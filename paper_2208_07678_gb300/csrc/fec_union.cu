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

// Whole-warp test of sub-cells a and b: is any point pair within d?  On the
// first hit lane 0 joins the two sets.
template <bool WIDE>
__device__ void warp_pair_test(uint32_t a, uint32_t b, const SubBox *__restrict__ box,
                               const Rec *__restrict__ rec, uint32_t *parent, const Metric<WIDE> &m,
                               uint32_t *status)
{
    const int lane = threadIdx.x & 31;
    SubBox A = box[a], B = box[b];
    if (A.count < B.count) {
        const SubBox t = A;
        A = B;
        B = t;
    }
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
            const bool hit = cand && m.within(p.x - q.x, p.y - q.y, p.z - q.z);
            if (__any_sync(0xffffffffu, hit)) {
                if (lane == 0 && !uf_unite(parent, a, b)) atomicOr(status, ST_UNION_CAP);
                return;
            }
        }
    }
}

template <bool WIDE>
__global__ void __launch_bounds__(kUnionThreads)
    k_union(Plan *plan, Params prm, const unsigned long long *__restrict__ cell_key,
            const uint32_t *__restrict__ cell_sc, const SubBox *__restrict__ box,
            const Rec *__restrict__ rec, uint32_t *parent, const uint32_t *__restrict__ slab_lo,
            const uint32_t *__restrict__ slab_hi)
{
    __shared__ uint32_t s_nb[kUnionWarps][16];
    __shared__ uint32_t s_pre[kUnionWarps][17];
    __shared__ SubBox s_own[kUnionWarps][8];

    const uint32_t M = plan->M_c;
    const uint32_t b1 = plan->bits[1], b2 = plan->bits[2];
    const unsigned long long m1 = (1ull << b1) - 1, m2 = (1ull << b2) - 1;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    uint32_t *status = &plan->status;
    Metric<WIDE> m;
    m.T2 = (typename Metric<WIDE>::T)prm.T2;
    m.R1 = prm.R + 1;

    for (uint32_t c = gw; c < M; c += nw) {
        const unsigned long long ck = cell_key[c];
        const unsigned long long c0 = ck >> (b1 + b2);
        const unsigned long long c1 = (ck >> b2) & m1, c2 = ck & m2;
        const uint32_t a_lo = cell_sc[c], na = cell_sc[c + 1] - a_lo;
        if (lane < (int)na) s_own[w][lane] = box[a_lo + lane];

        // Neighbour cells of the half stencil.  Lanes 0..3 search columns
        // (0,+1), (+1,-1), (+1,0), (+1,+1) over dz in {-1,0,+1}; lane 4
        // checks (0,0,+1), the next cell of the same column.
        uint32_t found[3];
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
                    found[nf++] = q;
                }
            }
        } else if (lane == 4) {
            if (c2 < m2 && c + 1 < M && cell_key[c + 1] == ck + 1) found[nf++] = c + 1;
        }
        int incl = nf;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        const int K = __shfl_sync(0xffffffffu, incl, 31);
        for (int i = 0; i < nf; ++i) s_nb[w][incl - nf + i] = found[i];
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
        const uint32_t P0 = na * (na - 1) / 2;
        const uint32_t P = P0 + na * T;

        for (uint32_t base = 0; base < P; base += 32) {
            const uint32_t i = base + lane;
            bool needs = false;
            uint32_t a = 0, b = 0;
            if (i < P) {
                uint32_t ia, ib;
                SubBox BB;
                if (i < P0) {
                    uint32_t rem = i;
                    ia = 0;
                    while (rem >= na - 1 - ia) {
                        rem -= na - 1 - ia;
                        ++ia;
                    }
                    ib = ia + 1 + rem;
                    b = a_lo + ib;
                    BB = s_own[w][ib];
                } else {
                    const uint32_t j = i - P0;
                    ia = j % na;
                    const uint32_t jb = j / na;
                    int k = 0;
                    while (k + 1 < K && s_pre[w][k + 1] <= jb) ++k;
                    const uint32_t q = s_nb[w][k];
                    b = cell_sc[q] + (jb - s_pre[w][k]);
                    BB = box[b];
                }
                a = a_lo + ia;
                const SubBox &AA = s_own[w][ia];
                if (m.box_gap(AA, BB)) {
                    if (m.box_diam(AA, BB)) {
                        if (!uf_unite(parent, a, b)) atomicOr(status, ST_UNION_CAP);
                    } else {
                        needs = true;
                    }
                }
            }
            uint32_t mask = __ballot_sync(0xffffffffu, needs);
            while (mask) {
                const int src = __ffs(mask) - 1;
                mask &= mask - 1;
                const uint32_t pa = __shfl_sync(0xffffffffu, a, src);
                const uint32_t pb = __shfl_sync(0xffffffffu, b, src);
                int same = 0;
                if (lane == 0) same = uf_find(parent, pa) == uf_find(parent, pb);
                same = __shfl_sync(0xffffffffu, same, 0);
                if (!same) warp_pair_test<WIDE>(pa, pb, box, rec, parent, m, status);
            }
        }
        __syncwarp();
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
    const int grid = ws.sms * 8;
    if (prm.R + 1 <= 26754)
        k_union<false><<<grid, kUnionThreads, 0, st>>>(ws.plan, prm, ws.cell_key, ws.cell_sc, ws.box,
                                                       ws.rec, ws.parent, ws.slab_lo, ws.slab_hi);
    else
        k_union<true><<<grid, kUnionThreads, 0, st>>>(ws.plan, prm, ws.cell_key, ws.cell_sc, ws.box,
                                                      ws.rec, ws.parent, ws.slab_lo, ws.slab_hi);
    FEC_MARK(ws, "k_union", st);
    k_flatten_stats<<<grid, 256, 0, st>>>(ws.plan, ws.box, ws.sminidx, ws.parent, ws.csize, ws.cmin);
    FEC_MARK(ws, "k_flatten_stats", st);
    k_kept<<<grid, 256, 0, st>>>(ws.plan, ws.parent, ws.csize, ws.cmin, min_size, max_size,
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
