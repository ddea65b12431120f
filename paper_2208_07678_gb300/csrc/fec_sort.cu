// fec_sort.cu -- LSD radix sort of (key, value) pairs (32- or 64-bit each),
// one kernel per 8-bit digit ("onesweep": every tile ranks its keys stably in
// shared memory, finds its global digit offsets by decoupled look-back over
// the preceding tiles, and writes each digit run coalesced).  Replaces the
// kd-tree build of Algorithm 1 (Section 2.2): sorting by grid-cell key groups
// every cell's points contiguously.
//
// Digit histograms of all passes are computed up front (by the key kernel
// for the main sort), so a pass reads each key and value once and writes them
// once; with packed payloads the main sort's first pass reads the point
// coordinates instead and computes each key and payload itself.  Look-back
// waits are bounded (SortCtl::wait_cap); a timeout sets ST_WAIT_TIMEOUT and
// the pass finishes with a wrong prefix (every store stays in bounds) instead
// of hanging; every later kernel of the call then returns at once.  Tile ids are taken from
// an atomic counter, so a tile only ever waits on tiles already owned by
// running blocks.
#include "fec_internal.cuh"

namespace fec {

namespace {

constexpr int kWarps = kSortThreads / 32;
static_assert(kSortThreads >= kRadixBins, "the digit loops need one thread per digit");
constexpr uint32_t kFlagAgg = 1u << 30;
constexpr uint32_t kFlagIncl = 2u << 30;
constexpr uint32_t kValMask = (1u << 30) - 1;
#ifndef FEC_SORT_LOOKWIN
#define FEC_SORT_LOOKWIN 4
#endif
constexpr int kLookWin = FEC_SORT_LOOKWIN;  // preceding tiles read per look-back step

template <typename KeyT, typename ValT>
struct SortSmem {
    KeyT keys[kSortTile];
    ValT vals[kSortTile];
    uint16_t wcnt[kWarps][kRadixBins];
    uint32_t gofs[kRadixBins];   // exclusive global offset of each digit (whole pass)
    uint32_t cnt[kRadixBins];    // tile count of each digit
    uint32_t excl[kRadixBins];   // tile-local exclusive offset of each digit
    uint32_t base[kRadixBins];   // output index = base[d] + tile-local position
    uint32_t warp_tot[kRadixBins / 32];
    uint32_t tile;
};

// Exclusive scan of in[0..255] into out[], by the first 256 threads.
__device__ __forceinline__ void scan256(const uint32_t *in, uint32_t *out, uint32_t *warp_tot)
{
    const int t = threadIdx.x;
    uint32_t v = 0, incl = 0;
    if (t < kRadixBins) {
        v = in[t];
        incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
            if ((t & 31) >= o) incl += u;
        }
        if ((t & 31) == 31) warp_tot[t >> 5] = incl;
    }
    __syncthreads();
    if (t < kRadixBins) {
        uint32_t add = 0;
        for (int w = 0; w < (t >> 5); ++w) add += warp_tot[w];
        out[t] = add + incl - v;
    }
    __syncthreads();
}

// XYZ: the first pass of the main sort in the packed layout, which reads the
// coordinates and computes each point's key and payload itself (the key
// kernel only made the histograms), instead of reading stored keys.
//
// SEG (the main sort of a call with several frames): every frame is sorted
// on its own, in its own positions: tiles never straddle two frames, a tile's
// digit offsets come from its frame's histograms, and the look-back stops at
// the frame's first tile.  Otherwise one run of ctl->n keys: the main sort
// of one frame (fr non-null: its histograms and input rows), or a plain
// sort of ctl->n keys (fr null: histograms in ctl).  Values of a first pass
// that has none are the points' input rows.
template <typename KeyT, typename ValT, bool XYZ, bool SEG>
__global__ void __launch_bounds__(kSortThreads, kSortMinBlocks)
    k_onesweep(SortCtl *__restrict__ ctl, const KeyT *__restrict__ kin,
               const ValT *__restrict__ vin, KeyT *__restrict__ kout,
               ValT *__restrict__ vout, uint32_t *__restrict__ tstat_base, size_t tstride,
               int pass, uint32_t *__restrict__ status, const float *__restrict__ xyz,
               const Plan *__restrict__ plan, Params prm, const Frame *__restrict__ fr,
               const uint32_t *__restrict__ fhist)
{
    grid_enter();
    // Two look-back status arrays alternate between passes: this pass reads
    // and publishes in `tstat`, and clears its own tiles' slots in the other
    // array for the next pass (which starts only after this one finishes).
    constexpr uint32_t want64 = sizeof(KeyT) == 8 ? 1u : 0u;
    if (ctl->key64 != want64 || (uint32_t)pass >= ctl->npasses) return;
    if (block_aborted(status)) return;  // an earlier stage gave up
    const uint32_t wait_cap = ctl->wait_cap;
    const uint32_t par = ctl->parity;
    uint32_t *__restrict__ tstat = tstat_base + (size_t)((pass + par) & 1) * tstride;
    uint32_t *__restrict__ tnext = tstat_base + (size_t)((pass + par + 1) & 1) * tstride;
    const uint32_t n = ctl->n;
    if (n == 0) return;
    const uint32_t nf = SEG ? prm.nf : 1u;
    const uint32_t ntiles = SEG ? prm.ntiles : (n + kSortTile - 1) / kSortTile;
    const int shift = pass * kRadixBits;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    SortSmem<KeyT, ValT> &S = *reinterpret_cast<SortSmem<KeyT, ValT> *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    __shared__ GridMap gm;  // read from shared memory: it would cost registers
    if (XYZ && tid == 0) gm.load(plan, prm, fr[0]);
    uint32_t cur = 0xffffffffu;  // frame whose digit offsets are in S.gofs (block-uniform)
    // the tile's frame: its positions [seg_lo, seg_lo + seg_n), its input
    // rows from row0, its first tile ftile0 (read once for a single frame)
    uint32_t f = 0, seg_lo = 0, seg_n = n, ftile0 = 0, row0 = 0;
    if (!SEG && fr) row0 = fr[0].in_off;

    for (;;) {
        if (tid == 0) S.tile = atomicAdd(&ctl->tile_counter[pass], 1u);
        for (int i = tid; i < kWarps * kRadixBins; i += kSortThreads)
            (&S.wcnt[0][0])[i] = 0;
        __syncthreads();
        const uint32_t tile = S.tile;
        if (tile >= ntiles) break;
        if (SEG) {
            f = frame_of_tile(fr, nf, tile);
            seg_lo = fr[f].pos_off;
            seg_n = fr[f].n;
            ftile0 = fr[f].tile0;
            row0 = fr[f].in_off;
        }
        if (f != cur) {  // the frame's exclusive digit offsets of this pass
            if (tid < kRadixBins)
                S.cnt[tid] = fr ? fhist[((size_t)f * kMaxPasses + pass) * kRadixBins + tid]
                                : ctl->hist[pass][tid];
            if (SEG && XYZ && tid == 0) gm.set_frame(fr[f]);
            __syncthreads();
            scan256(S.cnt, S.gofs, S.warp_tot);
            cur = f;
        }

        KeyT key[kSortIPT];
        ValT val[kSortIPT];
        uint32_t lrank[kSortIPT], dig[kSortIPT];
        // frame-local index of the warp's first key
        const uint32_t seg = (tile - ftile0) * (uint32_t)kSortTile + warp * (32u * kSortIPT);
        // all of the thread's loads first, so that they are in flight together
        // (the ranking loop below synchronises the warp after every item)
        if (XYZ) {
            float xf[3 * kSortIPT];
#pragma unroll
            for (int r = 0; r < kSortIPT; ++r) {
                const uint32_t li = seg + r * 32 + lane;
#pragma unroll
                for (int a = 0; a < 3; ++a)
                    xf[3 * r + a] = li < seg_n ? __ldcs(xyz + 3 * (size_t)(row0 + li) + a) : 0.0f;
            }
#pragma unroll
            for (int r = 0; r < kSortIPT; ++r) {
                const uint32_t li = seg + r * 32 + lane;
                int32_t q[3];
#pragma unroll
                for (int a = 0; a < 3; ++a) quantize1(xf[3 * r + a], q[a]);
                uint32_t c[3], off[3];
                gm.cell_of(q, c, off);
                key[r] = gm.key_of<KeyT>(c, off);
                val[r] = (ValT)gm.payload_of(off, row0 + li);
            }
        } else {
#pragma unroll
            for (int r = 0; r < kSortIPT; ++r) {
                const uint32_t li = seg + r * 32 + lane;
                const bool valid = li < seg_n;
                key[r] = valid ? kin[seg_lo + li] : KeyT(0);
                val[r] = valid ? (vin ? vin[seg_lo + li] : (ValT)(row0 + li)) : (ValT)0;
            }
        }
#pragma unroll
        for (int r = 0; r < kSortIPT; ++r) {
            const uint32_t li = seg + r * 32 + lane;
            const bool valid = li < seg_n;
            const uint32_t d = valid ? (uint32_t)(key[r] >> shift) & (kRadixBins - 1)
                                     : (uint32_t)kRadixBins + lane;
            dig[r] = d;
            const uint32_t peers = __match_any_sync(0xffffffffu, d);
            const int leader = __ffs(peers) - 1;
            uint32_t old = 0;
            if (valid && lane == leader) {
                old = S.wcnt[warp][d];
                S.wcnt[warp][d] = (uint16_t)(old + __popc(peers));
            }
            old = __shfl_sync(0xffffffffu, old, leader);
            lrank[r] = old + __popc(peers & lanemask_lt());
            __syncwarp();
        }
        __syncthreads();

        // Per digit: exclusive offsets of each warp inside the tile.
        if (tid < kRadixBins) {
            tnext[(size_t)tile * kRadixBins + tid] = 0;
            uint32_t run = 0;
            for (int w = 0; w < kWarps; ++w) {
                uint32_t c = S.wcnt[w][tid];
                S.wcnt[w][tid] = (uint16_t)run;
                run += c;
            }
            S.cnt[tid] = run;
            // publish this tile's digit count for later tiles of its frame
            st_relaxed(tstat + (size_t)tile * kRadixBins + tid,
                       (tile == ftile0 ? kFlagIncl : kFlagAgg) | run);
        }
        __syncthreads();
        scan256(S.cnt, S.excl, S.warp_tot);

        // Decoupled look-back: sum the digit counts of the frame's preceding tiles.
        if (tid < kRadixBins) {
            uint32_t prefix = 0;
            if (tile > ftile0) {  // ftile0 = 0 unless SEG
                // Windowed: the statuses of up to kLookWin preceding tiles are
                // loaded at once, so a walk over many tiles costs one memory
                // latency per window instead of one per tile.
                const int64_t first = (int64_t)ftile0;
                int64_t p = (int64_t)tile - 1;
                uint32_t it = 0;
                bool done = false;
                while (p >= first && !done) {
                    uint32_t win[kLookWin];
#pragma unroll
                    for (int j = 0; j < kLookWin; ++j)
                        win[j] = (p - j >= first) ? ld_relaxed(tstat + (size_t)(p - j) * kRadixBins + tid)
                                                  : kFlagIncl;
#pragma unroll
                    for (int j = 0; j < kLookWin; ++j) {
                        if (done) break;
                        uint32_t s = win[j];
                        while ((s & ~kValMask) == 0) {  // not published yet: wait for it
                            if (++it > wait_cap) {
                                atomicOr(status, ST_WAIT_TIMEOUT);
                                s = kFlagIncl;
                                break;
                            }
                            spin_pause(it);
                            s = ld_relaxed(tstat + (size_t)(p - j) * kRadixBins + tid);
                        }
                        if (p - j >= first) prefix += s & kValMask;
                        if ((s & ~kValMask) == kFlagIncl) done = true;
                    }
                    p -= kLookWin;
                }
                st_relaxed(tstat + (size_t)tile * kRadixBins + tid,
                           kFlagIncl | ((prefix + S.cnt[tid]) & kValMask));
            }
            S.base[tid] = S.gofs[tid] + prefix - S.excl[tid];
        }
        __syncthreads();

        // Stage in tile-sorted order, then write digit runs coalesced.
#pragma unroll
        for (int r = 0; r < kSortIPT; ++r) {
            const uint32_t li = seg + r * 32 + lane;
            if (li < seg_n) {
                const uint32_t d = dig[r];
                const uint32_t lp = S.excl[d] + S.wcnt[warp][d] + lrank[r];
                if (!FEC_IN_BOUNDS(status, lp, kSortTile)) continue;
                S.keys[lp] = key[r];
                S.vals[lp] = val[r];
            }
        }
        __syncthreads();
        const uint32_t tfirst = (tile - ftile0) * (uint32_t)kSortTile;
        const uint32_t tile_n = min((uint32_t)kSortTile, seg_n - tfirst);
        for (uint32_t i = tid; i < tile_n; i += kSortThreads) {
            const KeyT k = S.keys[i];
            const uint32_t d = (uint32_t)(k >> shift) & (kRadixBins - 1);
            const uint32_t o = S.base[d] + i;  // frame-local output position
            if (o < seg_n) {  // only false after a look-back timeout
                kout[seg_lo + o] = k;
                vout[seg_lo + o] = S.vals[i];
            }
        }
        __syncthreads();
    }
}

template <typename KeyT, typename ValT>
cudaError_t launch_sort_t(const Workspace &ws, const char *name, SortCtl *ctl, void *ka_, void *va_,
                          void *kb_, void *vb_, bool identity_vals, uint32_t *tile_status,
                          uint32_t tiles, int max_passes, int grid, cudaStream_t st,
                          uint32_t *status, const SortSource &src)
{
    const size_t smem = sizeof(SortSmem<KeyT, ValT>);
    static int per_sm = 0;  // resident blocks per SM (persistent grid)
    static std::atomic<unsigned long long> attr_ctx{0};  // context the attributes were set in
    constexpr bool kXyz = sizeof(ValT) == 8;  // keys from coordinates: packed payloads only
    if (!per_sm || ctx_setup_needed(attr_ctx)) {
        // every variant of this key / value width: its shared memory, and the
        // fewest resident blocks per SM of any of them
        int least = 1 << 30;
        cudaError_t e = cudaSuccess;
        auto setup = [&](const void *fn) {
            if (e != cudaSuccess) return;
            e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            int a = 0;
            if (e == cudaSuccess)
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, fn, kSortThreads, smem);
            if (e == cudaSuccess) least = a < least ? a : least;
        };
        setup((const void *)k_onesweep<KeyT, ValT, false, false>);
        setup((const void *)k_onesweep<KeyT, ValT, false, true>);
        if constexpr (kXyz) {
            setup((const void *)k_onesweep<KeyT, ValT, true, false>);
            setup((const void *)k_onesweep<KeyT, ValT, true, true>);
        }
        if (e != cudaSuccess) return e;
        per_sm = least < 1 ? 1 : least;
        ctx_setup_done(attr_ctx);
    }
    const bool seg = src.frames && src.prm.nf > 1;
    grid *= per_sm;
    if (grid > (int)tiles) grid = tiles > 0 ? (int)tiles : 1;  // a small sort needs fewer blocks
    // The look-back array the first pass uses is clear on entry: the key
    // kernel clears array 0 before the main sort, and every pass clears its
    // tiles' slots in the other array for the next pass.
    const size_t tstride = sort_tstride(ws);
    cudaError_t e = cudaSuccess;
    KeyT *kin = (KeyT *)ka_, *kout = (KeyT *)kb_;
    ValT *vin = (ValT *)va_, *vout = (ValT *)vb_;
    for (int p = 0; p < max_passes; ++p) {
        bool done = false;
        if constexpr (kXyz) {
            if (p == 0 && src.xyz) {
                if (seg)
                    launch(k_onesweep<KeyT, ValT, true, true>, grid, kSortThreads, smem, st,
                        ctl, nullptr, nullptr, kout, vout, tile_status, tstride, p, status, src.xyz,
                        src.plan, src.prm, src.frames, src.fhist);
                else
                    launch(k_onesweep<KeyT, ValT, true, false>, grid, kSortThreads, smem, st,
                        ctl, nullptr, nullptr, kout, vout, tile_status, tstride, p, status, src.xyz,
                        src.plan, src.prm, src.frames, src.fhist);
                done = true;
            }
        }
        const ValT *vsrc = (p == 0 && identity_vals) ? nullptr : vin;
        if (!done && seg)
            launch(k_onesweep<KeyT, ValT, false, true>, grid, kSortThreads, smem, st,
                ctl, kin, vsrc, kout, vout, tile_status, tstride, p, status, nullptr, nullptr,
                src.prm, src.frames, src.fhist);
        else if (!done)
            launch(k_onesweep<KeyT, ValT, false, false>, grid, kSortThreads, smem, st,
                ctl, kin, vsrc, kout, vout, tile_status, tstride, p, status, nullptr, nullptr,
                src.prm, src.frames, src.fhist);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        FEC_MARK(ws, name, st);
        KeyT *tk = kin;
        kin = kout;
        kout = tk;
        ValT *tv = vin;
        vin = vout;
        vout = tv;
    }
    return cudaSuccess;
}

}  // namespace

cudaError_t launch_sort(const Workspace &ws, const char *name, SortCtl *ctl, void *keys_a,
                        void *vals_a, void *keys_b, void *vals_b, bool key64, bool val64,
                        bool identity_vals, uint32_t *tile_status, uint32_t tiles, int max_passes,
                        int grid, cudaStream_t st, uint32_t *status, const SortSource &src)
{
    if (src.xyz && !val64) return cudaErrorInvalidValue;  // keys from xyz: packed payloads only
    using u32 = uint32_t;
    using u64 = unsigned long long;
    if (!key64 && !val64)
        return launch_sort_t<u32, u32>(ws, name, ctl, keys_a, vals_a, keys_b, vals_b, identity_vals,
                                       tile_status, tiles, max_passes, grid, st, status, src);
    if (!key64)
        return launch_sort_t<u32, u64>(ws, name, ctl, keys_a, vals_a, keys_b, vals_b, identity_vals,
                                       tile_status, tiles, max_passes, grid, st, status, src);
    if (!val64)
        return launch_sort_t<u64, u32>(ws, name, ctl, keys_a, vals_a, keys_b, vals_b, identity_vals,
                                       tile_status, tiles, max_passes, grid, st, status, src);
    return launch_sort_t<u64, u64>(ws, name, ctl, keys_a, vals_a, keys_b, vals_b, identity_vals,
                                   tile_status, tiles, max_passes, grid, st, status, src);
}

}  // namespace fec
