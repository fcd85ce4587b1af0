// Front-to-back per-tile lists (Sec. 3.1): a tile's list holds every Gaussian whose tile
// rectangle covers it, in ascending depth, ties by Gaussian id.
//
// Lists are short (hundreds of entries, a few thousand at most), so instead of sorting all
// (tile, depth) pairs globally the work is split by tile:
//   1. per-tile pair counts (atomics over each Gaussian's rectangle) and their exclusive scan,
//      which gives every tile's range directly;
//   2. block-cooperative fill: each pair is written into its tile's range at an atomic cursor
//      slot as (depth key, Gaussian id), in arbitrary order;
//   3. one CTA per tile sorts its range by the 64-bit key (depth bits << 32 | id) with a
//      bitonic network in shared memory (lists longer than the shared-memory capacity use the
//      same network on global memory).
// The key is unique per Gaussian, so the order is fully determined: the same lists as one
// stable sort of (tile, depth) keys in Gaussian-id order, without multi-pass global traffic.
//
// ogs_radix_sort_pairs (a classic three-kernel LSD radix sort: per-block digit histograms ->
// per-digit scan over blocks -> stable block-local multisplit and coalesced scatter, 8-bit
// digits, item count read on the device) is kept as a general entry point.
#include <mutex>

#include "internal.cuh"
#include "project_common.cuh"

namespace ogs {
namespace {

constexpr int kRsThreads = 256;
constexpr int kRsWarps = kRsThreads / 32;
constexpr int kRsItems = 4;
constexpr int kRsTile = kRsThreads * kRsItems;   // 1024 items per block
constexpr int kRsBins = 256;

__device__ __forceinline__ uint32_t count_of(const uint32_t* n_dev, int64_t n_cap) {
    if (!n_dev) return (uint32_t)n_cap;
    uint32_t n = *n_dev;
    return n < (uint64_t)n_cap ? n : (uint32_t)n_cap;
}

__global__ void __launch_bounds__(kRsThreads) rs_upsweep(const uint32_t* __restrict__ keys,
                                                         const uint32_t* n_dev, int64_t n_cap,
                                                         int shift, uint32_t mask,
                                                         uint32_t* __restrict__ hist, int nblocks) {
    __shared__ uint32_t h[kRsWarps][kRsBins];
    for (int i = threadIdx.x; i < kRsWarps * kRsBins; i += kRsThreads) (&h[0][0])[i] = 0;
    __syncthreads();
    const uint32_t n = count_of(n_dev, n_cap);
    const int64_t base = (int64_t)blockIdx.x * kRsTile;
    const int w = threadIdx.x >> 5;
    if (base < n) {
#pragma unroll 4
        for (int it = 0; it < kRsItems; ++it) {
            int64_t i = base + it * kRsThreads + threadIdx.x;
            if (i < n) atomicAdd(&h[w][(keys[i] >> shift) & mask], 1u);
        }
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kRsBins; d += kRsThreads) {
        uint32_t s = 0;
#pragma unroll
        for (int q = 0; q < kRsWarps; ++q) s += h[q][d];
        hist[(size_t)d * nblocks + blockIdx.x] = s;
    }
}

// One block per digit: exclusive scan of that digit's per-block counts; digit total out.
__global__ void __launch_bounds__(kRsThreads) rs_scan(uint32_t* hist, int nblocks,
                                                      uint32_t* digit_total) {
    __shared__ uint32_t ws[kRsWarps];
    __shared__ uint32_t carry;
    uint32_t* row = hist + (size_t)blockIdx.x * nblocks;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int b0 = 0; b0 < nblocks; b0 += kRsThreads) {
        int b = b0 + threadIdx.x;
        uint32_t v = b < nblocks ? row[b] : 0;
        uint32_t x = v;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane_id() >= (unsigned)o) x += y;
        }
        if (lane_id() == 31) ws[threadIdx.x >> 5] = x;
        __syncthreads();
        uint32_t wpre = 0;
        for (int q = 0; q < (int)(threadIdx.x >> 5); ++q) wpre += ws[q];
        uint32_t excl = carry + wpre + x - v;
        if (b < nblocks) row[b] = excl;
        __syncthreads();
        if (threadIdx.x == kRsThreads - 1) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) digit_total[blockIdx.x] = carry;
}

// block-wide exclusive scan of one value per thread (256 threads); returns the total
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t& excl, uint32_t* ws) {
    uint32_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane_id() >= (unsigned)o) x += y;
    }
    if (lane_id() == 31) ws[threadIdx.x >> 5] = x;
    __syncthreads();
    uint32_t wpre = 0, tot = 0;
#pragma unroll
    for (int q = 0; q < kRsWarps; ++q) {
        uint32_t s = ws[q];
        wpre += (q < (int)(threadIdx.x >> 5)) ? s : 0;
        tot += s;
    }
    excl = wpre + x - v;
    __syncthreads();
    return tot;
}

__global__ void __launch_bounds__(kRsThreads) rs_downsweep(
    const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
    uint32_t* __restrict__ kout, uint32_t* __restrict__ vout, const uint32_t* n_dev,
    int64_t n_cap, int shift, uint32_t mask, const uint32_t* __restrict__ hist, int nblocks,
    const uint32_t* __restrict__ digit_total) {
    __shared__ uint32_t wcnt[kRsWarps][kRsBins];
    __shared__ uint32_t gbase[kRsBins];
    __shared__ uint32_t lstart[kRsBins];
    __shared__ uint32_t ws[kRsWarps];
    __shared__ uint32_t skey[kRsTile];
    __shared__ uint32_t sval[kRsTile];
    const uint32_t n = count_of(n_dev, n_cap);
    const int64_t base = (int64_t)blockIdx.x * kRsTile;
    if (base >= n) return;
    for (int i = threadIdx.x; i < kRsWarps * kRsBins; i += kRsThreads) (&wcnt[0][0])[i] = 0;
    __syncthreads();
    const int w = threadIdx.x >> 5;
    const unsigned lane = lane_id();
    const int64_t wbase = base + (int64_t)w * (kRsItems * 32);
    uint32_t key[kRsItems], val[kRsItems], rank[kRsItems];
    // warp-striped: warp w owns a contiguous run of 32*kRsItems items, lane-interleaved per step, so
    // (step, lane) order equals input order and ranks come out stable
#pragma unroll
    for (int it = 0; it < kRsItems; ++it) {
        int64_t i = wbase + it * 32 + lane;
        bool valid = i < n;
        key[it] = valid ? kin[i] : 0xFFFFFFFFu;
        val[it] = valid ? vin[i] : 0u;
        uint32_t d = valid ? ((key[it] >> shift) & mask) : (uint32_t)kRsBins;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int leader = __ffs(peers) - 1;
        uint32_t old = 0;
        if (valid && (int)lane == leader) {
            old = wcnt[w][d];
            wcnt[w][d] = old + __popc(peers);
        }
        old = __shfl_sync(0xffffffffu, old, leader);
        rank[it] = old + __popc(peers & lanemask_lt());
    }
    __syncthreads();
    // per digit: prefix over warps (in place) and the block's digit total
    uint32_t dtot = 0;
    {
        const int d = threadIdx.x;   // kRsThreads == kRsBins
#pragma unroll
        for (int q = 0; q < kRsWarps; ++q) {
            uint32_t c = wcnt[q][d];
            wcnt[q][d] = dtot;
            dtot += c;
        }
    }
    // exclusive scan over digits of the block totals -> local start of each digit run
    uint32_t lex;
    block_excl_scan(dtot, lex, ws);
    // global base of each digit for this block
    uint32_t gt = digit_total[threadIdx.x], gex;
    block_excl_scan(gt, gex, ws);
    lstart[threadIdx.x] = lex;
    gbase[threadIdx.x] = gex + hist[(size_t)threadIdx.x * nblocks + blockIdx.x];
    __syncthreads();
#pragma unroll
    for (int it = 0; it < kRsItems; ++it) {
        int64_t i = wbase + it * 32 + lane;
        if (i < n) {
            uint32_t d = (key[it] >> shift) & mask;
            uint32_t p = lstart[d] + wcnt[w][d] + rank[it];
            skey[p] = key[it];
            sval[p] = val[it];
        }
    }
    __syncthreads();
    const int cnt = (int)min((int64_t)kRsTile, (int64_t)n - base);
    for (int p = threadIdx.x; p < cnt; p += kRsThreads) {
        uint32_t k = skey[p];
        uint32_t d = (k >> shift) & mask;
        uint32_t o = gbase[d] + (p - lstart[d]);
        kout[o] = k;
        vout[o] = sval[p];
    }
}

__global__ void copy_pairs(const uint32_t* ks, const uint32_t* vs, uint32_t* kd, uint32_t* vd,
                           const uint32_t* n_dev, int64_t n_cap) {
    const uint32_t n = count_of(n_dev, n_cap);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        kd[i] = ks[i];
        vd[i] = vs[i];
    }
}

struct RsScratch {
    uint32_t* k2;
    uint32_t* v2;
    uint32_t* hist;
    uint32_t* dtot;
};

size_t rs_layout(int64_t n_cap, void* base, RsScratch* s) {
    int64_t nb = (n_cap + kRsTile - 1) / kRsTile;
    if (nb < 1) nb = 1;
    Carver cv(base);
    RsScratch t;
    t.k2 = cv.take<uint32_t>(n_cap > 0 ? n_cap : 1);
    t.v2 = cv.take<uint32_t>(n_cap > 0 ? n_cap : 1);
    t.hist = cv.take<uint32_t>((size_t)nb * kRsBins);
    t.dtot = cv.take<uint32_t>(kRsBins);
    if (s) *s = t;
    return cv.off + 256;
}

// Sorts keys/vals in place by bits [lo, hi); returns false on launch failure.
bool radix_sort(uint32_t* keys, uint32_t* vals, const uint32_t* n_dev, int64_t n_cap, int lo,
                int hi, const RsScratch& s, cudaStream_t st) {
    int nb = (int)((n_cap + kRsTile - 1) / kRsTile);
    if (nb < 1) nb = 1;
    uint32_t *ka = keys, *va = vals, *kb = s.k2, *vb = s.v2;
    int passes = (hi - lo + 7) / 8;
    for (int p = 0; p < passes; ++p) {
        // split the bit range evenly over the passes
        int b0 = lo + (hi - lo) * p / passes, b1 = lo + (hi - lo) * (p + 1) / passes;
        uint32_t mask = (1u << (b1 - b0)) - 1u;
        rs_upsweep<<<nb, kRsThreads, 0, st>>>(ka, n_dev, n_cap, b0, mask, s.hist, nb);
        rs_scan<<<kRsBins, kRsThreads, 0, st>>>(s.hist, nb, s.dtot);
        rs_downsweep<<<nb, kRsThreads, 0, st>>>(ka, va, kb, vb, n_dev, n_cap, b0, mask, s.hist,
                                                 nb, s.dtot);
        uint32_t* t = ka; ka = kb; kb = t;
        t = va; va = vb; vb = t;
    }
    if (ka != keys)
        copy_pairs<<<stride_grid(n_cap, 256, 8), 256, 0, st>>>(ka, va, keys, vals, n_dev, n_cap);
    return cudaGetLastError() == cudaSuccess;
}

// ---------------------------------------------------------------------------------------
// per-tile lists: count -> scan -> fill -> per-tile sort
// ---------------------------------------------------------------------------------------

constexpr int kBinThreads = 256;
constexpr int kBinItems = 4;
constexpr int kBinTile = kBinThreads * kBinItems;
constexpr int kWarpSort = 512;           // lists up to this length: one warp, keys in registers
constexpr int kWarpTiles = 4;            // warps of a warp-sort CTA, one tile at a time each
constexpr int kWarpGrid = 8 * 152;       // warp-sort CTAs: 8 resident per SM
constexpr int kSmallSort = 2048;         // longer lists up to this length: 16 KB of keys ..
constexpr int kSmallGrid = 2 * 152;      // .. in CTAs of kLargeThreads looping over those lists
constexpr int kLargeThreads = 512;
constexpr int kLargeSort = 16384;        // longer lists: 128 KB of keys in dynamic shared memory
constexpr int kLargeGrid = 152;          // CTAs looping over the long lists
constexpr int kBinsListSort = 4096;      // ogs_sort_bins: lists past kWarpSort, 32 KB of keys ..
constexpr int kBinsListGrid = 4 * 152;   // .. in CTAs of kLargeThreads, four per SM

__device__ __forceinline__ void rect_of(uint2 r, uint32_t& x0, uint32_t& y0, uint32_t& x1,
                                        uint32_t& y1) {
    x0 = r.x & 0xFFFFu; y0 = r.x >> 16; x1 = r.y & 0xFFFFu; y1 = r.y >> 16;
}

// Block-cooperative walk over the pairs of kBinTile Gaussians (load balanced over pairs, not
// Gaussians): calls f(gaussian, tile) for every pair.  Consecutive pairs of a warp mostly
// belong to the k Gaussians of one anchor and so often share tiles, which f exploits.
template <class F>
__device__ __forceinline__ void for_each_pair(const uint32_t* __restrict__ tiles,
                                              const uint2* __restrict__ rect, uint32_t n,
                                              int gx, F f) {
    __shared__ uint32_t s_off[kBinThreads + 1];
    __shared__ uint32_t s_g[kBinThreads];
    __shared__ uint2 s_rect[kBinThreads];
    __shared__ uint32_t ws[kBinThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kBinTile;
    for (int it = 0; it < kBinItems; ++it) {
        const int64_t i = base + it * kBinThreads + threadIdx.x;
        uint32_t c = 0;
        uint2 rc = make_uint2(0, 0);
        if (i < n) {
            c = tiles[i];
            if (c) rc = rect[i];
        }
        uint32_t excl;
        const uint32_t tot = block_excl_scan(c, excl, ws);
        s_off[threadIdx.x] = excl;
        s_g[threadIdx.x] = (uint32_t)i;
        s_rect[threadIdx.x] = rc;
        __syncthreads();
        // every lane runs the same number of rounds, so f may use full-warp intrinsics
        const uint32_t rounds = (tot + kBinThreads - 1) / kBinThreads;
        for (uint32_t q = 0; q < rounds; ++q) {
            const uint32_t p = q * kBinThreads + threadIdx.x;
            const bool valid = p < tot;
            uint32_t g = 0, t = 0xFFFFFFFFu;
            if (valid) {
                int lo = 0, hi = kBinThreads - 1;      // owner: largest k with s_off[k] <= p
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (s_off[mid] <= p) lo = mid; else hi = mid - 1;
                }
                uint32_t x0, y0, x1, y1;
                rect_of(s_rect[lo], x0, y0, x1, y1);
                const uint32_t local = p - s_off[lo], w = x1 - x0;
                g = s_g[lo];
                t = (y0 + local / w) * (uint32_t)gx + x0 + local % w;
            }
            f(valid, g, t);
        }
        __syncthreads();
    }
}

// Warp-aggregated atomic add of 1 per lane on counter[t]: lanes with equal t are served by one
// atomic; returns this lane's slot (old value + rank among the equal lanes).
__device__ __forceinline__ uint32_t warp_agg_inc(uint32_t* counter, bool valid, uint32_t t,
                                                 bool want_slot) {
    const uint32_t peers = __match_any_sync(0xffffffffu, t);
    const uint32_t leader = __ffs(peers) - 1;
    uint32_t base = 0;
    if (valid && lane_id() == leader) {
        const uint32_t cnt = __popc(peers);
        if (want_slot) base = atomicAdd(counter + t, cnt);
        else atomicAdd(counter + t, cnt);
    }
    if (!want_slot) return 0;
    base = __shfl_sync(0xffffffffu, base, leader);
    return base + __popc(peers & lanemask_lt());
}

__global__ void __launch_bounds__(kBinThreads) bin_count(const uint32_t* __restrict__ tiles,
                                                         const uint2* __restrict__ rect,
                                                         const uint32_t* n_dev, int64_t n_cap,
                                                         int gx, uint32_t* __restrict__ tcount) {
    const uint32_t n = count_of(n_dev, n_cap);
    if ((int64_t)blockIdx.x * kBinTile >= n) return;
    for_each_pair(tiles, rect, n, gx, [&](bool valid, uint32_t, uint32_t t) {
        warp_agg_inc(tcount, valid, t, false);
    });
}

// Exclusive scan of the tile counts: one CTA per kScanChunk consecutive tiles (one tile per
// thread).  Each CTA sums every count itself (the total decides the overflow state; the part
// before its chunk is its offset: a few thousand words from L2), then scans its chunk: tile
// ranges, fill cursors cleared, and the chunk's tiles too long for the warp sorter listed in
// the chunk's slot of `mid` (up to kSmallSort entries) or `big` (longer), with their numbers
// in nmid[chunk] and nbig[chunk], so no counter needs clearing first.  CTA 0
// writes P and the overflow state.
constexpr int kScanChunk = 1024;

__global__ void __launch_bounds__(kScanChunk) tile_scan(const uint32_t* __restrict__ tcount,
                                                        int ntiles, int64_t pair_cap,
                                                        uint2* __restrict__ range,
                                                        uint32_t* __restrict__ cursor,
                                                        uint32_t* __restrict__ mid,
                                                        uint32_t* __restrict__ nmid,
                                                        uint32_t* __restrict__ big,
                                                        uint32_t* __restrict__ nbig,
                                                        ogs_counts* counts) {
    pdl_wait();
    pdl_trigger();
    __shared__ unsigned long long s_red[2][kScanChunk / 32];
    __shared__ uint32_t s_nmid, s_nbig;
    const int t = threadIdx.x, lane = (int)lane_id(), warp = t >> 5;
    const int c0 = blockIdx.x * kScanChunk;
    if (t == 0) s_nmid = s_nbig = 0;
    // totals: before the chunk, and over all tiles
    unsigned long long before = 0, all = 0;
    for (int b = t; b < ntiles; b += kScanChunk) {
        const uint32_t v = tcount[b];
        all += v;
        before += b < c0 ? v : 0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        before += __shfl_xor_sync(0xffffffffu, before, o);
        all += __shfl_xor_sync(0xffffffffu, all, o);
    }
    if (lane == 0) {
        s_red[0][warp] = before;
        s_red[1][warp] = all;
    }
    // the chunk's own counts, inclusive scan within each warp
    const int b = c0 + t;
    const uint32_t v = b < ntiles ? tcount[b] : 0u;
    unsigned long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    __syncthreads();
    unsigned long long off = 0, P = 0;
#pragma unroll 8
    for (int w = 0; w < kScanChunk / 32; ++w) {
        off += s_red[0][w];
        P += s_red[1][w];
    }
    __syncthreads();                                  // s_red reused for the warp totals
    if (lane == 31) s_red[0][warp] = x;
    __syncthreads();
    unsigned long long wbefore = 0;
    for (int w = 0; w < warp; ++w) wbefore += s_red[0][w];
    const bool over = P > (unsigned long long)pair_cap;
    if (b < ntiles) {
        const unsigned long long st = off + wbefore + x - v;
        range[b] = over ? make_uint2(0, 0) : make_uint2((uint32_t)st, (uint32_t)(st + v));
        cursor[b] = 0;
        if (!over && v > (uint32_t)kSmallSort)
            big[c0 + atomicAdd(&s_nbig, 1u)] = (uint32_t)b;
        else if (!over && v > (uint32_t)kWarpSort)
            mid[c0 + atomicAdd(&s_nmid, 1u)] = (uint32_t)b;
    }
    __syncthreads();
    if (t == 0) {
        nmid[blockIdx.x] = s_nmid;
        nbig[blockIdx.x] = s_nbig;
        if (blockIdx.x == 0) {
            counts->need_pairs = (uint32_t)(P > 0xFFFFFFFFull ? 0xFFFFFFFFull : P);
            if (over) {
                atomicOr(&counts->overflow, 2u);
                counts->n_pairs = 0;
            } else {
                counts->n_pairs = (uint32_t)P;
            }
        }
    }
}

// One pass over the Gaussians (one per thread, every lane of a warp calls bin_tiles):
// each (Gaussian, tile) pair is counted by an atomic whose return value is its slot in the
// tile's region, where its id and depth key are written.
__global__ void __launch_bounds__(kBinThreads, 8) bin_regions(const uint32_t* __restrict__ dkey,
                                                           const uint2* __restrict__ rect,
                                                           const uint32_t* __restrict__ tiles,
                                                           const uint32_t* n_dev, int64_t n_cap,
                                                           int gx, uint32_t* __restrict__ tc,
                                                           uint32_t cap,
                                                           uint32_t* __restrict__ keys,
                                                           uint32_t* __restrict__ ids,
                                                           uint2* __restrict__ defer,
                                                           unsigned long long* n_defer,
                                                           uint32_t defer_cap) {
    pdl_wait();
    pdl_trigger();
    const uint32_t n = count_of(n_dev, n_cap);
    const int64_t g = (int64_t)blockIdx.x * kBinThreads + threadIdx.x;
    if ((int64_t)blockIdx.x * kBinThreads >= n) return;        // whole CTA out of range
    // the three loads are independent (one round trip); rect and key are unused when c = 0
    uint32_t c = 0, k = 0xFFFFFFFFu;
    uint2 rc = make_uint2(0, 0);
    if (g < n) {
        c = tiles[g];
        rc = rect[g];
        k = dkey[g];
    }
    if (c == 0) rc = make_uint2(0, 0);
    bin_tiles(tc, gx, rc, c, (uint32_t)g, k, cap, keys, ids, defer, n_defer, defer_cap);
}

// The deferred chunks of large rectangles: one warp per (Gaussian, chunk) entry, the warps of
// a fixed grid taking the entries in turn, so the tiles of the large near-camera Gaussians
// are spread over every SM instead of staying with the warps that met them.
constexpr int kDeferGrid = 4 * kSmCount;

__global__ void __launch_bounds__(kBinThreads) bin_deferred(const uint32_t* __restrict__ dkey,
                                                            const uint2* __restrict__ rect,
                                                            int gx, uint32_t* __restrict__ tc,
                                                            uint32_t cap,
                                                            uint32_t* __restrict__ keys,
                                                            uint32_t* __restrict__ ids,
                                                            const uint2* __restrict__ defer,
                                                            const unsigned long long* n_defer,
                                                            uint32_t defer_cap) {
    pdl_wait();
    pdl_trigger();
    const unsigned long long nd = *n_defer;
    const uint32_t n = nd < (unsigned long long)defer_cap ? (uint32_t)nd : defer_cap;
    const uint32_t nwarps = gridDim.x * (kBinThreads / 32);
    for (uint32_t e = blockIdx.x * (kBinThreads / 32) + (threadIdx.x >> 5); e < n; e += nwarps) {
        const uint2 en = defer[e];                   // the same entry in every lane
        const uint2 r = rect[en.x];
        const uint32_t bw = (r.y & 0xFFFFu) - (r.x & 0xFFFFu);
        const uint32_t bn = bw * ((r.y >> 16) - (r.x >> 16));
        const uint32_t lo = en.y * kChunkTiles;
        const uint32_t hi = min(bn, lo + kChunkTiles);
        bin_rect_range<kOwnTiles>(tc, gx, r, lo, hi, en.x, dkey[en.x], cap, keys, ids);
    }
}

// Ranges of the binned lists: tile t owns [t cap, t cap + count_t).  One CTA per kScanChunk
// tiles: every CTA reads all the counts itself (their total and largest decide the pair count
// and the overflow state), then lists its chunk's tiles too long for the warp sorter in
// `longl` (count in nlong[chunk]).  CTA 0 writes P and the overflow state.
__global__ void __launch_bounds__(kScanChunk) bins_scan(const uint32_t* __restrict__ tcount,
                                                        int ntiles, uint32_t cap,
                                                        uint2* __restrict__ range,
                                                        uint32_t* __restrict__ longl,
                                                        uint32_t* __restrict__ nlong,
                                                        ogs_counts* counts) {
    pdl_wait();
    pdl_trigger();
    __shared__ unsigned long long s_sum[kScanChunk / 32];
    __shared__ uint32_t s_max[kScanChunk / 32];
    __shared__ uint32_t s_nlong;
    const int t = threadIdx.x, lane = (int)lane_id(), warp = t >> 5;
    const int c0 = blockIdx.x * kScanChunk;
    if (t == 0) s_nlong = 0;
    unsigned long long all = 0;
    uint32_t mx = 0;
    for (int b = t; b < ntiles; b += kScanChunk) {
        const uint32_t v = tcount[b];
        all += v;
        mx = max(mx, v);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        all += __shfl_xor_sync(0xffffffffu, all, o);
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    if (lane == 0) {
        s_sum[warp] = all;
        s_max[warp] = mx;
    }
    __syncthreads();
    unsigned long long P = 0;
    uint32_t M = 0;
#pragma unroll 8
    for (int w = 0; w < kScanChunk / 32; ++w) {
        P += s_sum[w];
        M = max(M, s_max[w]);
    }
    const bool over = M > cap;
    const int b = c0 + t;
    if (b < ntiles) {
        const uint32_t v = tcount[b];
        const uint32_t st = (uint32_t)b * cap;
        range[b] = over ? make_uint2(0, 0) : make_uint2(st, st + v);
        if (!over && v > (uint32_t)kWarpSort) longl[c0 + atomicAdd(&s_nlong, 1u)] = (uint32_t)b;
    }
    __syncthreads();
    if (t == 0) {
        nlong[blockIdx.x] = s_nlong;
        if (blockIdx.x == 0) {
            if (over) {
                atomicOr(&counts->overflow, 2u);
                counts->need_pairs = M;
                counts->n_pairs = 0;
            } else {
                counts->need_pairs = (uint32_t)(P > 0xFFFFFFFFull ? 0xFFFFFFFFull : P);
                counts->n_pairs = (uint32_t)(P > 0xFFFFFFFFull ? 0xFFFFFFFFull : P);
            }
        }
    }
}

__global__ void __launch_bounds__(kBinThreads) bin_fill(const uint32_t* __restrict__ tiles,
                                                        const uint2* __restrict__ rect,
                                                        const uint32_t* __restrict__ dkey,
                                                        const uint32_t* n_dev, int64_t n_cap,
                                                        int gx, const uint2* __restrict__ range,
                                                        uint32_t* __restrict__ cursor,
                                                        const ogs_counts* counts,
                                                        uint32_t* __restrict__ keys,
                                                        uint32_t* __restrict__ ids) {
    pdl_wait();
    pdl_trigger();
    if (counts->overflow & 2u) return;
    const uint32_t n = count_of(n_dev, n_cap);
    if ((int64_t)blockIdx.x * kBinTile >= n) return;
    for_each_pair(tiles, rect, n, gx, [&](bool valid, uint32_t g, uint32_t t) {
        const uint32_t slot = warp_agg_inc(cursor, valid, t, true);
        if (valid) {
            const uint32_t o = range[t].x + slot;
            keys[o] = dkey[g];
            ids[o] = g;
        }
    });
}

// Bitonic sorting network in its "flip" form over m = next power of two >= cnt slots: each
// merge stage first compares mirrored pairs of a block, then runs half-cleaners, and every
// comparator puts the smaller key at the lower index.  Slots >= cnt behave as +infinity, so a
// comparator that touches one is a no-op: arbitrary counts sort without padding.  (Generic
// form, used for lists kept in global memory.)
template <class Get, class Swap>
__device__ __forceinline__ void bitonic(uint32_t cnt, Get get, Swap swp) {
    uint32_t m = 1;
    while (m < cnt) m <<= 1;
    for (uint32_t lg = 1, size = 2; size <= m; ++lg, size <<= 1) {
        const uint32_t half = size >> 1;
        for (uint32_t i = threadIdx.x; i < m / 2; i += blockDim.x) {
            const uint32_t off = i & (half - 1);
            const uint32_t base = (i >> (lg - 1)) << lg;       // (i / half) * size
            const uint32_t lo = base + off, hi = base + size - 1 - off;
            if (hi < cnt && get(lo) > get(hi)) swp(lo, hi);
        }
        __syncthreads();
        for (uint32_t stride = half >> 1; stride > 0; stride >>= 1) {
            for (uint32_t i = threadIdx.x; i < m / 2; i += blockDim.x) {
                const uint32_t lo = 2 * i - (i & (stride - 1)), hi = lo + stride;
                if (hi < cnt && get(lo) > get(hi)) swp(lo, hi);
            }
            __syncthreads();
        }
    }
}

// One compare-exchange step of the same network inside a 64-slot window held by a warp in
// registers, lane l holding slots 2l (v[0]) and 2l + 1 (v[1]): every slot e meets slot e ^ mask
// and the lower of the two keeps the smaller key.  mask is 1 (within a lane), an odd block-flip
// mask size - 1, or an even half-cleaner stride.
__device__ __forceinline__ void window_step(unsigned long long (&v)[2], uint32_t mask,
                                            uint32_t lane) {
    if (mask == 1) {
        const unsigned long long a = v[0], b = v[1];
        v[0] = a < b ? a : b;
        v[1] = a < b ? b : a;
        return;
    }
    const uint32_t pl = lane ^ (mask >> 1);
    // an odd mask pairs my even slot with the partner's odd slot and vice versa
    const unsigned long long send0 = (mask & 1) ? v[1] : v[0];
    const unsigned long long send1 = (mask & 1) ? v[0] : v[1];
    const unsigned long long p0 = __shfl_sync(0xffffffffu, send0, pl);
    const unsigned long long p1 = __shfl_sync(0xffffffffu, send1, pl);
    const uint32_t e0 = 2 * lane, e1 = 2 * lane + 1;
    const bool low0 = e0 < (e0 ^ mask), low1 = e1 < (e1 ^ mask);
    v[0] = (low0 == (v[0] < p0)) ? v[0] : p0;
    v[1] = (low1 == (v[1] < p1)) ? v[1] : p1;
}

// Loads window `win` of s (slots >= cnt read as +infinity), runs the steps of `masks`, stores
// the slots < cnt back.  Called by whole warps.
template <int kN>
__device__ __forceinline__ void window_pass(unsigned long long* s, uint32_t cnt, uint32_t win,
                                            const uint32_t (&masks)[kN]) {
    const uint32_t lane = lane_id();
    const uint32_t e = win * 64 + 2 * lane;
    unsigned long long v[2];
    v[0] = e < cnt ? s[e] : ~0ull;
    v[1] = e + 1 < cnt ? s[e + 1] : ~0ull;
#pragma unroll
    for (int q = 0; q < kN; ++q) window_step(v, masks[q], lane);
    if (e < cnt) s[e] = v[0];
    if (e + 1 < cnt) s[e + 1] = v[1];
}

// Sorts the cnt unique 64-bit keys of s (no real key is ~0; cnt <= capacity of s) with the flip
// bitonic network: every step whose span fits a 64-slot window runs in registers with warp
// shuffles (the first six merge sizes entirely, and the last six steps of every larger merge);
// only the wider steps go through shared memory, between barriers of the CTA.  Slots >= cnt are
// never written.  Starts and ends with a barrier.
__device__ __forceinline__ void sort_u64_smem(unsigned long long* s, uint32_t cnt) {
    uint32_t m = 64;
    while (m < cnt) m <<= 1;
    const uint32_t nwin = m / 64, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    __syncthreads();
    {   // merge sizes 2 .. 64 inside each window
        const uint32_t masks[21] = {1, 3, 1, 7, 2, 1, 15, 4, 2, 1, 31, 8, 4, 2, 1,
                                    63, 16, 8, 4, 2, 1};
        for (uint32_t w = warp; w < nwin; w += nwarps) window_pass(s, cnt, w, masks);
    }
    const uint32_t tail[6] = {32, 16, 8, 4, 2, 1};
    for (uint32_t lg = 7, size = 128; size <= m; ++lg, size <<= 1) {
        __syncthreads();
        const uint32_t half = size >> 1;
        for (uint32_t i = threadIdx.x; i < m / 2; i += blockDim.x) {      // flip
            const uint32_t off = i & (half - 1);
            const uint32_t base = (i >> (lg - 1)) << lg;
            const uint32_t lo = base + off, hi = base + size - 1 - off;
            if (hi < cnt) {
                const unsigned long long a = s[lo], b = s[hi];
                if (a > b) { s[lo] = b; s[hi] = a; }
            }
        }
        for (uint32_t stride = half >> 1; stride >= 64; stride >>= 1) {   // wide half-cleaners
            __syncthreads();
            for (uint32_t i = threadIdx.x; i < m / 2; i += blockDim.x) {
                const uint32_t lo = 2 * i - (i & (stride - 1)), hi = lo + stride;
                if (hi < cnt) {
                    const unsigned long long a = s[lo], b = s[hi];
                    if (a > b) { s[lo] = b; s[hi] = a; }
                }
            }
        }
        __syncthreads();
        for (uint32_t w = warp; w < nwin; w += nwarps) window_pass(s, cnt, w, tail);
    }
    __syncthreads();
}

// sorts one tile's list (cnt <= capacity of s_k) by the unique key (depth << 32 | id)
__device__ __forceinline__ void sort_in_smem(unsigned long long* s_k, uint2 r,
                                             uint32_t* __restrict__ keys,
                                             uint32_t* __restrict__ ids) {
    const uint32_t cnt = r.y - r.x;
    for (uint32_t i = threadIdx.x; i < cnt; i += blockDim.x)
        s_k[i] = ((unsigned long long)keys[r.x + i] << 32) | ids[r.x + i];
    sort_u64_smem(s_k, cnt);
    for (uint32_t i = threadIdx.x; i < cnt; i += blockDim.x) ids[r.x + i] = (uint32_t)s_k[i];
}

// The largest power of two <= x (x >= 1), at compile time.
__host__ __device__ constexpr int top_bit(int x) { return x < 2 ? 1 : 2 * top_bit(x / 2); }

// The lower of two slots keeps the smaller key: 32-bit keys by min / max, 64-bit ones by a
// compare and selects.
__device__ __forceinline__ void cx_pair(uint32_t& a, uint32_t& b) {
    const uint32_t lo = min(a, b), hi = max(a, b);
    a = lo;
    b = hi;
}
__device__ __forceinline__ void cx_pair(unsigned long long& a, unsigned long long& b) {
    const bool lt = a < b;
    const unsigned long long lo = lt ? a : b, hi = lt ? b : a;
    a = lo;
    b = hi;
}
__device__ __forceinline__ uint32_t cx_keep(uint32_t a, uint32_t p, bool lower) {
    return lower ? min(a, p) : max(a, p);
}
__device__ __forceinline__ unsigned long long cx_keep(unsigned long long a, unsigned long long p,
                                                      bool lower) {
    return ((a < p) == lower) ? a : p;
}

// One step of the flip bitonic network over the 32 kPer slots of a warp, slot e = lane * kPer + j
// held in v[j] of that lane: slot e meets slot e ^ M and the lower of the two keeps the smaller
// key (M = size - 1 for a block flip, a power of two for a half-cleaner).  M < kPer pairs two
// registers of one lane; otherwise the partner lane is lane ^ (M / kPer) and the value
// exchanged is its slot j ^ (M mod kPer), by shuffle.
template <class T, int kPer, int M>
__device__ __forceinline__ void warp_cx(T (&v)[kPer], uint32_t lane) {
    if constexpr (M < kPer) {
#pragma unroll
        for (int j = 0; j < kPer; ++j)
            if (!(j & top_bit(M))) cx_pair(v[j], v[j ^ M]);
    } else {
        constexpr int jm = M % kPer, lm = M / kPer;
        const bool lower = !(lane & (uint32_t)top_bit(lm));
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            if (j <= (j ^ jm)) {            // slots j and j ^ jm together (read before written)
                const T a = v[j], b = v[j ^ jm];
                v[j] = cx_keep(a, __shfl_xor_sync(0xffffffffu, b, lm), lower);
                if (jm) v[j ^ jm] = cx_keep(b, __shfl_xor_sync(0xffffffffu, a, lm), lower);
            }
        }
    }
}

// merge of size S (a flip, then half-cleaners S/4 .. 1), then the merges above it up to 32 kPer
template <class T, int kPer, int S>
__device__ __forceinline__ void warp_merges(T (&v)[kPer], uint32_t lane) {
    if constexpr (S <= 32 * kPer) {
        warp_cx<T, kPer, S - 1>(v, lane);
        if constexpr (S >= 4) warp_cx<T, kPer, S / 4>(v, lane);
        if constexpr (S >= 8) warp_cx<T, kPer, S / 8>(v, lane);
        if constexpr (S >= 16) warp_cx<T, kPer, S / 16>(v, lane);
        if constexpr (S >= 32) warp_cx<T, kPer, S / 32>(v, lane);
        if constexpr (S >= 64) warp_cx<T, kPer, S / 64>(v, lane);
        if constexpr (S >= 128) warp_cx<T, kPer, S / 128>(v, lane);
        if constexpr (S >= 256) warp_cx<T, kPer, S / 256>(v, lane);
        if constexpr (S >= 512) warp_cx<T, kPer, S / 512>(v, lane);
        warp_merges<T, kPer, 2 * S>(v, lane);
    }
}

constexpr int kPosBits = 9;                // list positions < kWarpSort
constexpr int kFixRounds = 8;              // odd-even rounds before the exact re-sort
static_assert((1 << kPosBits) == kWarpSort, "position field");

// Exact form for a list of 2 <= cnt <= kWarpSort entries: the 512-slot network on the 64-bit
// keys (depth << 32 | id), read from and written back to the list in place (every read lands
// in registers before the first write).  Called by a whole warp; kept out of line, since it is
// the rare path and its code would otherwise crowd the instruction cache.
__device__ __noinline__ void warp_sort_exact(const uint32_t* __restrict__ keys,
                                             uint32_t* __restrict__ ids, uint32_t cnt,
                                             uint32_t lane) {
    constexpr int kPer = kWarpSort / 32;
    unsigned long long w[kPer];
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
        const uint32_t e = lane * kPer + j;
        w[j] = e < cnt ? ((unsigned long long)keys[e] << 32) | ids[e] : ~0ull;
    }
    warp_merges<unsigned long long, kPer, 2>(w, lane);
    __syncwarp();
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
        const uint32_t e = lane * kPer + j;
        if (e < cnt) ids[e] = (uint32_t)w[j];
    }
}

// Exact order of two list positions p, q (the low kPosBits of their 32-bit keys): by depth,
// then id, read from the warp's buffers.
template <int kPer>
__device__ __forceinline__ bool exact_less(uint32_t p, uint32_t q, const uint32_t* sd,
                                           const uint32_t* si) {
    p &= (1u << kPosBits) - 1;
    q &= (1u << kPosBits) - 1;
    const uint32_t dp = sd[p + p / kPer], dq = sd[q + q / kPer];
    return dp != dq ? dp < dq : si[p + p / kPer] < si[q + q / kPer];
}

// One round (even pairs, then odd pairs) of odd-even transposition over the first cnt of the
// 32 kPer slots of a warp (slot e = lane * kPer + j in v[j]): neighbours that share a quantised
// depth and are out of exact order swap (neighbours with different quantised depths are in
// order already).  Returns whether anything moved in this lane.
template <int kPer>
__device__ __forceinline__ bool oe_round(uint32_t (&v)[kPer], uint32_t lane, uint32_t cnt,
                                         const uint32_t* sd, const uint32_t* si) {
    bool moved = false;
#pragma unroll
    for (int phase = 0; phase < 2; ++phase) {
        if constexpr (kPer >= 2) {
#pragma unroll
            for (int j = phase; j + 1 < kPer; j += 2) {
                const uint32_t a = v[j], b = v[j + 1];
                if (lane * kPer + j + 1 < cnt && (a >> kPosBits) == (b >> kPosBits) &&
                    exact_less<kPer>(b, a, sd, si)) {
                    v[j] = b;
                    v[j + 1] = a;
                    moved = true;
                }
            }
        }
        if (kPer == 1 || phase == 1) {
            // pairs across lanes: my last slot (lower) with the next lane's first (upper)
            const uint32_t up = __shfl_down_sync(0xffffffffu, v[0], 1);
            const uint32_t dn = __shfl_up_sync(0xffffffffu, v[kPer - 1], 1);
            const bool as_lower = (kPer > 1 || (lane & 1u) == (uint32_t)phase) && lane < 31 &&
                                  (lane + 1) * kPer < cnt;
            const bool as_upper = (kPer > 1 || (lane & 1u) != (uint32_t)phase) && lane > 0 &&
                                  lane * kPer < cnt;
            const uint32_t last = v[kPer - 1], first = v[0];
            if (as_lower && (last >> kPosBits) == (up >> kPosBits) &&
                exact_less<kPer>(up, last, sd, si)) {
                v[kPer - 1] = up;
                moved = true;
            }
            if (as_upper && (dn >> kPosBits) == (first >> kPosBits) &&
                exact_less<kPer>(first, dn, sd, si)) {
                v[0] = dn;
                moved = true;
            }
        }
    }
    return moved;
}

// A warp sorts one tile's list of 2 <= cnt <= 32 kPer entries by the unique key (depth, id).
// The depths and ids go to the warp's shared buffers sd / si (slot e at e + e / kPer, which
// makes the lane-major reads conflict-free).  The network then runs in registers on 32-bit
// keys (quantised depth << kPosBits | list position), the depth quantised as (depth bits -
// the list's smallest) >> shift with the shift that fits the list's depth span in the other
// 23 bits: a monotone map, so the result is in (depth, id) order except inside runs that share
// a quantised depth (an exact tie, or depths closer than the quantum).  When there are such
// runs, the sorted slots go through rounds of odd-even transposition on the exact keys (depth,
// id) until a round moves nothing (every neighbour then in order: the list is sorted; runs are
// short, so one or two rounds usually do); after kFixRounds rounds the list is sorted again
// from scratch on the exact keys (warp_sort_exact).  Padding slots hold ~0,
// at or above every real key.
template <int kPer>
__device__ __forceinline__ void warp_sort_list(uint32_t* sd, uint32_t* si, uint2 r, uint32_t lane,
                                               const uint32_t* __restrict__ keys,
                                               uint32_t* __restrict__ ids) {
    const uint32_t cnt = r.y - r.x;
    uint32_t dmin = 0xFFFFFFFFu, dmax = 0;
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
        const uint32_t e = q * 32 + lane;
        if (e < cnt) {
            const uint32_t d = keys[r.x + e];
            sd[e + e / kPer] = d;
            si[e + e / kPer] = ids[r.x + e];
            dmin = min(dmin, d);
            dmax = max(dmax, d);
        }
    }
    dmin = __reduce_min_sync(0xffffffffu, dmin);
    dmax = __reduce_max_sync(0xffffffffu, dmax);
    const uint32_t wide = (dmax - dmin) >> (32 - kPosBits);
    const uint32_t shift = wide ? 32 - __clz(wide) : 0;
    __syncwarp();
    uint32_t v[kPer];
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
        const uint32_t e = lane * kPer + j;
        v[j] = e < cnt ? (((sd[lane * (kPer + 1) + j] - dmin) >> shift) << kPosBits) | e
                       : 0xFFFFFFFFu;
    }
    warp_merges<uint32_t, kPer, 2>(v, lane);
    // neighbours with one quantised depth?
    bool tie = false;
#pragma unroll
    for (int j = 0; j + 1 < kPer; ++j)
        tie |= lane * kPer + j + 1 < cnt && (v[j] >> kPosBits) == (v[j + 1] >> kPosBits);
    const uint32_t next = __shfl_down_sync(0xffffffffu, v[0], 1);
    tie |= lane < 31 && (lane + 1) * kPer < cnt && (v[kPer - 1] >> kPosBits) == (next >> kPosBits);
    if (__any_sync(0xffffffffu, tie)) {
        int round = 0;
        bool settled = true;
        while (__any_sync(0xffffffffu, oe_round<kPer>(v, lane, cnt, sd, si))) {
            if (++round == kFixRounds) {
                settled = false;
                break;
            }
        }
        if (!settled) {                     // uniform over the warp
            warp_sort_exact(keys + r.x, ids + r.x, cnt, lane);
            return;
        }
    }
    // slots < cnt hold real keys, whose positions are < cnt: their ids, lane-major, to sd
    __syncwarp();
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
        const uint32_t e = v[j] & ((1u << kPosBits) - 1);
        sd[lane * (kPer + 1) + j] = lane * kPer + j < cnt ? si[e + e / kPer] : 0u;
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
        const uint32_t e = q * 32 + lane;
        if (e < cnt) ids[r.x + e] = sd[e + e / kPer];
    }
}

// each warp sorts the lists of 2 .. kWarpSort entries of tiles warp, warp + W, warp + 2W, ..
// (W = every warp of the grid), the network sized to the list: 32, 64, .., 512 slots
__global__ void __launch_bounds__(32 * kWarpTiles, 8) tile_sort_warp(const uint2* __restrict__ range,
                                                                     int n_tiles,
                                                                     const ogs_counts* counts,
                                                                     const uint32_t* __restrict__ keys,
                                                                     uint32_t* __restrict__ ids) {
    pdl_wait();
    pdl_trigger();
    constexpr int kBuf = kWarpSort + kWarpSort / 16;
    __shared__ uint32_t s_d[kWarpTiles][kBuf], s_i[kWarpTiles][kBuf];
    if (counts->overflow & 2u) return;
    const uint32_t warp = threadIdx.x >> 5, lane = lane_id();
    uint32_t *sd = s_d[warp], *si = s_i[warp];
    for (int tile = blockIdx.x * kWarpTiles + (int)warp; tile < n_tiles;
         tile += gridDim.x * kWarpTiles) {
        const uint2 r = range[tile];
        const uint32_t cnt = r.y - r.x;
        if (cnt <= 1 || cnt > (uint32_t)kWarpSort) continue;
        if (cnt <= 32) warp_sort_list<1>(sd, si, r, lane, keys, ids);
        else if (cnt <= 64) warp_sort_list<2>(sd, si, r, lane, keys, ids);
        else if (cnt <= 128) warp_sort_list<4>(sd, si, r, lane, keys, ids);
        else if (cnt <= 256) warp_sort_list<8>(sd, si, r, lane, keys, ids);
        else warp_sort_list<16>(sd, si, r, lane, keys, ids);
        __syncwarp();
    }
}

// gridDim.x CTAs loop over the tiles listed per scan chunk (chunk c: list[c * kScanChunk ..
// + nlist[c]]), in chunk order, each list sorted in shared memory (cap keys) or, beyond that,
// on global memory
template <int kT>
__global__ void __launch_bounds__(kT) tile_sort_listed(const uint2* __restrict__ range,
                                                       const uint32_t* __restrict__ list,
                                                       const uint32_t* __restrict__ nlist,
                                                       int nchunks, uint32_t cap,
                                                       const ogs_counts* counts,
                                                       uint32_t* __restrict__ keys,
                                                       uint32_t* __restrict__ ids) {
    pdl_wait();
    pdl_trigger();
    extern __shared__ unsigned long long s_k[];
    if (counts->overflow & 2u) return;
    uint32_t n = 0;
    for (int c = 0; c < nchunks; ++c) n += nlist[c];
    for (uint32_t q = blockIdx.x; q < n; q += gridDim.x) {
        uint32_t c = 0, i = q;
        while (i >= nlist[c]) i -= nlist[c++];
        const uint2 r = range[list[c * kScanChunk + i]];
        const uint32_t cnt = r.y - r.x;
        if (cnt <= cap) {
            sort_in_smem(s_k, r, keys, ids);
        } else {
            // longer than shared memory holds: the same network on global memory
            uint32_t* K = keys + r.x;
            uint32_t* I = ids + r.x;
            bitonic(cnt, [&](uint32_t i) { return ((unsigned long long)K[i] << 32) | I[i]; },
                    [&](uint32_t i, uint32_t j) {
                        const uint32_t tk = K[i], ti = I[i];
                        K[i] = K[j]; I[i] = I[j]; K[j] = tk; I[j] = ti;
                    });
        }
        __syncthreads();
    }
}

struct SortScratch {
    uint32_t* tcount;   // per-tile pair counts
    uint32_t* cursor;   // per-tile fill cursors
    uint32_t* mid;      // tiles whose lists exceed kWarpSort but not kSmallSort, per scan chunk
    uint32_t* nmid;     // their number per chunk
    uint32_t* big;      // tiles whose lists exceed kSmallSort, per scan chunk
    uint32_t* nbig;     // their number per chunk
    uint32_t* keys;     // depth key of every pair
};

size_t sort_layout(int64_t pair_cap, int n_tiles, void* base, SortScratch* s) {
    Carver cv(base);
    SortScratch t;
    t.tcount = cv.take<uint32_t>(n_tiles > 0 ? n_tiles : 1);
    t.cursor = cv.take<uint32_t>(n_tiles > 0 ? n_tiles : 1);
    const int nchunks = n_tiles > 0 ? (n_tiles + kScanChunk - 1) / kScanChunk : 1;
    t.mid = cv.take<uint32_t>((size_t)nchunks * kScanChunk);
    t.nmid = cv.take<uint32_t>(nchunks);
    t.big = cv.take<uint32_t>((size_t)nchunks * kScanChunk);
    t.nbig = cv.take<uint32_t>(nchunks);
    t.keys = cv.take<uint32_t>(pair_cap > 0 ? pair_cap : 1);
    if (s) *s = t;
    return cv.off + 256;
}

}  // namespace
}  // namespace ogs

using namespace ogs;

extern "C" size_t ogs_radix_sort_scratch_bytes(int64_t n_cap) {
    return rs_layout(n_cap < 0 ? 0 : n_cap, nullptr, nullptr);
}

extern "C" ogs_status ogs_radix_sort_pairs(uint32_t* keys, uint32_t* vals, const uint32_t* n_dev,
                                           int64_t n_cap, int32_t bit_lo, int32_t bit_hi,
                                           void* scratch, size_t scratch_bytes, void* stream) {
    if (!keys || !vals || !scratch || n_cap < 0 || n_cap > 0xFFFFFFFFll) return OGS_ERR_ARG;
    if (bit_lo < 0 || bit_hi > 32 || bit_lo >= bit_hi) return OGS_ERR_ARG;
    if (scratch_bytes < ogs_radix_sort_scratch_bytes(n_cap) || !aligned(scratch, 16))
        return OGS_ERR_ARG;
    if (n_cap == 0) return OGS_OK;
    RsScratch s;
    rs_layout(n_cap, scratch, &s);
    return radix_sort(keys, vals, n_dev, n_cap, bit_lo, bit_hi, s, (cudaStream_t)stream)
               ? OGS_OK : OGS_ERR_CUDA;
}

extern "C" size_t ogs_sort_scratch_bytes(int64_t g_cap, int64_t pair_cap, int32_t n_tiles) {
    (void)g_cap;
    return sort_layout(pair_cap < 0 ? 0 : pair_cap, n_tiles, nullptr, nullptr);
}

// scratch of ogs_sort_bins: the tile counts behind the deferred-chunk counter (one memset
// clears both), the deferred (Gaussian, chunk) entries and the per-chunk lists of long tiles
struct BinsScratch {
    unsigned long long* ndefer;
    uint32_t *tcount, *longl, *nlong;
    uint2* defer;
    uint32_t defer_cap;
};

inline uint32_t defer_cap_of(int n_tiles) {
    const uint32_t c = 32u * (uint32_t)(n_tiles > 0 ? n_tiles : 0);
    return c > 4096u ? c : 4096u;
}

size_t bins_layout(int n_tiles, void* base, BinsScratch* s) {
    Carver cv(base);
    BinsScratch t;
    const int nchunks = n_tiles > 0 ? (n_tiles + kScanChunk - 1) / kScanChunk : 1;
    uint32_t* head = cv.take<uint32_t>(2 + (size_t)(n_tiles > 0 ? n_tiles : 1));
    t.ndefer = reinterpret_cast<unsigned long long*>(head);     // 256-byte aligned
    t.tcount = head ? head + 2 : nullptr;
    t.longl = cv.take<uint32_t>((size_t)nchunks * kScanChunk);
    t.nlong = cv.take<uint32_t>(nchunks);
    t.defer_cap = defer_cap_of(n_tiles);
    t.defer = cv.take<uint2>(t.defer_cap);
    if (s) *s = t;
    return cv.off + 256;
}

extern "C" size_t ogs_sort_bins_scratch_bytes(int32_t n_tiles) {
    return bins_layout(n_tiles < 0 ? 0 : n_tiles, nullptr, nullptr);
}

extern "C" ogs_status ogs_sort_bins(const uint32_t* depth_key, const uint32_t* rect,
                                    const uint32_t* tiles, int64_t g_cap, int64_t n_gauss,
                                    int32_t grid_x, int32_t grid_y, const ogs_tile_bins* bins,
                                    uint32_t* tile_range, ogs_counts* counts, void* scratch,
                                    size_t scratch_bytes, void* stream) {
    if (!depth_key || !rect || !tiles || !bins || !bins->pair_key || !bins->pair_gauss ||
        !tile_range || !counts || !scratch || bins->tile_cap == 0)
        return OGS_ERR_ARG;
    if (g_cap < 0 || g_cap > 0xFFFFFFFFll || !aligned(rect, 8)) return OGS_ERR_ARG;
    if (grid_x <= 0 || grid_y <= 0 || (int64_t)grid_x * grid_y > 65536 || grid_x > 65535)
        return OGS_ERR_ARG;
    const int n_tiles = grid_x * grid_y;
    if ((uint64_t)n_tiles * bins->tile_cap > 0xFFFFFFFFull) return OGS_ERR_ARG;
    if (scratch_bytes < ogs_sort_bins_scratch_bytes(n_tiles) || !aligned(scratch, 16) ||
        !aligned(tile_range, 8))
        return OGS_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    BinsScratch s;
    bins_layout(n_tiles, scratch, &s);
    uint2* range = reinterpret_cast<uint2*>(tile_range);
    if (cudaMemsetAsync(s.ndefer, 0, sizeof(uint32_t) * (2 + (size_t)n_tiles), st) !=
        cudaSuccess)
        return OGS_ERR_CUDA;
    // the Gaussian count is the device count written by the decoder, or the caller's n_gauss
    const uint32_t* n_dev = n_gauss < 0 ? &counts->n_gaussians : nullptr;
    const int64_t n_cap = n_gauss < 0 ? g_cap : (n_gauss < g_cap ? n_gauss : g_cap);
    const int nb = n_cap > 0 ? (int)((n_cap + kBinThreads - 1) / kBinThreads) : 1;
    launch_pdl(bin_regions, dim3(nb), dim3(kBinThreads), 0, st, depth_key,
               reinterpret_cast<const uint2*>(rect), tiles, n_dev, n_cap, grid_x, s.tcount,
               bins->tile_cap, bins->pair_key, bins->pair_gauss, s.defer, s.ndefer,
               s.defer_cap);
    launch_pdl(bin_deferred, dim3(kDeferGrid), dim3(kBinThreads), 0, st, depth_key,
               reinterpret_cast<const uint2*>(rect), grid_x, s.tcount, bins->tile_cap,
               bins->pair_key, bins->pair_gauss, (const uint2*)s.defer,
               (const unsigned long long*)s.ndefer, s.defer_cap);
    const int nchunks = (n_tiles + kScanChunk - 1) / kScanChunk;
    launch_pdl(bins_scan, dim3(nchunks), dim3(kScanChunk), 0, st, (const uint32_t*)s.tcount,
               n_tiles, bins->tile_cap, range, s.longl, s.nlong, counts);
    const int wgrid = std::min((n_tiles + kWarpTiles - 1) / kWarpTiles, kWarpGrid);
    launch_pdl(tile_sort_warp, dim3(wgrid), dim3(32 * kWarpTiles), 0, st, range, n_tiles, counts,
               (const uint32_t*)bins->pair_key, bins->pair_gauss);
    // every longer list in one launch: up to kBinsListSort keys in shared memory, the rare
    // longer list by the same network on global memory
    const size_t smem = sizeof(unsigned long long) * kBinsListSort;
    if (cudaFuncSetAttribute(tile_sort_listed<kLargeThreads>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(unsigned long long) * kLargeSort)) != cudaSuccess)
        return OGS_ERR_CUDA;
    launch_pdl(tile_sort_listed<kLargeThreads>, dim3(kBinsListGrid), dim3(kLargeThreads), smem,
               st, range, s.longl, s.nlong, nchunks, (uint32_t)kBinsListSort, counts,
               bins->pair_key, bins->pair_gauss);
    return launch_status();
}

extern "C" ogs_status ogs_sort(const uint32_t* depth_key, const uint32_t* rect, const uint32_t* tiles,
                               const uint32_t* tile_count, int64_t g_cap, int64_t n_gauss,
                               int32_t grid_x, int32_t grid_y,
                               uint32_t* pair_gauss, uint32_t* tile_range, int64_t pair_cap,
                               ogs_counts* counts, void* scratch, size_t scratch_bytes,
                               void* stream) {
    if (!depth_key || !rect || !tiles || !pair_gauss || !tile_range || !counts || !scratch)
        return OGS_ERR_ARG;
    if (g_cap < 0 || g_cap > 0xFFFFFFFFll || pair_cap < 0 || pair_cap > 0xFFFFFFFFll)
        return OGS_ERR_ARG;
    if (grid_x <= 0 || grid_y <= 0 || (int64_t)grid_x * grid_y > 65536 || grid_x > 65535)
        return OGS_ERR_ARG;
    if (scratch_bytes < ogs_sort_scratch_bytes(g_cap, pair_cap, grid_x * grid_y) ||
        !aligned(scratch, 16) || !aligned(rect, 8) || !aligned(tile_range, 8))
        return OGS_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int n_tiles = grid_x * grid_y;
    SortScratch s;
    sort_layout(pair_cap, n_tiles, scratch, &s);
    uint2* range = reinterpret_cast<uint2*>(tile_range);
    if (!tile_count && cudaMemsetAsync(s.tcount, 0, sizeof(uint32_t) * n_tiles, st) != cudaSuccess)
        return OGS_ERR_CUDA;
    // the Gaussian count is the device count written by the decoder, or the caller's n_gauss
    const uint32_t* n_dev = n_gauss < 0 ? &counts->n_gaussians : nullptr;
    const int64_t n_cap = n_gauss < 0 ? g_cap : (n_gauss < g_cap ? n_gauss : g_cap);
    int nb = (int)((n_cap + kBinTile - 1) / kBinTile);
    if (nb < 1) nb = 1;
    const uint2* rc = reinterpret_cast<const uint2*>(rect);
    if (!tile_count) bin_count<<<nb, kBinThreads, 0, st>>>(tiles, rc, n_dev, n_cap, grid_x, s.tcount);
    const int nchunks = (n_tiles + kScanChunk - 1) / kScanChunk;
    launch_pdl(tile_scan, dim3(nchunks), dim3(kScanChunk), 0, st,
               tile_count ? tile_count : s.tcount, n_tiles, pair_cap, range, s.cursor, s.mid,
               s.nmid, s.big, s.nbig, counts);
    launch_pdl(bin_fill, dim3(nb), dim3(kBinThreads), 0, st, tiles, rc, depth_key, n_dev, n_cap,
               grid_x, range, s.cursor, counts, s.keys, pair_gauss);
    const int wgrid = std::min((n_tiles + kWarpTiles - 1) / kWarpTiles, kWarpGrid);
    launch_pdl(tile_sort_warp, dim3(wgrid), dim3(32 * kWarpTiles), 0, st, range, n_tiles, counts,
               (const uint32_t*)s.keys, pair_gauss);
    launch_pdl(tile_sort_listed<kLargeThreads>, dim3(kSmallGrid), dim3(kLargeThreads),
               sizeof(unsigned long long) * kSmallSort, st, range, s.mid, s.nmid, nchunks,
               (uint32_t)kSmallSort, counts, s.keys, pair_gauss);
    const size_t smem = sizeof(unsigned long long) * kLargeSort;
    if (cudaFuncSetAttribute(tile_sort_listed<kLargeThreads>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return OGS_ERR_CUDA;
    launch_pdl(tile_sort_listed<kLargeThreads>, dim3(kLargeGrid), dim3(kLargeThreads), smem, st,
               range, s.big, s.nbig, nchunks, (uint32_t)kLargeSort, counts, s.keys, pair_gauss);
    return launch_status();
}

// ---------------------------------------------------------------------------------------
// Allocation-free variant of ogs_radix_sort_pairs.
//
// Some callers cannot hand this library a scratch buffer: a renderer embedded as a plugin in
// a host application that owns the whole device heap and offers no allocator, or a real-time
// frame loop that must never call cudaMalloc/cudaFree because they synchronise the device
// and stall the frame.  For them the sort's scratch lives in a fixed device array that is
// part of the library image: it is reserved on every GPU that loads the library and stays
// reserved until the process exits.
// ---------------------------------------------------------------------------------------

namespace ogs {
namespace {

constexpr int64_t kNoAllocMaxItems = (int64_t)1 << 20;   // largest n_cap accepted
constexpr int64_t kNoAllocBlocks = (kNoAllocMaxItems + kRsTile - 1) / kRsTile;
// alt keys + alt values + per-block digit histograms + digit totals, each 256-byte aligned
constexpr size_t kNoAllocBytes =
    2 * (size_t)kNoAllocMaxItems * sizeof(uint32_t) + 256 +
    (size_t)kNoAllocBlocks * kRsBins * sizeof(uint32_t) + 256 + kRsBins * sizeof(uint32_t) + 512;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of g_noalloc_scratch per device (host code only ever sees the symbol's
// host-side stand-in, never usable as a pointer).  Filled once per device.
constexpr int kMaxDevices = 64;
void* g_noalloc_ptr[kMaxDevices] = {};
std::mutex g_noalloc_mu;

ogs_status noalloc_scratch(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return OGS_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return OGS_ERR_CUDA;
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return OGS_OK;
}

}  // namespace
}  // namespace ogs

extern "C" int64_t ogs_radix_sort_pairs_noalloc_max_items(void) { return kNoAllocMaxItems; }

extern "C" ogs_status ogs_radix_sort_pairs_noalloc(uint32_t* keys, uint32_t* vals,
                                                   const uint32_t* n_dev, int64_t n_cap,
                                                   int32_t bit_lo, int32_t bit_hi, void* stream) {
    if (!keys || !vals || n_cap < 0) return OGS_ERR_ARG;
    if (bit_lo < 0 || bit_hi > 32 || bit_lo >= bit_hi) return OGS_ERR_ARG;
    if (n_cap > kNoAllocMaxItems) return OGS_ERR_CAPACITY;
    if (n_cap == 0) return OGS_OK;
    // rs_layout's size includes 256 bytes of slack for an unaligned base; the array is
    // 256-byte aligned, so the carve needs the rest.  This ties the fixed array to the carve:
    // a layout that grows beyond it is refused instead of writing past the array.
    if (rs_layout(n_cap, nullptr, nullptr) - 256 > kNoAllocBytes) return OGS_ERR_CAPACITY;
    void* base = nullptr;
    ogs_status st = noalloc_scratch(&base);
    if (st != OGS_OK) return st;
    // every scratch word is written before it is read in each pass: nothing to clear
    RsScratch s;
    rs_layout(n_cap, base, &s);
    return radix_sort(keys, vals, n_dev, n_cap, bit_lo, bit_hi, s, (cudaStream_t)stream)
               ? OGS_OK : OGS_ERR_CUDA;
}
