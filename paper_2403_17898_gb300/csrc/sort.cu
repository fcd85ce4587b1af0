// Front-to-back per-tile lists (Sec. 3.1): a tile's list holds every Gaussian whose tile
// rectangle covers it, in ascending depth, ties by Gaussian id.
//
// Instead of duplicating every Gaussian into 64-bit (tile, depth) keys and radix-sorting all
// ~45 key bits over all pairs, the work is factored:
//   1. stable radix sort of the G Gaussians by their 32-bit depth key (4 passes over G items);
//   2. exclusive scan of tile counts in depth order, fused with a block-cooperative emission of
//      (tile, Gaussian) pairs in depth order (load-balanced over pairs, not Gaussians);
//   3. stable radix sort of the P pairs by tile id only (ceil(log2 tiles) bits, 2 passes);
//   4. tile ranges from the boundaries of equal tile ids.
// Because step 3 is stable and step 2 emits in (depth, id) order, every tile list comes out in
// (depth, id) order, the same result as one stable sort of (tile << 32 | depth) keys, for
// about a third of the memory traffic when P is a few times G.
//
// The radix sort is a classic three-kernel LSD pass (per-block digit histograms -> per-digit
// scan over blocks -> stable block-local multisplit and coalesced scatter) with 8-bit digits;
// every item count is read on the device, so no host synchronisation is needed.
#include <mutex>

#include "internal.cuh"

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
// depth order -> pair emission
// ---------------------------------------------------------------------------------------

constexpr int kEmThreads = 256;
constexpr int kEmItems = 4;
constexpr int kEmTile = kEmThreads * kEmItems;

__global__ void iota_keys(const uint32_t* __restrict__ dkey, uint32_t* __restrict__ k,
                          uint32_t* __restrict__ v, const uint32_t* n_dev, int64_t n_cap) {
    const uint32_t n = count_of(n_dev, n_cap);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        k[i] = dkey[i];
        v[i] = (uint32_t)i;
    }
}

// per-block sums of tile counts, taken in depth order
__global__ void __launch_bounds__(kEmThreads) emit_count(const uint32_t* __restrict__ order,
                                                         const uint32_t* __restrict__ tiles,
                                                         const uint32_t* n_dev, int64_t n_cap,
                                                         uint32_t* block_sum) {
    __shared__ uint32_t ws[kEmThreads / 32];
    const uint32_t n = count_of(n_dev, n_cap);
    const int64_t base = (int64_t)blockIdx.x * kEmTile;
    uint64_t s = 0;
    for (int it = 0; it < kEmItems; ++it) {
        int64_t i = base + it * kEmThreads + threadIdx.x;
        if (i < n) s += tiles[order[i]];
    }
    // pair counts stay below 2^32 (pair capacity is 32-bit); saturate defensively
    uint32_t v = s > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)s;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane_id() == 0) ws[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint64_t t = 0;
        for (int q = 0; q < kEmThreads / 32; ++q) t += ws[q];
        block_sum[blockIdx.x] = t > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)t;
    }
}

// exclusive scan of block sums (one block); publishes P or the overflow state
__global__ void __launch_bounds__(1024) emit_scan(uint32_t* block_sum, int nb, int64_t pair_cap,
                                                  ogs_counts* counts) {
    __shared__ uint32_t ws[32];
    __shared__ unsigned long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int b0 = 0; b0 < nb; b0 += 1024) {
        int b = b0 + threadIdx.x;
        uint32_t v = b < nb ? block_sum[b] : 0;
        uint32_t x = v;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane_id() >= (unsigned)o) x += y;
        }
        if (lane_id() == 31) ws[threadIdx.x >> 5] = x;
        __syncthreads();
        uint32_t wpre = 0, tot = 0;
        for (int q = 0; q < 32; ++q) {
            uint32_t s = ws[q];
            wpre += (q < (int)(threadIdx.x >> 5)) ? s : 0;
            tot += s;
        }
        unsigned long long excl = carry + wpre + x - v;
        if (b < nb) block_sum[b] = (uint32_t)(excl > 0xFFFFFFFFull ? 0xFFFFFFFFull : excl);
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        unsigned long long P = carry;
        counts->need_pairs = (uint32_t)(P > 0xFFFFFFFFull ? 0xFFFFFFFFull : P);
        if (P > (unsigned long long)pair_cap) {
            atomicOr(&counts->overflow, 2u);
            counts->n_pairs = 0;
        } else {
            counts->n_pairs = (uint32_t)P;
        }
    }
}

// Block-cooperative emission: per step, the block scans 256 Gaussians' tile counts and then
// all 256 threads walk the step's pairs together (binary search for the owning Gaussian).
__global__ void __launch_bounds__(kEmThreads) emit_pairs(const uint32_t* __restrict__ order,
                                                         const uint32_t* __restrict__ tiles,
                                                         const uint2* __restrict__ rect,
                                                         const uint32_t* n_dev, int64_t n_cap,
                                                         const uint32_t* __restrict__ block_off,
                                                         const ogs_counts* counts, int gx,
                                                         uint32_t* __restrict__ pkey,
                                                         uint32_t* __restrict__ pval) {
    __shared__ uint32_t s_off[kEmThreads + 1];
    __shared__ uint32_t s_g[kEmThreads];
    __shared__ uint2 s_rect[kEmThreads];
    __shared__ uint32_t ws[kEmThreads / 32];
    if (counts->overflow & 2u) return;
    const uint32_t n = count_of(n_dev, n_cap);
    const int64_t base = (int64_t)blockIdx.x * kEmTile;
    if (base >= n) return;
    uint32_t running = block_off[blockIdx.x];
    for (int it = 0; it < kEmItems; ++it) {
        int64_t i = base + it * kEmThreads + threadIdx.x;
        uint32_t g = 0, c = 0;
        uint2 rc = make_uint2(0, 0);
        if (i < n) {
            g = order[i];
            c = tiles[g];
            if (c) rc = rect[g];
        }
        uint32_t excl;
        uint32_t tot = block_excl_scan(c, excl, ws);
        s_off[threadIdx.x] = excl;
        s_g[threadIdx.x] = g;
        s_rect[threadIdx.x] = rc;
        if (threadIdx.x == 0) s_off[kEmThreads] = tot;
        __syncthreads();
        for (uint32_t p = threadIdx.x; p < tot; p += kEmThreads) {
            // owner: largest k with s_off[k] <= p (entries with zero count share offsets)
            int lo = 0, hi = kEmThreads - 1;
            while (lo < hi) {
                int mid = (lo + hi + 1) >> 1;
                if (s_off[mid] <= p) lo = mid; else hi = mid - 1;
            }
            const uint32_t local = p - s_off[lo];
            const uint2 r = s_rect[lo];
            const uint32_t x0 = r.x & 0xFFFFu, y0 = r.x >> 16, x1 = r.y & 0xFFFFu;
            const uint32_t wdt = x1 - x0;
            const uint32_t ty = y0 + local / wdt, tx = x0 + local % wdt;
            const uint32_t o = running + p;
            pkey[o] = ty * (uint32_t)gx + tx;
            pval[o] = s_g[lo];
        }
        running += tot;
        __syncthreads();
    }
}

__global__ void tile_ranges(const uint32_t* __restrict__ pkey, const ogs_counts* counts,
                            uint2* __restrict__ range) {
    const uint32_t P = counts->n_pairs;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t t = pkey[i];
        if (i == 0 || pkey[i - 1] != t) range[t].x = (uint32_t)i;
        if (i == P - 1 || pkey[i + 1] != t) range[t].y = (uint32_t)(i + 1);
    }
}

struct SortScratch {
    uint32_t* dk;      // depth keys (sorted in place)
    uint32_t* order;   // Gaussian ids in depth order
    uint32_t* bsum;    // emission block offsets
    uint32_t* pkey;    // pair tile keys
    RsScratch rs;
};

size_t sort_layout(int64_t g_cap, int64_t pair_cap, void* base, SortScratch* s) {
    int64_t nbe = (g_cap + kEmTile - 1) / kEmTile;
    if (nbe < 1) nbe = 1;
    Carver cv(base);
    SortScratch t;
    t.dk = cv.take<uint32_t>(g_cap > 0 ? g_cap : 1);
    t.order = cv.take<uint32_t>(g_cap > 0 ? g_cap : 1);
    t.bsum = cv.take<uint32_t>(nbe);
    t.pkey = cv.take<uint32_t>(pair_cap > 0 ? pair_cap : 1);
    int64_t rs_cap = g_cap > pair_cap ? g_cap : pair_cap;
    size_t rs_bytes = rs_layout(rs_cap, nullptr, nullptr);
    char* rs_base = cv.take<char>(rs_bytes);
    rs_layout(rs_cap, rs_base, &t.rs);
    if (s) *s = t;
    return cv.off + 256;
}

int bits_for(int64_t n) {
    int b = 0;
    while (((int64_t)1 << b) < n) ++b;
    return b < 1 ? 1 : b;
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
    (void)n_tiles;
    return sort_layout(g_cap < 0 ? 0 : g_cap, pair_cap < 0 ? 0 : pair_cap, nullptr, nullptr);
}

extern "C" ogs_status ogs_sort(const uint32_t* depth_key, const uint32_t* rect, const uint32_t* tiles,
                               int64_t g_cap, int64_t n_gauss, int32_t grid_x, int32_t grid_y,
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
        !aligned(scratch, 16) || !aligned(rect, 8))
        return OGS_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int n_tiles = grid_x * grid_y;
    if (cudaMemsetAsync(tile_range, 0, sizeof(uint32_t) * 2 * (size_t)n_tiles, st) != cudaSuccess)
        return OGS_ERR_CUDA;
    if (g_cap == 0) return OGS_OK;
    SortScratch s;
    sort_layout(g_cap, pair_cap, scratch, &s);
    // the Gaussian count is the device count written by the decoder, or the caller's n_gauss
    const uint32_t* n_dev = n_gauss < 0 ? &counts->n_gaussians : nullptr;
    const int64_t n_cap = n_gauss < 0 ? g_cap : (n_gauss < g_cap ? n_gauss : g_cap);
    // 1. depth order
    iota_keys<<<stride_grid(n_cap, 256, 8), 256, 0, st>>>(depth_key, s.dk, s.order, n_dev, n_cap);
    if (!radix_sort(s.dk, s.order, n_dev, n_cap, 0, 32, s.rs, st)) return OGS_ERR_CUDA;
    // 2. pair emission in depth order
    int nbe = (int)((n_cap + kEmTile - 1) / kEmTile);
    if (nbe < 1) nbe = 1;
    emit_count<<<nbe, kEmThreads, 0, st>>>(s.order, tiles, n_dev, n_cap, s.bsum);
    emit_scan<<<1, 1024, 0, st>>>(s.bsum, nbe, pair_cap, counts);
    emit_pairs<<<nbe, kEmThreads, 0, st>>>(s.order, tiles, reinterpret_cast<const uint2*>(rect),
                                           n_dev, n_cap, s.bsum, counts, grid_x, s.pkey,
                                           pair_gauss);
    // 3. stable sort of pairs by tile id
    if (!radix_sort(s.pkey, pair_gauss, &counts->n_pairs, pair_cap, 0, bits_for(n_tiles), s.rs, st))
        return OGS_ERR_CUDA;
    // 4. tile ranges
    tile_ranges<<<stride_grid(pair_cap, 256, 8), 256, 0, st>>>(s.pkey, counts,
                                                                reinterpret_cast<uint2*>(tile_range));
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
    void* base = nullptr;
    ogs_status st = noalloc_scratch(&base);
    if (st != OGS_OK) return st;
    // every scratch word is written before it is read in each pass: nothing to clear
    RsScratch s;
    rs_layout(n_cap, base, &s);
    return radix_sort(keys, vals, n_dev, n_cap, bit_lo, bit_hi, s, (cudaStream_t)stream)
               ? OGS_OK : OGS_ERR_CUDA;
}
