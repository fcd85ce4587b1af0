// View-frequency anchor pruning (Sec. 4.2.2): the view frequency of an anchor is the fraction
// of training views that select it; anchors whose frequency is below the visibility
// threshold tau_v are removed.
//
//   ogs_count_selected  adds one to the counter of every anchor a view selected
//   ogs_prune_anchors   order-preserving list of the anchors with count >= min_count
//                       (count per 2048-anchor tile -> one-CTA scan -> ordered scatter)
//   ogs_gather_rows     compacts any per-anchor array (rows of bytes) by that list
//   ogs_opacity_accumulate, ogs_prune_by_opacity   the average-opacity rule of the same
//                       section: anchors whose Gaussians' average opacity over the counted
//                       views is below tau_o are removed (same compaction)
#include "internal.cuh"

namespace ogs {
namespace {

constexpr int kPrThreads = 256;
constexpr int kPrItems = 8;
constexpr int kPrChunk = kPrThreads * kPrItems;

__global__ void count_selected(const uint32_t* __restrict__ sel_idx, const ogs_counts* counts,
                               uint32_t* __restrict__ sel_count) {
    const uint32_t M = counts->n_selected;
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < M; r += gridDim.x * blockDim.x)
        sel_count[sel_idx[r]] += 1u;      // a view selects an anchor at most once
}

__global__ void __launch_bounds__(kPrThreads) prune_count(const uint32_t* __restrict__ cnt,
                                                          int64_t N, uint32_t min_count,
                                                          uint32_t* __restrict__ tile_count) {
    __shared__ uint32_t s_wc[kPrThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kPrChunk;
    uint32_t mine = 0;
#pragma unroll
    for (int it = 0; it < kPrItems; ++it) {
        const int64_t j = base + it * kPrThreads + threadIdx.x;
        mine += __popc(__ballot_sync(0xffffffffu, j < N && cnt[j] >= min_count));
    }
    if (lane_id() == 0) s_wc[threadIdx.x >> 5] = mine;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int i = 0; i < kPrThreads / 32; ++i) t += s_wc[i];
        tile_count[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(1024) prune_scan(uint32_t* __restrict__ tile_count, int nb,
                                                   uint32_t* __restrict__ n_kept) {
    __shared__ uint32_t ws[32];
    const int per = (nb + 1023) / 1024;
    const int b0 = threadIdx.x * per, b1 = min(b0 + per, nb);
    uint32_t local = 0;
    for (int b = b0; b < b1; ++b) local += tile_count[b];
    uint32_t x = local;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane_id() >= (unsigned)o) x += y;
    }
    if (lane_id() == 31) ws[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x < 32) {
        uint32_t v = ws[threadIdx.x];
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane_id() >= (unsigned)o) v += y;
        }
        ws[threadIdx.x] = v;
    }
    __syncthreads();
    uint32_t run = (threadIdx.x >= 32 ? ws[(threadIdx.x >> 5) - 1] : 0) + x - local;
    for (int b = b0; b < b1; ++b) {
        const uint32_t v = tile_count[b];
        tile_count[b] = run;
        run += v;
    }
    if (threadIdx.x == 0) *n_kept = ws[31];
}

__global__ void __launch_bounds__(kPrThreads) prune_scatter(const uint32_t* __restrict__ cnt,
                                                            int64_t N, uint32_t min_count,
                                                            const uint32_t* __restrict__ tile_off,
                                                            uint32_t* __restrict__ keep_idx) {
    __shared__ uint32_t s_wc[kPrThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kPrChunk;
    const unsigned warp = threadIdx.x >> 5;
    uint32_t off = tile_off[blockIdx.x];
    for (int it = 0; it < kPrItems; ++it) {
        const int64_t j = base + it * kPrThreads + threadIdx.x;
        const bool keep = j < N && cnt[j] >= min_count;
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        if (lane_id() == 0) s_wc[warp] = __popc(bal);
        __syncthreads();
        uint32_t before = 0, tot = 0;
#pragma unroll
        for (int i = 0; i < kPrThreads / 32; ++i) {
            before += (i < (int)warp) ? s_wc[i] : 0;
            tot += s_wc[i];
        }
        if (keep) keep_idx[off + before + __popc(bal & lanemask_lt())] = (uint32_t)j;
        off += tot;
        __syncthreads();
    }
}

// Average-opacity statistic (Sec. 4.2.2): thread per selected anchor of one view adds the
// opacities of its k Gaussians (dropped ones, opacity <= 0, as 0; summed in slot order) and
// one view.  An anchor appears once per view: no atomics.
__global__ void opacity_accumulate(const float* __restrict__ opac,
                                   const uint32_t* __restrict__ sel_idx, const ogs_counts* counts,
                                   int k, float* __restrict__ acc, uint32_t* __restrict__ views) {
    const uint32_t M = counts->n_selected;
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < M; r += gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int i = 0; i < k; ++i) s = __fadd_rn(s, fmaxf(opac[(size_t)r * k + i], 0.f));
        const uint32_t j = sel_idx[r];
        acc[j] = __fadd_rn(acc[j], s);
        views[j] += 1u;
    }
}

// keep[j] = 0 where an anchor seen in some view has average opacity acc / (views k) < tau
__global__ void opacity_keep(const float* __restrict__ acc, const uint32_t* __restrict__ views,
                             int64_t N, int k, float tau, uint32_t* __restrict__ keep) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < N;
         j += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t v = views[j];
        keep[j] = (v > 0 && __fdiv_rn(acc[j], (float)(v * (uint32_t)k)) < tau) ? 0u : 1u;
    }
}

// dst row r = src row idx[r] for r < n; rows of `row` bytes, copied in 4-byte words when
// the row size and both bases allow it
__global__ void gather_rows(const unsigned char* __restrict__ src, unsigned char* __restrict__ dst,
                            int64_t row, const uint32_t* __restrict__ idx,
                            const uint32_t* n_dev, int64_t n_cap, int words) {
    const int64_t n = n_dev ? min((int64_t)*n_dev, n_cap) : n_cap;
    const int64_t unit = words ? 4 : 1;
    const int64_t per = row / unit;
    const int64_t total = n * per;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / per, c = e % per;
        const int64_t s = (int64_t)idx[r];
        if (words)
            reinterpret_cast<uint32_t*>(dst)[r * per + c] =
                reinterpret_cast<const uint32_t*>(src)[s * per + c];
        else
            dst[r * per + c] = src[s * per + c];
    }
}

}  // namespace
}  // namespace ogs

using namespace ogs;

extern "C" ogs_status ogs_count_selected(const uint32_t* sel_idx, const ogs_counts* counts,
                                         uint32_t* sel_count, void* stream) {
    if (!sel_idx || !counts || !sel_count) return OGS_ERR_ARG;
    count_selected<<<2 * kSmCount, 256, 0, (cudaStream_t)stream>>>(sel_idx, counts, sel_count);
    return launch_status();
}

extern "C" size_t ogs_prune_scratch_bytes(int64_t N) {
    const int64_t nb = (N + kPrChunk - 1) / kPrChunk;
    return sizeof(uint32_t) * (size_t)(nb < 1 ? 1 : nb) + 256;
}

extern "C" ogs_status ogs_prune_anchors(const uint32_t* sel_count, int64_t N, uint32_t min_count,
                                        uint32_t* keep_idx, uint32_t* n_kept, void* scratch,
                                        size_t scratch_bytes, void* stream) {
    if (!sel_count || !keep_idx || !n_kept || !scratch || N < 0 || N > 0xFFFFFFFFll)
        return OGS_ERR_ARG;
    if (scratch_bytes < ogs_prune_scratch_bytes(N) || !aligned(scratch, 16)) return OGS_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int nb = (int)((N + kPrChunk - 1) / kPrChunk);
    if (nb < 1) nb = 1;
    uint32_t* tile = (uint32_t*)scratch;
    prune_count<<<nb, kPrThreads, 0, st>>>(sel_count, N, min_count, tile);
    prune_scan<<<1, 1024, 0, st>>>(tile, nb, n_kept);
    prune_scatter<<<nb, kPrThreads, 0, st>>>(sel_count, N, min_count, tile, keep_idx);
    return launch_status();
}

extern "C" ogs_status ogs_gather_rows(const void* src, void* dst, int64_t row_bytes,
                                      const uint32_t* idx, const uint32_t* n_dev, int64_t n_cap,
                                      void* stream) {
    if (!src || !dst || !idx || row_bytes <= 0 || n_cap < 0) return OGS_ERR_ARG;
    if (src == dst) return OGS_ERR_ARG;
    if (n_cap == 0) return OGS_OK;
    const int words = (row_bytes % 4 == 0) && aligned(src, 4) && aligned(dst, 4);
    const int64_t units = n_cap * (words ? row_bytes / 4 : row_bytes);
    gather_rows<<<stride_grid(units, 256, 8), 256, 0, (cudaStream_t)stream>>>(
        (const unsigned char*)src, (unsigned char*)dst, row_bytes, idx, n_dev, n_cap, words);
    return launch_status();
}

extern "C" ogs_status ogs_opacity_accumulate(const float* opac, const uint32_t* sel_idx,
                                             const ogs_counts* counts, int32_t k,
                                             float* opac_sum, uint32_t* opac_views,
                                             void* stream) {
    if (!opac || !sel_idx || !counts || !opac_sum || !opac_views || k < 1 || k > 16)
        return OGS_ERR_ARG;
    opacity_accumulate<<<2 * kSmCount, 256, 0, (cudaStream_t)stream>>>(opac, sel_idx, counts, k,
                                                                       opac_sum, opac_views);
    return launch_status();
}

extern "C" size_t ogs_prune_opacity_scratch_bytes(int64_t N) {
    if (N < 0) return 0;
    const size_t flags = (sizeof(uint32_t) * (size_t)(N > 0 ? N : 1) + 255) / 256 * 256;
    return flags + ogs_prune_scratch_bytes(N);
}

extern "C" ogs_status ogs_prune_by_opacity(const float* opac_sum, const uint32_t* opac_views,
                                           int64_t N, int32_t k, float tau_o,
                                           uint32_t* keep_idx, uint32_t* n_kept, void* scratch,
                                           size_t scratch_bytes, void* stream) {
    if (!opac_sum || !opac_views || !keep_idx || !n_kept || !scratch || N < 0 ||
        N > 0xFFFFFFFFll || k < 1 || k > 16)
        return OGS_ERR_ARG;
    if (scratch_bytes < ogs_prune_opacity_scratch_bytes(N) || !aligned(scratch, 16))
        return OGS_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    uint32_t* keep = (uint32_t*)scratch;
    const size_t flags = (sizeof(uint32_t) * (size_t)(N > 0 ? N : 1) + 255) / 256 * 256;
    if (N > 0)
        opacity_keep<<<stride_grid(N, 256, 8), 256, 0, st>>>(opac_sum, opac_views, N, k, tau_o,
                                                             keep);
    return ogs_prune_anchors(keep, N, 1u, keep_idx, n_kept, (unsigned char*)scratch + flags,
                             scratch_bytes - flags, stream);
}
