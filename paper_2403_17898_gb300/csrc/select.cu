// Anchor selection by octree level (Sec. 4.1.3, Eq. for L_hat) with the inference-time
// opacity blending of the next level, followed by an order-preserving compaction.
//
// HBM-bound streaming pass over the anchor SoA (pos 12 B + level 1 B + dL 4 B per anchor),
// read once, then an order-preserving compaction: each CTA stages one tile of anchors in
// shared memory with TMA bulk copies (so the whole tile's bytes are in flight at once) and
// writes every anchor's weight (4 B) and the tile's kept count; one CTA scans the counts; the
// scatter re-reads only the weights, ranks kept anchors with warp scans and writes them in
// ascending anchor order.  No CTA waits on another, so every tile streams at full rate.
#include "gate_common.cuh"

namespace ogs {
namespace {

constexpr int kSelThreads = 256;
constexpr int kSelItems = 8;
constexpr int kSelWarps = kSelThreads / 32;
constexpr int kSelChunk = kSelThreads * kSelItems;   // anchors per tile (one CTA)
struct SelArgs {
    const float* pos;
    const uint8_t* level;
    const float* dL;
    int64_t N;
    int NL;
    int k;
    int infer;
    Cam cam;
};

// Returns true if an anchor at (px, py, pz) with level `lvl` and LOD bias `dl` is kept; w
// receives its opacity weight.
__device__ __forceinline__ bool keep_anchor(const SelArgs& a, float px, float py, float pz,
                                           uint32_t lvl, float dl, float& w) {
    const Cam& c = a.cam;
    float dx = px - c.c[0];
    float dy = py - c.c[1];
    float dz = pz - c.c[2];
    // visibility of the anchor centre: in front of the near plane, within 1.3x half-fov
    float zc = c.R[6] * dx + c.R[7] * dy + c.R[8] * dz;
    float xc = c.R[0] * dx + c.R[1] * dy + c.R[2] * dz;
    float yc = c.R[3] * dx + c.R[4] * dy + c.R[5] * dz;
    if (!(zc > c.znear) || fabsf(xc) > c.limx * zc || fabsf(yc) > c.limy * zc) return false;
    // fractional level from the viewing distance plus the anchor's LOD bias, clamped
    float d = sqrtf(dx * dx + dy * dy + dz * dz);
    float Lraw = log2f(c.d_max / (d * c.s)) + dl;
    float Ls = fminf(fmaxf(Lraw, 0.0f), (float)(a.NL - 1));
    float Lh = floorf(Ls);
    float L = (float)lvl;
    if (L <= Lh) {
        w = 1.0f;
        return true;
    }
    if (a.infer && L == Lh + 1.0f && Ls > Lh) {
        w = Ls - Lh;
        return true;
    }
    return false;
}

// Pass 1 (tile of kSelChunk anchors per CTA): the tile's anchor SoA lands in shared memory by
// three TMA bulk copies (plain loads for a partial tile or unaligned arrays); the predicate
// writes each anchor's opacity weight (0 = not kept, kept weights are > 0) and the tile's
// kept count.
__global__ void __launch_bounds__(kSelThreads) select_eval(SelArgs a, float* __restrict__ wsel,
                                                           uint32_t* __restrict__ tile_count,
                                                           ogs_counts* counts, int bulk) {
    pdl_wait();
    pdl_trigger();
    __shared__ __align__(16) float s_pos[3 * kSelChunk];
    __shared__ __align__(16) float s_dl[kSelChunk];
    __shared__ __align__(16) uint8_t s_lvl[kSelChunk];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t s_wc[kSelWarps];
    const int64_t base = (int64_t)blockIdx.x * kSelChunk;
    const int n_here = (int)min((int64_t)kSelChunk, a.N - base);
    if (bulk && n_here == kSelChunk) {
        if (threadIdx.x == 0) {
            tc::mbar_init(&mbar, 1);
            tc::mbar_expect_tx(&mbar, (3 * 4 + 4 + 1) * kSelChunk);
            tc::bulk_load(s_pos, a.pos + 3 * base, 3 * 4 * kSelChunk, &mbar);
            tc::bulk_load(s_dl, a.dL + base, 4 * kSelChunk, &mbar);
            tc::bulk_load(s_lvl, a.level + base, kSelChunk, &mbar);
        }
        __syncthreads();                              // barrier initialised before anyone polls
        if (!tc::mbar_wait(&mbar, 0, kSpinLimit)) {
            if (threadIdx.x == 0) atomicExch(&counts->timeout, 1u);
            tc::mbar_wait(&mbar, 0, kSpinLimit);      // copies may still be landing
        }
    } else {
        for (int e = threadIdx.x; e < 3 * n_here; e += kSelThreads) s_pos[e] = a.pos[3 * base + e];
        for (int e = threadIdx.x; e < n_here; e += kSelThreads) {
            s_dl[e] = a.dL[base + e];
            s_lvl[e] = a.level[base + e];
        }
        __syncthreads();
    }
    uint32_t mine = 0;
#pragma unroll
    for (int it = 0; it < kSelItems; ++it) {
        const int l = it * kSelThreads + threadIdx.x;
        float w = 0.0f;
        const bool keep = l < n_here && keep_anchor(a, s_pos[3 * l], s_pos[3 * l + 1],
                                                    s_pos[3 * l + 2], s_lvl[l], s_dl[l], w);
        if (l < n_here) wsel[base + l] = keep ? w : 0.0f;
        mine += __popc(__ballot_sync(0xffffffffu, keep));
    }
    if (lane_id() == 0) s_wc[threadIdx.x >> 5] = mine;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
#pragma unroll
        for (int i = 0; i < kSelWarps; ++i) t += s_wc[i];
        tile_count[blockIdx.x] = t;
    }
}

// Pass 1 of the gated selection (same tiles): the LOD predicate as in select_eval, then the
// learned gate on the tile's kept anchors in chunks of 128 rows (tensor-core network shared
// with ogs_proposal_gate_bf16, so the keep decisions are the same bits); an anchor the gate
// drops gets weight 0, so passes 2 and 3 build the gated list directly.  Persistent CTAs
// (three per SM) take tiles round-robin: the network image and the tensor memory are set up
// once per CTA, and the next tile's bulk copy is issued as soon as the current tile's staged
// arrays are no longer read (once the last chunk's gate inputs are built), so it lands while
// the gate runs.
constexpr int kSgOffImg = 0;                              // network image
constexpr int kSgOffA = gate::kGImgBytes;                 // gate A operand
constexpr int kSgSmem = kSgOffA + gate::kGABytes;

__device__ __forceinline__ void sg_issue_tile(const SelArgs& a, int64_t tile, float* s_pos,
                                              float* s_dl, uint8_t* s_lvl, uint64_t* mbar) {
    const int64_t base = tile * kSelChunk;
    tc::mbar_expect_tx(mbar, (3 * 4 + 4 + 1) * kSelChunk);
    tc::bulk_load(s_pos, a.pos + 3 * base, 3 * 4 * kSelChunk, mbar);
    tc::bulk_load(s_dl, a.dL + base, 4 * kSelChunk, mbar);
    tc::bulk_load(s_lvl, a.level + base, kSelChunk, mbar);
}

__global__ void __launch_bounds__(kSelThreads, 3) select_eval_gated(
    SelArgs a, const float* __restrict__ feat, const unsigned char* __restrict__ img,
    float p_star, float* __restrict__ wsel, uint32_t* __restrict__ tile_count,
    ogs_counts* counts, int bulk) {
    pdl_wait();
    pdl_trigger();
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(16) float s_pos[3 * kSelChunk];
    __shared__ __align__(16) float s_dl[kSelChunk];
    __shared__ __align__(16) uint8_t s_lvl[kSelChunk];
    __shared__ uint16_t s_list[kSelChunk];
    __shared__ uint8_t s_drop[kSelChunk];
    __shared__ __align__(8) uint64_t mbar, wbar, gbar;
    __shared__ uint32_t s_wc[kSelWarps];
    __shared__ uint32_t s_n;
    __shared__ uint32_t tmem_base;
    const int t = threadIdx.x;
    const int64_t nb = (a.N + kSelChunk - 1) / kSelChunk;
    // a tile is copied in bulk when it is full and the arrays are aligned
    auto full = [&](int64_t tile) { return bulk && (tile + 1) * kSelChunk <= a.N; };
    if (t == 0) {
        tc::mbar_init(&mbar, 1);
        tc::mbar_init(&wbar, 1);
        tc::mbar_init(&gbar, 1);
        tc::mbar_expect_tx(&wbar, gate::kGImgBytes);
        tc::bulk_load(sm + kSgOffImg, img, gate::kGImgBytes, &wbar);
        if (full(blockIdx.x)) sg_issue_tile(a, blockIdx.x, s_pos, s_dl, s_lvl, &mbar);
    }
    if ((t >> 5) == 0) {
        tc::tmem_alloc(&tmem_base, gate::kGTmemCols);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = tmem_base;
    bool net_ok = tc::mbar_wait(&wbar, 0, gate::kGWaitLimit);
    if (!net_ok) {
        if (t == 0) atomicExch(&counts->timeout, 1u);
        tc::mbar_wait(&wbar, 0, gate::kGWaitLimit);   // the copy may still be landing
    }
    uint32_t tma_phase = 0, phase = 0;
    bool mma_ok = true;
    unsigned char* sA = sm + kSgOffA;
    for (int64_t tile = blockIdx.x; tile < nb; tile += gridDim.x) {
        const int64_t base = tile * kSelChunk;
        const int n_here = (int)min((int64_t)kSelChunk, a.N - base);
        if (full(tile)) {
            if (!tc::mbar_wait(&mbar, tma_phase, kSpinLimit)) {
                if (t == 0) atomicExch(&counts->timeout, 1u);
                tc::mbar_wait(&mbar, tma_phase, kSpinLimit);   // copies may still be landing
            }
            tma_phase ^= 1;
        } else {
            for (int e = t; e < 3 * n_here; e += kSelThreads) s_pos[e] = a.pos[3 * base + e];
            for (int e = t; e < n_here; e += kSelThreads) {
                s_dl[e] = a.dL[base + e];
                s_lvl[e] = a.level[base + e];
            }
        }
        if (t == 0) s_n = 0;
        __syncthreads();
        // LOD predicate; kept anchors listed (in any order) for the gate
        float wv[kSelItems];
#pragma unroll
        for (int it = 0; it < kSelItems; ++it) {
            const int l = it * kSelThreads + t;
            float w = 0.0f;
            const bool keep = l < n_here && keep_anchor(a, s_pos[3 * l], s_pos[3 * l + 1],
                                                        s_pos[3 * l + 2], s_lvl[l], s_dl[l], w);
            wv[it] = keep ? w : 0.0f;
            if (keep) {
                s_drop[l] = 0;
                s_list[atomicAdd(&s_n, 1u)] = (uint16_t)l;
            }
        }
        __syncthreads();
        const uint32_t K = s_n;
        const int64_t next = tile + gridDim.x;
        const bool prefetch = next < nb && full(next);
        bool issued = false;
        if (K == 0) {                                 // staged arrays no longer read
            if (t == 0 && prefetch) sg_issue_tile(a, next, s_pos, s_dl, s_lvl, &mbar);
            issued = true;
        }
        bool gated = mma_ok;
        for (uint32_t c0 = 0; gated && c0 < K; c0 += 128) {
            // gate inputs: two threads per row (t and t + 128)
            const uint32_t r = c0 + (uint32_t)(t & 127);
            if (r < K) {
                const int l = s_list[r];
                gate::put_input_half(sA, t & 127, t >> 7, feat + (size_t)(base + l) * 32,
                                     s_pos[3 * l], s_pos[3 * l + 1], s_pos[3 * l + 2], s_lvl[l],
                                     a.NL, a.cam);
            } else {
                gate::put_input_half(sA, t & 127, t >> 7, nullptr, 0.f, 0.f, 0.f, 0u, a.NL,
                                     a.cam);
            }
            if (c0 + 128 >= K) {                      // last chunk: staged arrays now free
                __syncthreads();
                if (t == 0 && prefetch) sg_issue_tile(a, next, s_pos, s_dl, s_lvl, &mbar);
                issued = true;
            }
            float z;
            if (!gate::gate_hidden(sA, sm + kSgOffImg, tbase, &gbar, phase, z)) {
                gated = mma_ok = false;               // this and later tiles keep the LOD list
                if (t == 0) atomicExch(&counts->timeout, 1u);
                tc::mbar_wait(&gbar, phase, gate::kGWaitLimit);   // product still in flight
                break;
            }
            if (t < 128 && r < K) s_drop[s_list[r]] = gate::keep_prob(z) >= p_star ? 0 : 1;
        }
        tc::fence_before_sync();
        __syncthreads();                              // s_drop complete; TMEM reads done
        tc::fence_after_sync();
        uint32_t mine = 0;
#pragma unroll
        for (int it = 0; it < kSelItems; ++it) {
            const int l = it * kSelThreads + t;
            const bool keep = wv[it] > 0.0f && !(gated && s_drop[l]);
            if (l < n_here) wsel[base + l] = keep ? wv[it] : 0.0f;
            mine += __popc(__ballot_sync(0xffffffffu, keep));
        }
        if (lane_id() == 0) s_wc[t >> 5] = mine;
        // a gate that stopped early: the staged arrays are free only now
        if (!issued && t == 0 && prefetch) sg_issue_tile(a, next, s_pos, s_dl, s_lvl, &mbar);
        __syncthreads();
        if (t == 0) {
            uint32_t tot = 0;
#pragma unroll
            for (int i = 0; i < kSelWarps; ++i) tot += s_wc[i];
            tile_count[tile] = tot;
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if ((t >> 5) == 0) tc::tmem_dealloc(tbase, gate::kGTmemCols);
}

// Pass 2 (one CTA): exclusive scan of the tile counts in place; M and the overflow state.
__global__ void __launch_bounds__(1024) select_scan(uint32_t* __restrict__ tile_count, int nb,
                                                    int64_t cap, int k, ogs_counts* counts) {
    pdl_wait();
    pdl_trigger();
    __shared__ unsigned long long ws[32];
    const int per = (nb + 1023) / 1024;
    const int b0 = threadIdx.x * per, b1 = min(b0 + per, nb);
    unsigned long long local = 0;
    for (int b = b0; b < b1; ++b) local += tile_count[b];
    unsigned long long x = local;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane_id() >= (unsigned)o) x += y;
    }
    if (lane_id() == 31) ws[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x < 32) {
        unsigned long long v = ws[threadIdx.x];
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane_id() >= (unsigned)o) v += y;
        }
        ws[threadIdx.x] = v;                          // inclusive warp totals
    }
    __syncthreads();
    unsigned long long run = (threadIdx.x >= 32 ? ws[(threadIdx.x >> 5) - 1] : 0) + x - local;
    for (int b = b0; b < b1; ++b) {
        const uint32_t v = tile_count[b];
        tile_count[b] = (uint32_t)min(run, 0xFFFFFFFFull);
        run += v;
    }
    if (threadIdx.x == 0) {
        const unsigned long long total = ws[31];
        const uint32_t m = total > (unsigned long long)cap ? (uint32_t)cap : (uint32_t)total;
        counts->n_selected = m;
        counts->n_gaussians = m * (uint32_t)k;
        counts->need_selected = total > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)total;
        if (total > (unsigned long long)cap) atomicOr(&counts->overflow, 1u);
    }
}

// Pass 3 (same tiles as pass 1): kept anchors ranked by warp ballots and written in
// ascending order at the tile's offset (16-byte weight loads, four anchors per thread and
// round).
__global__ void __launch_bounds__(kSelThreads) select_scatter(const float* __restrict__ wsel,
                                                              const uint32_t* __restrict__ tile_off,
                                                              int64_t N, uint32_t* sel_idx,
                                                              float* sel_w, int64_t cap) {
    pdl_wait();
    pdl_trigger();
    __shared__ uint32_t s_cnt[kSelItems / 4][kSelWarps];
    const int64_t base = (int64_t)blockIdx.x * kSelChunk;
    const int n_here = (int)min((int64_t)kSelChunk, N - base);
    const unsigned warp = threadIdx.x >> 5;
    constexpr int kRounds = kSelItems / 4;
    float4 wv[kRounds];
    uint32_t cnt[kRounds];
#pragma unroll
    for (int q = 0; q < kRounds; ++q) {
        const int l = 4 * (q * kSelThreads + threadIdx.x);   // four consecutive anchors
        float v[4];
        if (l + 4 <= n_here && ((base & 3) == 0)) {
            const float4 u = *reinterpret_cast<const float4*>(wsel + base + l);
            v[0] = u.x; v[1] = u.y; v[2] = u.z; v[3] = u.w;
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e) v[e] = l + e < n_here ? wsel[base + l + e] : 0.f;
        }
        wv[q] = make_float4(v[0], v[1], v[2], v[3]);
        cnt[q] = (v[0] > 0.f) + (v[1] > 0.f) + (v[2] > 0.f) + (v[3] > 0.f);
        // warp-inclusive scan of the per-thread counts
        uint32_t x = cnt[q];
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane_id() >= (unsigned)o) x += y;
        }
        if (lane_id() == 31) s_cnt[q][warp] = x;
        cnt[q] = x - cnt[q];                           // exclusive within the warp
    }
    __syncthreads();
    unsigned long long off = tile_off[blockIdx.x];
#pragma unroll
    for (int q = 0; q < kRounds; ++q) {
        uint32_t before = 0, tot = 0;
#pragma unroll
        for (int i = 0; i < kSelWarps; ++i) {
            const uint32_t c = s_cnt[q][i];
            before += (i < (int)warp) ? c : 0;
            tot += c;
        }
        unsigned long long p = off + before + cnt[q];
        const int l = 4 * (q * kSelThreads + threadIdx.x);
        const float v[4] = {wv[q].x, wv[q].y, wv[q].z, wv[q].w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            if (v[e] > 0.f) {
                if (p < (unsigned long long)cap) {
                    sel_idx[p] = (uint32_t)(base + l + e);
                    sel_w[p] = v[e];
                }
                ++p;
            }
        }
        off += tot;
    }
}

}  // namespace
}  // namespace ogs

using namespace ogs;

extern "C" size_t ogs_lod_select_scratch_bytes(int64_t N) {
    int64_t nb = (N + kSelChunk - 1) / kSelChunk;
    Carver cv(nullptr);
    cv.take<uint32_t>((size_t)(nb < 1 ? 1 : nb));
    cv.take<float>((size_t)(N > 0 ? N : 1));
    return cv.off + 256;
}

extern "C" ogs_status ogs_lod_select(const float* pos, const uint8_t* level, const float* dL,
                                     int64_t N, int32_t NL, int32_t k, const ogs_camera* cam,
                                     int32_t infer, uint32_t* sel_idx, float* sel_w,
                                     int64_t sel_cap, ogs_counts* counts, void* scratch,
                                     size_t scratch_bytes, void* stream) {
    if (!pos || !level || !dL || !cam || !sel_idx || !sel_w || !counts || !scratch)
        return OGS_ERR_ARG;
    if (N < 0 || N > 0xFFFFFFFFll || NL < 1 || NL > 255 || k < 1 || sel_cap < 0)
        return OGS_ERR_ARG;
    if (cam->width <= 0 || cam->height <= 0 || !(cam->d_max > 0) || !(cam->s > 0))
        return OGS_ERR_ARG;
    if (scratch_bytes < ogs_lod_select_scratch_bytes(N) || !aligned(scratch, 16)) return OGS_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    SelArgs a{pos, level, dL, N, NL, k, infer, make_cam(*cam)};
    int nb = (int)((N + kSelChunk - 1) / kSelChunk);
    if (nb < 1) nb = 1;
    Carver cv(scratch);
    uint32_t* tile_count = cv.take<uint32_t>((size_t)nb);
    float* wsel = cv.take<float>((size_t)(N > 0 ? N : 1));
    const int bulk = aligned(pos, 16) && aligned(dL, 16) && aligned(level, 16);
    launch_pdl(select_eval, dim3(nb), dim3(kSelThreads), 0, st, a, wsel, tile_count, counts, bulk);
    launch_pdl(select_scan, dim3(1), dim3(1024), 0, st, tile_count, nb, sel_cap, k, counts);
    launch_pdl(select_scatter, dim3(nb), dim3(kSelThreads), 0, st,
               wsel, tile_count, N, sel_idx, sel_w, sel_cap);
    return launch_status();
}

extern "C" size_t ogs_lod_select_gated_scratch_bytes(int64_t N) {
    return ogs_lod_select_scratch_bytes(N) + gate::kGImgBytes + 256;
}

extern "C" ogs_status ogs_lod_select_gated(const float* pos, const uint8_t* level,
                                           const float* dL, const float* feat, int64_t N,
                                           int32_t NL, int32_t k, const ogs_camera* cam,
                                           int32_t infer, const ogs_proposal* net,
                                           float p_star, uint32_t* sel_idx, float* sel_w,
                                           int64_t sel_cap, ogs_counts* counts, void* scratch,
                                           size_t scratch_bytes, void* stream) {
    if (!pos || !level || !dL || !feat || !cam || !net || !sel_idx || !sel_w || !counts ||
        !scratch)
        return OGS_ERR_ARG;
    if (!net->w1 || !net->b1 || !net->w2 || !net->b2 || !net->w3 || !net->b3) return OGS_ERR_ARG;
    if (N < 0 || N > 0xFFFFFFFFll || NL < 1 || NL > 255 || k < 1 || sel_cap < 0)
        return OGS_ERR_ARG;
    if (cam->width <= 0 || cam->height <= 0 || !(cam->d_max > 0) || !(cam->s > 0))
        return OGS_ERR_ARG;
    if (scratch_bytes < ogs_lod_select_gated_scratch_bytes(N) || !aligned(scratch, 16) ||
        !aligned(feat, 16))
        return OGS_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    SelArgs a{pos, level, dL, N, NL, k, infer, make_cam(*cam)};
    int nb = (int)((N + kSelChunk - 1) / kSelChunk);
    if (nb < 1) nb = 1;
    Carver cv(scratch);
    uint32_t* tile_count = cv.take<uint32_t>((size_t)nb);
    float* wsel = cv.take<float>((size_t)(N > 0 ? N : 1));
    unsigned char* img = cv.take<unsigned char>(gate::kGImgBytes);
    // the packing launch also resets the frame's counters, so no separate clear runs first
    static_assert(sizeof(ogs_counts) % 8 == 0, "counters cleared as 64-bit words");
    if (aligned(counts, 8)) {
        if (gate::pack_image(*net, img, reinterpret_cast<unsigned long long*>(counts),
                             (int)(sizeof(ogs_counts) / 8), st) != OGS_OK)
            return OGS_ERR_CUDA;
    } else {
        if (cudaMemsetAsync(counts, 0, sizeof(ogs_counts), st) != cudaSuccess) return OGS_ERR_CUDA;
        if (gate::pack_image(*net, img, nullptr, 0, st) != OGS_OK) return OGS_ERR_CUDA;
    }
    if (cudaFuncSetAttribute(select_eval_gated, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kSgSmem) != cudaSuccess)
        return OGS_ERR_CUDA;
    const int bulk = aligned(pos, 16) && aligned(dL, 16) && aligned(level, 16);
    const int grid = nb < 3 * kSmCount ? nb : 3 * kSmCount;
    launch_pdl(select_eval_gated, dim3(grid), dim3(kSelThreads), kSgSmem, st,
               a, feat, img, p_star, wsel, tile_count, counts, bulk);
    launch_pdl(select_scan, dim3(1), dim3(1024), 0, st, tile_count, nb, sel_cap, k, counts);
    launch_pdl(select_scatter, dim3(nb), dim3(kSelThreads), 0, st,
               wsel, tile_count, N, sel_idx, sel_w, sel_cap);
    return launch_status();
}

extern "C" const char* ogs_version(void) { return "ogs-gb300 0.1 (sm_103a)"; }
