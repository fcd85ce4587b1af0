// Anchor selection by octree level (Sec. 4.1.3, Eq. for L_hat) with the inference-time
// opacity blending of the next level, followed by an order-preserving compaction.
//
// HBM-bound streaming pass over the anchor SoA (pos 12 B + level 1 B + dL 4 B per anchor),
// read once, in two kernels:
//   select_tiles  persistent CTAs (three per SM) walk 2048-anchor tiles; each tile's arrays
//                 land in shared memory by TMA bulk copies, double-buffered so that the next
//                 tile's copy is in flight while the current one is evaluated; the tile's kept
//                 anchors (index and weight) are written compacted, in ascending order, to the
//                 tile's slot of a staging area, with the tile's count;
//   select_emit   one CTA per tile sums the counts of the tiles before it (its output offset)
//                 and copies its staged entries into place; tile 0 also writes the totals.
// No CTA waits on another, so every tile streams at full rate, and only kept anchors (a few
// percent) are written twice.
#include <cmath>

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
    float lod0;     // log2(d_max / s), formed on the host in double precision
};

// Opacity weight of an anchor at (px, py, pz) with level `lvl` and LOD bias `dl`: 0 if it is
// not kept.  Branch-free (every lane of a warp takes the same path).  The distance enters as
// L* = log2(d_max / (d s)) + dL = log2(d_max / s) - log2(d^2) / 2 + dL: no square root and no
// division, and the fast log2 is within ~1e-7 (absolute) of log2, far inside the decision
// margins the oracle reports.
__device__ __forceinline__ float anchor_weight(const SelArgs& a, float px, float py, float pz,
                                               uint32_t lvl, float dl) {
    const Cam& c = a.cam;
    const float dx = px - c.c[0];
    const float dy = py - c.c[1];
    const float dz = pz - c.c[2];
    // visibility of the anchor centre: in front of the near plane, within 1.3x half-fov
    const float zc = c.R[6] * dx + c.R[7] * dy + c.R[8] * dz;
    const float xc = c.R[0] * dx + c.R[1] * dy + c.R[2] * dz;
    const float yc = c.R[3] * dx + c.R[4] * dy + c.R[5] * dz;
    const bool vis = zc > c.znear && !(fabsf(xc) > c.limx * zc) && !(fabsf(yc) > c.limy * zc);
    // fractional level from the viewing distance plus the anchor's LOD bias, clamped
    const float d2 = dx * dx + dy * dy + dz * dz;
    const float Lraw = fmaf(-0.5f, __log2f(d2), a.lod0) + dl;
    const float Ls = fminf(fmaxf(Lraw, 0.0f), (float)(a.NL - 1));
    const float Lh = floorf(Ls);
    const float L = (float)lvl;
    const float wnext = (a.infer && L == Lh + 1.0f && Ls > Lh) ? Ls - Lh : 0.0f;
    const float w = L <= Lh ? 1.0f : wnext;
    return vis ? w : 0.0f;
}

// Thread t of a tile owns its kSelItems consecutive anchors kSelItems * t + it.
// Their opacity weights (0 = not kept) from the staged SoA: positions as six 16-byte shared
// loads, LOD biases as two and levels as one 8-byte load.
__device__ __forceinline__ void tile_weights(const SelArgs& a, const float* s_pos,
                                             const float* s_dl, const uint8_t* s_lvl, int n_here,
                                             float (&wv)[kSelItems]) {
    static_assert(kSelItems == 8, "eight consecutive anchors per thread");
    const int l0 = kSelItems * threadIdx.x;
    float p[3 * kSelItems], dl[kSelItems];
    const float4* p4 = reinterpret_cast<const float4*>(s_pos + 3 * l0);
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        const float4 v = p4[q];
        p[4 * q] = v.x; p[4 * q + 1] = v.y; p[4 * q + 2] = v.z; p[4 * q + 3] = v.w;
    }
    const float4 d0 = reinterpret_cast<const float4*>(s_dl + l0)[0];
    const float4 d1 = reinterpret_cast<const float4*>(s_dl + l0)[1];
    dl[0] = d0.x; dl[1] = d0.y; dl[2] = d0.z; dl[3] = d0.w;
    dl[4] = d1.x; dl[5] = d1.y; dl[6] = d1.z; dl[7] = d1.w;
    const uint2 lv = *reinterpret_cast<const uint2*>(s_lvl + l0);
#pragma unroll
    for (int it = 0; it < kSelItems; ++it) {
        const uint32_t lvl = ((it < 4 ? lv.x : lv.y) >> (8 * (it & 3))) & 0xFFu;
        const float w = anchor_weight(a, p[3 * it], p[3 * it + 1], p[3 * it + 2], lvl, dl[it]);
        wv[it] = l0 + it < n_here ? w : 0.0f;
    }
}

// Writes a tile's kept anchors (weight > 0) compacted in ascending order: thread t owns the
// consecutive anchors kSelItems * t + it, so its rank is the block's exclusive scan of the
// per-thread counts.  s_wc (kSelWarps + 1 words) is scratch; ends with a barrier.
__device__ __forceinline__ uint32_t stage_tile(const float (&wv)[kSelItems], int64_t base,
                                               uint32_t* __restrict__ st_idx,
                                               float* __restrict__ st_w, uint32_t* s_wc) {
    const int t = threadIdx.x;
    const unsigned warp = t >> 5, lane = lane_id();
    uint32_t cnt = 0;
#pragma unroll
    for (int it = 0; it < kSelItems; ++it) cnt += wv[it] > 0.0f ? 1u : 0u;
    uint32_t x = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= (unsigned)o) x += y;
    }
    if (lane == 31) s_wc[warp] = x;
    __syncthreads();
    uint32_t r = x - cnt, total = 0;
#pragma unroll
    for (int w = 0; w < kSelWarps; ++w) {
        const uint32_t c = s_wc[w];
        r += w < (int)warp ? c : 0u;
        total += c;
    }
    const int64_t a0 = base + kSelItems * t;
#pragma unroll
    for (int it = 0; it < kSelItems; ++it) {
        if (wv[it] > 0.0f) {
            st_idx[r] = (uint32_t)(a0 + it);
            st_w[r] = wv[it];
            ++r;
        }
    }
    __syncthreads();                                  // s_wc free for the next tile
    return total;
}

// Pass 1: persistent CTAs walk the tiles tile = blockIdx.x + i * gridDim.x.  Full tiles of
// aligned arrays arrive by three bulk copies into one of two shared-memory stages: the copy of
// tile i + 1 is issued before tile i is evaluated (its stage was released by the barrier that
// ended tile i - 1).  Partial tiles and unaligned arrays use plain loads.
constexpr int kStStageBytes = (3 * 4 + 4 + 1) * kSelChunk;      // pos, dL, level
constexpr int kStSmem = 2 * kStStageBytes;

struct Stage {
    float* pos;
    float* dl;
    uint8_t* lvl;
};

__device__ __forceinline__ Stage stage_of(unsigned char* sm, int s) {
    unsigned char* b = sm + s * kStStageBytes;
    return Stage{reinterpret_cast<float*>(b), reinterpret_cast<float*>(b + 12 * kSelChunk),
                 b + 16 * kSelChunk};
}

__device__ __forceinline__ void issue_tile(const SelArgs& a, int64_t tile, const Stage& st,
                                           uint64_t* mbar) {
    const int64_t base = tile * kSelChunk;
    tc::mbar_expect_tx(mbar, kStStageBytes);
    tc::bulk_load(st.pos, a.pos + 3 * base, 3 * 4 * kSelChunk, mbar);
    tc::bulk_load(st.dl, a.dL + base, 4 * kSelChunk, mbar);
    tc::bulk_load(st.lvl, a.level + base, kSelChunk, mbar);
}

// Waits for a tile's copies (bounded; on expiry flags the timeout and waits once more, as the
// copies may still be landing) or loads a partial / unaligned tile with plain loads.
// `phases` holds the parity to wait for of stage s in bit s.
__device__ __forceinline__ void land_tile(const SelArgs& a, int64_t base, int n_here, bool full,
                                          const Stage& st, uint64_t* mbar, int s,
                                          uint32_t& phases, ogs_counts* counts) {
    if (full) {
        const uint32_t parity = (phases >> s) & 1u;
        if (!tc::mbar_wait(mbar, parity, kSpinLimit)) {
            if (threadIdx.x == 0) atomicExch(&counts->timeout, 1u);
            tc::mbar_wait(mbar, parity, kSpinLimit);
        }
        phases ^= 1u << s;
    } else {
        for (int e = threadIdx.x; e < 3 * n_here; e += kSelThreads) st.pos[e] = a.pos[3 * base + e];
        for (int e = threadIdx.x; e < n_here; e += kSelThreads) {
            st.dl[e] = a.dL[base + e];
            st.lvl[e] = a.level[base + e];
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kSelThreads, 3) select_tiles(SelArgs a,
                                                               uint32_t* __restrict__ st_idx,
                                                               float* __restrict__ st_w,
                                                               uint32_t* __restrict__ tile_count,
                                                               ogs_counts* counts, int bulk) {
    pdl_wait();
    pdl_trigger();
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t s_wc[kSelWarps];
    const int t = threadIdx.x;
    const int64_t nb = (a.N + kSelChunk - 1) / kSelChunk;
    auto full = [&](int64_t tile) { return bulk && (tile + 1) * kSelChunk <= a.N; };
    if (t == 0) {
        tc::mbar_init(&mbar[0], 1);
        tc::mbar_init(&mbar[1], 1);
        if (blockIdx.x < nb && full(blockIdx.x)) issue_tile(a, blockIdx.x, stage_of(sm, 0), &mbar[0]);
    }
    __syncthreads();
    uint32_t phases = 0u;
    int s = 0;
    for (int64_t tile = blockIdx.x; tile < nb; tile += gridDim.x, s ^= 1) {
        const int64_t next = tile + gridDim.x;
        if (t == 0 && next < nb && full(next)) issue_tile(a, next, stage_of(sm, s ^ 1), &mbar[s ^ 1]);
        const int64_t base = tile * kSelChunk;
        const int n_here = (int)min((int64_t)kSelChunk, a.N - base);
        const Stage st = stage_of(sm, s);
        land_tile(a, base, n_here, full(tile), st, &mbar[s], s, phases, counts);
        float wv[kSelItems];
        tile_weights(a, st.pos, st.dl, st.lvl, n_here, wv);
        const uint32_t n = stage_tile(wv, base, st_idx + base, st_w + base, s_wc);
        if (t == 0) tile_count[tile] = n;
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
    float p_star, uint32_t* __restrict__ st_idx, float* __restrict__ st_w,
    uint32_t* __restrict__ tile_count, ogs_counts* counts, int bulk) {
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
        tile_weights(a, s_pos, s_dl, s_lvl, n_here, wv);
#pragma unroll
        for (int it = 0; it < kSelItems; ++it) {
            if (wv[it] > 0.0f) {
                const int l = kSelItems * t + it;
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
#pragma unroll
        for (int it = 0; it < kSelItems; ++it)
            if (gated && wv[it] > 0.0f && s_drop[kSelItems * t + it]) wv[it] = 0.0f;
        // a gate that stopped early: the staged arrays are free only now
        if (!issued && t == 0 && prefetch) sg_issue_tile(a, next, s_pos, s_dl, s_lvl, &mbar);
        const uint32_t n = stage_tile(wv, base, st_idx + base, st_w + base, s_wc);
        if (t == 0) tile_count[tile] = n;
    }
    tc::fence_before_sync();
    __syncthreads();
    if ((t >> 5) == 0) tc::tmem_dealloc(tbase, gate::kGTmemCols);
}

// Pass 2: one CTA per tile.  Its output offset is the sum of the counts of the tiles before
// it (each CTA reads them itself: at most a few thousand words, from L2); its staged entries
// are copied to sel_idx / sel_w at that offset, up to the capacity.  Tile 0 also sums every
// count and writes M, the Gaussian count and the overflow state.
constexpr int kEmitThreads = 256;

__global__ void __launch_bounds__(kEmitThreads) select_emit(const uint32_t* __restrict__ tile_count,
                                                            int nb,
                                                            const uint32_t* __restrict__ st_idx,
                                                            const float* __restrict__ st_w,
                                                            uint32_t* __restrict__ sel_idx,
                                                            float* __restrict__ sel_w, int64_t cap,
                                                            int k, ogs_counts* counts) {
    pdl_wait();
    pdl_trigger();
    __shared__ unsigned long long s_part[kEmitThreads / 32];
    const int tile = blockIdx.x;
    const uint32_t n = tile_count[tile];
    if (n == 0 && tile != 0) return;
    const int upto = tile == 0 ? nb : tile;       // tile 0 sums everything (the total)
    unsigned long long part = 0;
    for (int i = threadIdx.x; i < upto; i += kEmitThreads) part += tile_count[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if (lane_id() == 0) s_part[threadIdx.x >> 5] = part;
    __syncthreads();
    unsigned long long sum = 0;
#pragma unroll
    for (int w = 0; w < kEmitThreads / 32; ++w) sum += s_part[w];
    const unsigned long long off = tile == 0 ? 0 : sum;
    if (tile == 0 && threadIdx.x == 0) {
        const unsigned long long total = sum;
        const uint32_t m = total > (unsigned long long)cap ? (uint32_t)cap : (uint32_t)total;
        counts->n_selected = m;
        counts->n_gaussians = m * (uint32_t)k;
        counts->need_selected = total > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)total;
        if (total > (unsigned long long)cap) atomicOr(&counts->overflow, 1u);
    }
    const size_t src = (size_t)tile * kSelChunk;
    for (uint32_t r = threadIdx.x; r < n; r += kEmitThreads) {
        const unsigned long long p = off + r;
        if (p < (unsigned long long)cap) {
            sel_idx[p] = st_idx[src + r];
            sel_w[p] = st_w[src + r];
        }
    }
}

}  // namespace
}  // namespace ogs

using namespace ogs;

namespace ogs {
namespace {

// scratch: per-tile counts, then the staging area (one 2048-entry slot per tile) of indices
// and weights
struct SelScratch {
    uint32_t* tile_count;
    uint32_t* st_idx;
    float* st_w;
};

size_t sel_layout(int64_t N, void* base, SelScratch* s) {
    const int64_t nb = (N + kSelChunk - 1) / kSelChunk;
    const size_t slots = (size_t)(nb < 1 ? 1 : nb) * kSelChunk;
    Carver cv(base);
    SelScratch t;
    t.tile_count = cv.take<uint32_t>((size_t)(nb < 1 ? 1 : nb));
    t.st_idx = cv.take<uint32_t>(slots);
    t.st_w = cv.take<float>(slots);
    if (s) *s = t;
    return cv.off + 256;
}

// persistent grid of the tile passes: three CTAs per SM, never more than the tiles
int tile_grid(int nb) { return nb < 3 * kSmCount ? nb : 3 * kSmCount; }

}  // namespace
}  // namespace ogs

extern "C" size_t ogs_lod_select_scratch_bytes(int64_t N) {
    return sel_layout(N < 0 ? 0 : N, nullptr, nullptr);
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
    SelArgs a{pos, level, dL, N, NL, k, infer, make_cam(*cam),
              (float)std::log2((double)cam->d_max / (double)cam->s)};
    int nb = (int)((N + kSelChunk - 1) / kSelChunk);
    if (nb < 1) nb = 1;
    SelScratch sc;
    sel_layout(N, scratch, &sc);
    const int bulk = aligned(pos, 16) && aligned(dL, 16) && aligned(level, 16);
    if (cudaFuncSetAttribute(select_tiles, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kStSmem) != cudaSuccess)
        return OGS_ERR_CUDA;
    if (N == 0 &&
        cudaMemsetAsync(sc.tile_count, 0, sizeof(uint32_t), st) != cudaSuccess)
        return OGS_ERR_CUDA;
    launch_pdl(select_tiles, dim3(tile_grid(nb)), dim3(kSelThreads), kStSmem, st, a, sc.st_idx,
               sc.st_w, sc.tile_count, counts, bulk);
    launch_pdl(select_emit, dim3(nb), dim3(kEmitThreads), 0, st, (const uint32_t*)sc.tile_count,
               nb, (const uint32_t*)sc.st_idx, (const float*)sc.st_w, sel_idx, sel_w, sel_cap, k,
               counts);
    return launch_status();
}

extern "C" size_t ogs_lod_select_gated_scratch_bytes(int64_t N) {
    return ((ogs_lod_select_scratch_bytes(N) + 255) & ~(size_t)255) + gate::kGImgBytes + 256;
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
    SelArgs a{pos, level, dL, N, NL, k, infer, make_cam(*cam),
              (float)std::log2((double)cam->d_max / (double)cam->s)};
    int nb = (int)((N + kSelChunk - 1) / kSelChunk);
    if (nb < 1) nb = 1;
    SelScratch sc;
    const size_t sel_bytes = sel_layout(N, scratch, &sc);
    unsigned char* img = static_cast<unsigned char*>(scratch) + ((sel_bytes + 255) & ~(size_t)255);
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
    if (N == 0 &&
        cudaMemsetAsync(sc.tile_count, 0, sizeof(uint32_t), st) != cudaSuccess)
        return OGS_ERR_CUDA;
    launch_pdl(select_eval_gated, dim3(tile_grid(nb)), dim3(kSelThreads), kSgSmem, st,
               a, feat, img, p_star, sc.st_idx, sc.st_w, sc.tile_count, counts, bulk);
    launch_pdl(select_emit, dim3(nb), dim3(kEmitThreads), 0, st, (const uint32_t*)sc.tile_count,
               nb, (const uint32_t*)sc.st_idx, (const float*)sc.st_w, sel_idx, sel_w, sel_cap, k,
               counts);
    return launch_status();
}

extern "C" const char* ogs_version(void) { return "ogs-gb300 0.1 (sm_103a)"; }
