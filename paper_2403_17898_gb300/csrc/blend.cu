// Front-to-back alpha blending per 16x16 tile (Sec. 3.1, Eq. 2).
//
// One CTA of 4 warps per tile; each thread blends two vertically adjacent pixels (warps cover
// compact 8x8 blocks, so pixels that saturate together share a warp).  The tile's list is
// consumed in batches of 256 records gathered into shared memory, converted once per batch to
// pre-scaled coefficients and to a mask of the 8x8 blocks that the record's alpha >= 1/255
// ellipse can reach; each warp then walks, in list order, only the records whose mask holds
// its block.  One (pixel, Gaussian) evaluation is: offset, a 5-operation quadratic form, the
// exponent-bound skip test, one ex2 and the compositing update, done branch-free: a pixel that
// skips the Gaussian (or saturates on it) adds a zero weight and keeps its transmittance, which
// leaves its sums bit-for-bit as a skipped update would.  Lanes of a warp therefore never
// diverge inside the walk.  A warp stops walking once all its pixels have saturated (checked
// every 128 records) and the CTA stops loading batches once all of its pixels have.  The
// kernel is bound by instruction issue (FP32 + MUFU), not by memory.  The optional n_eval
// output counts, per pixel, the (pixel, Gaussian) tests the kernel made while the pixel still
// needed them: the entries of its warp block's list up to the one it saturated on.
#include "blend_common.cuh"

namespace ogs {
namespace {

using namespace blend;

constexpr int kExitEvery = 128;  // records walked between two warp-wide saturation checks

// One pixel's compositing step with Gaussian `idx - 1` of the list, branch-free.  Returns the
// weight alpha T added to the pixel (0 when it skipped the Gaussian or saturated on it).
template <bool kEval, bool kLast>
__device__ __forceinline__ float composite(float p2, float o, float cr, float cg, float cb,
                                           float pskip2, int idx, bool& done, float& T,
                                           float& C0, float& C1, float& C2, int& last,
                                           int& tests) {
    if (kEval) tests += done ? 0 : 1;               // a test this pixel still needed
    // skip if power > 0 or alpha < 1/255 (power2 < pskip2)
    const bool pass = !done && p2 <= 0.f && p2 >= pskip2;
    const float alpha = fminf(0.99f, raw_alpha(o, p2));
    const float w = alpha * T;
    const float Tn = T - w;                         // T (1 - alpha)
    const bool sat = pass && Tn < 1e-4f;            // this Gaussian would saturate the pixel
    const bool apply = pass && !sat;
    const float wgt = apply ? w : 0.0f;
    C0 = fmaf(cr, wgt, C0);
    C1 = fmaf(cg, wgt, C1);
    C2 = fmaf(cb, wgt, C2);
    T = apply ? Tn : T;
    if (kLast) last = apply ? idx : last;
    done = done || sat;
    return wgt;
}

template <bool kMaxC, bool kEval, bool kLast>
__global__ void __launch_bounds__(kThreads) blend_fwd_kernel(
    const float4* __restrict__ rec, const uint32_t* __restrict__ pair_gauss,
    const uint2* __restrict__ tile_range, int W, int H, int gx, float bg0, float bg1, float bg2,
    float* __restrict__ img, float* __restrict__ T_final, uint32_t* __restrict__ n_last,
    uint32_t* __restrict__ n_eval, const uint32_t* __restrict__ sel_idx, int k,
    uint32_t* __restrict__ maxc) {
    pdl_wait();
    pdl_trigger();
    __shared__ float4 s_a[kBatch];
    __shared__ float4 s_b[kBatch];
    __shared__ float2 s_c[kBatch];
    __shared__ uint8_t s_m[kBatch];
    __shared__ uint8_t s_list[kThreads / 32][kBatch];
    __shared__ uint32_t s_anchor[kMaxC ? kBatch : 1];
    const int tile = blockIdx.x;
    int lx, ly;
    pixels_of(threadIdx.x, lx, ly);
    const int tx0 = (tile % gx) * kTile, ty0 = (tile / gx) * kTile;
    const int px = tx0 + lx;
    const int py = ty0 + ly;
    const bool in0 = px < W && py < H, in1 = px < W && py + 1 < H;
    const float fx = (float)px, fy = (float)py;
    const uint2 range = tile_range[tile];
    const int n = (int)(range.y - range.x);
    uint8_t* list = s_list[threadIdx.x >> 5];
    float T0 = 1.f, T1 = 1.f, C00 = 0.f, C01 = 0.f, C02 = 0.f, C10 = 0.f, C11 = 0.f, C12 = 0.f;
    int last0 = 0, last1 = 0, tests0 = 0, tests1 = 0;
    bool done0 = !in0, done1 = !in1;
    for (int b0 = 0; b0 < n; b0 += kBatch) {
        if (__syncthreads_count(done0 && done1) == kThreads) break;
        for (int e = threadIdx.x; e < kBatch && b0 + e < n; e += kThreads) {
            const uint32_t g = pair_gauss[range.x + b0 + e];
            const Rec r = load_rec(rec, g, (float)tx0, (float)ty0);
            s_a[e] = r.A;
            s_b[e] = r.B;
            s_c[e] = r.C;
            s_m[e] = (uint8_t)r.blocks;
            if (kMaxC) s_anchor[e] = sel_idx[g / (uint32_t)k];
        }
        __syncthreads();
        const int cnt = min(kBatch, n - b0);
        const int nw = warp_list(s_m, cnt, list);
        for (int q0 = 0; q0 < nw; q0 += kExitEvery) {
            if (__all_sync(0xffffffffu, done0 && done1)) break;
            const int q1 = min(q0 + kExitEvery, nw);
            for (int q = q0; q < q1; ++q) {
                const int j = list[q];
                const float4 A = s_a[j];
                const float4 B = s_b[j];
                const float2 Cc = s_c[j];
                const float dx = A.x - fx;
                const float dy0 = A.y - fy, dy1 = dy0 - 1.0f;
                const float ax = __fmul_rn(A.z, dx);
                const float p0 = power2(ax, dx, dy0, A.w, B.x);
                const float p1 = power2(ax, dx, dy1, A.w, B.x);
                const int idx = b0 + j + 1;
                const float c0 = composite<kEval, kLast>(p0, B.y, B.z, B.w, Cc.x, Cc.y, idx, done0, T0,
                                                  C00, C01, C02, last0, tests0);
                const float c1 = composite<kEval, kLast>(p1, B.y, B.z, B.w, Cc.x, Cc.y, idx, done1, T1,
                                                  C10, C11, C12, last1, tests1);
                if (kMaxC) {
                    // contributions are >= 0, so their float bits order like unsigned ints
                    const uint32_t m = __reduce_max_sync(0xffffffffu,
                                                         __float_as_uint(fmaxf(c0, c1)));
                    if (lane_id() == 0 && m) atomicMax(&maxc[s_anchor[j]], m);
                }
            }
        }
    }
    const size_t plane = (size_t)W * H;
    if (in0) {
        const size_t pix = (size_t)py * W + px;
        img[pix] = C00 + T0 * bg0;
        img[plane + pix] = C01 + T0 * bg1;
        img[2 * plane + pix] = C02 + T0 * bg2;
        T_final[pix] = T0;
        if (kLast) n_last[pix] = (uint32_t)last0;
        if (kEval) n_eval[pix] = (uint32_t)tests0;
    }
    if (in1) {
        const size_t pix = (size_t)(py + 1) * W + px;
        img[pix] = C10 + T1 * bg0;
        img[plane + pix] = C11 + T1 * bg1;
        img[2 * plane + pix] = C12 + T1 * bg2;
        T_final[pix] = T1;
        if (kLast) n_last[pix] = (uint32_t)last1;
        if (kEval) n_eval[pix] = (uint32_t)tests1;
    }
}

}  // namespace
}  // namespace ogs

using namespace ogs;

extern "C" ogs_status ogs_blend_fwd(const ogs_rec2d* rec, const uint32_t* pair_gauss,
                                    const uint32_t* tile_range, int32_t width, int32_t height,
                                    const float* bg, float* img, float* T_final,
                                    uint32_t* n_last, uint32_t* n_eval, const uint32_t* sel_idx,
                                    int32_t k, uint32_t* maxc, void* stream) {
    if (!rec || !pair_gauss || !tile_range || !bg || !img || !T_final) return OGS_ERR_ARG;
    if (width <= 0 || height <= 0 || !aligned(rec, 16) || !aligned(tile_range, 8)) return OGS_ERR_ARG;
    if (maxc && (!sel_idx || k <= 0)) return OGS_ERR_ARG;
    const int gx = (width + kTile - 1) / kTile, gy = (height + kTile - 1) / kTile;
    cudaStream_t st = (cudaStream_t)stream;
    const float4* r = reinterpret_cast<const float4*>(rec);
    const uint2* tr = reinterpret_cast<const uint2*>(tile_range);
    const dim3 grid(gx * gy), block(blend::kThreads);
    const int variant = (maxc ? 4 : 0) | (n_eval ? 2 : 0) | (n_last ? 1 : 0);
#define OGS_BLEND(M, E, L)                                                                     \
    launch_pdl(blend_fwd_kernel<M, E, L>, grid, block, 0, st, r, pair_gauss, tr, width, height, \
               gx, bg[0], bg[1], bg[2], img, T_final, n_last, n_eval, sel_idx, k, maxc)
    switch (variant) {
        case 0: OGS_BLEND(false, false, false); break;
        case 1: OGS_BLEND(false, false, true); break;
        case 2: OGS_BLEND(false, true, false); break;
        case 3: OGS_BLEND(false, true, true); break;
        case 4: OGS_BLEND(true, false, false); break;
        case 5: OGS_BLEND(true, false, true); break;
        case 6: OGS_BLEND(true, true, false); break;
        default: OGS_BLEND(true, true, true); break;
    }
#undef OGS_BLEND
    return launch_status();
}
