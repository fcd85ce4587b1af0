// Front-to-back alpha blending per 16x16 tile (Sec. 3.1, Eq. 2).
//
// One CTA per tile, one thread per pixel.  The tile's list is consumed in batches of 256
// records staged through shared memory (one coalesced gather per batch), and the CTA leaves
// as soon as every pixel has saturated (barrier vote).  The inner loop is FP32 FMA plus one
// MUFU ex2 per (pixel, Gaussian) evaluation, so it is bound by issue slots, not HBM.
#include "internal.cuh"

namespace ogs {
namespace {

constexpr int kBlendThreads = kTile * kTile;   // 256

template <bool kMaxC>
__global__ void __launch_bounds__(kBlendThreads) blend_fwd_kernel(
    const float4* __restrict__ rec, const uint32_t* __restrict__ pair_gauss,
    const uint2* __restrict__ tile_range, int W, int H, int gx, float bg0, float bg1, float bg2,
    float* __restrict__ img, float* __restrict__ T_final, uint32_t* __restrict__ n_last,
    uint32_t* __restrict__ n_eval, const uint32_t* __restrict__ sel_idx, int k,
    uint32_t* __restrict__ maxc) {
    __shared__ float4 s_a[kBlendThreads];   // u, v, conic a, conic b
    __shared__ float4 s_b[kBlendThreads];   // conic c, opacity, r, g
    __shared__ float s_c[kBlendThreads];    // b
    __shared__ float s_p[kBlendThreads];    // exponent below which alpha < 1/255
    __shared__ uint32_t s_anchor[kMaxC ? kBlendThreads : 1];
    const int tile = blockIdx.x;
    const int tx = tile % gx, ty = tile / gx;
    const int px = tx * kTile + (threadIdx.x & (kTile - 1));
    const int py = ty * kTile + (threadIdx.x >> 4);
    const bool inside = px < W && py < H;
    const float fx = (float)px, fy = (float)py;
    const uint2 range = tile_range[tile];
    const int n = (int)(range.y - range.x);
    float T = 1.0f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
    uint32_t contributor = 0, last = 0;
    bool done = !inside;
    for (int b0 = 0; b0 < n; b0 += kBlendThreads) {
        if (__syncthreads_count(done) == kBlendThreads) break;
        const int e = b0 + threadIdx.x;
        if (e < n) {
            const uint32_t g = pair_gauss[range.x + e];
            s_a[threadIdx.x] = rec[3 * (size_t)g];
            s_b[threadIdx.x] = rec[3 * (size_t)g + 1];
            const float4 C = rec[3 * (size_t)g + 2];
            s_c[threadIdx.x] = C.x;
            s_p[threadIdx.x] = C.w;
            if (kMaxC) s_anchor[threadIdx.x] = sel_idx[g / (uint32_t)k];
        }
        __syncthreads();
        const int cnt = min(kBlendThreads, n - b0);
        if (!kMaxC) {
            for (int j = 0; !done && j < cnt; ++j) {
                ++contributor;
                const float4 A = s_a[j];
                const float dx = A.x - fx, dy = A.y - fy;
                const float4 B = s_b[j];
                const float power = -0.5f * (A.z * dx * dx + B.x * dy * dy) - A.w * dx * dy;
                if (!(power <= 0.0f && power >= s_p[j])) continue;   // power > 0 or alpha < 1/255
                const float alpha = fminf(0.99f, B.y * __expf(power));
                const float Tn = T * (1.0f - alpha);
                if (Tn < 1e-4f) { done = true; continue; }
                const float wgt = alpha * T;
                C0 = fmaf(B.z, wgt, C0);
                C1 = fmaf(B.w, wgt, C1);
                C2 = fmaf(s_c[j], wgt, C2);
                T = Tn;
                last = contributor;
            }
        } else {
            // warp-uniform loop so that the per-anchor max can be reduced across the warp
            for (int j = 0; j < cnt; ++j) {
                float contrib = 0.0f;
                if (!done) {
                    ++contributor;
                    const float4 A = s_a[j];
                    const float dx = A.x - fx, dy = A.y - fy;
                    const float4 B = s_b[j];
                    const float power = -0.5f * (A.z * dx * dx + B.x * dy * dy) - A.w * dx * dy;
                    if (power <= 0.0f && power >= s_p[j]) {
                        const float alpha = fminf(0.99f, B.y * __expf(power));
                        const float Tn = T * (1.0f - alpha);
                        if (Tn < 1e-4f) {
                            done = true;
                        } else {
                            const float wgt = alpha * T;
                            C0 = fmaf(B.z, wgt, C0);
                            C1 = fmaf(B.w, wgt, C1);
                            C2 = fmaf(s_c[j], wgt, C2);
                            contrib = wgt;
                            T = Tn;
                            last = contributor;
                        }
                    }
                }
                // contributions are >= 0, so their float bits order like unsigned ints
                const uint32_t m = __reduce_max_sync(0xffffffffu, __float_as_uint(contrib));
                if (lane_id() == 0 && m) atomicMax(&maxc[s_anchor[j]], m);
                if (__all_sync(0xffffffffu, done)) break;
            }
        }
    }
    if (inside) {
        const size_t pix = (size_t)py * W + px;
        const size_t plane = (size_t)W * H;
        img[pix] = C0 + T * bg0;
        img[plane + pix] = C1 + T * bg1;
        img[2 * plane + pix] = C2 + T * bg2;
        T_final[pix] = T;
        n_last[pix] = last;
        if (n_eval) n_eval[pix] = contributor;
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
    if (!rec || !pair_gauss || !tile_range || !bg || !img || !T_final || !n_last) return OGS_ERR_ARG;
    if (width <= 0 || height <= 0 || !aligned(rec, 16) || !aligned(tile_range, 8)) return OGS_ERR_ARG;
    if (maxc && (!sel_idx || k <= 0)) return OGS_ERR_ARG;
    const int gx = (width + kTile - 1) / kTile, gy = (height + kTile - 1) / kTile;
    cudaStream_t st = (cudaStream_t)stream;
    const float4* r = reinterpret_cast<const float4*>(rec);
    const uint2* tr = reinterpret_cast<const uint2*>(tile_range);
    if (maxc)
        blend_fwd_kernel<true><<<gx * gy, kBlendThreads, 0, st>>>(
            r, pair_gauss, tr, width, height, gx, bg[0], bg[1], bg[2], img, T_final, n_last,
            n_eval, sel_idx, k, maxc);
    else
        blend_fwd_kernel<false><<<gx * gy, kBlendThreads, 0, st>>>(
            r, pair_gauss, tr, width, height, gx, bg[0], bg[1], bg[2], img, T_final, n_last,
            n_eval, nullptr, 1, nullptr);
    return launch_status();
}
