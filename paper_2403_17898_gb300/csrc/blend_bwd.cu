// Backward of the front-to-back blending (Sec. 3.1, Eq. 2).
//
// With C = sum_i c_i a_i T_i + T_{n+1} bg:  dC/dc_i = a_i T_i and dC/da_i = T_i (c_i - S_i),
// where S_i is the colour accumulated behind Gaussian i (S_n = bg, S_{i-1} = a_i c_i +
// (1 - a_i) S_i).  Each pixel replays its list back to front from its last blended entry,
// recovering T_i = T_{i+1} / (1 - a_i) from the final transmittance instead of storing
// per-pair values (1 - a_i >= 0.01 because a is clamped to 0.99).  a = min(0.99, o G) has
// zero derivative where clamped.  Per-Gaussian gradients of one warp are summed with
// shuffles before a single atomic add per warp and Gaussian.
#include "internal.cuh"

namespace ogs {
namespace {

constexpr int kBwdThreads = kTile * kTile;

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(kBwdThreads) blend_bwd_kernel(
    const float4* __restrict__ rec, const uint32_t* __restrict__ pair_gauss,
    const uint2* __restrict__ tile_range, int W, int H, int gx, float bg0, float bg1, float bg2,
    const float* __restrict__ T_final, const uint32_t* __restrict__ n_last,
    const float* __restrict__ dimg, float* __restrict__ drec) {
    __shared__ float4 s_a[kBwdThreads];
    __shared__ float4 s_b[kBwdThreads];
    __shared__ float s_c[kBwdThreads];
    __shared__ float s_p[kBwdThreads];
    __shared__ uint32_t s_g[kBwdThreads];
    __shared__ int s_maxlast;
    const int tile = blockIdx.x;
    const int tx = tile % gx, ty = tile / gx;
    const int px = tx * kTile + (threadIdx.x & (kTile - 1));
    const int py = ty * kTile + (threadIdx.x >> 4);
    const bool inside = px < W && py < H;
    const float fx = (float)px, fy = (float)py;
    const uint2 range = tile_range[tile];
    const size_t pix = (size_t)py * W + px, plane = (size_t)W * H;
    int last = 0;
    float T = 1.0f, d0 = 0.f, d1 = 0.f, d2 = 0.f;
    if (inside) {
        last = (int)n_last[pix];
        T = T_final[pix];
        d0 = dimg[pix]; d1 = dimg[plane + pix]; d2 = dimg[2 * plane + pix];
    }
    if (threadIdx.x == 0) s_maxlast = 0;
    __syncthreads();
    atomicMax(&s_maxlast, last);
    __syncthreads();
    const int n = s_maxlast;           // entries beyond every pixel's last blend are unused
    float S0 = bg0, S1 = bg1, S2 = bg2;
    const unsigned lane = lane_id();
    for (int top = n; top > 0; top -= kBwdThreads) {
        const int lo = max(top - kBwdThreads, 0);
        const int e = lo + threadIdx.x;
        __syncthreads();
        if (e < top) {
            const uint32_t g = pair_gauss[range.x + e];
            s_g[threadIdx.x] = g;
            s_a[threadIdx.x] = rec[3 * (size_t)g];
            s_b[threadIdx.x] = rec[3 * (size_t)g + 1];
            const float4 C = rec[3 * (size_t)g + 2];
            s_c[threadIdx.x] = C.x;
            s_p[threadIdx.x] = C.w;
        }
        __syncthreads();
        for (int j = top - lo - 1; j >= 0; --j) {
            const int idx = lo + j;        // list position of this entry
            float gu = 0.f, gv = 0.f, ga = 0.f, gb = 0.f, gc = 0.f, go = 0.f;
            float gr = 0.f, gg = 0.f, gbl = 0.f;
            bool act = false;
            if (idx < last) {
                const float4 A = s_a[j];
                const float4 B = s_b[j];
                const float dx = A.x - fx, dy = A.y - fy;
                const float power = -0.5f * (A.z * dx * dx + B.x * dy * dy) - A.w * dx * dy;
                // the forward's skip test, bit for bit: power > 0 or alpha < 1/255
                if (power <= 0.0f && power >= s_p[j]) {
                    const float G = __expf(power);
                    const float raw = B.y * G;
                    const float alpha = fminf(0.99f, raw);
                    {
                        act = true;
                        T = T / (1.0f - alpha);               // T_i, before this Gaussian
                        const float cb = s_c[j];
                        const float wgt = alpha * T;
                        gr = wgt * d0; gg = wgt * d1; gbl = wgt * d2;
                        const float dalpha = T * ((B.z - S0) * d0 + (B.w - S1) * d1 + (cb - S2) * d2);
                        S0 = alpha * B.z + (1.0f - alpha) * S0;
                        S1 = alpha * B.w + (1.0f - alpha) * S1;
                        S2 = alpha * cb + (1.0f - alpha) * S2;
                        if (raw < 0.99f) {
                            go = dalpha * G;
                            const float dp = dalpha * alpha;
                            gu = -dp * (A.z * dx + A.w * dy);
                            gv = -dp * (B.x * dy + A.w * dx);
                            ga = -0.5f * dp * dx * dx;
                            gb = -dp * dx * dy;
                            gc = -0.5f * dp * dy * dy;
                        }
                    }
                }
            }
            if (__any_sync(0xffffffffu, act)) {
                gu = warp_sum(gu); gv = warp_sum(gv); ga = warp_sum(ga); gb = warp_sum(gb);
                gc = warp_sum(gc); go = warp_sum(go); gr = warp_sum(gr); gg = warp_sum(gg);
                gbl = warp_sum(gbl);
                if (lane == 0) {
                    float* d = drec + 9 * (size_t)s_g[j];
                    atomicAdd(d + 0, gu); atomicAdd(d + 1, gv); atomicAdd(d + 2, ga);
                    atomicAdd(d + 3, gb); atomicAdd(d + 4, gc); atomicAdd(d + 5, go);
                    atomicAdd(d + 6, gr); atomicAdd(d + 7, gg); atomicAdd(d + 8, gbl);
                }
            }
        }
    }
}

}  // namespace
}  // namespace ogs

using namespace ogs;

extern "C" ogs_status ogs_blend_bwd(const ogs_rec2d* rec, const uint32_t* pair_gauss,
                                    const uint32_t* tile_range, int32_t width, int32_t height,
                                    const float* bg, const float* T_final, const uint32_t* n_last,
                                    const float* dimg, float* drec, void* stream) {
    if (!rec || !pair_gauss || !tile_range || !bg || !T_final || !n_last || !dimg || !drec)
        return OGS_ERR_ARG;
    if (width <= 0 || height <= 0 || !aligned(rec, 16) || !aligned(tile_range, 8)) return OGS_ERR_ARG;
    const int gx = (width + kTile - 1) / kTile, gy = (height + kTile - 1) / kTile;
    blend_bwd_kernel<<<gx * gy, kBwdThreads, 0, (cudaStream_t)stream>>>(
        reinterpret_cast<const float4*>(rec), pair_gauss,
        reinterpret_cast<const uint2*>(tile_range), width, height, gx, bg[0], bg[1], bg[2],
        T_final, n_last, dimg, drec);
    return launch_status();
}
