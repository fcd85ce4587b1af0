// Backward of the front-to-back blending (Sec. 3.1, Eq. 2).
//
// With C = sum_i c_i a_i T_i + T_{n+1} bg:  dC/dc_i = a_i T_i and dC/da_i = T_i (c_i - S_i),
// where S_i is the colour accumulated behind Gaussian i (S_n = bg, S_{i-1} = a_i c_i +
// (1 - a_i) S_i).  Each pixel replays its list back to front from its last blended entry,
// recovering T_i = T_{i+1} / (1 - a_i) from the final transmittance instead of storing
// per-pair values (1 - a_i >= 0.01 because a is clamped to 0.99).  a = min(0.99, o G) has
// zero derivative where clamped.  Same tile/pixel mapping and skip test as the forward (two
// pixels per thread, each warp walking only the records whose alpha >= 1/255 ellipse can
// reach its 8x8 block); a thread's two contributions are summed, then a warp's nine sums
// with a recursive-halving shuffle reduction, and nine lanes add them with one atomic
// instruction per warp and Gaussian.
#include "blend_common.cuh"

namespace ogs {
namespace {

using namespace blend;

// Sums each of 16 per-lane values over the warp by recursive halving: at every step a lane
// keeps half of its values and sends the other half to its partner, so 8 + 4 + 2 + 1 + 1
// shuffles replace 16 x 5.  On return, lane 2k holds the warp total of value k.
__device__ __forceinline__ float warp_sum16(float (&v)[16]) {
    const unsigned lane = lane_id();
#pragma unroll
    for (int half = 8; half >= 1; half >>= 1) {
        const bool upper = lane & (2u * half);          // partner at xor 2*half
#pragma unroll
        for (int i = 0; i < half; ++i) {
            const float send = upper ? v[i] : v[half + i];
            const float keep = upper ? v[half + i] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 2 * half);
        }
    }
    return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

// one pixel's contribution of one Gaussian, accumulated into g[0..8] (g[9..15] stay 0):
// du dv da db dc do dr dg db (w.r.t. the unscaled record)
struct PixState {
    float T, S0, S1, S2, d0, d1, d2;
    int last;
};

__device__ __forceinline__ bool pixel_step(PixState& s, int idx, float p2, const float4& A,
                                           const float4& B, const float2& Cc, float dx, float dy,
                                           float (&g)[16]) {
    if (idx >= s.last || !(p2 <= 0.f && p2 >= Cc.y)) return false;
    const float G = ex2(p2);
    const float raw = __fmul_rn(B.y, G);            // the forward's raw_alpha(o, p2)
    const float alpha = fminf(0.99f, raw);
    s.T = __fdividef(s.T, 1.0f - alpha);            // T_i, before this Gaussian
    const float wgt = alpha * s.T;
    g[6] += wgt * s.d0; g[7] += wgt * s.d1; g[8] += wgt * s.d2;
    const float dalpha = s.T * ((B.z - s.S0) * s.d0 + (B.w - s.S1) * s.d1 + (Cc.x - s.S2) * s.d2);
    s.S0 = alpha * B.z + (1.0f - alpha) * s.S0;
    s.S1 = alpha * B.w + (1.0f - alpha) * s.S1;
    s.S2 = alpha * Cc.x + (1.0f - alpha) * s.S2;
    if (raw < 0.99f) {
        // d alpha / d power = alpha, d alpha / d o = G; the record's conic is (a, b, c) with
        // power = -0.5 (a dx^2 + c dy^2) - b dx dy, recovered from a2 = -0.5 a log2e,
        // b2 = -b log2e, c2 = -0.5 c log2e
        g[5] += dalpha * G;
        const float dp = dalpha * alpha;
        constexpr float kA = -1.3862943611198906f;     // -2 / log2(e) = -2 ln 2
        constexpr float kB = -0.6931471805599453f;     // -1 / log2(e) = -ln 2
        const float a = A.z * kA, b = A.w * kB, c = B.x * kA;
        g[0] += -dp * (a * dx + b * dy);
        g[1] += -dp * (c * dy + b * dx);
        g[2] += -0.5f * dp * dx * dx;
        g[3] += -dp * dx * dy;
        g[4] += -0.5f * dp * dy * dy;
    }
    return true;
}

__global__ void __launch_bounds__(kThreads) blend_bwd_kernel(
    const float4* __restrict__ rec, const uint32_t* __restrict__ pair_gauss,
    const uint2* __restrict__ tile_range, int W, int H, int gx, float bg0, float bg1, float bg2,
    const float* __restrict__ T_final, const uint32_t* __restrict__ n_last,
    const float* __restrict__ dimg, float* __restrict__ drec) {
    __shared__ float4 s_a[kBatch];
    __shared__ float4 s_b[kBatch];
    __shared__ float2 s_c[kBatch];
    __shared__ uint32_t s_g[kBatch];
    __shared__ uint8_t s_m[kBatch];
    __shared__ uint8_t s_list[kThreads / 32][kBatch];
    __shared__ int s_maxlast;
    const int tile = blockIdx.x;
    int lx, ly;
    pixels_of(threadIdx.x, lx, ly);
    const int tx0 = (tile % gx) * kTile, ty0 = (tile / gx) * kTile;
    const int px = tx0 + lx;
    const int py = ty0 + ly;
    uint8_t* list = s_list[threadIdx.x >> 5];
    const float fx = (float)px, fy = (float)py;
    const uint2 range = tile_range[tile];
    const size_t plane = (size_t)W * H;
    PixState q[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        q[i] = PixState{1.f, bg0, bg1, bg2, 0.f, 0.f, 0.f, 0};
        if (px < W && py + i < H) {
            const size_t pix = (size_t)(py + i) * W + px;
            q[i].last = (int)n_last[pix];
            q[i].T = T_final[pix];
            q[i].d0 = dimg[pix]; q[i].d1 = dimg[plane + pix]; q[i].d2 = dimg[2 * plane + pix];
        }
    }
    if (threadIdx.x == 0) s_maxlast = 0;
    __syncthreads();
    atomicMax(&s_maxlast, max(q[0].last, q[1].last));
    __syncthreads();
    const int n = s_maxlast;           // entries beyond every pixel's last blend are unused
    const unsigned lane = lane_id();
    for (int top = n; top > 0; top -= kBatch) {
        const int lo = max(top - kBatch, 0);
        __syncthreads();
        for (int e = threadIdx.x; lo + e < top; e += kThreads) {
            const uint32_t g = pair_gauss[range.x + lo + e];
            const Rec r = load_rec(rec, g, (float)tx0, (float)ty0);
            s_g[e] = g;
            s_a[e] = r.A;
            s_b[e] = r.B;
            s_c[e] = r.C;
            s_m[e] = (uint8_t)r.blocks;
        }
        __syncthreads();
        const int nw = warp_list(s_m, top - lo, list);
        for (int it = nw - 1; it >= 0; --it) {
            const int j = list[it];
            const int idx = lo + j;        // list position of this entry
            const float4 A = s_a[j];
            const float4 B = s_b[j];
            const float2 Cc = s_c[j];
            const float dx = A.x - fx;
            const float dy0 = A.y - fy, dy1 = dy0 - 1.0f;
            const float ax = __fmul_rn(A.z, dx);
            float g[16] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f,
                           0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            bool act = pixel_step(q[0], idx, power2(ax, dx, dy0, A.w, B.x), A, B, Cc, dx, dy0, g);
            act |= pixel_step(q[1], idx, power2(ax, dx, dy1, A.w, B.x), A, B, Cc, dx, dy1, g);
            if (__any_sync(0xffffffffu, act)) {
                const float tot = warp_sum16(g);
                // lane 2c adds component c: one atomic instruction for the nine sums
                if ((lane & 1u) == 0 && (lane >> 1) < 9)
                    atomicAdd(drec + 9 * (size_t)s_g[j] + (lane >> 1), tot);
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
    blend_bwd_kernel<<<gx * gy, blend::kThreads, 0, (cudaStream_t)stream>>>(
        reinterpret_cast<const float4*>(rec), pair_gauss,
        reinterpret_cast<const uint2*>(tile_range), width, height, gx, bg[0], bg[1], bg[2],
        T_final, n_last, dimg, drec);
    return launch_status();
}
