// Per-tile blending conventions shared by the forward and backward blend kernels, so both
// take every skip decision with the same operations in the same order.  Each warp blends an
// 8x8 block of the tile and walks only the records whose alpha >= 1/255 ellipse can reach it.
#pragma once

#include "internal.cuh"

namespace ogs {
namespace blend {

constexpr int kThreads = 128;            // 4 warps per 16x16 tile
constexpr int kBatch = 256;              // records staged per shared-memory batch
constexpr float kLog2e = 1.4426950408889634f;

// Pixel mapping: warp w covers the 8x8 block (w % 2, w / 2) of the tile; lane l owns the two
// vertically adjacent pixels (l % 8, 2 (l / 8)) and (l % 8, 2 (l / 8) + 1) of that block.
__device__ __forceinline__ void pixels_of(int tid, int& lx, int& ly) {
    const int w = tid >> 5, l = tid & 31;
    lx = (w & 1) * 8 + (l & 7);
    ly = (w >> 1) * 8 + (l >> 3) * 2;
}

// power2 at offset (dx, dy); ax = a2 * dx is shared by the thread's two pixels
__device__ __forceinline__ float power2(float ax, float dx, float dy, float b2, float c2) {
    return __fmaf_rn(__fmul_rn(c2, dy), dy, __fmul_rn(dx, __fmaf_rn(b2, dy, ax)));
}

__device__ __forceinline__ float ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// raw opacity o G and the clamped alpha
__device__ __forceinline__ float raw_alpha(float o, float p2) { return __fmul_rn(o, ex2(p2)); }

// Which 8x8 warp blocks of the tile at (tx0, ty0) can hold a pixel with alpha >= 1/255: those
// met by the bounding box of the ellipse d^T Q d <= 2 ln(255 o), Q = [[a, b], [b, c]] the conic
// of record r0/r1/r2 (half extents sqrt(2 ln(255 o) (Q^-1)_xx) and sqrt(... (Q^-1)_yy)).  The
// box is widened by 1e-4 relative + 1e-3 px, far more than the rounding of its computation
// (the determinant is formed without cancellation), so every pixel inside the ellipse keeps its
// per-pixel test; a pixel outside the box would fail it.  Bit w stands for warp w.
__device__ __forceinline__ uint32_t warp_blocks(const float4& r0, const float4& r1, float pskip,
                                                float tx0, float ty0) {
    const float t2 = -2.0f * pskip;                   // 2 ln(255 o)
    if (!(t2 >= 0.0f)) return 0u;                     // o < 1/255: no pixel passes
    const float a = r0.z, b = r0.w, c = r1.x;
    const float bb = b * b;
    const float det = fmaf(a, c, -bb) - fmaf(b, b, -bb);
    if (!(det > 0.0f)) return 0xFu;
    const float k = t2 / det;
    const float ex = fmaf(sqrtf(k * c), 1.0001f, 1e-3f), ey = fmaf(sqrtf(k * a), 1.0001f, 1e-3f);
    uint32_t m = 0;
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        const float qx = tx0 + 8.0f * (w & 1), qy = ty0 + 8.0f * (w >> 1);
        if (r0.x - ex <= qx + 7.0f && r0.x + ex >= qx && r0.y - ey <= qy + 7.0f && r0.y + ey >= qy)
            m |= 1u << w;
    }
    return m;
}

// A record in the form the inner loop wants: the conic pre-scaled so that
// power2 = log2(e) * power = dx (a2 dx + b2 dy) + c2 dy^2 and G = ex2(power2), and the skip
// bound alpha < 1/255 <=> power2 < pskip2.
struct Rec {
    float4 A;   // u, v, a2 = -0.5 a log2e, b2 = -b log2e
    float4 B;   // c2 = -0.5 c log2e, opacity, r, g
    float2 C;   // b (blue), pskip2 = p_skip log2e
    uint32_t blocks;   // warp_blocks() of the record for the tile being blended
};

__device__ __forceinline__ Rec load_rec(const float4* __restrict__ rec, uint32_t g, float tx0,
                                        float ty0) {
    const float4 r0 = rec[3 * (size_t)g], r1 = rec[3 * (size_t)g + 1], r2 = rec[3 * (size_t)g + 2];
    Rec o;
    o.A = make_float4(r0.x, r0.y, -0.5f * kLog2e * r0.z, -kLog2e * r0.w);
    o.B = make_float4(-0.5f * kLog2e * r1.x, r1.y, r1.z, r1.w);
    o.C = make_float2(r2.x, r2.w * kLog2e);
    o.blocks = warp_blocks(r0, r1, r2.w, tx0, ty0);
    return o;
}

// Warp-local list of the batch entries (in order) whose block mask has this warp's bit.
__device__ __forceinline__ int warp_list(const uint8_t* s_m, int cnt, uint8_t* list) {
    const unsigned lane = lane_id(), w = threadIdx.x >> 5;
    int nw = 0;
    for (int base = 0; base < cnt; base += 32) {
        const int e = base + (int)lane;
        const bool hit = e < cnt && ((s_m[e] >> w) & 1u);
        const uint32_t bal = __ballot_sync(0xffffffffu, hit);
        if (hit) list[nw + __popc(bal & lanemask_lt())] = (uint8_t)e;
        nw += __popc(bal);
    }
    __syncwarp();
    return nw;
}

}  // namespace blend
}  // namespace ogs
