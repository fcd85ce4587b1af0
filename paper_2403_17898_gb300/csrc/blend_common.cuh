// Per-tile blending conventions shared by the forward and backward blend kernels, so both
// take every skip decision with the same operations in the same order.
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

// A record in the form the inner loop wants: the conic pre-scaled so that
// power2 = log2(e) * power = dx (a2 dx + b2 dy) + c2 dy^2 and G = ex2(power2), and the skip
// bound alpha < 1/255 <=> power2 < pskip2.
struct Rec {
    float4 A;   // u, v, a2 = -0.5 a log2e, b2 = -b log2e
    float4 B;   // c2 = -0.5 c log2e, opacity, r, g
    float2 C;   // b (blue), pskip2 = p_skip log2e
};

__device__ __forceinline__ Rec load_rec(const float4* __restrict__ rec, uint32_t g) {
    const float4 r0 = rec[3 * (size_t)g], r1 = rec[3 * (size_t)g + 1], r2 = rec[3 * (size_t)g + 2];
    Rec o;
    o.A = make_float4(r0.x, r0.y, -0.5f * kLog2e * r0.z, -kLog2e * r0.w);
    o.B = make_float4(-0.5f * kLog2e * r1.x, r1.y, r1.z, r1.w);
    o.C = make_float2(r2.x, r2.w * kLog2e);
    return o;
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

}  // namespace blend
}  // namespace ogs
