// Tensor-core neural-Gaussian decoder pieces shared by ogs_decode_bf16 and the fused decode +
// projection (Sec. 3.2, Eq. offsets and Eq. mlp): tile shapes, the BF16 operand images of the
// two decoder layers and the FP32 output activations, written once so that both kernels
// produce the same bits.
#pragma once

#include "internal.cuh"
#include "tc.cuh"

namespace ogs {
namespace dec {

constexpr int kTM = 128;            // anchors per tile (MMA M)
constexpr int kF = 32;
constexpr int kH = 32;
constexpr int kDin = kF + 4;        // 36
constexpr int kK1 = 48;             // padded layer-1 K
constexpr int kN1 = 3 * kH;         // 96 hidden (layer-1 N, layer-2 K)
constexpr int kK = 10;              // Gaussians per anchor
constexpr int kN2 = 112;            // 110 outputs padded to a multiple of 16
constexpr uint32_t kWaitLimit = 1u << 24;

__device__ __forceinline__ float sigm(float x) { return 1.0f / (1.0f + __expf(-x)); }

// 8 consecutive K values of one row = one 16-byte core-matrix row: a single vector store
__device__ __forceinline__ void put8(unsigned char* base, int row, int kc, int Kpad,
                                     const float (&v)[8]) {
    __nv_bfloat162 h[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) h[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
    *reinterpret_cast<uint4*>(base + tc::core_offset(row, 8 * kc, Kpad)) =
        *reinterpret_cast<const uint4*>(h);
}

constexpr int kAppCol = 40;         // layer-1 K column of an appearance code's first value
static_assert(kAppCol + kMaxApp == kK1, "the code fills the last K chunk");

// Element (n, k) of the layer-1 B operand: W1 [96][36] with K zero-padded to 48; with
// appearance codes (Sec. 4.4) the colour rows 32..63 hold w1_app in columns 40..40+A.
__device__ __forceinline__ float w1_elem(const ogs_mlp& m, int n, int k) {
    if (k < kDin) return m.w1[n * kDin + k];
    const int c = k - kAppCol;
    if (c >= 0 && c < m.A && n >= kH && n < 2 * kH) return m.w1_app[(n - kH) * m.A + c];
    return 0.f;
}

// Layer-1 K columns 40..47 of anchor j's input row: its appearance code, zero-padded (all
// zero without codes).  app: f32[N][A] codes, A: their width (0..8).
__device__ __forceinline__ void app_chunk(const float* __restrict__ app, int A, uint32_t j,
                                          float (&v)[8]) {
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = i < A ? app[(size_t)j * A + i] : 0.f;
}

// Element (n, k) of the block-diagonal layer-2 B operand [112][96]: output rows 0..9 (opacity)
// see hidden units 0..31, rows 10..39 (colour) units 32..63, rows 40..109 (covariance) units
// 64..95; rows 110, 111 are zero.
__device__ __forceinline__ float w2_elem(const ogs_mlp& m, int n, int k) {
    if (n < kK) return k < kH ? m.w2_op[n * kH + k] : 0.f;
    if (n < 4 * kK) return (k >= kH && k < 2 * kH) ? m.w2_col[(n - kK) * kH + (k - kH)] : 0.f;
    if (n < 11 * kK) return k >= 2 * kH ? m.w2_cov[(n - 4 * kK) * kH + (k - 2 * kH)] : 0.f;
    return 0.f;
}

__device__ __forceinline__ float b2_elem(const ogs_mlp& m, int e) {
    return e < kK ? m.b2_op[e] : (e < 4 * kK ? m.b2_col[e - kK]
                                             : (e < 11 * kK ? m.b2_cov[e - 4 * kK] : 0.f));
}

// Camera-relative anchor position dv = x_v - campos and its distance d (explicit
// round-to-nearest operations: the same bits in every kernel that inlines it).
__device__ __forceinline__ float anchor_offset(const float* p, const float* campos,
                                               float (&dv)[3]) {
#pragma unroll
    for (int q = 0; q < 3; ++q) dv[q] = __fsub_rn(p[q], campos[q]);
    return __fsqrt_rn(__fmaf_rn(dv[2], dv[2], __fmaf_rn(dv[1], dv[1], __fmul_rn(dv[0], dv[0]))));
}

// Output activations of Gaussian i of an anchor from its bias-added layer-2 outputs y.
__device__ __forceinline__ float act_opacity(float wgt, float y) { return wgt * tanhf(y); }
__device__ __forceinline__ float act_color(float y) { return sigm(y); }
__device__ __forceinline__ float act_scale(float lv, float y) { return lv * sigm(y); }
__device__ __forceinline__ float act_qinv(const float* yc) {
    const float n2 = __fmaf_rn(yc[3], yc[3], __fmaf_rn(yc[2], yc[2],
                               __fmaf_rn(yc[1], yc[1], __fmul_rn(yc[0], yc[0]))));
    return __frcp_rn(__fsqrt_rn(n2));
}
__device__ __forceinline__ float act_mean(float dv, float o, float lv) {
    return __fmaf_rn(o, lv, dv);
}

}  // namespace dec
}  // namespace ogs
