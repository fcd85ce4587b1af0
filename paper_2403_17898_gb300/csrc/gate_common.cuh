// The learned anchor-visibility gate's network on the tensor cores, shared by the standalone
// gate (ogs_proposal_gate_bf16) and the gated selection (ogs_lod_select_gated), so that both
// take every keep decision with the same bits: the input vector of an anchor, the BF16 operand
// image of the network, and the two hidden layers of a 128-anchor tile as tcgen05 products
// with their FP32 epilogues.
#pragma once

#include "internal.cuh"
#include "tc.cuh"

namespace ogs {
namespace gate {

constexpr int kPIn = 37;                 // inputs: f_v (32), level, camera-frame direction, ln d
constexpr int kPInPad = 40;
constexpr int kPH = 64;                  // hidden width
constexpr int kGK1 = 48;                 // layer-1 K (inputs zero-padded)
constexpr uint32_t kGTmemCols = 64;
constexpr uint32_t kGWaitLimit = 1u << 24;
// network image (global scratch, packed once per call, and the head of shared memory)
constexpr int kGOffB1 = 0;                               // 64 x 48 bf16
constexpr int kGOffB2 = kGOffB1 + kPH * kGK1 * 2;        // 64 x 64 bf16
constexpr int kGOffVec = kGOffB2 + kPH * kPH * 2;        // b1, b2, w3 (f32), b3 (+ pad)
constexpr int kGImgBytes = kGOffVec + (3 * kPH + 4) * 4;
constexpr int kGABytes = 128 * kPH * 2;                  // A operand: 128 x 64 bf16 (A1 is x 48)
static_assert(kGImgBytes % 16 == 0, "bulk copy granularity");

__device__ __forceinline__ void gput8(unsigned char* base, int row, int kc, int Kpad,
                                      const float (&v)[8]) {
    __nv_bfloat162 h[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) h[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
    *reinterpret_cast<uint4*>(base + tc::core_offset(row, 8 * kc, Kpad)) =
        *reinterpret_cast<const uint4*>(h);
}

// Inputs 32..39 of an anchor's vector: L / (NL - 1), the unit viewing direction in the camera
// frame, ln(d / d_max), zeros.  Every operation is an explicit round-to-nearest intrinsic, so
// each kernel that inlines this computes the same bits.
__device__ __forceinline__ void prop_extras(float p0, float p1, float p2, uint32_t level, int NL,
                                            const Cam& c, float (&e)[8]) {
    const float dx = __fsub_rn(p0, c.c[0]), dy = __fsub_rn(p1, c.c[1]), dz = __fsub_rn(p2, c.c[2]);
    const float d = __fsqrt_rn(__fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx))));
    e[0] = __fdiv_rn((float)level, (float)max(NL - 1, 1));
#pragma unroll
    for (int r = 0; r < 3; ++r)
        e[1 + r] = __fdiv_rn(__fmaf_rn(c.R[3 * r + 2], dz,
                                       __fmaf_rn(c.R[3 * r + 1], dy, __fmul_rn(c.R[3 * r], dx))),
                             d);
    e[4] = logf(__fdiv_rn(d, c.d_max));
    e[5] = e[6] = e[7] = 0.f;
}

// Input vector of an anchor: [f_v, L / (NL - 1), unit viewing direction in the camera frame,
// ln(d / d_max)], padded with zeros to 40.  feat: the anchor's 32 features (16-byte aligned);
// p: its position.
__device__ __forceinline__ void prop_input_vals(const float* __restrict__ feat, float p0,
                                                float p1, float p2, uint32_t level, int NL,
                                                const Cam& c, float (&x)[kPInPad]) {
    const float4* f4 = reinterpret_cast<const float4*>(feat);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const float4 v = f4[i];
        x[4 * i] = v.x; x[4 * i + 1] = v.y; x[4 * i + 2] = v.z; x[4 * i + 3] = v.w;
    }
    float e[8];
    prop_extras(p0, p1, p2, level, NL, c, e);
#pragma unroll
    for (int i = 0; i < 8; ++i) x[32 + i] = e[i];
}

// Writes row `row` of the layer-1 A operand (K = 48) from an input vector (inputs 40..47 zero).
__device__ __forceinline__ void put_input_row(unsigned char* sA, int row, const float (&x)[kPInPad]) {
#pragma unroll
    for (int kc = 0; kc < kPInPad / 8; ++kc) {
        const float v[8] = {x[8 * kc], x[8 * kc + 1], x[8 * kc + 2], x[8 * kc + 3],
                            x[8 * kc + 4], x[8 * kc + 5], x[8 * kc + 6], x[8 * kc + 7]};
        gput8(sA, row, kc, kGK1, v);
    }
    const float z8[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    gput8(sA, row, kGK1 / 8 - 1, kGK1, z8);
}

// Half `half` (0 or 1) of row `row` of the layer-1 A operand, written by one of two threads:
// half 0 writes features 0..15 and inputs 32..39 (extras), half 1 features 16..31 and the zero
// inputs 40..47.  feat: the anchor's features, or null for an empty row.  The same bits as
// put_input_row of the full vector.
__device__ __forceinline__ void put_input_half(unsigned char* sA, int row, int half,
                                               const float* __restrict__ feat, float p0,
                                               float p1, float p2, uint32_t level, int NL,
                                               const Cam& c) {
    float v0[8], v1[8], e[8];
    if (feat) {
        const float4* f4 = reinterpret_cast<const float4*>(feat) + 4 * half;
        const float4 u0 = f4[0], u1 = f4[1], u2 = f4[2], u3 = f4[3];
        v0[0] = u0.x; v0[1] = u0.y; v0[2] = u0.z; v0[3] = u0.w;
        v0[4] = u1.x; v0[5] = u1.y; v0[6] = u1.z; v0[7] = u1.w;
        v1[0] = u2.x; v1[1] = u2.y; v1[2] = u2.z; v1[3] = u2.w;
        v1[4] = u3.x; v1[5] = u3.y; v1[6] = u3.z; v1[7] = u3.w;
        if (half == 0) {
            prop_extras(p0, p1, p2, level, NL, c, e);
        } else {
#pragma unroll
            for (int i = 0; i < 8; ++i) e[i] = 0.f;
        }
    } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) v0[i] = v1[i] = e[i] = 0.f;
    }
    gput8(sA, row, 2 * half, kGK1, v0);
    gput8(sA, row, 2 * half + 1, kGK1, v1);
    gput8(sA, row, half == 0 ? kPInPad / 8 - 1 : kGK1 / 8 - 1, kGK1, e);
}

// Both hidden layers of the network for the 128 rows of the layer-1 operand in sA (written by
// the caller): D = A1 W1^T (64 TMEM columns), bias + ReLU -> BF16 A2 (over A1, which the first
// product has consumed), D = A2 W2^T, then the FP32 output logit w3 . relu(D + b2) + b3 of row
// threadIdx.x.  Called by every thread of the CTA (it holds the barriers); threads 0..127
// (warps 0..3, one TMEM lane quarter each) do the epilogues, the others return 0.  img: the
// network image in shared memory; tbase: 64 allocated TMEM columns; mbar: the product barrier
// with its running phase.  Returns false (in every thread) if a product's wait expired; the
// caller must then wait (bounded) on mbar at `phase` before releasing TMEM.
__device__ __forceinline__ bool gate_hidden(unsigned char* sA, const unsigned char* img,
                                            uint32_t tbase, uint64_t* mbar, uint32_t& phase,
                                            float& z) {
    const int t = threadIdx.x, w = t >> 5;
    const unsigned char* sB1 = img + kGOffB1;
    const unsigned char* sB2 = img + kGOffB2;
    const float* sb1 = reinterpret_cast<const float*>(img + kGOffVec);
    const float* sb2 = sb1 + kPH;
    const float* sw3 = sb2 + kPH;
    const uint32_t id = tc::idesc_bf16(128, kPH);
    const uint32_t lane_addr = tbase + ((uint32_t)(32 * (w & 3)) << 16);
    z = 0.f;
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (t == 0) {
#pragma unroll
        for (int kk = 0; kk < kGK1 / 16; ++kk)
            tc::mma_bf16(tbase, tc::smem_desc(tc::smem_u32(sA + kk * 256), 128, 16 * kGK1),
                         tc::smem_desc(tc::smem_u32(sB1 + kk * 256), 128, 16 * kGK1), id, kk > 0);
        tc::commit(mbar);
    }
    bool ok = tc::mbar_wait(mbar, phase, kGWaitLimit);
    if (__syncthreads_or(!ok)) return false;
    phase ^= 1;
    tc::fence_after_sync();
    if (t < 128) {
#pragma unroll
        for (int c0 = 0; c0 < kPH; c0 += 32) {
            float v[32];
            tc::tmem_ld32(lane_addr + c0, v);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float h8[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) h8[i] = fmaxf(v[8 * q + i] + sb1[c0 + 8 * q + i], 0.f);
                gput8(sA, t, c0 / 8 + q, kPH, h8);
            }
        }
    }
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (t == 0) {
#pragma unroll
        for (int kk = 0; kk < kPH / 16; ++kk)
            tc::mma_bf16(tbase, tc::smem_desc(tc::smem_u32(sA + kk * 256), 128, 16 * kPH),
                         tc::smem_desc(tc::smem_u32(sB2 + kk * 256), 128, 16 * kPH), id, kk > 0);
        tc::commit(mbar);
    }
    ok = tc::mbar_wait(mbar, phase, kGWaitLimit);
    if (__syncthreads_or(!ok)) return false;
    phase ^= 1;
    tc::fence_after_sync();
    if (t < 128) {
        float acc = sb1[3 * kPH];                  // b3
#pragma unroll
        for (int c0 = 0; c0 < kPH; c0 += 32) {
            float v[32];
            tc::tmem_ld32(lane_addr + c0, v);
#pragma unroll
            for (int i = 0; i < 32; ++i) acc = fmaf(sw3[c0 + i], fmaxf(v[i] + sb2[c0 + i], 0.f), acc);
        }
        z = acc;
    }
    return true;
}

// Keep probability from the logit (the same expression in every gate form).
__device__ __forceinline__ float keep_prob(float z) { return 1.0f / (1.0f + __expf(-z)); }

// Enqueues the packing of the network's BF16 operand image (kGImgBytes, 16-byte aligned) into
// img; with n_words > 0 the same launch also zeroes the 64-bit words status[0 .. n_words).
ogs_status pack_image(const ogs_proposal& net, unsigned char* img, unsigned long long* status,
                      int n_words, cudaStream_t st);

}  // namespace gate
}  // namespace ogs
