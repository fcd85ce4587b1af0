// Neural-Gaussian decoding (Sec. 3.2, Eq. offsets and Eq. mlp) on the 5th-generation tensor
// cores: both decoder layers as BF16 x BF16 -> FP32 tcgen05 MMAs, 128 anchors per tile.
//
//   layer 1:  D1[128 x 96]  = Z[128 x 48] . W1^T       (3 decoders stacked along N;
//                                                        K = 36 inputs padded to 48)
//   layer 2:  D2[128 x 112] = H[128 x 96] . W2blk^T    (block-diagonal: each decoder's
//                                                        outputs only see its own hidden)
// Operands live in shared memory in the no-swizzle K-major core-matrix layout (8 rows x 16
// bytes per core matrix); accumulators live in tensor memory (128 columns: layer 2 reuses the
// columns of layer 1 once its epilogue has read them), so three CTAs share an SM.  One thread
// issues the MMAs and commits them to an mbarrier; the four warps read their 32 accumulator
// rows each (one anchor per thread) for the bias/ReLU epilogue of layer 1 and the activation
// epilogue of layer 2 (FP32).  Each output array of a tile is staged in the (then free)
// layer-2 operand buffer and written with one TMA bulk copy, so global stores are
// contiguous.  Every mbarrier wait is bounded; on expiry the kernel flags ogs_counts.timeout,
// releases its tensor memory and exits.
#include "decode_common.cuh"

namespace ogs {
namespace {

using namespace dec;

constexpr int kTcThreads = 128;     // 4 warps, one anchor (TMEM lane) per thread
constexpr uint32_t kTmemCols = 128;
constexpr uint32_t kD2Col = 0;          // layer 2 overwrites layer 1's (already read) columns

// shared-memory carve (bytes)
constexpr int kOffA1 = 0;                               // 128 x 48 bf16
constexpr int kOffB1 = kOffA1 + kTM * kK1 * 2;          // 96 x 48 bf16
constexpr int kOffA2 = kOffB1 + kN1 * kK1 * 2;          // 128 x 96 bf16
constexpr int kOffB2 = kOffA2 + kTM * kN1 * 2;          // 112 x 96 bf16
constexpr int kOffBias = kOffB2 + kN2 * kN1 * 2;        // 96 + 112 f32
constexpr int kSmemUsed = kOffBias + (kN1 + kN2) * 4;
// three CTAs per SM: 3 x 72 KB of shared memory and 3 x 128 of the 512 TMEM columns
constexpr int kSmemRequest = 72 * 1024;
static_assert(kTM * kK * 4 * 4 <= kTM * kN1 * 2, "largest staged output (quats) fits in A2");
static_assert(kSmemUsed <= kSmemRequest, "shared memory carve");

struct TcArgs {
    const float* pos;
    const float* feat;
    const float* offs;
    const float* lv;
    const uint32_t* sel_idx;
    const float* sel_w;
    ogs_counts* counts;
    ogs_mlp mlp;
    ogs_gaussians out;
    Cam cam;
};

__global__ void __launch_bounds__(kTcThreads, 3) decode_bf16_tc(TcArgs a) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    unsigned char* sA1 = sm + kOffA1;
    unsigned char* sB1 = sm + kOffB1;
    unsigned char* sA2 = sm + kOffA2;
    unsigned char* sB2 = sm + kOffB2;
    float* sb1 = reinterpret_cast<float*>(sm + kOffBias);
    float* sb2 = sb1 + kN1;
    const int t = threadIdx.x, w = t >> 5;

    // weights -> bf16 operand tiles (zero padding included), one 8-value chunk per store
    for (int e = t; e < kN1 * (kK1 / 8); e += kTcThreads) {
        const int n = e / (kK1 / 8), kc = e % (kK1 / 8);
        float v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = w1_elem(a.mlp, n, 8 * kc + i);
        put8(sB1, n, kc, kK1, v);
    }
    for (int e = t; e < kN2 * (kN1 / 8); e += kTcThreads) {
        const int n = e / (kN1 / 8), kc = e % (kN1 / 8);
        float v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = w2_elem(a.mlp, n, 8 * kc + i);
        put8(sB2, n, kc, kN1, v);
    }
    for (int e = t; e < kN1; e += kTcThreads) sb1[e] = a.mlp.b1[e];
    for (int e = t; e < kN2; e += kTcThreads) sb2[e] = b2_elem(a.mlp, e);
    {   // the last K chunk (columns 40..47) of the input tile: zero unless codes are used
        const float z8[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        put8(sA1, t, kK1 / 8 - 1, kK1, z8);
    }
    const bool app = a.mlp.A > 0;
    if (t == 0) tc::mbar_init(&mbar, 1);
    if (w == 0) {
        tc::tmem_alloc(&tmem_base, kTmemCols);
        tc::tmem_relinquish();
    }
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = tmem_base;
    const uint32_t lane_addr = tbase + ((uint32_t)(32 * w) << 16);
    const uint32_t id1 = tc::idesc_bf16(kTM, kN1), id2 = tc::idesc_bf16(kTM, kN2);
    const uint32_t M = a.counts->n_selected;
    const uint32_t ntiles = (M + kTM - 1) / kTM;
    const Cam& c = a.cam;
    uint32_t phase = 0;
    bool aborted = false;

    for (uint32_t tile = blockIdx.x; tile < ntiles && !aborted; tile += gridDim.x) {
        const uint32_t r = tile * kTM + t;
        const bool valid = r < M;
        uint32_t j = 0;
        float wgt = 0.f, dv[3] = {0.f, 0.f, 0.f};
        float zc[8];
        if (valid) {
            j = a.sel_idx[r];
            wgt = a.sel_w[r];
            const float d = anchor_offset(a.pos + 3 * (size_t)j, c.c, dv);
            const float4* f4 = reinterpret_cast<const float4*>(a.feat + (size_t)j * kF);
#pragma unroll
            for (int kc = 0; kc < kF / 8; ++kc) {
                const float4 u0 = f4[2 * kc], u1 = f4[2 * kc + 1];
                const float v[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
                put8(sA1, t, kc, kK1, v);
            }
            zc[0] = dv[0] / d; zc[1] = dv[1] / d; zc[2] = dv[2] / d; zc[3] = d;
            if (app) {
                float code[8];
                app_chunk(a.mlp.app, a.mlp.A, j, code);
                put8(sA1, t, kK1 / 8 - 1, kK1, code);
            }
        } else {
            const float z8[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int kc = 0; kc < kF / 8; ++kc) put8(sA1, t, kc, kK1, z8);
            if (app) put8(sA1, t, kK1 / 8 - 1, kK1, z8);
            zc[0] = zc[1] = zc[2] = zc[3] = 0.f;
        }
        zc[4] = zc[5] = zc[6] = zc[7] = 0.f;
        put8(sA1, t, kF / 8, kK1, zc);
        tc::fence_smem_to_async();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (t == 0) {
#pragma unroll
            for (int kk = 0; kk < kK1 / 16; ++kk)
                tc::mma_bf16(tbase, tc::smem_desc(tc::smem_u32(sA1 + kk * 256), 128, 16 * kK1),
                             tc::smem_desc(tc::smem_u32(sB1 + kk * 256), 128, 16 * kK1), id1, kk > 0);
            tc::commit(&mbar);
        }
        bool ok = tc::mbar_wait(&mbar, phase, kWaitLimit);
        if (__syncthreads_or(!ok)) { aborted = true; break; }
        phase ^= 1;
        tc::fence_after_sync();
        // layer-1 epilogue: bias, ReLU, bf16 -> layer-2 A tile (row t)
#pragma unroll
        for (int c0 = 0; c0 < kN1; c0 += 32) {
            float v[32];
            tc::tmem_ld32(lane_addr + c0, v);
#pragma unroll
            for (int i = 0; i < 32; ++i) v[i] = fmaxf(v[i] + sb1[c0 + i], 0.f);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float h8[8] = {v[8 * q], v[8 * q + 1], v[8 * q + 2], v[8 * q + 3],
                                     v[8 * q + 4], v[8 * q + 5], v[8 * q + 6], v[8 * q + 7]};
                put8(sA2, t, c0 / 8 + q, kN1, h8);
            }
        }
        tc::fence_smem_to_async();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (t == 0) {
#pragma unroll
            for (int kk = 0; kk < kN1 / 16; ++kk)
                tc::mma_bf16(tbase + kD2Col, tc::smem_desc(tc::smem_u32(sA2 + kk * 256), 128, 16 * kN1),
                             tc::smem_desc(tc::smem_u32(sB2 + kk * 256), 128, 16 * kN1), id2, kk > 0);
            tc::commit(&mbar);
        }
        ok = tc::mbar_wait(&mbar, phase, kWaitLimit);
        if (__syncthreads_or(!ok)) { aborted = true; break; }
        phase ^= 1;
        tc::fence_after_sync();
        // layer-2 epilogue (FP32): activations, positions.  The 112 accumulator columns of
        // this anchor are read once; each output array is staged row-major for the tile in the
        // layer-2 operand buffer (free now) and written with one bulk copy.
        float y[128];
#pragma unroll
        for (int c0 = 0; c0 < 128; c0 += 32) {
            float v[32];
            tc::tmem_ld32(lane_addr + kD2Col + c0, v);
#pragma unroll
            for (int i = 0; i < 32; ++i) y[c0 + i] = v[i];
        }
        float lvv[3] = {0.f, 0.f, 0.f};
        if (valid) {
#pragma unroll
            for (int i = 0; i < kN2; ++i) y[i] += sb2[i];
#pragma unroll
            for (int q = 0; q < 3; ++q) lvv[q] = a.lv[3 * (size_t)j + q];
        }
        const uint32_t nvalid = min((uint32_t)kTM, M - tile * kTM);
        const size_t g0 = (size_t)tile * kTM * kK;        // first Gaussian of the tile
        float* stage = reinterpret_cast<float*>(sA2);
        // (array, floats per Gaussian): opacity 1, colours 3, scales 3, quats 4, means 3
        for (int arr = 0; arr < 5; ++arr) {
            const int per = arr == 0 ? 1 : (arr == 3 ? 4 : 3);
            float* rowp = stage + (size_t)t * kK * per;
            if (valid) {
#pragma unroll
                for (int i = 0; i < kK; ++i) {
                    if (arr == 0) {
                        rowp[i] = act_opacity(wgt, y[i]);
                    } else if (arr == 1) {
#pragma unroll
                        for (int q = 0; q < 3; ++q) rowp[3 * i + q] = act_color(y[kK + 3 * i + q]);
                    } else if (arr == 2) {
#pragma unroll
                        for (int q = 0; q < 3; ++q)
                            rowp[3 * i + q] = act_scale(lvv[q], y[4 * kK + 7 * i + q]);
                    } else if (arr == 3) {
                        const float* yc = y + 4 * kK + 7 * i + 3;
                        const float inv = act_qinv(yc);
#pragma unroll
                        for (int q = 0; q < 4; ++q) rowp[4 * i + q] = yc[q] * inv;
                    } else {
                        const float* O = a.offs + ((size_t)j * kK + i) * 3;
#pragma unroll
                        for (int q = 0; q < 3; ++q) rowp[3 * i + q] = act_mean(dv[q], O[q], lvv[q]);
                    }
                }
            }
            tc::fence_smem_to_async();
            __syncthreads();
            float* dst = arr == 0 ? a.out.opac : (arr == 1 ? a.out.colors :
                         (arr == 2 ? a.out.scales : (arr == 3 ? a.out.quats : a.out.means)));
            const uint32_t bytes = nvalid * kK * per * 4u;
            if ((bytes & 15u) == 0 && (((uintptr_t)(dst + g0 * per)) & 15u) == 0) {
                if (t == 0) {
                    tc::bulk_store(dst + g0 * per, stage, bytes);
                    tc::bulk_commit();
                    tc::bulk_wait_read();
                }
            } else {
                for (uint32_t e = t; e < nvalid * kK * per; e += kTcThreads) dst[g0 * per + e] = stage[e];
            }
            __syncthreads();
        }
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
    }
    if (aborted) {
        if (t == 0) atomicExch(&a.counts->timeout, 1u);
        // wait (bounded) for the MMA group that may still be in flight before releasing TMEM
        tc::mbar_wait(&mbar, phase, kWaitLimit);
    }
    if (t == 0) tc::bulk_wait_all();
    tc::fence_before_sync();
    __syncthreads();
    if (w == 0) tc::tmem_dealloc(tbase, kTmemCols);
}

}  // namespace
}  // namespace ogs

using namespace ogs;

extern "C" ogs_status ogs_decode_bf16(const float* pos, const float* feat, const float* offs,
                                      const float* lv, int64_t N, const ogs_mlp* mlp,
                                      const ogs_camera* cam, const uint32_t* sel_idx,
                                      const float* sel_w, int64_t sel_cap, ogs_counts* counts,
                                      const ogs_gaussians* out, void* stream) {
    if (!pos || !feat || !offs || !lv || !mlp || !cam || !sel_idx || !sel_w || !counts || !out)
        return OGS_ERR_ARG;
    if (mlp->F != kF || mlp->H != kH || mlp->k != kK || N < 0 || sel_cap < 0 || !app_ok(*mlp))
        return OGS_ERR_ARG;
    if (!mlp->w1 || !mlp->b1 || !mlp->w2_op || !mlp->b2_op || !mlp->w2_col || !mlp->b2_col ||
        !mlp->w2_cov || !mlp->b2_cov)
        return OGS_ERR_ARG;
    if (!out->means || !out->scales || !out->quats || !out->opac || !out->colors)
        return OGS_ERR_ARG;
    if (!aligned(feat, 16) || !aligned(out->quats, 16)) return OGS_ERR_ARG;
    if (sel_cap == 0) return OGS_OK;
    if (cudaFuncSetAttribute(decode_bf16_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kSmemRequest) != cudaSuccess)
        return OGS_ERR_CUDA;
    TcArgs args{pos, feat, offs, lv, sel_idx, sel_w, counts, *mlp, *out, make_cam(*cam)};
    int64_t tiles = (sel_cap + kTM - 1) / kTM;
    int grid = (int)(tiles < 2 * kSmCount ? tiles : 2 * kSmCount);
    decode_bf16_tc<<<grid, kTcThreads, kSmemRequest, (cudaStream_t)stream>>>(args);
    return launch_status();
}
