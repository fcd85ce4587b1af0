// Fused neural-Gaussian decoding and EWA projection (Sec. 3.2, Eq. offsets and Eq. mlp, then
// Sec. 3.1, Eq. 1) on the tensor cores: the decoded Gaussians of a 128-anchor tile go straight
// from tensor memory to screen-space records, so the Gaussian attributes never travel through
// HBM between the two steps.  Results are bit-for-bit those of ogs_decode_bf16 followed by
// ogs_project_bin (same decoder operands, activations and projection code).
//
// Per tile (8 warps; warps w and w + 4 share TMEM lane quarter w % 4, one anchor row per lane):
//   gather     the anchor inputs (two threads per row) -> BF16 A1 in shared memory
//   layer 1    D[128 x 96]  = A1 . W1^T     (tcgen05, FP32 in TMEM)
//   epilogue   bias, ReLU -> BF16 A2 (the two warps of a lane quarter split the columns)
//   layer 2    D[128 x 112] = A2 . W2blk^T  (block-diagonal decoders; reuses the columns)
//   in two rounds of 64 anchors (so that three CTAs share an SM):
//   stage      the 112 FP32 outputs of each anchor of the round -> shared memory (over the
//              consumed operands)
//   project    one thread per Gaussian, consecutive Gaussians on consecutive threads: bias,
//              activations, mean, projection, tile extent; coalesced record writes and the
//              per-tile pair counts
// The network's BF16 operand image is packed once per call by dp_pack (which also zeroes the
// tile counts) and fetched by every CTA with one bulk copy.  Every mbarrier wait is bounded;
// on expiry the kernel flags ogs_counts.timeout, releases its tensor memory and exits.
#include "decode_common.cuh"
#include "project_common.cuh"

namespace ogs {
namespace {

using namespace dec;

constexpr int kDpThreads = 256;
constexpr uint32_t kDpTmemCols = 128;
constexpr int kYStride = 113;                             // staged outputs per row (odd stride)
constexpr int kRowWords = 8;                              // j, w, dv[3], l_v[3] per row

// network image (global scratch and the head of shared memory)
constexpr int kImgB1 = 0;                                 // 96 x 48 bf16
constexpr int kImgB2 = kImgB1 + kN1 * kK1 * 2;            // 112 x 96 bf16
constexpr int kImgBias1 = kImgB2 + kN2 * kN1 * 2;         // b1 f32[96]
constexpr int kImgBias2 = kImgBias1 + kN1 * 4;            // b2 f32[112] (block order)
constexpr int kImgBytes = kImgBias2 + kN2 * 4;
// shared memory: image | work (A1 + A2 during the products, staged outputs after) | rows
constexpr int kOffWork = kImgBytes;
constexpr int kOffA1 = kOffWork;                          // 128 x 48 bf16
constexpr int kOffA2 = kOffA1 + kTM * kK1 * 2;            // 128 x 96 bf16
constexpr int kOperandBytes = kTM * kK1 * 2 + kTM * kN1 * 2;
constexpr int kRoundRows = kTM / 2;                      // anchors staged per round
constexpr int kStageBytes = kRoundRows * kYStride * 4;
constexpr int kWorkBytes = kOperandBytes > kStageBytes ? kOperandBytes : kStageBytes;
constexpr int kOffRows = kOffWork + kWorkBytes;
constexpr int kDpSmem = kOffRows + kTM * kRowWords * 4;
static_assert(kImgBytes % 16 == 0 && kOffWork % 16 == 0 && kOffA2 % 16 == 0, "alignment");
constexpr int kRoundGauss = kRoundRows * kK;               // 640 Gaussians per round

constexpr int kPackThreads = 256;
constexpr int kPackG1 = kN1 * (kK1 / 8), kPackG2 = kN2 * (kN1 / 8);
constexpr int kPackItems = kPackG1 + kPackG2 + kN1 + kN2;
constexpr int kPackCtas = (kPackItems + kPackThreads - 1) / kPackThreads;

struct DpArgs {
    const float* pos;
    const float* feat;
    const float* offs;
    const float* lv;
    const uint32_t* sel_idx;
    const float* sel_w;
    ogs_counts* counts;
    ogs_gaussians out;          // written when write_gauss != 0
    int write_gauss;
    float4* rec;
    uint32_t* depth_key;
    uint2* rect;
    uint32_t* tiles;
    uint32_t* tile_count;       // may be null
    const unsigned char* img;
    const float* app;           // appearance codes f32[N][n_app] (n_app = 0: none)
    int n_app;
    Cam cam;
};

// The first kPackCtas CTAs write the network image, one 8-element operand row chunk or bias
// per thread; the others zero the n_tc per-tile counts.
__global__ void __launch_bounds__(kPackThreads) dp_pack(ogs_mlp m, unsigned char* img,
                                                        uint32_t* tile_count, int n_tc) {
    pdl_wait();
    pdl_trigger();
    if (blockIdx.x < kPackCtas) {
        const int e = blockIdx.x * kPackThreads + threadIdx.x;
        float v[8];
        if (e < kPackG1) {
            const int n = e / (kK1 / 8), kc = e % (kK1 / 8);
#pragma unroll
            for (int i = 0; i < 8; ++i) v[i] = w1_elem(m, n, 8 * kc + i);
            put8(img + kImgB1, n, kc, kK1, v);
        } else if (e < kPackG1 + kPackG2) {
            const int f = e - kPackG1;
            const int n = f / (kN1 / 8), kc = f % (kN1 / 8);
#pragma unroll
            for (int i = 0; i < 8; ++i) v[i] = w2_elem(m, n, 8 * kc + i);
            put8(img + kImgB2, n, kc, kN1, v);
        } else if (e < kPackG1 + kPackG2 + kN1) {
            const int f = e - kPackG1 - kPackG2;
            reinterpret_cast<float*>(img + kImgBias1)[f] = m.b1[f];
        } else if (e < kPackItems) {
            const int f = e - kPackG1 - kPackG2 - kN1;
            reinterpret_cast<float*>(img + kImgBias2)[f] = b2_elem(m, f);
        }
        return;
    }
    const int nz = gridDim.x - kPackCtas;
    for (int e = (blockIdx.x - kPackCtas) * kPackThreads + threadIdx.x; e < n_tc;
         e += nz * kPackThreads)
        tile_count[e] = 0u;
}

__global__ void __launch_bounds__(kDpThreads, 3) decode_project_tc(DpArgs a) {
    pdl_wait();
    pdl_trigger();
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ __align__(8) uint64_t wbar;
    __shared__ uint32_t tmem_base;
    unsigned char* sB1 = sm + kImgB1;
    unsigned char* sB2 = sm + kImgB2;
    const float* sb1 = reinterpret_cast<const float*>(sm + kImgBias1);
    const float* sb2 = reinterpret_cast<const float*>(sm + kImgBias2);
    unsigned char* sA1 = sm + kOffA1;
    unsigned char* sA2 = sm + kOffA2;
    float* stage = reinterpret_cast<float*>(sm + kOffWork);
    float* rows = reinterpret_cast<float*>(sm + kOffRows);
    const int t = threadIdx.x, w = t >> 5, half = w >> 2;
    const int row = t & (kTM - 1);                       // = 32 (w % 4) + lane
    const uint32_t M = a.counts->n_selected;
    const uint32_t ntiles = (M + kTM - 1) / kTM;
    if (blockIdx.x >= ntiles) return;                    // uniform: no TMEM, no copies
    const Cam& c = a.cam;

    if (t == 0) {
        tc::mbar_init(&mbar, 1);
        tc::mbar_init(&wbar, 1);
        tc::mbar_expect_tx(&wbar, kImgBytes);
        tc::bulk_load(sm, a.img, kImgBytes, &wbar);      // lands while the inputs are gathered
    }
    if (w == 0) {
        tc::tmem_alloc(&tmem_base, kDpTmemCols);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = tmem_base;
    const uint32_t lane_addr = tbase + ((uint32_t)(32 * (w & 3)) << 16);
    const uint32_t id1 = tc::idesc_bf16(kTM, kN1), id2 = tc::idesc_bf16(kTM, kN2);
    uint32_t phase = 0;
    bool aborted = false, have_net = false;

    for (uint32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        // ---- gather: half 0 writes features 0..15 and [dir, d], half 1 features 16..31 ----
        const uint32_t r = tile * kTM + row;
        const bool valid = r < M;
        {
            const float z8[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            if (valid) {
                const uint32_t j = a.sel_idx[r];
                const float4* f4 = reinterpret_cast<const float4*>(a.feat + (size_t)j * kF) + 4 * half;
                const float4 u0 = f4[0], u1 = f4[1], u2 = f4[2], u3 = f4[3];
                const float v0[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
                const float v1[8] = {u2.x, u2.y, u2.z, u2.w, u3.x, u3.y, u3.z, u3.w};
                put8(sA1, row, 2 * half, kK1, v0);
                put8(sA1, row, 2 * half + 1, kK1, v1);
                if (half == 0) {
                    float dv[3];
                    const float d = anchor_offset(a.pos + 3 * (size_t)j, c.c, dv);
                    const float zc[8] = {dv[0] / d, dv[1] / d, dv[2] / d, d, 0.f, 0.f, 0.f, 0.f};
                    put8(sA1, row, kF / 8, kK1, zc);
                    float* rw = rows + row * kRowWords;
                    rw[0] = __uint_as_float(j);
                    rw[1] = a.sel_w[r];
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        rw[2 + q] = dv[q];
                        rw[5 + q] = a.lv[3 * (size_t)j + q];
                    }
                } else {
                    float code[8];
                    app_chunk(a.app, a.n_app, j, code);
                    put8(sA1, row, kK1 / 8 - 1, kK1, code);
                }
            } else {
                put8(sA1, row, 2 * half, kK1, z8);
                put8(sA1, row, 2 * half + 1, kK1, z8);
                put8(sA1, row, half == 0 ? kF / 8 : kK1 / 8 - 1, kK1, z8);
            }
        }
        if (!have_net) {                                 // the network image, once per CTA
            have_net = true;
            if (!tc::mbar_wait(&wbar, 0, kWaitLimit)) {
                if (t == 0) atomicExch(&a.counts->timeout, 1u);
                tc::mbar_wait(&wbar, 0, kWaitLimit);     // copy may still be landing
            }
        }
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
        // ---- layer-1 epilogue: half 0 columns 0..63, half 1 columns 64..95 ----
        for (int c0 = half * 64; c0 < (half ? kN1 : 64); c0 += 32) {
            float v[32];
            tc::tmem_ld32(lane_addr + c0, v);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float h8[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) h8[i] = fmaxf(v[8 * q + i] + sb1[c0 + 8 * q + i], 0.f);
                put8(sA2, row, c0 / 8 + q, kN1, h8);
            }
        }
        tc::fence_smem_to_async();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (t == 0) {
#pragma unroll
            for (int kk = 0; kk < kN1 / 16; ++kk)
                tc::mma_bf16(tbase, tc::smem_desc(tc::smem_u32(sA2 + kk * 256), 128, 16 * kN1),
                             tc::smem_desc(tc::smem_u32(sB2 + kk * 256), 128, 16 * kN1), id2, kk > 0);
            tc::commit(&mbar);
        }
        ok = tc::mbar_wait(&mbar, phase, kWaitLimit);
        if (__syncthreads_or(!ok)) { aborted = true; break; }
        phase ^= 1;
        tc::fence_after_sync();
        const size_t g_base = (size_t)tile * kTM * kK;
        for (int round = 0; round < 2; ++round) {
            // ---- stage the layer-2 outputs of anchors 64 round .. + 63 over the consumed
            //      operands (lane quarters 2 round, 2 round + 1): half 0 columns 0..63, half 1
            //      columns 64..111 ----
            if (((w & 3) >> 1) == round) {
                for (int c0 = half * 64; c0 < half * 64 + 64; c0 += 32) {
                    float v[32];
                    tc::tmem_ld32(lane_addr + c0, v);
                    float* y = stage + (row - kRoundRows * round) * kYStride + c0;
#pragma unroll
                    for (int i = 0; i < 32; ++i)
                        if (c0 + i < kN2) y[i] = v[i];
                }
            }
            tc::fence_before_sync();
            __syncthreads();
            tc::fence_after_sync();
            // ---- project: Gaussian g of the round on thread g % 256 (the same trip count for
            //      every lane of a warp, for the tile counting).  The offsets of the thread's
            //      Gaussians (the only global reads of this phase) are all loaded first, so
            //      their latencies overlap ----
            constexpr int kIters = (kRoundGauss + kDpThreads - 1) / kDpThreads;
            float Opre[kIters][3];
#pragma unroll
            for (int it = 0; it < kIters; ++it) {
                const int gr = it * kDpThreads + t;
                const int gl = kRoundGauss * round + gr;
                const int rl = gl / kK, i = gl - rl * kK;
                if (gr < kRoundGauss && tile * kTM + rl < M) {
                    const uint32_t j = __float_as_uint(rows[rl * kRowWords]);
                    const float* O = a.offs + ((size_t)j * kK + i) * 3;
#pragma unroll
                    for (int q = 0; q < 3; ++q) Opre[it][q] = O[q];
                }
            }
#pragma unroll
            for (int it = 0; it < kIters; ++it) {
                const int gr = it * kDpThreads + t;                 // Gaussian of the round
                const int gl = kRoundGauss * round + gr;            // Gaussian of the tile
                const int rl = gl / kK, i = gl - rl * kK;
                const bool gv = gr < kRoundGauss && tile * kTM + rl < M;
                ProjOut p;
                if (gv) {
                    const float* y = stage + (rl - kRoundRows * round) * kYStride;
                    const float* rw = rows + rl * kRowWords;
                    const uint32_t j = __float_as_uint(rw[0]);
                    const float wgt = rw[1];
                    const float dv[3] = {rw[2], rw[3], rw[4]};
                    const float lvv[3] = {rw[5], rw[6], rw[7]};
                    const float o = act_opacity(wgt, y[i] + sb2[i]);
                    float col[3], scl[3], yc[4], mu[3];
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        col[q] = act_color(y[kK + 3 * i + q] + sb2[kK + 3 * i + q]);
                        scl[q] = act_scale(lvv[q], y[4 * kK + 7 * i + q] + sb2[4 * kK + 7 * i + q]);
                    }
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        yc[q] = y[4 * kK + 7 * i + 3 + q] + sb2[4 * kK + 7 * i + 3 + q];
                    const float inv = act_qinv(yc);
                    const float4 qu = make_float4(yc[0] * inv, yc[1] * inv, yc[2] * inv, yc[3] * inv);
#pragma unroll
                    for (int q = 0; q < 3; ++q) mu[q] = act_mean(dv[q], Opre[it][q], lvv[q]);
                    const size_t gi = g_base + gl;
                    if (a.write_gauss) {
                        a.out.opac[gi] = o;
#pragma unroll
                        for (int q = 0; q < 3; ++q) {
                            a.out.colors[3 * gi + q] = col[q];
                            a.out.scales[3 * gi + q] = scl[q];
                            a.out.means[3 * gi + q] = mu[q];
                        }
                        *reinterpret_cast<float4*>(a.out.quats + 4 * gi) = qu;
                    }
                    p = project_one(c, mu[0], mu[1], mu[2], qu, scl[0], scl[1], scl[2], o,
                                    col[0], col[1], col[2]);
                    a.rec[3 * gi] = p.r0;
                    a.rec[3 * gi + 1] = p.r1;
                    a.rec[3 * gi + 2] = p.r2;
                    a.depth_key[gi] = p.dkey;
                    a.rect[gi] = p.rc;
                    a.tiles[gi] = p.ntiles;
                } else {
                    p.rc = make_uint2(0, 0);
                    p.ntiles = 0;
                }
                if (a.tile_count) count_tiles(a.tile_count, c.gx, p.rc, p.ntiles);
            }
            // the staged round is overwritten by the next round or tile
            __syncthreads();
        }
        // staged outputs and rows are rewritten by the next tile
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
    }
    if (aborted) {
        if (t == 0) atomicExch(&a.counts->timeout, 1u);
        // wait (bounded) for the product that may still be in flight before releasing TMEM
        tc::mbar_wait(&mbar, phase, kWaitLimit);
    }
    if (!have_net) tc::mbar_wait(&wbar, 0, kWaitLimit);   // no tile: let the copy land
    tc::fence_before_sync();
    __syncthreads();
    if (w == 0) tc::tmem_dealloc(tbase, kDpTmemCols);
}

}  // namespace
}  // namespace ogs

using namespace ogs;

extern "C" size_t ogs_decode_project_scratch_bytes(void) { return (size_t)kImgBytes + 256; }

extern "C" ogs_status ogs_decode_project_bf16(
    const float* pos, const float* feat, const float* offs, const float* lv, int64_t N,
    const ogs_mlp* mlp, const ogs_camera* cam, const uint32_t* sel_idx, const float* sel_w,
    int64_t sel_cap, ogs_counts* counts, const ogs_gaussians* out, ogs_rec2d* rec,
    uint32_t* depth_key, uint32_t* rect, uint32_t* tiles, uint32_t* tile_count, void* scratch,
    size_t scratch_bytes, void* stream) {
    if (!pos || !feat || !offs || !lv || !mlp || !cam || !sel_idx || !sel_w || !counts || !rec ||
        !depth_key || !rect || !tiles || !scratch)
        return OGS_ERR_ARG;
    if (mlp->F != kF || mlp->H != kH || mlp->k != kK || N < 0 || sel_cap < 0 || !app_ok(*mlp))
        return OGS_ERR_ARG;
    if (!mlp->w1 || !mlp->b1 || !mlp->w2_op || !mlp->b2_op || !mlp->w2_col || !mlp->b2_col ||
        !mlp->w2_cov || !mlp->b2_cov)
        return OGS_ERR_ARG;
    const bool write_gauss = out != nullptr;
    if (write_gauss && (!out->means || !out->scales || !out->quats || !out->opac ||
                        !out->colors || !aligned(out->quats, 16)))
        return OGS_ERR_ARG;
    if (!aligned(feat, 16) || !aligned(rec, 16) || !aligned(rect, 8) || !aligned(scratch, 16) ||
        scratch_bytes < ogs_decode_project_scratch_bytes())
        return OGS_ERR_ARG;
    if (cam->width <= 0 || cam->height <= 0 || cam->width > 16 * 65535 || cam->height > 16 * 65535)
        return OGS_ERR_ARG;
    const Cam cm = make_cam(*cam);
    cudaStream_t st = (cudaStream_t)stream;
    const int n_tc = tile_count ? cm.gx * cm.gy : 0;
    unsigned char* img = (unsigned char*)scratch;
    const int pack_grid = kPackCtas + (n_tc + 4 * kPackThreads - 1) / (4 * kPackThreads);
    launch_pdl(dp_pack, dim3(pack_grid), dim3(kPackThreads), 0, st, *mlp, img, tile_count, n_tc);
    if (sel_cap == 0) return launch_status();
    if (cudaFuncSetAttribute(decode_project_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kDpSmem) != cudaSuccess)
        return OGS_ERR_CUDA;
    DpArgs a{pos, feat, offs, lv, sel_idx, sel_w, counts,
             write_gauss ? *out : ogs_gaussians{nullptr, nullptr, nullptr, nullptr, nullptr},
             write_gauss ? 1 : 0, reinterpret_cast<float4*>(rec), depth_key,
             reinterpret_cast<uint2*>(rect), tiles, tile_count, img, mlp->app, mlp->A, cm};
    const int64_t tiles_cap = (sel_cap + kTM - 1) / kTM;
    const int grid = (int)(tiles_cap < 3 * kSmCount ? tiles_cap : 3 * kSmCount);
    launch_pdl(decode_project_tc, dim3(grid), dim3(kDpThreads), kDpSmem, st, a);
    return launch_status();
}
