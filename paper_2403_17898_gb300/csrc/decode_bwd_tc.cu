// Backward of the neural-Gaussian decoders (Sec. 3.2, Eq. offsets and Eq. mlp) with the
// per-anchor products on the 5th-generation tensor cores (BF16 x BF16 -> FP32 in TMEM), 128
// anchors per tile, two threads per anchor (TMEM lane; warps w and w + 4 share a lane
// quarter and split the epilogue columns and Gaussians):
//
//   MMA 1:  D[128 x 96]  = Z[128 x 48]  . W1^T     hidden pre-activations (recomputed)
//   MMA 2:  D[128 x 112] = H[128 x 96]  . W2^T     decoder outputs (block-diagonal W2)
//   MMA 3:  D[128 x 96]  = dY[128 x 112] . W2      hidden gradients
//   MMA 4:  D[128 x 32]  = dP[128 x 96]  . W1f     feature gradients (W1 restricted to f_v)
//
// Between them the FP32 epilogues apply bias/ReLU, compute the output gradients dy of every
// Gaussian (shared with the FP32 row pass), mask dh by the ReLU and accumulate dfeat, doffs
// and dlv.  With appearance codes (Sec. 4.4) the code fills Z's zero-padded columns 40..47
// and the colour rows of W1 carry its weights there; the code gradient W_app^T dp is formed
// on the CUDA cores in epilogue 3.  The f32 rows z, h, dy, dp go to scratch for the weight
// pass, which is the FP32 split-over-anchors product of grad.cu.  Operands live in shared memory in the no-swizzle
// K-major core-matrix layout; every mbarrier wait is bounded and on expiry the kernel sets
// ogs_counts.timeout, waits (bounded) for the MMAs in flight, releases TMEM and exits.
#include "decode_bwd.cuh"
#include "tc.cuh"

namespace ogs {
namespace {

using namespace db;

constexpr int kTM = 128;
constexpr int kThreads = 256;            // two threads per anchor (TMEM lane): halves 0 and 1
constexpr int kK1 = 48;                  // 36 inputs padded
constexpr int kN1 = 96;                  // hidden units of the three decoders
constexpr int kN2 = 112;                 // 110 outputs padded
constexpr uint32_t kTmemCols = 256;
constexpr uint32_t kColD1 = 0;           // MMA 1 and MMA 3 (96 columns)
constexpr uint32_t kColD4 = 96;          // MMA 4 (32 columns)
constexpr uint32_t kColD2 = 128;         // MMA 2 (112 columns)
constexpr uint32_t kWaitLimit = 1u << 24;
constexpr int kAppK = 40;                // layer-1 K column of an appearance code's first value

constexpr int kOffA1 = 0;                               // Z   128 x 48
constexpr int kOffB1 = kOffA1 + kTM * kK1 * 2;          // W1   96 x 48
constexpr int kOffA2 = kOffB1 + kN1 * kK1 * 2;          // H, later dP  128 x 96
constexpr int kOffB2 = kOffA2 + kTM * kN1 * 2;          // W2  112 x 96
constexpr int kOffA3 = kOffB2 + kN2 * kN1 * 2;          // dY  128 x 112
constexpr int kOffB3 = kOffA3 + kTM * kN2 * 2;          // W2^T 96 x 112
constexpr int kOffB4 = kOffB3 + kN1 * kN2 * 2;          // W1f^T 32 x 96
constexpr int kOffBias = kOffB4 + kF * kN1 * 2;         // b1 (96) + b2 (112) f32
constexpr int kDyPitch = kN2 + 1;                       // f32 staging of dy per anchor
constexpr int kOffDy = kOffBias + (kN1 + kN2) * 4;
constexpr int kOffDlv = kOffDy + kTM * kDyPitch * 4;    // half 1's dlv partial (3 per anchor)
constexpr int kSmem = kOffDlv + kTM * 3 * 4;
static_assert(kSmem <= 220 * 1024, "shared memory carve");

__device__ __forceinline__ void put8(unsigned char* base, int row, int kc, int Kpad,
                                     const float (&v)[8]) {
    __nv_bfloat162 h[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) h[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
    *reinterpret_cast<uint4*>(base + tc::core_offset(row, 8 * kc, Kpad)) =
        *reinterpret_cast<const uint4*>(h);
}

// stacked output row n of the block-diagonal second layer, hidden unit o: W2[n][o] or 0
__device__ __forceinline__ float w2_blk(const ogs_mlp& w, int n, int o) {
    if (n >= kNOut) return 0.f;
    const int d = dec_of(n);
    if (o / kH != d) return 0.f;
    const int ol = o % kH;
    if (d == 0) return w.w2_op[n * kH + ol];
    if (d == 1) return w.w2_col[(n - kK) * kH + ol];
    return w.w2_cov[(n - 4 * kK) * kH + ol];
}

__device__ __forceinline__ void mma_chain(uint32_t d, const unsigned char* a, const unsigned char* b,
                                          int Kpad, uint32_t idesc) {
    for (int kk = 0; kk < Kpad / 16; ++kk)
        tc::mma_bf16(d, tc::smem_desc(tc::smem_u32(a + kk * 256), 128, 16 * Kpad),
                     tc::smem_desc(tc::smem_u32(b + kk * 256), 128, 16 * Kpad), idesc, kk > 0);
}

// dy of Gaussians [5 kHalf, 5 kHalf + 5) of one anchor from its outputs y, into its f32 staging
// row (compile-time Gaussian indices keep y in registers)
template <int kHalf>
__device__ __forceinline__ void dy_half(const DbArgs& a, const float (&y)[kN2], float* dyrow,
                                        size_t g0, uint32_t j, float wgt, const float (&lvv)[3],
                                        float (&dlv)[3], bool valid) {
#pragma unroll
    for (int ii = 0; ii < kK / 2; ++ii) {
        const int i = kHalf * (kK / 2) + ii;
        float dyv[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        float ys[7];
        if (valid) {
            ys[0] = y[i];
            gaussian_dy(a, 0, g0 + i, j, i, wgt, lvv, ys, dyv, dlv);
        }
        dyrow[i] = dyv[0];
        if (valid) {
#pragma unroll
            for (int e = 0; e < 3; ++e) ys[e] = y[kK + 3 * i + e];
            gaussian_dy(a, 1, g0 + i, j, i, wgt, lvv, ys, dyv, dlv);
        }
#pragma unroll
        for (int e = 0; e < 3; ++e) dyrow[kK + 3 * i + e] = dyv[e];
        if (valid) {
#pragma unroll
            for (int e = 0; e < 7; ++e) ys[e] = y[4 * kK + 7 * i + e];
            gaussian_dy(a, 2, g0 + i, j, i, wgt, lvv, ys, dyv, dlv);
        }
#pragma unroll
        for (int e = 0; e < 7; ++e) dyrow[4 * kK + 7 * i + e] = dyv[e];
    }
}

struct TcBwdArgs {
    DbArgs a;
    uint32_t* timeout;
};

__global__ void __launch_bounds__(kThreads, 1) decode_bwd_rows_tc(TcBwdArgs args) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    __shared__ float sWa[kH * kMaxApp];            // appearance weights [o][c], zero-padded
    const DbArgs& a = args.a;
    unsigned char* sA1 = sm + kOffA1;
    unsigned char* sB1 = sm + kOffB1;
    unsigned char* sA2 = sm + kOffA2;
    unsigned char* sB2 = sm + kOffB2;
    unsigned char* sA3 = sm + kOffA3;
    unsigned char* sB3 = sm + kOffB3;
    unsigned char* sB4 = sm + kOffB4;
    float* sb1 = reinterpret_cast<float*>(sm + kOffBias);
    float* sb2 = sb1 + kN1;
    float* sDy = reinterpret_cast<float*>(sm + kOffDy);
    float* sDlv = reinterpret_cast<float*>(sm + kOffDlv);
    const int t = threadIdx.x, w = t >> 5;
    const int half = w >> 2;                     // warp-uniform
    const int al = t & (kTM - 1);                // anchor (TMEM lane) of this thread
    const uint32_t M = a.counts->n_selected;
    const uint32_t ntiles = (M + kTM - 1) / kTM;
    if (blockIdx.x >= ntiles) return;                      // uniform, before any TMEM use
    const int napp = a.mlp.A;                              // appearance code width (0: none)

    // weights -> bf16 operand tiles, one 8-value chunk per store
    for (int e = t; e < kN1 * (kK1 / 8); e += kThreads) {  // W1 [o][k]
        const int n = e / (kK1 / 8), kc = e % (kK1 / 8);
        float v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int k = 8 * kc + i, ca = k - kAppK;
            // columns 40..47: the colour decoder's appearance weights (Sec. 4.4), else zero
            v[i] = k < kDin ? a.mlp.w1[n * kDin + k]
                            : (ca >= 0 && ca < napp && n >= kH && n < 2 * kH
                                   ? a.mlp.w1_app[(n - kH) * napp + ca] : 0.f);
        }
        put8(sB1, n, kc, kK1, v);
    }
    for (int e = t; e < kH * kMaxApp; e += kThreads) {
        const int o = e / kMaxApp, ca = e % kMaxApp;
        sWa[e] = ca < napp ? a.mlp.w1_app[o * napp + ca] : 0.f;
    }
    for (int e = t; e < kN2 * (kN1 / 8); e += kThreads) {  // W2 block-diagonal [n][o]
        const int n = e / (kN1 / 8), kc = e % (kN1 / 8);
        float v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = w2_blk(a.mlp, n, 8 * kc + i);
        put8(sB2, n, kc, kN1, v);
    }
    for (int e = t; e < kN1 * (kN2 / 8); e += kThreads) {  // W2^T [o][n]
        const int o = e / (kN2 / 8), kc = e % (kN2 / 8);
        float v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = w2_blk(a.mlp, 8 * kc + i, o);
        put8(sB3, o, kc, kN2, v);
    }
    for (int e = t; e < kF * (kN1 / 8); e += kThreads) {   // W1 restricted to f_v, [i][o]
        const int i = e / (kN1 / 8), kc = e % (kN1 / 8);
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = a.mlp.w1[(8 * kc + u) * kDin + i];
        put8(sB4, i, kc, kN1, v);
    }
    for (int e = t; e < kN1; e += kThreads) sb1[e] = a.mlp.b1[e];
    for (int e = t; e < kN2; e += kThreads)
        sb2[e] = e < kK ? a.mlp.b2_op[e]
                        : (e < 4 * kK ? a.mlp.b2_col[e - kK]
                                      : (e < kNOut ? a.mlp.b2_cov[e - 4 * kK] : 0.f));
    if (half == 0) {   // the last K chunk of the input tile (inputs 40..47): zero or the code
        const float z8[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        put8(sA1, al, kK1 / 8 - 1, kK1, z8);
    }
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
    const uint32_t lane_addr = tbase + ((uint32_t)(32 * (w & 3)) << 16);
    const uint32_t id96 = tc::idesc_bf16(kTM, kN1), id112 = tc::idesc_bf16(kTM, kN2),
                   id32 = tc::idesc_bf16(kTM, kF);
    const Cam& c = a.cam;
    uint32_t phase = 0;
    bool aborted = false;

    // issue (thread 0), then all threads wait on the MMA group; false if the wait expired
    auto run = [&](auto issue) -> bool {
        tc::fence_smem_to_async();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (t == 0) {
            issue();
            tc::commit(&mbar);
        }
        const bool ok = tc::mbar_wait(&mbar, phase, kWaitLimit);
        if (__syncthreads_or(!ok)) return false;
        phase ^= 1;
        tc::fence_after_sync();
        return true;
    };
    // columns [32 q0, 32 q1) of a 96-column accumulator belong to this half
    const int q0 = half == 0 ? 0 : 2, q1 = half == 0 ? 2 : 3;

    for (uint32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const uint32_t r = tile * kTM + al;
        const bool valid = r < M;
        uint32_t j = 0;
        float wgt = 0.f, lvv[3] = {0.f, 0.f, 0.f}, dlv[3] = {0.f, 0.f, 0.f};
        if (valid) {
            j = a.sel_idx[r];
            wgt = a.sel_w[r];
#pragma unroll
            for (int q = 0; q < 3; ++q) lvv[q] = a.lv[3 * (size_t)j + q];
        }
        if (half == 0) {
            float zc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            if (valid) {
                float dv[3];
#pragma unroll
                for (int q = 0; q < 3; ++q) dv[q] = a.pos[3 * (size_t)j + q] - c.c[q];
                const float d = sqrtf(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
                zc[0] = dv[0] / d; zc[1] = dv[1] / d; zc[2] = dv[2] / d; zc[3] = d;
                const float4* f4 = reinterpret_cast<const float4*>(a.feat + (size_t)j * kF);
                float4* zr = reinterpret_cast<float4*>(a.rowZ + (size_t)r * kRowZ);
#pragma unroll
                for (int kc = 0; kc < kF / 8; ++kc) {
                    const float4 u0 = f4[2 * kc], u1 = f4[2 * kc + 1];
                    zr[2 * kc] = u0;
                    zr[2 * kc + 1] = u1;
                    const float v[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
                    put8(sA1, al, kc, kK1, v);
                }
                zr[kF / 4] = make_float4(zc[0], zc[1], zc[2], zc[3]);
                zr[kF / 4 + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
            } else {
                const float z8[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int kc = 0; kc < kF / 8; ++kc) put8(sA1, al, kc, kK1, z8);
            }
            put8(sA1, al, kF / 8, kK1, zc);
            if (napp > 0) {
                float code[8];
#pragma unroll
                for (int ca = 0; ca < 8; ++ca)
                    code[ca] = valid && ca < napp ? a.mlp.app[(size_t)j * napp + ca] : 0.f;
                put8(sA1, al, kK1 / 8 - 1, kK1, code);
            }
        }
        if (!run([&] { mma_chain(tbase + kColD1, sA1, sB1, kK1, id96); })) { aborted = true; break; }

        // epilogue 1 (this half's columns): bias, ReLU (mask kept), H -> bf16 operand, f32 row
        uint32_t mask[2] = {0u, 0u};
#pragma unroll
        for (int qq = 0; qq < 2; ++qq) {
            const int q = q0 + qq;
            if (q >= q1) break;
            float v[32];
            tc::tmem_ld32(lane_addr + kColD1 + 32 * q, v);
            uint32_t mk = 0;
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                const float p = v[i] + sb1[32 * q + i];
                mk |= (p > 0.f ? 1u : 0u) << i;
                v[i] = fmaxf(p, 0.f);
            }
            mask[qq] = mk;
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) {
                const float h8[8] = {v[8 * cc], v[8 * cc + 1], v[8 * cc + 2], v[8 * cc + 3],
                                     v[8 * cc + 4], v[8 * cc + 5], v[8 * cc + 6], v[8 * cc + 7]};
                put8(sA2, al, 4 * q + cc, kN1, h8);
            }
            if (valid) {
                float4* hr = reinterpret_cast<float4*>(a.rowH + (size_t)r * kRowH + 32 * q);
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    hr[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
            }
        }
        if (!run([&] { mma_chain(tbase + kColD2, sA2, sB2, kN1, id112); })) { aborted = true; break; }

        // epilogue 2: outputs y -> per-Gaussian gradients dy of this half's five Gaussians,
        // staged in f32 shared memory
        {
            float y[kN2];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float v[32];
                tc::tmem_ld32(lane_addr + kColD2 + 32 * q, v);
#pragma unroll
                for (int i = 0; i < 32; ++i)
                    if (32 * q + i < kN2) y[32 * q + i] = v[i] + sb2[32 * q + i];
            }
            float* dyrow = sDy + al * kDyPitch;
            const size_t g0 = (size_t)r * kK;
            if (half == 0) dy_half<0>(a, y, dyrow, g0, j, wgt, lvv, dlv, valid);
            else dy_half<1>(a, y, dyrow, g0, j, wgt, lvv, dlv, valid);
            if (half == 1) {
#pragma unroll
                for (int e = 0; e < 3; ++e) sDlv[3 * al + e] = dlv[e];
                dyrow[kNOut] = 0.f;
                dyrow[kNOut + 1] = 0.f;
            }
        }
        __syncthreads();
        if (half == 0 && valid) {
#pragma unroll
            for (int e = 0; e < 3; ++e) a.dlv[3 * (size_t)j + e] += dlv[e] + sDlv[3 * al + e];
        }
        {   // dy rows -> bf16 operand and f32 row, chunks split between the halves
            const float* dyrow = sDy + al * kDyPitch;
            for (int cc = half * 7; cc < half * 7 + 7; ++cc) {
                float d8[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) d8[u] = dyrow[8 * cc + u];
                put8(sA3, al, cc, kN2, d8);
                if (valid) {
                    float4* yr = reinterpret_cast<float4*>(a.rowY + (size_t)r * kRowY + 8 * cc);
                    yr[0] = make_float4(d8[0], d8[1], d8[2], d8[3]);
                    yr[1] = make_float4(d8[4], d8[5], d8[6], d8[7]);
                }
            }
        }
        if (!run([&] { mma_chain(tbase + kColD1, sA3, sB3, kN2, id96); })) { aborted = true; break; }

        // epilogue 3 (this half's columns): through the ReLU -> dP (bf16 operand in the H
        // buffer, f32 row)
#pragma unroll
        for (int qq = 0; qq < 2; ++qq) {
            const int q = q0 + qq;
            if (q >= q1) break;
            float v[32];
            tc::tmem_ld32(lane_addr + kColD1 + 32 * q, v);
#pragma unroll
            for (int i = 0; i < 32; ++i) v[i] = ((mask[qq] >> i) & 1u) && valid ? v[i] : 0.f;
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) {
                const float p8[8] = {v[8 * cc], v[8 * cc + 1], v[8 * cc + 2], v[8 * cc + 3],
                                     v[8 * cc + 4], v[8 * cc + 5], v[8 * cc + 6], v[8 * cc + 7]};
                put8(sA2, al, 4 * q + cc, kN1, p8);
            }
            if (valid) {
                float4* pr = reinterpret_cast<float4*>(a.rowP + (size_t)r * kRowP + 32 * q);
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    pr[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
                if (q == 1 && napp > 0) {   // code gradient: dapp_c += sum_o Wa[o][c] dp_o
                    for (int ca = 0; ca < napp; ++ca) {
                        float g = 0.f;
#pragma unroll
                        for (int o = 0; o < kH; ++o) g = fmaf(sWa[o * kMaxApp + ca], v[o], g);
                        a.dapp[(size_t)j * napp + ca] += g;
                    }
                }
            }
        }
        if (!run([&] { mma_chain(tbase + kColD4, sA2, sB4, kN1, id32); })) { aborted = true; break; }

        // epilogue 4: feature gradients
        if (half == 0) {
            float v[32];
            tc::tmem_ld32(lane_addr + kColD4, v);
            if (valid) {
                float4* df = reinterpret_cast<float4*>(a.dfeat + (size_t)j * kF);
#pragma unroll
                for (int i = 0; i < kF / 4; ++i) {
                    float4 u = df[i];
                    u.x += v[4 * i]; u.y += v[4 * i + 1]; u.z += v[4 * i + 2]; u.w += v[4 * i + 3];
                    df[i] = u;
                }
            }
        }
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
    }
    if (aborted) {
        if (t == 0) atomicExch(args.timeout, 1u);
        tc::mbar_wait(&mbar, phase, kWaitLimit);           // the group that may be in flight
    }
    tc::fence_before_sync();
    __syncthreads();
    if (w == 0) tc::tmem_dealloc(tbase, kTmemCols);
}

}  // namespace
}  // namespace ogs

using namespace ogs;
using namespace ogs::db;

extern "C" ogs_status ogs_decode_bwd_bf16(const float* pos, const float* feat, const float* offs,
                                          const float* lv, int64_t N, const ogs_mlp* mlp,
                                          const ogs_camera* cam, const uint32_t* sel_idx,
                                          const float* sel_w, int64_t sel_cap,
                                          ogs_counts* counts, const float* dmeans,
                                          const float* dscales, const float* dquats,
                                          const float* drec, float* dfeat, float* doffs,
                                          float* dlv, const ogs_mlp* dmlp, void* scratch,
                                          size_t scratch_bytes, void* stream) {
    if (!pos || !feat || !offs || !lv || !mlp || !cam || !sel_idx || !sel_w || !counts ||
        !dmeans || !dscales || !dquats || !drec || !dfeat || !doffs || !dlv || !dmlp || !scratch)
        return OGS_ERR_ARG;
    if (mlp->F != kF || mlp->H != kH || mlp->k != kK || N < 0 || sel_cap < 0 || !app_ok(*mlp))
        return OGS_ERR_ARG;
    if (mlp->A > 0 && (!dmlp->w1_app || !dmlp->app)) return OGS_ERR_ARG;
    if (!dmlp->w1 || !dmlp->b1 || !dmlp->w2_op || !dmlp->b2_op || !dmlp->w2_col ||
        !dmlp->b2_col || !dmlp->w2_cov || !dmlp->b2_cov)
        return OGS_ERR_ARG;
    if (scratch_bytes < db_layout(sel_cap, nullptr, nullptr) || !aligned(scratch, 16) ||
        !aligned(dquats, 16) || !aligned(feat, 16) || !aligned(dfeat, 16))
        return OGS_ERR_ARG;
    if (sel_cap == 0) return OGS_OK;
    cudaStream_t st = (cudaStream_t)stream;
    DbScratch sc;
    db_layout(sel_cap, scratch, &sc);
    TcBwdArgs args{{pos, feat, offs, lv, sel_idx, sel_w, counts, *mlp, make_cam(*cam), dmeans,
                    dscales, dquats, drec, dfeat, doffs, dlv, sc.rowY, sc.rowH, sc.rowP, sc.rowZ,
                    sc.partial, const_cast<float*>(dmlp->app)},
                   &counts->timeout};
    if (cudaFuncSetAttribute(decode_bwd_rows_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kSmem) != cudaSuccess)
        return OGS_ERR_CUDA;
    const int64_t tiles = (sel_cap + kTM - 1) / kTM;
    const int grid = (int)(tiles < kSmCount ? tiles : kSmCount);
    decode_bwd_rows_tc<<<grid, kThreads, kSmem, st>>>(args);
    if (launch_weight_pass(args.a, sc, *dmlp, st) != cudaSuccess) return OGS_ERR_CUDA;
    return launch_status();
}
