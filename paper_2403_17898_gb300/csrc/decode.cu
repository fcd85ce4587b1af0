// Neural-Gaussian decoding (Sec. 3.2): per selected anchor, the three attribute MLPs
// (Eq. mlp) and the offset positions (Eq. offsets), FP32 on the CUDA cores.
//
// One thread per selected anchor; decoder weights (~30 KB, second layers transposed) live in
// shared memory and every weight read is a warp-wide broadcast.  Each decoder runs in
// outer-product form (loop over hidden units, all outputs accumulated in registers), so only
// the 36-wide input and one decoder's outputs are live.  Means are written camera-relative
// (x_v - campos + O_i * l_v) so FP32 keeps them accurate far from the world origin.  With
// appearance codes (Sec. 4.4) the colour decoder's hidden units also see the anchor's code.
#include "internal.cuh"

namespace ogs {
namespace {

constexpr int kDecThreads = 128;
constexpr int kF = 32;
constexpr int kH = 32;
constexpr int kDin = kF + 4;

struct DecArgs {
    const float* pos;
    const float* feat;
    const float* offs;
    const float* lv;
    const uint32_t* sel_idx;
    const float* sel_w;
    const ogs_counts* counts;
    int64_t sel_cap;
    ogs_mlp mlp;
    ogs_gaussians out;
    Cam cam;
};

__device__ __forceinline__ float sigmoidf_(float x) { return 1.0f / (1.0f + __expf(-x)); }

// Padded output widths of the three decoders (rows of the transposed second layer are kept
// 16-byte aligned in shared memory).
template <int K> struct Widths {
    static constexpr int op = (K + 3) / 4 * 4;
    static constexpr int col = (3 * K + 3) / 4 * 4;
    static constexpr int cov = (7 * K + 3) / 4 * 4;
};

// One decoder: y = W2 relu(W1 z + b1 [+ Wa code]) + b2.  w2t is the transposed second layer
// [H][NP]; with APP the hidden unit o also adds wa[o][0..8) . code (Sec. 4.4, zero-padded).
template <int NOUT, int NP, bool APP = false>
__device__ __forceinline__ void decoder(const float* __restrict__ w1, const float* __restrict__ b1,
                                        const float* __restrict__ w2t, const float* __restrict__ b2,
                                        const float (&z)[kDin], float (&y)[NOUT],
                                        const float* __restrict__ wa = nullptr,
                                        const float* code = nullptr) {
#pragma unroll
    for (int i = 0; i < NOUT; ++i) y[i] = b2[i];
#pragma unroll 1
    for (int o = 0; o < kH; ++o) {
        const float4* row = reinterpret_cast<const float4*>(w1 + o * kDin);
        float a = b1[o];
#pragma unroll
        for (int i = 0; i < kDin / 4; ++i) {
            const float4 w = row[i];
            a = fmaf(w.x, z[4 * i], a);
            a = fmaf(w.y, z[4 * i + 1], a);
            a = fmaf(w.z, z[4 * i + 2], a);
            a = fmaf(w.w, z[4 * i + 3], a);
        }
        if (APP) {
#pragma unroll
            for (int c = 0; c < kMaxApp; ++c) a = fmaf(wa[o * kMaxApp + c], code[c], a);
        }
        a = fmaxf(a, 0.0f);
        const float4* col = reinterpret_cast<const float4*>(w2t + o * NP);
#pragma unroll
        for (int i = 0; i < NOUT / 4; ++i) {
            const float4 w = col[i];
            y[4 * i] = fmaf(w.x, a, y[4 * i]);
            y[4 * i + 1] = fmaf(w.y, a, y[4 * i + 1]);
            y[4 * i + 2] = fmaf(w.z, a, y[4 * i + 2]);
            y[4 * i + 3] = fmaf(w.w, a, y[4 * i + 3]);
        }
#pragma unroll
        for (int i = NOUT / 4 * 4; i < NOUT; ++i) y[i] = fmaf(w2t[o * NP + i], a, y[i]);
    }
}

template <int K, bool APP>
__global__ void __launch_bounds__(kDecThreads) decode_fp32(DecArgs a) {
    using Wd = Widths<K>;
    extern __shared__ __align__(16) float sm[];
    float* w1 = sm;                                  // [3][H][Din]
    float* b1 = w1 + 3 * kH * kDin;                  // [3][H]
    float* t_op = b1 + 3 * kH;                       // [H][op]   transposed layer 2
    float* t_col = t_op + kH * Wd::op;               // [H][col]
    float* t_cov = t_col + kH * Wd::col;             // [H][cov]
    float* b_op = t_cov + kH * Wd::cov;              // [op]
    float* b_col = b_op + Wd::op;                    // [col]
    float* b_cov = b_col + Wd::col;                  // [cov]
    float* w_app = b_cov + Wd::cov;                  // [H][8] appearance weights (APP only)
    for (int i = threadIdx.x; i < 3 * kH * kDin; i += blockDim.x) w1[i] = a.mlp.w1[i];
    for (int i = threadIdx.x; i < 3 * kH; i += blockDim.x) b1[i] = a.mlp.b1[i];
    for (int i = threadIdx.x; i < kH * Wd::op; i += blockDim.x) {
        int o = i / Wd::op, r = i % Wd::op;
        t_op[i] = r < K ? a.mlp.w2_op[r * kH + o] : 0.f;
    }
    for (int i = threadIdx.x; i < kH * Wd::col; i += blockDim.x) {
        int o = i / Wd::col, r = i % Wd::col;
        t_col[i] = r < 3 * K ? a.mlp.w2_col[r * kH + o] : 0.f;
    }
    for (int i = threadIdx.x; i < kH * Wd::cov; i += blockDim.x) {
        int o = i / Wd::cov, r = i % Wd::cov;
        t_cov[i] = r < 7 * K ? a.mlp.w2_cov[r * kH + o] : 0.f;
    }
    for (int i = threadIdx.x; i < Wd::op; i += blockDim.x) b_op[i] = i < K ? a.mlp.b2_op[i] : 0.f;
    for (int i = threadIdx.x; i < Wd::col; i += blockDim.x) b_col[i] = i < 3 * K ? a.mlp.b2_col[i] : 0.f;
    for (int i = threadIdx.x; i < Wd::cov; i += blockDim.x) b_cov[i] = i < 7 * K ? a.mlp.b2_cov[i] : 0.f;
    if (APP) {
        for (int i = threadIdx.x; i < kH * kMaxApp; i += blockDim.x) {
            const int o = i / kMaxApp, q = i % kMaxApp;
            w_app[i] = q < a.mlp.A ? a.mlp.w1_app[o * a.mlp.A + q] : 0.f;
        }
    }
    __syncthreads();
    const uint32_t M = a.counts->n_selected;
    const Cam& c = a.cam;
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < M; r += gridDim.x * blockDim.x) {
        const uint32_t j = a.sel_idx[r];
        const float w = a.sel_w[r];
        float z[kDin];
        const float4* f4 = reinterpret_cast<const float4*>(a.feat + (size_t)j * kF);
#pragma unroll
        for (int i = 0; i < kF / 4; ++i) {
            const float4 v = f4[i];
            z[4 * i] = v.x; z[4 * i + 1] = v.y; z[4 * i + 2] = v.z; z[4 * i + 3] = v.w;
        }
        float dv[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) dv[q] = a.pos[3 * (size_t)j + q] - c.c[q];
        const float d = sqrtf(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
        z[kF] = dv[0] / d; z[kF + 1] = dv[1] / d; z[kF + 2] = dv[2] / d; z[kF + 3] = d;
        const size_t g0 = (size_t)r * K;
        {   // opacity: w * tanh (a Gaussian with opacity <= 0 is dropped by the projection)
            float y[K];
            decoder<K, Wd::op>(w1, b1, t_op, b_op, z, y);
#pragma unroll
            for (int i = 0; i < K; ++i) a.out.opac[g0 + i] = w * tanhf(y[i]);
        }
        {   // colour: sigmoid
            float y[3 * K];
            if (APP) {
                float code[kMaxApp];
#pragma unroll
                for (int q = 0; q < kMaxApp; ++q)
                    code[q] = q < a.mlp.A ? a.mlp.app[(size_t)j * a.mlp.A + q] : 0.f;
                decoder<3 * K, Wd::col, true>(w1 + kH * kDin, b1 + kH, t_col, b_col, z, y, w_app,
                                              code);
            } else {
                decoder<3 * K, Wd::col>(w1 + kH * kDin, b1 + kH, t_col, b_col, z, y);
            }
#pragma unroll
            for (int i = 0; i < 3 * K; ++i) a.out.colors[3 * g0 + i] = sigmoidf_(y[i]);
        }
        {   // covariance: scale = l_v * sigmoid, quaternion normalised; and positions
            float y[7 * K];
            decoder<7 * K, Wd::cov>(w1 + 2 * kH * kDin, b1 + 2 * kH, t_cov, b_cov, z, y);
            float lv[3];
#pragma unroll
            for (int q = 0; q < 3; ++q) lv[q] = a.lv[3 * (size_t)j + q];
#pragma unroll
            for (int i = 0; i < K; ++i) {
                const size_t g = g0 + i;
#pragma unroll
                for (int q = 0; q < 3; ++q) a.out.scales[3 * g + q] = lv[q] * sigmoidf_(y[7 * i + q]);
                const float q0 = y[7 * i + 3], q1 = y[7 * i + 4], q2 = y[7 * i + 5], q3 = y[7 * i + 6];
                const float inv = 1.0f / sqrtf(q0 * q0 + q1 * q1 + q2 * q2 + q3 * q3);
                *reinterpret_cast<float4*>(a.out.quats + 4 * g) =
                    make_float4(q0 * inv, q1 * inv, q2 * inv, q3 * inv);
                const float* O = a.offs + ((size_t)j * K + i) * 3;
#pragma unroll
                for (int q = 0; q < 3; ++q) a.out.means[3 * g + q] = dv[q] + O[q] * lv[q];
            }
        }
    }
}

template <int K, bool APP>
ogs_status launch_decode(const DecArgs& a, cudaStream_t st) {
    using Wd = Widths<K>;
    size_t smem = sizeof(float) * (3 * kH * kDin + 3 * kH + (kH + 1) * (Wd::op + Wd::col + Wd::cov) +
                                   (APP ? kH * kMaxApp : 0));
    if (cudaFuncSetAttribute(decode_fp32<K, APP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return OGS_ERR_CUDA;
    int grid = stride_grid(a.sel_cap, kDecThreads, 4);
    decode_fp32<K, APP><<<grid, kDecThreads, smem, st>>>(a);
    return launch_status();
}

}  // namespace
}  // namespace ogs

using namespace ogs;

extern "C" ogs_status ogs_decode(const float* pos, const float* feat, const float* offs,
                                 const float* lv, int64_t N, const ogs_mlp* mlp,
                                 const ogs_camera* cam, const uint32_t* sel_idx,
                                 const float* sel_w, int64_t sel_cap, const ogs_counts* counts,
                                 const ogs_gaussians* out, void* stream) {
    if (!pos || !feat || !offs || !lv || !mlp || !cam || !sel_idx || !sel_w || !counts || !out)
        return OGS_ERR_ARG;
    if (mlp->F != kF || mlp->H != kH || mlp->k != 10 || N < 0 || sel_cap < 0 || !app_ok(*mlp))
        return OGS_ERR_ARG;
    if (!mlp->w1 || !mlp->b1 || !mlp->w2_op || !mlp->b2_op || !mlp->w2_col || !mlp->b2_col ||
        !mlp->w2_cov || !mlp->b2_cov)
        return OGS_ERR_ARG;
    if (!out->means || !out->scales || !out->quats || !out->opac || !out->colors)
        return OGS_ERR_ARG;
    if (!aligned(feat, 16) || !aligned(out->quats, 16) || !aligned(mlp->w1, 16)) return OGS_ERR_ARG;
    if (sel_cap == 0) return OGS_OK;
    DecArgs a{pos, feat, offs, lv, sel_idx, sel_w, counts, sel_cap, *mlp, *out, make_cam(*cam)};
    return mlp->A > 0 ? launch_decode<10, true>(a, (cudaStream_t)stream)
                      : launch_decode<10, false>(a, (cudaStream_t)stream);
}
